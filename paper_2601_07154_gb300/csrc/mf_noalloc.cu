// mf_render_noalloc: the motion-focus path for callers that must not allocate.
//
// Some callers cannot let a library call cudaMalloc: real-time loops that
// must never hit an allocation (cudaMalloc can synchronise the device and
// has no latency bound), plugins that run inside a host framework owning all
// device memory through its own pool, and processes held to a fixed memory
// budget.  This entry point runs the same kernels as a stream (ingest,
// motion points, map, records) but keeps its scratch -- the pose copies,
// their rigidity flags and the per-frame records -- in the file-scope device
// array below, sized for MF_NOALLOC_MAX_FRAMES rendered frames.  Every GPU
// that loads the library holds that array until the process exits.  The
// caller still passes (and owns) the inputs and the outputs.
#include <atomic>
#include <cstring>

#include "mf_internal.h"

namespace {

constexpr int kRingSlots = 512;  // power of two >= MF_NOALLOC_MAX_POSES
static_assert(kRingSlots >= MF_NOALLOC_MAX_POSES, "pose ring too small");
constexpr int kRecSlots = MF_NOALLOC_MAX_FRAMES;  // power of two
static_assert((kRecSlots & (kRecSlots - 1)) == 0, "record ring must be a power of two");

constexpr size_t kRecBytes = sizeof(mf::FrameRec) * kRecSlots;
constexpr size_t kPoseOff = (kRecBytes + 255) / 256 * 256;
constexpr size_t kPoseBytes = sizeof(double) * 12 * kRingSlots;
constexpr size_t kBadOff = kPoseOff + (kPoseBytes + 255) / 256 * 256;
constexpr size_t kSchedOff = kBadOff + (sizeof(int32_t) * kRingSlots + 255) / 256 * 256;
constexpr size_t kFaultOff = kSchedOff + sizeof(unsigned int);
constexpr size_t kScratchBytes = kFaultOff + sizeof(unsigned int);

// The shared scratch: frame records, then pose copies, then rigidity flags,
// then the map kernels' work counter (zero from load, and every map launch
// leaves it at zero), then the fault word a map kernel sets when a bounded
// device wait runs out (this entry point reports that per frame, as
// MF_FRAME_TIMEOUT in the records).
static __device__ __align__(256) unsigned char mf_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::atomic<unsigned char*> g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device.  The symbol
// named in host code is only a host-side stand-in, so the address is looked
// up once per device (with that device current) and cached.
int scratch_on_current_device(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return mf::host_fail(MF_ERR_NO_DEVICE, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return mf::host_fail(MF_ERR_NO_DEVICE, "device id out of range", cudaSuccess);
  unsigned char* p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    void* addr = nullptr;
    e = cudaGetSymbolAddress(&addr, mf_noalloc_scratch);
    if (e != cudaSuccess || !addr)
      return mf::host_fail(MF_ERR_CUDA, "cudaGetSymbolAddress of the scratch array", e);
    p = static_cast<unsigned char*>(addr);
    g_scratch_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return MF_OK;
}

}  // namespace

extern "C" int mf_render_noalloc(const mf_stream_desc* d, int32_t n_poses,
                                 const double* poses_w2c_3x4, int32_t n_render,
                                 const void* depth, const double* K, void* focus_map,
                                 void* guided_depth, mf_frame_info* info) {
  mf::NvtxRange range("mf_render_noalloc");
  int rc = mf::host_validate_desc(d);
  if (rc) return rc;
  if (d->pose_frame != MF_POSES_WORLD)
    return mf::host_fail(MF_ERR_INVALID_ARG, "mf_render_noalloc takes world-frame poses only", cudaSuccess);
  if (n_render < 1 || n_render > n_poses)
    return mf::host_fail(MF_ERR_INVALID_ARG, "need 1 <= n_render <= n_poses", cudaSuccess);
  if (n_render > MF_NOALLOC_MAX_FRAMES)
    return mf::host_fail(MF_ERR_INVALID_ARG,
                         "n_render exceeds MF_NOALLOC_MAX_FRAMES (256): split the call", cudaSuccess);
  if (n_poses > MF_NOALLOC_MAX_POSES)
    return mf::host_fail(MF_ERR_INVALID_ARG,
                         "n_poses exceeds MF_NOALLOC_MAX_POSES (319): pass at most "
                         "window + smooth_len - 2 poses of history", cudaSuccess);
  if (!poses_w2c_3x4 || !K) return mf::host_fail(MF_ERR_INVALID_ARG, "NULL poses or K", cudaSuccess);
  for (int k = 0; k < 4; ++k)
    if (!(K[k] == K[k]) || K[k] - K[k] != 0.0)
      return mf::host_fail(MF_ERR_INVALID_ARG, "non-finite intrinsics", cudaSuccess);
  if (!(K[0] > 0.0) || !(K[1] > 0.0)) return mf::host_fail(MF_ERR_INVALID_ARG, "fx, fy must be > 0", cudaSuccess);
  // every pointer must be device memory of the current device: the kernels
  // run there, and another GPU's memory would fault them
  int dev = -1;
  cudaError_t de = cudaGetDevice(&dev);
  if (de != cudaSuccess) return mf::host_fail(MF_ERR_NO_DEVICE, "cudaGetDevice", de);
  const void* ptrs[5] = {poses_w2c_3x4, depth, focus_map, guided_depth, info};
  for (const void* p : ptrs)
    if (p && mf::host_pointer_kind(p, dev) != mf::kPtrDevice)
      return mf::host_fail(MF_ERR_INVALID_ARG,
                           "mf_render_noalloc takes device pointers of the current device only",
                           cudaSuccess);

  double w[MF_MAX_HISTORY] = {};
  if (!mf::host_ls_weights(d->smooth_len, d->mode, w))
    return mf::host_fail(MF_ERR_INVALID_ARG, "least-squares weights not representable", cudaSuccess);
  unsigned char* scratch = nullptr;
  rc = scratch_on_current_device(&scratch);
  if (rc) return rc;
  mf::FrameRec* recs = reinterpret_cast<mf::FrameRec*>(scratch);
  double* ring = reinterpret_cast<double*>(scratch + kPoseOff);
  int32_t* bad = reinterpret_cast<int32_t*>(scratch + kBadOff);
  unsigned int* sched = reinterpret_cast<unsigned int*>(scratch + kSchedOff);
  cudaStream_t st = static_cast<cudaStream_t>(d->cuda_stream);
  int64_t launches = 0;

  // rigidity check + copy of all poses (frames 0 .. n_poses-1)
  mf::IngestParams ip{};
  ip.in = poses_w2c_3x4;
  ip.n = n_poses;
  ip.first = 0;
  ip.anchor = 0;
  ip.ring = ring;
  ip.ring_bad = bad;
  ip.ring_mask = kRingSlots - 1;
  ip.e0 = 0;
  cudaError_t e = mf::launch_ingest(ip, st, &launches);
  // motion points of the rendered frames (every field, the argmax key
  // included, is rewritten, so nothing from an earlier call survives)
  const int64_t e0 = (int64_t)n_poses - n_render;
  if (e == cudaSuccess) {
    mf::PointsParams pp{};
    pp.ring = ring;
    pp.ring_bad = bad;
    pp.ring_mask = kRingSlots - 1;
    pp.recs = recs;
    pp.rec_mask = kRecSlots - 1;
    pp.e0 = e0;
    pp.n_frames = n_render;
    pp.window = d->window;
    pp.smooth_len = d->smooth_len;
    pp.width = d->width;
    pp.height = d->height;
    pp.calib_width = d->calib_width;
    pp.calib_height = d->calib_height;
    for (int k = 0; k < 4; ++k) pp.K[k] = K[k];
    pp.sigma_rel = d->sigma_rel;
    pp.s_lo = d->s_lo;
    pp.s_hi = d->s_hi;
    std::memcpy(pp.w, w, sizeof(pp.w));
    pp.d0 = d->depth_ref_m;
    e = mf::launch_points(pp, st, &launches);
  }
  if (e == cudaSuccess) {
    mf::MapParams mp{};
    mp.recs = recs;
    mp.rec_mask = kRecSlots - 1;
    mp.f0 = e0;
    mp.n_frames = n_render;
    mp.width = d->width;
    mp.height = d->height;
    mp.tile_h = mf::map_tile_h(d->width, d->height, d->window);
    mp.tiles_x = (d->width + mf::kTileW - 1) / mf::kTileW;
    mp.tiles_y = (d->height + mp.tile_h - 1) / mp.tile_h;
    mp.depth = depth;
    mp.M = focus_map;
    mp.G = guided_depth;
    mp.path = mf::host_map_path(d->flags);
    mp.sched = sched;
    mp.fault = reinterpret_cast<unsigned int*>(scratch + kFaultOff);
    e = mf::launch_map(mp, d->window, d->depth_dtype, d->map_dtype, d->normalize, st, &launches);
  }
  if (e == cudaSuccess && info) {
    mf::FinalizeParams fp{};
    fp.recs = recs;
    fp.rec_mask = kRecSlots - 1;
    fp.f0 = e0;
    fp.n_frames = n_render;
    fp.width = d->width;
    fp.window = d->window;
    fp.info = info;
    fp.points = nullptr;
    fp.normalize = d->normalize;
    e = mf::launch_finalize(fp, st, &launches);
  }
  mf::host_count_launches(launches);
  if (e != cudaSuccess) return mf::host_fail(MF_ERR_CUDA, "mf_render_noalloc launch", e);
  return MF_OK;
}
