// Internal interfaces between the host engine (mf_stream.cpp) and the CUDA
// kernels (mf_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mf.h"
#include "mf_ptr_kind.h"

namespace mf {

constexpr int kMaxPts = MF_MAX_WINDOW;   // N motion points per frame
constexpr int kMaxHist = MF_MAX_HISTORY; // W + K - 1 poses per frame
constexpr int kTileW = 128;              // map-kernel tile width (32 lanes x 4 px)
constexpr int kMapThreads = 256;         // 8 warps per CTA of the tiled map kernel
constexpr int kStages = 4;               // depth ring rows per map warp at 16 B per lane (power of 2)
constexpr int kBandMax = 256;            // largest rows per map unit
constexpr int kGroupStrips = 8;          // strips (one per warp) per map unit
constexpr int kUnitThreads = 32 * kGroupStrips;  // threads per CTA of the unit map kernels

// Thresholds of the motion-point validity test (Section 2.3, Eq. 6 readings).
constexpr double kRigidTol = 1e-6;
constexpr double kStaticRel = 1e-12;
constexpr double kValidRelNorm = 1e-9;
constexpr double kValidRelZ = 1e-3;

// One emitted frame's motion points and per-frame results.  Written by the
// window-points kernel, read by the map and finalize kernels.  The first
// block holds the map kernel's operands for the valid points, compacted in
// slot order: u = ux_hi + ux_lo and v = vy_hi + vy_lo split so that the
// integer pixel coordinate minus the high part is exact in FP32, and the
// Gaussian's log2(e) / (2 sigma^2) as a float pair c_hi + c_lo (the map
// kernels take exp(-d^2 / (2 sigma^2)) as 2^-(d^2 c)).
struct alignas(16) FrameRec {
  float ux_hi[kMaxPts], ux_lo[kMaxPts];
  float vy_hi[kMaxPts], vy_lo[kMaxPts];
  float c_hi[kMaxPts], c_lo[kMaxPts];
  int32_t n_valid;
  float inv_n;                 // 1 / Z of Eq. 7
  uint32_t valid_mask;
  int32_t status;
  int64_t frame_index;
  unsigned long long argmax_key;  // (bits of M << 32) | ~(y*W+x), max-reduced
  double focus_u, focus_v;
  int32_t focus_valid, focus_px_x, focus_px_y;
  float d0;                    // reference depth of G, in this frame's depth scale
  float depth_scale;           // the batch's depth alignment scale (reported)
  // slot-ordered FP64 records (slot s <-> frame n - W + 1 + s)
  double u[kMaxPts], v[kMaxPts], sigma[kMaxPts], s[kMaxPts];
  int32_t valid[kMaxPts];
};

struct IngestParams {
  const double* in;        // n x 12 pushed poses (device)
  int n;                   // frames in the push
  int first;               // first emitted push frame (= overlap or 0)
  int anchor;              // 1: gravity-locked anchoring against the history
  double* ring;            // world-pose history, ring_mask+1 slots x 12
  int32_t* ring_bad;
  int64_t ring_mask;
  int64_t e0;              // global index of the first emitted frame
  // Depth alignment: the push's batch scale (device; NULL = 1), applied to
  // every translation of the push before anchoring.
  const double* scale;
};

struct PointsParams {
  const double* ring;
  const int32_t* ring_bad;
  int64_t ring_mask;
  FrameRec* recs;
  int64_t rec_mask;
  int64_t e0;              // global index of the first frame to process
  int n_frames;
  int window, smooth_len;
  int width, height, calib_width, calib_height;
  double K[4];             // fx, fy, cx, cy at the calibration resolution
  double sigma_rel, s_lo, s_hi;
  double w[kMaxHist];      // least-squares weights, w[k] multiplies q_{i-k}
  double d0;               // reference depth of the motion-guided depth (m)
  const double* scale;     // the push's batch depth scale (device; NULL = 1)
};

struct MapParams {
  const FrameRec* recs;
  int64_t rec_mask;
  int64_t f0;              // global index of the first frame of the launch
  int n_frames;
  int width, height;
  int tiles_x, tiles_y, tile_h;
  const void* depth;       // plane of frame f0, frames contiguous; may be NULL
  void* M;                 // plane of frame f0 (may be NULL)
  void* G;                 // (may be NULL)
  int path;                // kMapAuto, kMapCudaCores or kMapTensorCores
  // Work counter of the persistent map kernels' dynamic unit schedule: 0 at
  // launch and left at 0; no two launches in flight may share it.
  unsigned int* sched;
  // Set to 1 by a kernel whose bounded device wait ran out (device-visible;
  // may be NULL).  The frames concerned are also marked MF_FRAME_TIMEOUT.
  unsigned int* fault;
};

// MF_NORM_MAX applies to frames whose count-normalised map maximum is at
// least this (smaller maxima: every point lies far outside the image).
constexpr float kNormFloor = 0x1p-20f;

// Map kernel selection (MapParams::path).
constexpr int kMapAuto = 0;
constexpr int kMapCudaCores = 1;
constexpr int kMapTensorCores = 2;

struct FinalizeParams {
  const FrameRec* recs;
  int64_t rec_mask;
  int64_t f0;
  int n_frames;
  int width, window;
  int normalize;           // mf_norm: report the map maximum after scaling
  mf_frame_info* info;     // may be NULL
  mf_motion_point* points; // may be NULL
};

// In-place MF_NORM_MAX scaling of M and G by 1 / (the frame's map maximum).
struct NormalizeParams {
  const FrameRec* recs;
  int64_t rec_mask;
  int64_t f0;
  int n_frames;
  int64_t plane;           // pixels per frame
  void* M;                 // plane of frame f0 (may be NULL)
  void* G;                 // (may be NULL)
};

// Launchers (return the CUDA launch status).  `launches` is incremented by
// the number of kernels launched.
cudaError_t launch_ingest(const IngestParams& p, cudaStream_t st, int64_t* launches);
cudaError_t launch_points(const PointsParams& p, cudaStream_t st, int64_t* launches);
// Whether launch_map runs the tensor-core kernel for a launch path.
bool map_uses_tensor_cores(int path);
// Tensor-core map kernel (mf_map_tc.cu); any width, any plane alignment.
cudaError_t launch_map_tc(const MapParams& p, int window, int depth_dtype, int map_dtype,
                          cudaStream_t st, int64_t* launches);
// launch_map renders the maps of p's frames with Z of Eq. 7 as `normalize`
// (mf_norm) selects.
cudaError_t launch_map(const MapParams& p, int window, int in_dtype, int out_dtype, int normalize,
                       cudaStream_t st, int64_t* launches);
cudaError_t launch_finalize(const FinalizeParams& p, cudaStream_t st, int64_t* launches);

// Depth alignment of one batch against the previous one (Section 2.2,
// Fig. 3; mf_align.cu): *scale *= the lower median of the single-precision
// ratios prev / cur over the `count` pixels where both depths are finite and
// > 0 (unchanged when none qualifies).  Radix selection over the ratios'
// bit patterns in three histogram passes; `work` holds kAlignWorkWords
// words, and the launches leave nothing in it that the next call needs.
constexpr int kAlignBins = 2048;
constexpr int kAlignWorkWords = 3 * kAlignBins + 8;
struct AlignParams {
  const void* prev;        // previous batch's last overlap planes
  const void* cur;         // this batch's first overlap planes
  int64_t count;           // pixels compared (overlap frames x plane)
  unsigned int* work;      // kAlignWorkWords words (zeroed by the launcher)
  double* scale;           // batch scale, updated in place
};
cudaError_t launch_depth_align(const AlignParams& p, int depth_dtype, cudaStream_t st, int64_t* launches);
cudaError_t launch_normalize(const NormalizeParams& p, int map_dtype, cudaStream_t st,
                             int64_t* launches);
cudaError_t launch_ring_copy(const double* src, const int32_t* src_bad, int64_t src_mask,
                             double* dst, int32_t* dst_bad, int64_t dst_mask, int64_t first,
                             int count, cudaStream_t st, int64_t* launches);

// Map-kernel tile height used by the plain path.
int map_tile_h(int width, int height, int window);

// Checked build (compiled with -DMF_CHECKED, libmf_checked.so): the map
// kernels test every global access against its plane before making it.  An
// access outside sets the launch's fault word to kFaultOutOfRange and is
// skipped, so an index error is reported instead of faulting the GPU (a
// stand-in for a memory checker where none can run).  Release builds test
// nothing.
constexpr unsigned int kFaultWaitExpired = 1u;
constexpr unsigned int kFaultOutOfRange = 2u;
#ifdef MF_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// An NVTX range over one host call (push, get, tick, render): the timeline
// of a profiler shows the path's calls around their kernels.  Costs a
// function-pointer test when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Host helpers defined in mf_stream.cpp.
bool host_ls_weights(int K, int mode, double* w);
int host_validate_desc(const mf_stream_desc* d);
int host_map_path(uint32_t flags);
int host_fail(int status, const char* what, cudaError_t e);
void host_count_launches(int64_t n);
// Where a caller's pointer lives, for work launched on device `dev`
// (kPtrHost, kPtrDevice or kPtrOtherDevice of mf_ptr_kind.h).
int host_pointer_kind(const void* p, int dev);
// Launch facts of a kernel on the current device: its SM count and the CTAs
// of `threads` threads with `smem_launch` bytes of dynamic shared memory that
// fit on one SM.  On first use per (kernel, limit, launch size, device) --
// with that device current -- the kernel's dynamic shared memory limit is
// raised to `smem_limit` (and its carveout set when carveout >= 0) on that
// device; the result is cached under a lock.
struct KernelFit {
  int sms = 1;
  int per_sm = 1;
};
KernelFit host_kernel_fit(const void* kernel, int threads, size_t smem_limit, size_t smem_launch,
                          int carveout = -1);

// Host-side fault injection (mf_fault.cpp; MF_FAULT or mf_set_fault).
// fault_fires(kind) counts one occurrence of the guarded event and returns
// true when the installed rule makes this occurrence fail.
constexpr int kFaultAllocFail = 0;     // a library device allocation returns NULL
constexpr int kFaultBadPose = 1;       // a host pose is made non-rigid before upload
constexpr int kFaultDropPush = 2;      // a serving push is accepted, then dropped
constexpr int kFaultAdmissionFull = 3; // an engine admission is refused
constexpr int kFaultWaitTimeout = 4;   // a stream wait reports a device wait that ran out
constexpr int kFaultKinds = 5;
bool fault_fires(int kind);

}  // namespace mf
