// Batched kernels of the engine: one tick processes the pushes of many
// streams (any resolution, any window) with four launches.  The per-frame
// and per-unit bodies are the same device functions the single-stream
// kernels run (mf_pose_device.cuh, mf_map_unit.cuh), so results do not
// depend on what else is in the batch.
#include <algorithm>

#include "mf_engine_internal.h"
#include "mf_map_unit.cuh"

namespace mf {

namespace {

__device__ __forceinline__ const TickFrame* tick_frames(const TickHeader* t) {
  return reinterpret_cast<const TickFrame*>(reinterpret_cast<const char*>(t) + t->frames_off);
}
__device__ __forceinline__ const TickPush* tick_pushes(const TickHeader* t) {
  return reinterpret_cast<const TickPush*>(reinterpret_cast<const char*>(t) + t->pushes_off);
}
__device__ __forceinline__ const double* tick_poses(const TickHeader* t) {
  return reinterpret_cast<const double*>(reinterpret_cast<const char*>(t) + t->poses_off);
}

}  // namespace

// Section 2.2: one thread per emitted frame of the tick.
__global__ void __launch_bounds__(128) engine_ingest_kernel(EngineKernelArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.table->n_frames) return;
  const TickFrame& fr = tick_frames(a.table)[t];
  const TickPush& ps = tick_pushes(a.table)[fr.push];
  const SlotParams& sp = a.slots[ps.slot];
  ingest_frame(tick_poses(a.table) + ps.pose_off * 12, ps.first, fr.k, ps.anchor, sp.ring,
               sp.ring_bad, sp.ring_mask, ps.e0);
}

// Eqs. 1-6: one warp per emitted frame of the tick.
constexpr int kEngPtsWarps = 4;
__global__ void __launch_bounds__(kEngPtsWarps * 32) engine_points_kernel(EngineKernelArgs a) {
  __shared__ PointsScratch S[kEngPtsWarps];
  const int wi = threadIdx.x >> 5;
  const int t = blockIdx.x * kEngPtsWarps + wi;
  if (t >= a.table->n_frames) return;  // warp-uniform
  const TickFrame& fr = tick_frames(a.table)[t];
  const TickPush& ps = tick_pushes(a.table)[fr.push];
  const SlotParams& sp = a.slots[ps.slot];
  frame_points(sp.ring, sp.ring_bad, sp.ring_mask, ps.e0 + fr.k, sp.fp, ps.K, sp.w, a.recs + t, S[wi]);
}

// Eq. 7 + guided depth: persistent CTAs over every frame's units.  One path
// serves every window (up to 32 points, 2 columns per lane): a kernel holding
// the 8/16-point paths as well would not fit the register budget.
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kMapThreads, 2) engine_map_kernel(EngineKernelArgs a) {
  extern __shared__ float4 smem4[];
  __shared__ PointsSmem<kMaxPts> P;
  __shared__ int s_kept;
  const TickHeader* tab = a.table;
  const int nf = tab->n_frames;
  const long long units = tab->n_units;
  const TickFrame* frames = tick_frames(tab);
  const TickPush* pushes = tick_pushes(tab);
  float* Ey = reinterpret_cast<float*>(smem4);
  uint4* ring = reinterpret_cast<uint4*>(Ey + (size_t)kBandMax * kMaxPts);
  uint4* my_ring = ring + (size_t)(threadIdx.x >> 5) * ring_stages(kEngineCPT) * 32;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    // frame owning unit u: the last frame whose unit_begin <= u
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (frames[mid].unit_begin <= u)
        lo = mid;
      else
        hi = mid - 1;
    }
    const TickFrame& fr = frames[lo];
    const SlotParams& sp = a.slots[pushes[fr.push].slot];
    const int local = (int)(u - fr.unit_begin);
    const int b = local / fr.groups_x, g = local - b * fr.groups_x;
    UnitGeom ug;
    ug.rec = a.recs + lo;
    ug.depth = fr.depth;
    ug.M = fr.M;
    ug.G = fr.G;
    ug.width = sp.fp.width;
    ug.height = sp.fp.height;
    ug.y0 = b * fr.band_h;
    ug.rows = min(fr.band_h, ug.height - ug.y0);
    ug.d0 = sp.d0;
    ug.gx0 = g * kEngineGroupW;
    map_unit<kMaxPts, kEngineCPT, TIn, TOut>(ug, Ey, my_ring, P, s_kept);
  }
}

__global__ void engine_finalize_kernel(EngineKernelArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.table->n_frames) return;
  const TickFrame& fr = tick_frames(a.table)[t];
  if (!fr.info) return;
  const SlotParams& sp = a.slots[tick_pushes(a.table)[fr.push].slot];
  finalize_frame(a.recs + t, sp.fp.width, fr.info);
}

size_t engine_map_smem() { return unit_smem_bytes(kMaxPts, kBandMax, kEngineCPT); }

namespace {

template <typename TIn, typename TOut>
struct MapKernel {
  static int grid() {
    static int g = 0;
    if (!g) {
      auto k = engine_map_kernel<TIn, TOut>;
      int dev = 0, sms = 0, per = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)engine_map_smem());
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kMapThreads, engine_map_smem());
      g = sms * std::max(per, 1);
    }
    return g;
  }
  static void launch(const EngineKernelArgs& a, int grid, cudaStream_t st) {
    engine_map_kernel<TIn, TOut><<<grid, kMapThreads, engine_map_smem(), st>>>(a);
  }
};

template <typename F>
bool with_types(int din, int dout, F&& f) {
  auto inner = [&](auto tin) {
    using TI = decltype(tin);
    switch (dout) {
      case MF_F32: f(TI{}, float{}); return true;
      case MF_BF16: f(TI{}, __nv_bfloat16{}); return true;
      case MF_F16: f(TI{}, __half{}); return true;
    }
    return false;
  };
  switch (din) {
    case MF_F32: return inner(float{});
    case MF_BF16: return inner(__nv_bfloat16{});
    case MF_F16: return inner(__half{});
  }
  return false;
}

}  // namespace

int engine_map_grid(int din, int dout) {
  int g = 0;
  with_types(din, dout, [&](auto ti, auto to) {
    g = MapKernel<decltype(ti), decltype(to)>::grid();
  });
  return g;
}

cudaError_t launch_engine_map_only(const EngineKernelArgs& a, int din, int dout, int map_grid,
                                   cudaStream_t st) {
  if (!with_types(din, dout, [&](auto ti, auto to) {
        MapKernel<decltype(ti), decltype(to)>::launch(a, map_grid, st);
      }))
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_engine_tick(const EngineKernelArgs& a, int din, int dout, int map_grid,
                               cudaStream_t st, int64_t* launches) {
  const int mf = a.max_frames;
  engine_ingest_kernel<<<(mf + 127) / 128, 128, 0, st>>>(a);
  engine_points_kernel<<<(mf + kEngPtsWarps - 1) / kEngPtsWarps, kEngPtsWarps * 32, 0, st>>>(a);
  cudaError_t e = launch_engine_map_only(a, din, dout, map_grid, st);
  if (e != cudaSuccess) return e;
  engine_finalize_kernel<<<(mf + 255) / 256, 256, 0, st>>>(a);
  *launches += 4;
  return cudaGetLastError();
}

}  // namespace mf
