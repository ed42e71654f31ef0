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
__device__ __forceinline__ const int32_t* tick_order(const TickHeader* t) {
  return reinterpret_cast<const int32_t*>(reinterpret_cast<const char*>(t) + t->order_off);
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

// Eq. 7 + guided depth: persistent CTAs over the units of one map path's
// frames.  Each path is its own kernel: one kernel holding both the 16- and
// the 32-point unit would not fit the register budget.
template <typename TIn, typename TOut, int NMAX, int CPT, int PATH>
__global__ void __launch_bounds__(kUnitThreads, unit_ctas_per_sm(NMAX, CPT)) engine_map_kernel(EngineKernelArgs a) {
  extern __shared__ float4 smem4[];
  __shared__ PointsSmem<kMaxPts> P[kGroupStrips];
  __shared__ uint4 zeros[kZeroBytes / 16];
  init_zero_source(zeros);
  constexpr int kGroupW = kGroupStrips * 32 * CPT;
  const TickHeader* tab = a.table;
  const int nf = tab->n_frames_path[PATH];
  const long long units = tab->n_units_path[PATH];
  const TickFrame* frames = tick_frames(tab);
  const int32_t* order = tick_order(tab) + (PATH ? tab->n_frames_path[0] : 0);
  const TickPush* pushes = tick_pushes(tab);
  float* Ey = reinterpret_cast<float*>(smem4);
  uint4* ring = reinterpret_cast<uint4*>(Ey + (size_t)kBandMax * NMAX);
  // this warp's ring: S rows of 32 lanes x CPT depth elements (uint4 units)
  uint4* my_ring = ring + (size_t)(threadIdx.x >> 5) * ring_stages(CPT, (int)sizeof(TIn), NMAX) * 2 * CPT *
                             (int)sizeof(TIn);
  __shared__ long long s_next[2];
  long long u = blockIdx.x;
  for (int k = 0; u < units; ++k) {
    const unsigned claim = claim_unit(a.sched + PATH);
    // frame owning unit u: the last of the path's frames whose unit_begin <= u
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (frames[order[mid]].unit_begin <= u)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int t = order[lo];
    const TickFrame& fr = frames[t];
    const SlotParams& sp = a.slots[pushes[fr.push].slot];
    const int local = (int)(u - fr.unit_begin);
    const int b = local / fr.groups_x, g = local - b * fr.groups_x;
    UnitGeom ug;
    ug.rec = a.recs + t;
    ug.depth = fr.depth;
    ug.M = fr.M;
    ug.G = fr.G;
    ug.width = sp.fp.width;
    ug.fault = a.fault;
    ug.height = sp.fp.height;
    ug.y0 = b * fr.band_h;
    ug.rows = min(fr.band_h, ug.height - ug.y0);
    ug.d0 = sp.d0;
    ug.gx0 = g * kGroupW;
    map_unit<NMAX, CPT, TIn, TOut>(ug, Ey, my_ring, P, zeros);
    u = next_unit(a.sched + PATH, claim, units, s_next, k);
  }
  bulk_wait_all();
}

__global__ void engine_finalize_kernel(EngineKernelArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.table->n_frames) return;
  const TickFrame& fr = tick_frames(a.table)[t];
  if (!fr.info) return;
  const SlotParams& sp = a.slots[tick_pushes(a.table)[fr.push].slot];
  finalize_frame(a.recs + t, sp.fp.width, fr.info);
}

namespace {

template <typename TIn, typename TOut, int PATH>
struct MapKernel {
  static constexpr int kN = PATH ? kEngineWideNMAX : kMaxPts;
  static constexpr int kC = PATH ? engine_wide_cpt((int)sizeof(TOut)) : kEngineCPT;
  static size_t smem() { return unit_smem_bytes(kN, kBandMax, kC, (int)sizeof(TIn)); }
  // resident CTAs on the current device (shared memory limit raised there)
  static int grid() {
    const KernelFit f = host_kernel_fit(
        reinterpret_cast<const void*>(engine_map_kernel<TIn, TOut, kN, kC, PATH>), kUnitThreads, smem(),
        smem());
    return f.sms * f.per_sm;
  }
  static void launch(const EngineKernelArgs& a, int grid, cudaStream_t st) {
    engine_map_kernel<TIn, TOut, kN, kC, PATH><<<grid, kUnitThreads, smem(), st>>>(a);
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

EngineGrids engine_map_grids(int din, int dout) {
  EngineGrids g{};
  with_types(din, dout, [&](auto ti, auto to) {
    g.g[0] = MapKernel<decltype(ti), decltype(to), 0>::grid();
    g.g[1] = MapKernel<decltype(ti), decltype(to), 1>::grid();
  });
  return g;
}

cudaError_t launch_engine_map_only(const EngineKernelArgs& a, int din, int dout,
                                   const EngineGrids& grids, cudaStream_t st) {
  if (!with_types(din, dout, [&](auto ti, auto to) {
        MapKernel<decltype(ti), decltype(to), 0>::launch(a, grids.g[0], st);
        MapKernel<decltype(ti), decltype(to), 1>::launch(a, grids.g[1], st);
      }))
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_engine_tick(const EngineKernelArgs& a, int din, int dout, const EngineGrids& grids,
                               cudaStream_t st, const EngineFork& fk, int64_t* launches) {
  const int mf = a.max_frames;
  engine_ingest_kernel<<<(mf + 127) / 128, 128, 0, st>>>(a);
  engine_points_kernel<<<(mf + kEngPtsWarps - 1) / kEngPtsWarps, kEngPtsWarps * 32, 0, st>>>(a);
  cudaError_t e = cudaEventRecord(fk.fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(fk.side, fk.fork, 0);
  if (e != cudaSuccess) return e;
  // the two persistent map kernels share the GPU: the tail of one overlaps
  // the other instead of following it
  if (!with_types(din, dout, [&](auto ti, auto to) {
        MapKernel<decltype(ti), decltype(to), 1>::launch(a, grids.g[1], fk.side);
        MapKernel<decltype(ti), decltype(to), 0>::launch(a, grids.g[0], st);
      }))
    return cudaErrorInvalidValue;
  e = cudaEventRecord(fk.join, fk.side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, fk.join, 0);
  if (e != cudaSuccess) return e;
  engine_finalize_kernel<<<(mf + 255) / 256, 256, 0, st>>>(a);
  *launches += kEngineTickLaunches;
  return cudaGetLastError();
}

}  // namespace mf
