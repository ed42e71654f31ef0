// Per-pixel kernels of the motion-focus path (templates; instantiated by
// mf_map_n8.cu, mf_map_n16.cu and mf_map_n32.cu, one window bucket each, so
// that the build compiles them in parallel): the motion-focus map of Eq. 7
// and the motion-guided depth (Fig. 1(iii), Fig. 5), fused, with the
// per-frame argmax of the map.
//
// The map is a sum of N isotropic Gaussians, so each term factors into a
// column factor and a row factor:
//     exp(-((x-u)^2 + (y-v)^2) c) = exp(-(x-u)^2 c) * exp(-(y-v)^2 c),
// c = 1 / (2 sigma_i^2).  A CTA owns a 128-column x tile_h-row tile of one
// frame: it evaluates the N x 128 column factors and tile_h x N row factors
// (with 1/Z folded into the row factors) in shared memory, then every pixel
// costs N FP32 FMAs, issued two pixels at a time with fma.rn.f32x2, summed in
// fixed point order so results do not depend on the tiling.  Depth is read
// and both maps are written with 128-bit (FP32) or 64-bit (16-bit storage)
// streaming accesses, 4 pixels per thread per row; each warp covers 128
// contiguous pixels of a row (512 B of FP32), so every access is coalesced.
//
// Accuracy: the exponent is formed from an exact FP32 coordinate difference
// (u is split into a hi part on a 2^-8 grid plus a lo part) and a float pair
// for c, so its relative error stays near one FP32 rounding; expf (full
// precision) then costs at most 2 ulp per factor.
#pragma once

#include <algorithm>
#include <type_traits>

#include "mf_map_unit.cuh"
#include "mf_pose_device.cuh"

namespace mf {


namespace {

// Storage types: 4 consecutive pixels per access.
template <typename T>
struct Px;

template <>
struct Px<float> {
  static __device__ __forceinline__ float4 load4(const void* b, size_t i) {
    return __ldcs(reinterpret_cast<const float4*>(static_cast<const float*>(b) + i));
  }
  static __device__ __forceinline__ float load1(const void* b, size_t i) {
    return __ldcs(static_cast<const float*>(b) + i);
  }
  static __device__ __forceinline__ void store4(void* b, size_t i, float4 v) {
    __stcs(reinterpret_cast<float4*>(static_cast<float*>(b) + i), v);
  }
  static __device__ __forceinline__ void store1(void* b, size_t i, float v) {
    __stcs(static_cast<float*>(b) + i, v);
  }
};

template <>
struct Px<__nv_bfloat16> {
  static __device__ __forceinline__ float4 load4(const void* b, size_t i) {
    uint2 r = __ldcs(reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(b) + i));
    const float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&r.x));
    const float2 c = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&r.y));
    return make_float4(a.x, a.y, c.x, c.y);
  }
  static __device__ __forceinline__ float load1(const void* b, size_t i) {
    return __bfloat162float(static_cast<const __nv_bfloat16*>(b)[i]);
  }
  static __device__ __forceinline__ void store4(void* b, size_t i, float4 v) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
    __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
    uint2 r;
    r.x = *reinterpret_cast<unsigned*>(&lo);
    r.y = *reinterpret_cast<unsigned*>(&hi);
    __stcs(reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(b) + i), r);
  }
  static __device__ __forceinline__ void store1(void* b, size_t i, float v) {
    static_cast<__nv_bfloat16*>(b)[i] = __float2bfloat16_rn(v);
  }
};

template <>
struct Px<__half> {
  static __device__ __forceinline__ float4 load4(const void* b, size_t i) {
    uint2 r = __ldcs(reinterpret_cast<const uint2*>(static_cast<const __half*>(b) + i));
    const float2 a = __half22float2(*reinterpret_cast<__half2*>(&r.x));
    const float2 c = __half22float2(*reinterpret_cast<__half2*>(&r.y));
    return make_float4(a.x, a.y, c.x, c.y);
  }
  static __device__ __forceinline__ float load1(const void* b, size_t i) {
    return __half2float(static_cast<const __half*>(b)[i]);
  }
  static __device__ __forceinline__ void store4(void* b, size_t i, float4 v) {
    __half2 lo = __floats2half2_rn(v.x, v.y);
    __half2 hi = __floats2half2_rn(v.z, v.w);
    uint2 r;
    r.x = *reinterpret_cast<unsigned*>(&lo);
    r.y = *reinterpret_cast<unsigned*>(&hi);
    __stcs(reinterpret_cast<uint2*>(static_cast<__half*>(b) + i), r);
  }
  static __device__ __forceinline__ void store1(void* b, size_t i, float v) {
    static_cast<__half*>(b)[i] = __float2half_rn(v);
  }
};

template <typename TIn, bool VEC>
__device__ __forceinline__ float4 load_depth(const void* base, size_t idx, int xc, int width) {
  if (VEC) return Px<TIn>::load4(base, idx);
  float4 d;
  d.x = (xc + 0 < width) ? Px<TIn>::load1(base, idx + 0) : 0.0f;
  d.y = (xc + 1 < width) ? Px<TIn>::load1(base, idx + 1) : 0.0f;
  d.z = (xc + 2 < width) ? Px<TIn>::load1(base, idx + 2) : 0.0f;
  d.w = (xc + 3 < width) ? Px<TIn>::load1(base, idx + 3) : 0.0f;
  return d;
}

template <typename TOut, bool VEC>
__device__ __forceinline__ void store_px(void* base, size_t idx, float4 v, int xc, int width) {
  if (VEC) {
    Px<TOut>::store4(base, idx, v);
    return;
  }
  if (xc + 0 < width) Px<TOut>::store1(base, idx + 0, v.x);
  if (xc + 1 < width) Px<TOut>::store1(base, idx + 1, v.y);
  if (xc + 2 < width) Px<TOut>::store1(base, idx + 2, v.z);
  if (xc + 3 < width) Px<TOut>::store1(base, idx + 3, v.w);
}

}  // namespace

template <int NMAX, typename TIn, typename TOut, bool VEC>
__global__ void __launch_bounds__(kMapThreads) map_kernel(MapParams p) {
  extern __shared__ float4 smem4[];
  float* Ex = reinterpret_cast<float*>(smem4);   // [NMAX][kTileW]
  float* Ey = Ex + NMAX * kTileW;                // [tile_h][NMAX]
  __shared__ PointsSmem<NMAX> P;
  __shared__ unsigned long long s_key[kMapThreads / 32];

  const int tpf = p.tiles_x * p.tiles_y;
  const int f = blockIdx.x / tpf;
  const int rem = blockIdx.x - f * tpf;
  const int ty = rem / p.tiles_x;
  const int tx = rem - ty * p.tiles_x;
  FrameRec* rec = const_cast<FrameRec*>(p.recs) + ((p.f0 + f) & p.rec_mask);
  const int n = rec->n_valid;                       // block-uniform
  const int nc = min(NMAX, (n + 3) & ~3);           // padded to a multiple of 4
  const float inv_n = rec->inv_n;
  const int x0 = tx * kTileW, y0 = ty * p.tile_h;
  const int rows = min(p.tile_h, p.height - y0);
  const int tid = threadIdx.x;

  if (tid < n) {
    P.uhi[tid] = rec->ux_hi[tid];
    P.ulo[tid] = rec->ux_lo[tid];
    P.vhi[tid] = rec->vy_hi[tid];
    P.vlo[tid] = rec->vy_lo[tid];
    P.chi[tid] = rec->c_hi[tid];
    P.clo[tid] = rec->c_lo[tid];
  }
  __syncthreads();
  // Column factors Ex[i][c] and row factors Ey[r][i] (1/Z folded in); zero
  // for the padding points n <= i < nc.
  for (int e = tid; e < nc * kTileW; e += kMapThreads) {
    const int i = e >> 7, c = e & (kTileW - 1);
    Ex[e] = i < n ? gauss_factor((float)(x0 + c), P.uhi[i], P.ulo[i], P.chi[i], P.clo[i]) : 0.0f;
  }
  for (int r = tid >> 5; r < rows; r += kMapThreads / 32) {
    for (int i = tid & 31; i < nc; i += 32) {
      Ey[r * NMAX + i] =
          i < n ? gauss_factor((float)(y0 + r), P.vhi[i], P.vlo[i], P.chi[i], P.clo[i]) * inv_n
                : 0.0f;
    }
  }
  __syncthreads();

  const int lane = tid & 31, warp = tid >> 5;
  const int xc = x0 + lane * 4;
  const bool col_ok = xc < p.width;
  float2 ex01[NMAX], ex23[NMAX];
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
    if (i < nc) {
      const float4 e = *reinterpret_cast<const float4*>(Ex + i * kTileW + lane * 4);
      ex01[i] = make_float2(e.x, e.y);
      ex23[i] = make_float2(e.z, e.w);
    }
  }

  const size_t plane = (size_t)p.width * (size_t)p.height;
  const size_t fbase = (size_t)f * plane;
  const void* dep = p.depth;
  float best = -1.0f;
  unsigned bidx = 0;
  const bool has_depth = dep != nullptr;
  float4 dnext = make_float4(0.f, 0.f, 0.f, 0.f);
  int r = warp;
  if (has_depth && col_ok && r < rows)
    dnext = load_depth<TIn, VEC>(dep, fbase + (size_t)(y0 + r) * p.width + xc, xc, p.width);
  for (; r < rows; r += kMapThreads / 32) {
    const float4 dv = dnext;
    const int rn = r + kMapThreads / 32;
    const size_t idx = fbase + (size_t)(y0 + r) * p.width + xc;
    if (has_depth && col_ok && rn < rows)
      dnext = load_depth<TIn, VEC>(dep, idx + (size_t)(kMapThreads / 32) * p.width, xc, p.width);
    float2 a01 = make_float2(0.f, 0.f), a23 = make_float2(0.f, 0.f);
    const float4* ey4 = reinterpret_cast<const float4*>(Ey + r * NMAX);
#pragma unroll
    for (int i = 0; i < NMAX; i += 4) {
      if (i >= nc) break;
      const float4 e = ey4[i >> 2];
      a01 = ffma2(ex01[i + 0], e.x, a01);
      a23 = ffma2(ex23[i + 0], e.x, a23);
      a01 = ffma2(ex01[i + 1], e.y, a01);
      a23 = ffma2(ex23[i + 1], e.y, a23);
      a01 = ffma2(ex01[i + 2], e.z, a01);
      a23 = ffma2(ex23[i + 2], e.z, a23);
      a01 = ffma2(ex01[i + 3], e.w, a01);
      a23 = ffma2(ex23[i + 3], e.w, a23);
    }
    if (!col_ok) continue;
    const float4 m = make_float4(a01.x, a01.y, a23.x, a23.y);
    if (p.M) store_px<TOut, VEC>(p.M, idx, m, xc, p.width);
    if (p.G) {
      float4 g;
      if (has_depth) {
        g.x = m.x * depth_weight(dv.x, rec->d0);
        g.y = m.y * depth_weight(dv.y, rec->d0);
        g.z = m.z * depth_weight(dv.z, rec->d0);
        g.w = m.w * depth_weight(dv.w, rec->d0);
      } else {
        g = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      store_px<TOut, VEC>(p.G, idx, g, xc, p.width);
    }
    const unsigned pix = (unsigned)((y0 + r) * p.width + xc);
    if (m.x > best) { best = m.x; bidx = pix; }
    if (m.y > best && (VEC || xc + 1 < p.width)) { best = m.y; bidx = pix + 1; }
    if (m.z > best && (VEC || xc + 2 < p.width)) { best = m.z; bidx = pix + 2; }
    if (m.w > best && (VEC || xc + 3 < p.width)) { best = m.w; bidx = pix + 3; }
  }

  // Per-frame argmax: largest M, ties to the lowest linear index.
  unsigned long long key =
      best >= 0.0f ? ((unsigned long long)__float_as_uint(best) << 32) | (0xffffffffu - bidx) : 0ull;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
    key = k2 > key ? k2 : key;
  }
  if (lane == 0) s_key[warp] = key;
  __syncthreads();
  if (tid == 0 && n > 0) {
    unsigned long long k = s_key[0];
    for (int w = 1; w < kMapThreads / 32; ++w) k = s_key[w] > k ? s_key[w] : k;
    if (k) atomicMax(&rec->argmax_key, k);
  }
}

// ---------------------------------------------------------------------------
// Streaming kernel for frames whose rows allow CPT-pixel vector access (the
// common case): persistent CTAs of 8 warps take the frames' units (band of
// up to 256 rows x group of 8 strips) in frame order from the dynamic
// schedule; map_unit does the work.
template <int NMAX, int CPT, typename TIn, typename TOut, int MODE>
__global__ void __launch_bounds__(kUnitThreads, unit_ctas_per_sm(NMAX, CPT))
    map_stream_kernel(MapParams p, int band_h) {
  extern __shared__ float4 smem4[];
  float* Ey = reinterpret_cast<float*>(smem4);                          // [band_h][NMAX]
  uint4* ring = reinterpret_cast<uint4*>(Ey + (size_t)band_h * NMAX);   // [8][stages][32]
  __shared__ PointsSmem<kMaxPts> P[kGroupStrips];
  __shared__ uint4 zeros[kZeroBytes / 16];
  init_zero_source(zeros);
  constexpr int kGroupW = kGroupStrips * 32 * CPT;
  const int groups_x = (p.width + kGroupW - 1) / kGroupW;
  const int bands = (p.height + band_h - 1) / band_h;
  const long long units = (long long)p.n_frames * bands * groups_x;
  const size_t plane = (size_t)p.width * (size_t)p.height;
  // this warp's ring: S rows of 32 lanes x CPT depth elements (uint4 units)
  uint4* my_ring = ring + (size_t)(threadIdx.x >> 5) * ring_stages(CPT, (int)sizeof(TIn), NMAX) * 2 * CPT *
                             (int)sizeof(TIn);
  __shared__ long long s_next[2];
  long long u = blockIdx.x;
  for (int k = 0; u < units; ++k) {
    const unsigned claim = claim_unit(p.sched);
    const int f = (int)(u / ((long long)bands * groups_x));
    const int rem = (int)(u - (long long)f * bands * groups_x);
    const int b = rem / groups_x, g = rem - b * groups_x;
    UnitGeom ug;
    ug.rec = const_cast<FrameRec*>(p.recs) + ((p.f0 + f) & p.rec_mask);
    ug.depth = p.depth ? static_cast<const char*>(p.depth) + (size_t)f * plane * sizeof(TIn) : nullptr;
    ug.M = p.M ? static_cast<char*>(p.M) + (size_t)f * plane * sizeof(TOut) : nullptr;
    ug.G = p.G ? static_cast<char*>(p.G) + (size_t)f * plane * sizeof(TOut) : nullptr;
    ug.width = p.width;
    ug.fault = p.fault;
    ug.height = p.height;
    ug.y0 = b * band_h;
    ug.rows = min(band_h, p.height - ug.y0);
    ug.gx0 = g * kGroupW;
    ug.d0 = ug.rec->d0;
    map_unit<NMAX, CPT, TIn, TOut, MODE>(ug, Ey, my_ring, P, zeros);
    u = next_unit(p.sched, claim, units, s_next, k);
  }
  bulk_wait_all();
}

// ---------------------------------------------------------------------------
// MF_NORM_MAX (Eq. 7 with Z = the frame's largest point sum): divides a
// frame's M and G in place by its map maximum (from the fused argmax).
// blockIdx.y is the frame; the CTAs of a frame stride over its pixels, four
// at a time when the planes allow vector access.
namespace mapk {

template <typename T>
constexpr int out_dtype_of() {
  return std::is_same<T, float>::value ? MF_F32 : std::is_same<T, __half>::value ? MF_F16 : MF_BF16;
}

// Parameters of the in-place MF_NORM_MAX pass over p's planes (mf_map_kernel.cu).
NormalizeParams normalize_params(const MapParams& p);

// Launches the persistent kernel k over `units` units: one CTA per unit up
// to the CTAs the device holds at the band's largest shared memory.
template <typename K>
void launch_persistent(K k, size_t smem_max, long long units, size_t smem, const MapParams& p,
                       int band_h, cudaStream_t st) {
  const KernelFit f = host_kernel_fit(reinterpret_cast<const void*>(k), kUnitThreads, smem_max, smem_max);
  const long long grid = std::min<long long>(units, (long long)f.sms * f.per_sm);
  k<<<(unsigned)grid, kUnitThreads, smem, st>>>(p, band_h);
}

// One launch (or, for MF_NORM_MAX, a max-only pass then a scaled pass) of
// the map kernel for NMAX-point windows; *nl receives the launch count.
// The persistent unit kernel with CPT columns per lane over p's frames (one
// launch, or for MF_NORM_MAX a max-only pass then a scaled pass).
template <int NMAX, int CPT, typename TIn, typename TOut>
void launch_units(const MapParams& p, bool norm_max, cudaStream_t st, int64_t* nl) {
  // Rows per unit: bands of at most 128 rows at up to 16 points skip depth
  // and factors at a finer grain (1080p x 304 frames, window 16, against 256
  // rows: ACCEL FP32 1.20 -> 1.24 of measured HBM, HEADING unchanged; 64 rows
  // reach 1.27 but lose 4 % on HEADING).  At 32 points the Ey table per row
  // is twice as costly and 256 rows stay faster.
  constexpr int kBand = NMAX <= 16 ? 128 : kBandMax;
  const int bands = (p.height + kBand - 1) / kBand;
  const int band_h = (p.height + bands - 1) / bands;
  constexpr int kGroupW = kGroupStrips * 32 * CPT;
  const long long units = (long long)p.n_frames * bands * ((p.width + kGroupW - 1) / kGroupW);
  const size_t smem_max = unit_smem_bytes(NMAX, kBand, CPT, (int)sizeof(TIn)),
               smem = unit_smem_bytes(NMAX, band_h, CPT, (int)sizeof(TIn));
  if (!norm_max) {
    launch_persistent(map_stream_kernel<NMAX, CPT, TIn, TOut, kUnitFull>, smem_max, units, smem, p, band_h,
                      st);
    *nl += 1;
  } else {
    // same units, same sums: the first pass only finds each frame's maximum
    launch_persistent(map_stream_kernel<NMAX, CPT, float, float, kUnitMaxOnly>, smem_max, units, smem, p,
                      band_h, st);
    launch_persistent(map_stream_kernel<NMAX, CPT, TIn, TOut, kUnitScaled>, smem_max, units, smem, p,
                      band_h, st);
    *nl += 2;
  }
}

template <int NMAX, typename TIn, typename TOut>
cudaError_t launch_typed(const MapParams& p, bool norm_max, cudaStream_t st, int64_t* nl) {
  const long long tiles = (long long)p.n_frames * p.tiles_x * p.tiles_y;
  if (tiles <= 0) return cudaSuccess;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  // Pixels per lane.  FP32 maps: 2, so that windows of up to 16 points fit
  // three CTAs (24 warps) per SM, whose extra loads in flight beat the wider
  // rows (1080p ACCEL, window 16: 1.20 vs 1.16 of measured HBM).  16-bit maps:
  // 4 (8-byte stores; 2 pixels lose 20 % at up to 16 points), also above 16
  // points, where the column factors alone take 128 registers and one CTA
  // fits per SM (HEADING BF16 window 32: 0.49 -> 0.52 against 2 pixels per
  // lane); widths or planes that do not allow 4 take 2, then the tiled
  // kernel.
  auto aligned = [](const void* q, size_t a) { return q == nullptr || ((uintptr_t)q % a) == 0; };
  auto fits = [&](int cpt) {
    return (p.width % cpt) == 0 && aligned(p.depth, cpt * sizeof(TIn)) && aligned(p.M, cpt * sizeof(TOut)) &&
           aligned(p.G, cpt * sizeof(TOut));
  };
  bool done = false;
  if constexpr (sizeof(TOut) == 2) {
    if (fits(4)) {
      launch_units<NMAX, 4, TIn, TOut>(p, norm_max, st, nl);
      done = true;
    }
  }
  if (done) {
  } else if (fits(2)) {
    launch_units<NMAX, 2, TIn, TOut>(p, norm_max, st, nl);
  } else {
    const size_t smem = (size_t)NMAX * kTileW * 4 + (size_t)p.tile_h * NMAX * 4;
    auto k = map_kernel<NMAX, TIn, TOut, false>;
    if (smem > 48 * 1024) host_kernel_fit(reinterpret_cast<const void*>(k), kMapThreads, smem, smem);
    k<<<(unsigned)tiles, kMapThreads, smem, st>>>(p);
    *nl += 1;
    if (norm_max) {
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      return launch_normalize(normalize_params(p), out_dtype_of<TOut>(), st, nl);
    }
  }
  return cudaGetLastError();
}

template <int NMAX>
cudaError_t launch_n(const MapParams& p, int in_dtype, int out_dtype, bool mx, cudaStream_t st,
                     int64_t* nl) {
  switch (in_dtype * 3 + out_dtype) {
    case MF_F32 * 3 + MF_F32: return launch_typed<NMAX, float, float>(p, mx, st, nl);
    case MF_F32 * 3 + MF_BF16: return launch_typed<NMAX, float, __nv_bfloat16>(p, mx, st, nl);
    case MF_F32 * 3 + MF_F16: return launch_typed<NMAX, float, __half>(p, mx, st, nl);
    case MF_BF16 * 3 + MF_F32: return launch_typed<NMAX, __nv_bfloat16, float>(p, mx, st, nl);
    case MF_BF16 * 3 + MF_BF16: return launch_typed<NMAX, __nv_bfloat16, __nv_bfloat16>(p, mx, st, nl);
    case MF_BF16 * 3 + MF_F16: return launch_typed<NMAX, __nv_bfloat16, __half>(p, mx, st, nl);
    case MF_F16 * 3 + MF_F32: return launch_typed<NMAX, __half, float>(p, mx, st, nl);
    case MF_F16 * 3 + MF_BF16: return launch_typed<NMAX, __half, __nv_bfloat16>(p, mx, st, nl);
    case MF_F16 * 3 + MF_F16: return launch_typed<NMAX, __half, __half>(p, mx, st, nl);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mapk
}  // namespace mf
