// Per-pixel kernel of the motion-focus path: the motion-focus map of Eq. 7
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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>

#include "mf_internal.h"

namespace mf {

namespace {

template <int NMAX>
struct PointsSmem {
  float uhi[NMAX], ulo[NMAX], vhi[NMAX], vlo[NMAX], chi[NMAX], clo[NMAX];
};

// exp(-(q - hi - lo)^2 * (chi + clo)) for an integer-valued q.
__device__ __forceinline__ float gauss_factor(float q, float hi, float lo, float chi, float clo) {
  const float dh = q - hi;                 // exact (hi on a 2^-8 grid, |q|, |hi| < 2^15)
  const float p2 = dh * dh;
  const float e2 = fmaf(dh, dh, -p2);      // dh^2 = p2 + e2 exactly
  float qq = fmaf(-2.0f * dh, lo, e2);     // (dh - lo)^2 = p2 + qq
  qq = fmaf(lo, lo, qq);
  const float t1 = fmaf(clo, p2, chi * qq);
  const float a = fmaf(chi, p2, t1);
  return expf(-a);
}

__device__ __forceinline__ float2 ffma2(float2 a, float b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %4};\n\t"
      "mov.b64 rc, {%5, %6};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b), "f"(c.x), "f"(c.y));
  return d;
}

__device__ __forceinline__ float depth_weight(float D, float d0) {
  // min(1, d0 / D) for finite D > 0, else 0 (NaN fails both comparisons)
  return (D > 0.0f && D <= 3.402823466e38f) ? fminf(1.0f, __fdividef(d0, D)) : 0.0f;
}

// Storage types: 4 consecutive pixels per access.
template <typename T>
struct Px;

template <>
struct Px<float> {
  static constexpr int kAlign = 16;
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
  static constexpr int kAlign = 8;
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
  static constexpr int kAlign = 8;
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
        g.x = m.x * depth_weight(dv.x, p.d0);
        g.y = m.y * depth_weight(dv.y, p.d0);
        g.z = m.z * depth_weight(dv.z, p.d0);
        g.w = m.w * depth_weight(dv.w, p.d0);
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
// Streaming variant for frames whose rows allow 4-pixel vector access (the
// common case).  Persistent CTAs of 8 warps walk a list of units (frame, band
// of up to 256 rows, group of 8 adjacent 128-column strips).  Per unit:
//   * warp 0 keeps only the points whose Gaussian can reach the unit: a
//     point whose largest column factor over the unit times its largest row
//     factor (times 1/Z) is below 2^-40 contributes less than 2^-40 to every
//     pixel of it, far inside the 1e-10 absolute floor of the map tolerance;
//     the kept points stay in their original order;
//   * the CTA builds the band's row factors once in shared memory (one
//     barrier per unit, none per row);
//   * each warp owns one strip: it keeps its 4 columns' factors for the kept
//     points in registers and streams the band's rows two at a time (four
//     independent FMA chains), depth arriving through a per-warp ring of
//     kStages cp.async stages (no registers held by loads in flight), maps
//     leaving through 128-bit streaming stores.
// Per pixel and point the arithmetic is the same FMA chain, in the same point
// order, as the tiled kernel above.
namespace {

constexpr int kStages = 6;     // depth rows in flight per warp
constexpr int kBandMax = 256;  // rows per unit
constexpr float kCullBelow = 9.094947017729282e-13f;  // 2^-40

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  if (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <typename T>
__device__ __forceinline__ float4 unpack4(const uint4& raw);
template <>
__device__ __forceinline__ float4 unpack4<float>(const uint4& raw) {
  return make_float4(__uint_as_float(raw.x), __uint_as_float(raw.y), __uint_as_float(raw.z),
                     __uint_as_float(raw.w));
}
template <>
__device__ __forceinline__ float4 unpack4<__nv_bfloat16>(const uint4& raw) {
  uint2 r = make_uint2(raw.x, raw.y);
  const float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&r.x));
  const float2 c = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&r.y));
  return make_float4(a.x, a.y, c.x, c.y);
}
template <>
__device__ __forceinline__ float4 unpack4<__half>(const uint4& raw) {
  uint2 r = make_uint2(raw.x, raw.y);
  const float2 a = __half22float2(*reinterpret_cast<__half2*>(&r.x));
  const float2 c = __half22float2(*reinterpret_cast<__half2*>(&r.y));
  return make_float4(a.x, a.y, c.x, c.y);
}

// Two rows' N-term sums for one thread's 4 columns, points in order 0..nc-1.
// NC > 0 fixes the trip count at compile time (all NMAX points kept).
template <int NMAX, int NC>
__device__ __forceinline__ void accum_two_rows(const float2* ex01, const float2* ex23,
                                               const float* ey0, const float* ey1, int nc,
                                               float2& a01, float2& a23, float2& b01, float2& b23) {
  const float4* e0p = reinterpret_cast<const float4*>(ey0);
  const float4* e1p = reinterpret_cast<const float4*>(ey1);
#pragma unroll
  for (int i = 0; i < NMAX; i += 4) {
    if (NC == 0 && i >= nc) break;
    const float4 e = e0p[i >> 2];
    const float4 f = e1p[i >> 2];
    a01 = ffma2(ex01[i + 0], e.x, a01);
    a23 = ffma2(ex23[i + 0], e.x, a23);
    b01 = ffma2(ex01[i + 0], f.x, b01);
    b23 = ffma2(ex23[i + 0], f.x, b23);
    a01 = ffma2(ex01[i + 1], e.y, a01);
    a23 = ffma2(ex23[i + 1], e.y, a23);
    b01 = ffma2(ex01[i + 1], f.y, b01);
    b23 = ffma2(ex23[i + 1], f.y, b23);
    a01 = ffma2(ex01[i + 2], e.z, a01);
    a23 = ffma2(ex23[i + 2], e.z, a23);
    b01 = ffma2(ex01[i + 2], f.z, b01);
    b23 = ffma2(ex23[i + 2], f.z, b23);
    a01 = ffma2(ex01[i + 3], e.w, a01);
    a23 = ffma2(ex23[i + 3], e.w, a23);
    b01 = ffma2(ex01[i + 3], f.w, b01);
    b23 = ffma2(ex23[i + 3], f.w, b23);
  }
}

}  // namespace

template <int NMAX, typename TIn, typename TOut>
__global__ void __launch_bounds__(kMapThreads, NMAX <= 16 ? 2 : 1)
    map_stream_kernel(MapParams p, int band_h) {
  extern __shared__ float4 smem4[];
  float* Ey = reinterpret_cast<float*>(smem4);                            // [band_h][NMAX]
  uint4* ring = reinterpret_cast<uint4*>(Ey + (size_t)band_h * NMAX);     // [8][kStages][32]
  __shared__ PointsSmem<NMAX> P;
  __shared__ int s_kept;

  constexpr int kInBytes = 4 * (int)sizeof(TIn);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int groups_x = (p.tiles_x + 7) / 8;
  const int bands = (p.height + band_h - 1) / band_h;
  const long long units = (long long)p.n_frames * bands * groups_x;
  const size_t plane = (size_t)p.width * (size_t)p.height;
  const bool has_depth = p.depth != nullptr;
  uint4* my_ring = ring + (size_t)warp * kStages * 32;

  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const int f = (int)(u / ((long long)bands * groups_x));
    const int rem = (int)(u - (long long)f * bands * groups_x);
    const int b = rem / groups_x, g = rem - b * groups_x;
    FrameRec* rec = const_cast<FrameRec*>(p.recs) + ((p.f0 + f) & p.rec_mask);
    const int y0 = b * band_h;
    const int rows = min(band_h, p.height - y0);
    const int gx0 = g * 8 * kTileW;
    const int gx1 = min(p.width, gx0 + 8 * kTileW) - 1;
    const int x0 = gx0 + warp * kTileW;
    const int xc = x0 + lane * 4;
    const bool col_ok = xc < p.width;
    const size_t row0 = (size_t)f * plane + (size_t)y0 * p.width + xc;
    const char* dsrc = has_depth ? static_cast<const char*>(p.depth) + row0 * sizeof(TIn) : nullptr;
    const size_t dstride = (size_t)p.width * sizeof(TIn);
    auto issue = [&](int r) {
      if (r < rows && col_ok && has_depth)
        cp_async<kInBytes>(my_ring + (r % kStages) * 32 + lane, dsrc + (size_t)r * dstride);
      cp_async_commit();
    };
    // The first depth rows are requested before the unit's set-up, so the
    // copies are in flight while the factors are computed.  Each warp's ring
    // is its own; the previous unit drained it.
#pragma unroll
    for (int s = 0; s < kStages - 2; ++s) issue(s);
    __syncthreads();  // the previous unit is done with P and Ey
    const int n = rec->n_valid;
    const float inv_n = rec->inv_n;
    if (warp == 0) {
      bool keep = false;
      float uh = 0.f, ul = 0.f, vh = 0.f, vl = 0.f, ch = 0.f, cl = 0.f;
      if (lane < n) {
        uh = rec->ux_hi[lane];
        ul = rec->ux_lo[lane];
        vh = rec->vy_hi[lane];
        vl = rec->vy_lo[lane];
        ch = rec->c_hi[lane];
        cl = rec->c_lo[lane];
        // the factors peak at the unit's pixel nearest (u, v)
        const float xn = fminf(fmaxf(rintf(uh + ul), (float)gx0), (float)gx1);
        const float yn = fminf(fmaxf(rintf(vh + vl), (float)y0), (float)(y0 + rows - 1));
        const float peak = gauss_factor(xn, uh, ul, ch, cl) * gauss_factor(yn, vh, vl, ch, cl);
        keep = peak * inv_n >= kCullBelow;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int pos = __popc(mask & ((1u << lane) - 1u));
        P.uhi[pos] = uh;
        P.ulo[pos] = ul;
        P.vhi[pos] = vh;
        P.vlo[pos] = vl;
        P.chi[pos] = ch;
        P.clo[pos] = cl;
      }
      if (lane == 0) s_kept = __popc(mask);
    }
    __syncthreads();
    const int nk = s_kept;
    const int nc = min(NMAX, (nk + 3) & ~3);
    for (int r = warp; r < rows; r += kMapThreads / 32)
      for (int i = lane; i < nc; i += 32)
        Ey[r * NMAX + i] =
            i < nk ? gauss_factor((float)(y0 + r), P.vhi[i], P.vlo[i], P.chi[i], P.clo[i]) * inv_n
                   : 0.0f;
    float2 ex01[NMAX], ex23[NMAX];
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
      if (i < nc) {
        float e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f;
        if (i < nk && col_ok) {
          e0 = gauss_factor((float)(xc + 0), P.uhi[i], P.ulo[i], P.chi[i], P.clo[i]);
          e1 = gauss_factor((float)(xc + 1), P.uhi[i], P.ulo[i], P.chi[i], P.clo[i]);
          e2 = gauss_factor((float)(xc + 2), P.uhi[i], P.ulo[i], P.chi[i], P.clo[i]);
          e3 = gauss_factor((float)(xc + 3), P.uhi[i], P.ulo[i], P.chi[i], P.clo[i]);
        }
        ex01[i] = make_float2(e0, e1);
        ex23[i] = make_float2(e2, e3);
      }
    }
    __syncthreads();  // Ey complete
    if (x0 >= p.width) continue;  // warp-uniform: this strip lies past the frame
    float best = -1.0f;
    unsigned bidx = 0;
    auto emit = [&](const float2& a01, const float2& a23, const float4& dv, int r) {
      const float4 m = make_float4(a01.x, a01.y, a23.x, a23.y);
      const size_t idx = row0 + (size_t)r * p.width;
      if (p.M) Px<TOut>::store4(p.M, idx, m);
      if (p.G) {
        float4 gv;
        gv.x = m.x * depth_weight(dv.x, p.d0);
        gv.y = m.y * depth_weight(dv.y, p.d0);
        gv.z = m.z * depth_weight(dv.z, p.d0);
        gv.w = m.w * depth_weight(dv.w, p.d0);
        Px<TOut>::store4(p.G, idx, gv);
      }
      const float m4 = fmaxf(fmaxf(m.x, m.y), fmaxf(m.z, m.w));
      if (m4 > best) {
        best = m4;
        const unsigned pix = (unsigned)((y0 + r) * p.width + xc);
        bidx = m.x == m4 ? pix : (m.y == m4 ? pix + 1 : (m.z == m4 ? pix + 2 : pix + 3));
      }
    };
    // Rows r and r+1 per iteration: the ring slots of rows r-2 and r-1 were
    // consumed by the previous iteration, so rows r+kStages-2 and
    // r+kStages-1 can be requested before rows r, r+1 are read.
    for (int r = 0; r < rows; r += 2) {
      issue(r + kStages - 2);
      issue(r + kStages - 1);
      cp_async_wait<kStages - 2>();
      const bool two = r + 1 < rows;
      float4 d0v = make_float4(0.f, 0.f, 0.f, 0.f), d1v = d0v;
      if (has_depth) {
        d0v = unpack4<TIn>(my_ring[(r % kStages) * 32 + lane]);
        if (two) d1v = unpack4<TIn>(my_ring[((r + 1) % kStages) * 32 + lane]);
      }
      float2 a01 = make_float2(0.f, 0.f), a23 = a01, b01 = a01, b23 = a01;
      const float* ey0 = Ey + r * NMAX;
      const float* ey1 = Ey + (two ? r + 1 : r) * NMAX;
      if (nc == NMAX)
        accum_two_rows<NMAX, NMAX>(ex01, ex23, ey0, ey1, nc, a01, a23, b01, b23);
      else
        accum_two_rows<NMAX, 0>(ex01, ex23, ey0, ey1, nc, a01, a23, b01, b23);
      if (!col_ok) continue;
      emit(a01, a23, d0v, r);
      if (two) emit(b01, b23, d1v, r + 1);
    }
    cp_async_wait<0>();
    unsigned long long key =
        best >= 0.0f ? ((unsigned long long)__float_as_uint(best) << 32) | (0xffffffffu - bidx) : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
      key = k2 > key ? k2 : key;
    }
    if (lane == 0 && n > 0 && key) atomicMax(&rec->argmax_key, key);
  }
}

int map_tile_h(int width, int height, int window) {
  (void)width;
  (void)window;
  return height < 64 ? ((height + 7) / 8) * 8 : 64;
}

namespace {

template <int NMAX, typename TIn, typename TOut>
cudaError_t launch_typed(const MapParams& p, cudaStream_t st) {
  const size_t smem = (size_t)NMAX * kTileW * 4 + (size_t)p.tile_h * NMAX * 4;
  const long long blocks = (long long)p.n_frames * p.tiles_x * p.tiles_y;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  auto aligned = [](const void* q, int a) { return q == nullptr || ((uintptr_t)q % a) == 0; };
  const bool vec = (p.width % 4) == 0 && aligned(p.depth, Px<TIn>::kAlign) &&
                   aligned(p.M, Px<TOut>::kAlign) && aligned(p.G, Px<TOut>::kAlign);
  if (vec) {
    // streaming kernel: persistent grid of (SMs x resident CTAs)
    const int bands = (p.height + kBandMax - 1) / kBandMax;
    const int band_h = (p.height + bands - 1) / bands;
    const size_t smem2 = (size_t)band_h * NMAX * 4 + (size_t)(kMapThreads / 32) * kStages * 32 * 16;
    auto k = map_stream_kernel<NMAX, TIn, TOut>;
    static int per_sm = -1, sms = 0;
    if (per_sm < 0) {
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kBandMax * NMAX * 4 + (kMapThreads / 32) * kStages * 32 * 16));
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kMapThreads,
                                                    (size_t)kBandMax * NMAX * 4 +
                                                        (kMapThreads / 32) * kStages * 32 * 16);
      if (per_sm < 1) per_sm = 1;
    }
    const long long units = (long long)p.n_frames * ((p.height + band_h - 1) / band_h) *
                            ((p.tiles_x + 7) / 8);
    const long long grid = std::min<long long>(units, (long long)sms * per_sm);
    k<<<(unsigned)grid, kMapThreads, smem2, st>>>(p, band_h);
  } else {
    auto k = map_kernel<NMAX, TIn, TOut, false>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<(unsigned)blocks, kMapThreads, smem, st>>>(p);
  }
  return cudaGetLastError();
}

template <int NMAX>
cudaError_t launch_n(const MapParams& p, int in_dtype, int out_dtype, cudaStream_t st) {
  switch (in_dtype * 3 + out_dtype) {
    case MF_F32 * 3 + MF_F32: return launch_typed<NMAX, float, float>(p, st);
    case MF_F32 * 3 + MF_BF16: return launch_typed<NMAX, float, __nv_bfloat16>(p, st);
    case MF_F32 * 3 + MF_F16: return launch_typed<NMAX, float, __half>(p, st);
    case MF_BF16 * 3 + MF_F32: return launch_typed<NMAX, __nv_bfloat16, float>(p, st);
    case MF_BF16 * 3 + MF_BF16: return launch_typed<NMAX, __nv_bfloat16, __nv_bfloat16>(p, st);
    case MF_BF16 * 3 + MF_F16: return launch_typed<NMAX, __nv_bfloat16, __half>(p, st);
    case MF_F16 * 3 + MF_F32: return launch_typed<NMAX, __half, float>(p, st);
    case MF_F16 * 3 + MF_BF16: return launch_typed<NMAX, __half, __nv_bfloat16>(p, st);
    case MF_F16 * 3 + MF_F16: return launch_typed<NMAX, __half, __half>(p, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_map(const MapParams& p, int window, int in_dtype, int out_dtype,
                       cudaStream_t st, int64_t* launches) {
  if (p.n_frames <= 0) return cudaSuccess;
  cudaError_t e;
  if (window <= 8)
    e = launch_n<8>(p, in_dtype, out_dtype, st);
  else if (window <= 16)
    e = launch_n<16>(p, in_dtype, out_dtype, st);
  else
    e = launch_n<32>(p, in_dtype, out_dtype, st);
  if (e == cudaSuccess) ++*launches;
  return e;
}

}  // namespace mf
