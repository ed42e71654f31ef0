// Device code shared by the per-stream and the batched map kernels: the
// motion-focus map of Eq. 7 and the motion-guided depth over one "unit" (a
// band of up to 256 rows of one frame, across a group of 8 adjacent strips of
// 32*CPT columns), with the frame's argmax.  Both launch paths run exactly
// this code, so a frame's maps do not depend on which path, batch or tile
// schedule produced them.
//
// Per unit:
//   * warp 0 keeps only the points whose Gaussian can reach the unit: a point
//     whose largest column factor over the unit times its largest row factor
//     (times 1/Z) is below 2^-40 contributes less than 2^-40 to every pixel
//     of it, far inside the 1e-10 absolute floor of the map tolerance; kept
//     points keep their order;
//   * each warp applies the same rule to its own strip: a strip that no
//     kept point reaches reads no depth and writes zeros (at most 32 points
//     are dropped from any pixel, each below 2^-40, together below 2^-35);
//   * the CTA evaluates the band's row factors once in shared memory;
//   * each warp owns one strip: every lane holds its CPT columns' factors for
//     the kept points in registers and streams the band's rows two at a time
//     (CPT/2 x 2 independent FMA chains), depth arriving through the warp's
//     ring of cp.async stages, maps leaving through streaming stores.
// The map is a sum of N isotropic Gaussians, so each term factors as
//     exp(-((x-u)^2 + (y-v)^2) c) = exp(-(x-u)^2 c) * exp(-(y-v)^2 c),
// c = 1/(2 sigma_i^2); every pixel then costs one FP32 FMA per kept point,
// issued two pixels at a time (fma.rn.f32x2), in point order.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <type_traits>

#include "mf_internal.h"

namespace mf {

constexpr float kCullBelow = 9.094947017729282e-13f;  // 2^-40

// Resident warps per SM the persistent map kernels are compiled for: 24
// where 2 pixels per lane and at most 16 points keep the unit within 85
// registers; 8 for 4 pixels per lane above 16 points (the column factors
// alone take 128 registers); else 16 (the 128-register unit).  CTAs per SM:
// that over the warps of a CTA.
__host__ __device__ constexpr int unit_warps_per_sm(int nmax, int cpt) {
  return cpt == 2 && nmax <= 16 ? 24 : (cpt == 4 && nmax > 16 ? 8 : 16);
}
__host__ __device__ constexpr int unit_ctas_per_sm(int nmax, int cpt) {
  return unit_warps_per_sm(nmax, cpt) / kGroupStrips;
}

// Depth rows in flight per warp; the ring packs a row at CPT x in_bytes
// bytes per lane.  Rows of 16 bytes per lane: kStages.  Narrower rows: 2 KB
// per warp where 24 warps share an SM, 4 KB where 16 or 8 do (1080p frames:
// the 4 KB ring gains 2-6 % at 16 warps per SM and loses about 1 % at
// 24).
__host__ __device__ constexpr int ring_stages(int cpt, int in_bytes, int nmax) {
  return cpt * in_bytes >= 16 ? kStages
                              : (unit_warps_per_sm(nmax, cpt) == 24 ? 2048 : 4096) / (32 * cpt * in_bytes);
}

// A lane's depth bytes of ring row slot `slot` (rows packed at BYTES per lane).
template <int BYTES>
__device__ __forceinline__ uint4 ring_row(const uint4* ring, int slot) {
  const char* q = reinterpret_cast<const char*>(ring) + slot * BYTES;
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (BYTES == 16) {
    v = *reinterpret_cast<const uint4*>(q);
  } else if (BYTES == 8) {
    const uint2 t = *reinterpret_cast<const uint2*>(q);
    v.x = t.x;
    v.y = t.y;
  } else {
    v.x = *reinterpret_cast<const unsigned*>(q);
  }
  return v;
}

template <int NMAX>
struct PointsSmem {
  float uhi[NMAX], ulo[NMAX], vhi[NMAX], vlo[NMAX], chi[NMAX], clo[NMAX];
  int kept;  // entries in use (the map unit's lists)
};

// 2^x by the hardware base-2 exponential (PTX ex2.approx.ftz: relative
// error of a few ulp; results below 2^-126 flush to 0).
__device__ __forceinline__ float exp2_hw(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// exp(-(q - hi - lo)^2 / (2 sigma^2)) = 2^-((q - hi - lo)^2 (chi + clo)) for an
// integer-valued q, with chi + clo = log2(e) / (2 sigma^2) as a float pair.
// hi lies on a 2^-8 grid with |hi| < 2^15, so q - hi is exact; the square is
// carried as a compensated pair, which keeps the exponent's relative error
// near one FP32 rounding before the base-2 exponential.
__device__ __forceinline__ float gauss_factor(float q, float hi, float lo, float chi, float clo) {
  const float dh = q - hi;
  const float p2 = dh * dh;
  const float e2 = fmaf(dh, dh, -p2);   // dh^2 = p2 + e2 exactly
  float qq = fmaf(-2.0f * dh, lo, e2);  // (dh - lo)^2 = p2 + qq
  qq = fmaf(lo, lo, qq);
  const float t1 = fmaf(clo, p2, chi * qq);
  const float a = fmaf(chi, p2, t1);
  return exp2_hw(-a);
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

// a * b on both lanes of a (the first term of a sum: a product rounds
// exactly as a fused multiply-add onto +0 does when the product is >= +0).
__device__ __forceinline__ float2 fmul2(float2 a, float b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %4};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b));
  return d;
}

// Lane-wise a + b, a * b and fma(a, b, c) on f32x2 pairs (IEEE round to
// nearest on each lane: the values of the scalar operations).
__device__ __forceinline__ float2 fadd2v(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 fmul2v(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 ffma2v(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// gauss_factor at columns q0 and q0 + 1 (q0 integer-valued), the exponent's
// steps on f32x2 pairs: the same operations in the same order on each lane,
// with the signs carried through exact negations, so the same values.
__device__ __forceinline__ float2 gauss_pair(float q0, float hi, float lo, float chi, float clo) {
  const float2 dh = fadd2v(make_float2(q0, q0 + 1.0f), make_float2(-hi, -hi));  // exact
  const float2 p2 = fmul2v(dh, dh);
  const float2 e2 = ffma2v(dh, dh, fmul2v(p2, make_float2(-1.0f, -1.0f)));        // dh^2 - p2
  float2 qq = ffma2v(fmul2v(dh, make_float2(-2.0f, -2.0f)), make_float2(lo, lo), e2);
  qq = ffma2v(make_float2(lo, lo), make_float2(lo, lo), qq);
  const float2 nt1 = ffma2v(make_float2(-clo, -clo), p2, fmul2v(make_float2(-chi, -chi), qq));
  const float2 na = ffma2v(make_float2(-chi, -chi), p2, nt1);                      // -a
  return make_float2(exp2_hw(na.x), exp2_hw(na.y));
}

// max(a, b, c) in one instruction (three-input max.f32 of sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Largest of one lane's CPT pixels of rows a and b (b only when `two`).
template <int CPT>
__device__ __forceinline__ float lane_max(const float2 (&a)[CPT / 2], const float2 (&b)[CPT / 2], bool two) {
  float m = fmax3(a[0].x, a[0].y, two ? fmaxf(b[0].x, b[0].y) : a[0].x);
#pragma unroll
  for (int c = 1; c < CPT / 2; ++c) m = fmax3(m, fmaxf(a[c].x, a[c].y), two ? fmaxf(b[c].x, b[c].y) : m);
  return m;
}

// min(1, d0 / x) for x = D - 2^-149, as one approximate reciprocal (PTX
// rcp.approx.ftz, within about an ulp) and one saturating product, with no
// compare or select.  Subtracting the smallest denormal leaves every normal
// D unchanged and moves D = +0 and -0 below zero; the flush to zero of the
// reciprocal's input then gives:
//   normal D > 0        -> min(1, d0 / D);
//   positive denormal D -> 1/x = +inf -> 1 (the clamp of a huge quotient);
//   D = +-0, D < 0      -> 1/x <= -0 -> 0 ("no depth");
//   D = NaN             -> NaN, which the saturation turns into 0;
//   D = +inf            -> 0;  D = -inf -> -0 -> 0.
__device__ __forceinline__ float weight_of(float x, float d0) {
  float r, w;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  asm("mul.rn.sat.f32 %0, %1, %2;" : "=f"(w) : "f"(d0), "f"(r));
  return w;
}
__device__ __forceinline__ float depth_weight(float D, float d0) { return weight_of(D - 0x1p-149f, d0); }

// G = M min(1, d0 / D) for one lane's CPT pixels.
template <int CPT>
__device__ __forceinline__ void guided(const float (&m)[CPT], const float (&D)[CPT], float d0, float (&g)[CPT]) {
#pragma unroll
  for (int c = 0; c < CPT; c += 2) {
    float x0, x1;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %4};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(x0), "=f"(x1) : "f"(D[c]), "f"(D[c + 1]), "f"(-0x1p-149f));
    const float w0 = weight_of(x0, d0), w1 = weight_of(x1, d0);
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(g[c]), "=f"(g[c + 1]) : "f"(m[c]), "f"(m[c + 1]), "f"(w0), "f"(w1));
  }
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  if (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
  else if (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

// Zero rows through the bulk-copy engine: a shared-memory source of zeros,
// at least one unit row wide (kGroupStrips strips x 32 lanes x 4 columns x
// 4 bytes).
constexpr int kZeroBytes = kGroupStrips * 32 * 4 * 4;
__device__ __forceinline__ void bulk_copy_s2g(void* dst, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"((uint32_t)__cvta_generic_to_shared(src_smem)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Every bulk copy this thread issued has written global memory.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Fills a kernel's zero source (every thread of the CTA calls this once,
// before its first unit) and makes it visible to the bulk-copy engine.
__device__ __forceinline__ void init_zero_source(uint4* zeros) {
  for (int i = threadIdx.x; i < kZeroBytes / 16; i += blockDim.x) zeros[i] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// CPT consecutive storage elements <-> floats.
template <typename T, int CPT>
struct Vec;

template <int CPT>
struct Vec<float, CPT> {
  static __device__ __forceinline__ void unpack(const uint4& r, float (&d)[CPT]) {
    d[0] = __uint_as_float(r.x);
    d[1] = __uint_as_float(r.y);
    if (CPT == 4) {
      d[CPT > 2 ? 2 : 0] = __uint_as_float(r.z);
      d[CPT > 3 ? 3 : 0] = __uint_as_float(r.w);
    }
  }
  static __device__ __forceinline__ void store(void* plane, size_t i, const float (&v)[CPT]) {
    float* q = static_cast<float*>(plane) + i;
    if (CPT == 4)
      __stcs(reinterpret_cast<float4*>(q), make_float4(v[0], v[1], v[CPT > 2 ? 2 : 0], v[CPT > 3 ? 3 : 0]));
    else
      __stcs(reinterpret_cast<float2*>(q), make_float2(v[0], v[1]));
  }
};

template <typename H>
struct Half2Of;
template <>
struct Half2Of<__nv_bfloat16> {
  static __device__ __forceinline__ float2 to_f2(unsigned w) {
    return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&w));
  }
  static __device__ __forceinline__ unsigned from_f2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<unsigned*>(&h);
  }
};
template <>
struct Half2Of<__half> {
  static __device__ __forceinline__ float2 to_f2(unsigned w) {
    return __half22float2(*reinterpret_cast<__half2*>(&w));
  }
  static __device__ __forceinline__ unsigned from_f2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned*>(&h);
  }
};

template <typename H, int CPT>
struct Vec16 {
  static __device__ __forceinline__ void unpack(const uint4& r, float (&d)[CPT]) {
    const float2 a = Half2Of<H>::to_f2(r.x);
    d[0] = a.x;
    d[1] = a.y;
    if (CPT == 4) {
      const float2 c = Half2Of<H>::to_f2(r.y);
      d[CPT > 2 ? 2 : 0] = c.x;
      d[CPT > 3 ? 3 : 0] = c.y;
    }
  }
  static __device__ __forceinline__ void store(void* plane, size_t i, const float (&v)[CPT]) {
    H* q = static_cast<H*>(plane) + i;
    if (CPT == 4) {
      uint2 w;
      w.x = Half2Of<H>::from_f2(v[0], v[1]);
      w.y = Half2Of<H>::from_f2(v[CPT > 2 ? 2 : 0], v[CPT > 3 ? 3 : 0]);
      __stcs(reinterpret_cast<uint2*>(q), w);
    } else {
      __stcs(reinterpret_cast<unsigned*>(q), Half2Of<H>::from_f2(v[0], v[1]));
    }
  }
};
template <int CPT>
struct Vec<__nv_bfloat16, CPT> : Vec16<__nv_bfloat16, CPT> {};
template <int CPT>
struct Vec<__half, CPT> : Vec16<__half, CPT> {};

// Two rows' sums for one lane's CPT columns, points 0..nc-1 in order.  NC > 0
// fixes the trip count at compile time (all NMAX points kept).  INIT: the
// sums start with the first point's product (nc >= 1; no zeroed
// accumulators), else they add onto a and b as given.  Both give the same
// bits: every term is >= +0.
template <int NMAX, int CPT, int NC, bool INIT = false>
__device__ __forceinline__ void accum_two_rows(const float2 (&ex)[NMAX][CPT / 2], const float* ey0,
                                               const float* ey1, int nc, float2 (&a)[CPT / 2],
                                               float2 (&b)[CPT / 2]) {
  const float4* e0p = reinterpret_cast<const float4*>(ey0);
  const float4* e1p = reinterpret_cast<const float4*>(ey1);
#pragma unroll
  for (int i = 0; i < (NC ? NC : NMAX); i += 4) {
    if (NC == 0 && i >= nc) break;
    const float4 e = e0p[i >> 2];
    const float4 f = e1p[i >> 2];
    const float es[4] = {e.x, e.y, e.z, e.w};
    const float fs[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int c = 0; c < CPT / 2; ++c) {
        if (INIT && i == 0 && k == 0) {
          a[c] = fmul2(ex[0][c], es[0]);
          b[c] = fmul2(ex[0][c], fs[0]);
        } else {
          a[c] = ffma2(ex[i + k][c], es[k], a[c]);
          b[c] = ffma2(ex[i + k][c], fs[k], b[c]);
        }
      }
    }
  }
}

// Warp-wide maximum of the lanes' argmax keys, published to the frame's
// record by lane 0 (frames without valid points keep key 0).
__device__ __forceinline__ void publish_key(FrameRec* rec, unsigned long long key, bool any_points) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
    key = k2 > key ? k2 : key;
  }
  if ((threadIdx.x & 31) == 0 && any_points && key) atomicMax(&rec->argmax_key, key);
}

// Trip count of the fast row loop for q groups of 4 kept points (1 <= q):
// 4 q, except that above 16 points counts up to 16 take 8 or 16 (fewer
// compiled copies of the loop where they are rare).
__host__ __device__ constexpr int padded_count(int nmax, int q) {
  return 4 * q >= nmax ? nmax : (nmax > 16 && q <= 4 ? (q <= 2 ? 8 : 16) : 4 * q);
}

// One unit of one frame.  planes point at the frame's first pixel; the
// caller guarantees width % CPT == 0 and CPT-element alignment of all
// planes.  Every thread of the CTA must call this (it holds barriers).
struct UnitGeom {
  FrameRec* rec;
  const char* depth;  // frame plane or NULL
  char* M;            // frame plane or NULL
  char* G;            // frame plane or NULL
  int width, height;
  int y0, rows;       // band
  int gx0;            // first column of the strip group
  float d0;
  unsigned int* fault;  // checked builds: reports an access outside the planes (may be NULL)
};

// Checked builds: rows y of columns x .. x + n - 1 lie in the unit's
// planes (else the fault word is set and the caller skips the access).
// Release builds: always true, and the test compiles away.
__device__ __forceinline__ bool in_plane(const UnitGeom& ug, int y, int x, int n) {
  if (!kChecked) return true;
  const bool ok = y >= 0 && y < ug.height && x >= 0 && n >= 0 && x + n <= ug.width;
  if (!ok && ug.fault) atomicExch_system(ug.fault, kFaultOutOfRange);
  return ok;
}

// What a pass over a unit produces.  Full: M, G and the frame's argmax.
// MaxOnly: the argmax alone (no memory traffic), the first pass of
// MF_NORM_MAX.  Scaled: M and G of the map divided by the frame's maximum
// from that first pass -- the same FP32 sums, so the pixel holding the
// maximum becomes exactly 1.
constexpr int kUnitFull = 0;
constexpr int kUnitMaxOnly = 1;
constexpr int kUnitScaled = 2;

template <int NMAX, int CPT, typename TIn, typename TOut, int MODE = kUnitFull>
__device__ __forceinline__ void map_unit(const UnitGeom& ug, float* Ey, uint4* my_ring,
                                         PointsSmem<kMaxPts>* Pw, const uint4* zeros) {
  constexpr int kInBytes = CPT * (int)sizeof(TIn);
  constexpr int kStrip = 32 * CPT;
  constexpr int S = ring_stages(CPT, (int)sizeof(TIn), NMAX);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rows = ug.rows, y0 = ug.y0;
  const int x0 = ug.gx0 + warp * kStrip;
  const int xc = x0 + lane * CPT;
  const bool col_ok = xc < ug.width;
  const int gx1 = min(ug.width, ug.gx0 + kGroupStrips * kStrip) - 1;
  const size_t row0 = (size_t)y0 * ug.width + xc;
  const char* dsrc = (MODE != kUnitMaxOnly && ug.depth) ? ug.depth + row0 * sizeof(TIn) : nullptr;
  const size_t dstride = (size_t)ug.width * sizeof(TIn);
  static_assert((S & (S - 1)) == 0, "ring stages must be a power of two");
  // Depth rows are requested in order, one group per row: rq is the next
  // row to request and dq its source (a running pointer, no per-row
  // multiply).  `sure`: the caller knows that dsrc is set and the lane's
  // columns lie inside the frame.
  int rq = 0;
  uintptr_t dq = reinterpret_cast<uintptr_t>(dsrc);
  auto issue = [&](bool sure) {
    if (rq < rows && (sure || (col_ok && dsrc)) && in_plane(ug, y0 + rq, xc, CPT))
      cp_async<kInBytes>(reinterpret_cast<char*>(my_ring) + ((rq & (S - 1)) * 32 + lane) * kInBytes,
                         reinterpret_cast<const char*>(dq));
    cp_async_commit();
    ++rq;
    dq += dstride;
  };
  // The ring is this warp's own and the previous unit drained it.  Every
  // warp culls the points itself into its own copy of the kept list (the
  // same list in every warp), so no warp waits for another before the row
  // factors; the caller's barrier between units (next_unit) ordered every
  // warp's last use of the previous unit's tables before the writes below.
  // The one-CTA-per-SM unit (4 columns per lane above 16 points) keeps one
  // list, culled by warp 0 between two barriers: its register-bound code
  // measured 5 % slower with per-warp lists (HEADING BF16, window 32),
  // where the others gained up to 2 %.
  constexpr bool kOwnList = !(CPT == 4 && NMAX > 16);
  if (!kOwnList) __syncthreads();  // the previous unit is done with P and Ey

  FrameRec* rec = ug.rec;
  const int n = rec->n_valid;
  const float inv_n = rec->inv_n;
  // This warp's strip as zeros: its rows (when write_rows; plain CPT-element
  // stores, or with bulk one bulk copy per row and map, which needs 16-byte
  // aligned rows) and its argmax candidate, the strip's first pixel (0).
  auto zero_strip = [&](bool write_rows, bool bulk) {
    if (write_rows && MODE != kUnitMaxOnly) {
      if (bulk) {
        const uint32_t bytes = (uint32_t)(min(kStrip, ug.width - x0) * (int)sizeof(TOut));
        const size_t first = (size_t)y0 * ug.width + x0;
        for (int r = lane; r < rows; r += 32) {
          const size_t at = (first + (size_t)r * ug.width) * sizeof(TOut);
          if (!in_plane(ug, y0 + r, x0, (int)(bytes / sizeof(TOut)))) continue;
          if (ug.M) bulk_copy_s2g(ug.M + at, zeros, bytes);
          if (ug.G) bulk_copy_s2g(ug.G + at, zeros, bytes);
        }
        bulk_commit();
      } else if (col_ok) {
        const float z[CPT] = {};
        const size_t ostride = (size_t)ug.width * sizeof(TOut);
        char* qm = ug.M ? ug.M + row0 * sizeof(TOut) : nullptr;
        char* qg = ug.G ? ug.G + row0 * sizeof(TOut) : nullptr;
        int ry = y0;
        for (size_t off = 0, end = (size_t)rows * ostride; off < end; off += ostride, ++ry) {
          if (!in_plane(ug, ry, xc, CPT)) continue;
          if (qm) Vec<TOut, CPT>::store(qm + off, 0, z);
          if (qg) Vec<TOut, CPT>::store(qg + off, 0, z);
        }
      }
    }
    if (MODE != kUnitScaled)
      publish_key(rec, col_ok ? (unsigned long long)(0xffffffffu - (unsigned)(y0 * ug.width + xc)) : 0ull, n > 0);
  };
  PointsSmem<kMaxPts>& P = Pw[kOwnList ? warp : 0];
  int nk;  // <= NMAX: n never exceeds the window's bucket
  if (kOwnList || warp == 0) {
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
      const float xn = fminf(fmaxf(rintf(uh + ul), (float)ug.gx0), (float)gx1);
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
    nk = __popc(mask);
    if (!kOwnList && lane == 0) P.kept = nk;
    __syncwarp();
  }
  if (!kOwnList) {
    __syncthreads();  // warp 0's list is complete
    nk = P.kept;
  }
  // Zero rows by bulk copy need 16-byte aligned rows in both map planes.
  const bool bulk = zeros != nullptr && ((size_t)ug.width * sizeof(TOut)) % 16 == 0 &&
                    ((uintptr_t)ug.M % 16) == 0 && ((uintptr_t)ug.G % 16) == 0;
  if (nk == 0 && (bulk || sizeof(TOut) == 2)) {
    // No point reaches the unit: M = 0 and G = M min(1, d0/D) = 0 on every
    // pixel, whatever the depth holds, and each lane's maximum is that 0 at
    // its first pixel.  The zero rows leave through the bulk-copy engine
    // (one copy per row and map, issued across the CTA), or with 16-bit
    // maps and unaligned rows through plain stores: no depth copies, factor
    // tables or per-row bookkeeping.  (Measured on 1080p ACCEL frames: FP32
    // maps with plain zero stores lose about 1 % against the general loop,
    // so FP32 without bulk copies keeps that loop.)
    if (bulk && MODE != kUnitMaxOnly) {
      const int cols = min(kGroupStrips * kStrip, ug.width - ug.gx0);
      const uint32_t bytes = (uint32_t)(cols * (int)sizeof(TOut));
      const size_t first = (size_t)y0 * ug.width + ug.gx0;
      for (int r = tid; r < rows; r += kUnitThreads) {
        const size_t at = (first + (size_t)r * ug.width) * sizeof(TOut);
        if (!in_plane(ug, y0 + r, ug.gx0, cols)) continue;
        if (ug.M) bulk_copy_s2g(ug.M + at, zeros, bytes);
        if (ug.G) bulk_copy_s2g(ug.G + at, zeros, bytes);
      }
      bulk_commit();
    }
    if (x0 >= ug.width) return;  // warp-uniform: this strip lies past the frame
    zero_strip(!bulk, false);  // with bulk the CTA's copies above wrote the rows
    return;
  }
  // Depth only scales G: with no G output, or no point kept (M = 0, so G = 0
  // whatever D holds), its rows are not read.
  if (nk == 0 || !ug.G) dsrc = nullptr;
  // A warp whose strip none of the kept points reaches (the same 2^-40 rule
  // over the strip's columns and the band's rows) has M = 0 and G = 0 there:
  // it reads no depth and writes zeros.
  bool strip_zero = false;
  {
    const int sx1 = min(ug.width, x0 + kStrip) - 1;
    bool reach = false;
    if (lane < nk && x0 <= sx1) {
      const float xn = fminf(fmaxf(rintf(P.uhi[lane] + P.ulo[lane]), (float)x0), (float)sx1);
      const float yn = fminf(fmaxf(rintf(P.vhi[lane] + P.vlo[lane]), (float)y0), (float)(y0 + rows - 1));
      const float peak = gauss_factor(xn, P.uhi[lane], P.ulo[lane], P.chi[lane], P.clo[lane]) *
                         gauss_factor(yn, P.vhi[lane], P.vlo[lane], P.chi[lane], P.clo[lane]);
      reach = peak * inv_n >= kCullBelow;
    }
    strip_zero = __ballot_sync(0xffffffffu, reach) == 0u;
  }
  if (strip_zero) dsrc = nullptr;
  // the first depth rows are in flight while the factors are computed
  dq = reinterpret_cast<uintptr_t>(dsrc);  // after the strip test (dsrc may have been dropped)
#pragma unroll
  for (int s = 0; s < S - 2; ++s) issue(false);
  const int nc = min(NMAX, (nk + 3) & ~3);
  // Row factors times 1/Z, two rows per entry and NMAX entries per row
  // pair, so that every lane has work also below 32 points: entry k is point
  // k % NMAX of rows 2 (k / NMAX) and 2 (k / NMAX) + 1.
  for (int k = tid; k < ((rows + 1) >> 1) * NMAX; k += kUnitThreads) {
    const int i = k & (NMAX - 1), r = 2 * (k / NMAX);
    float2 g = make_float2(0.0f, 0.0f);  // zeros past the kept points (padded trip counts)
    if (i < nk) {
      g = gauss_pair((float)(y0 + r), P.vhi[i], P.vlo[i], P.chi[i], P.clo[i]);
      g.x *= inv_n;
      g.y *= inv_n;
    }
    Ey[r * NMAX + i] = g.x;
    if (r + 1 < rows) Ey[(r + 1) * NMAX + i] = g.y;
  }
  float2 ex[NMAX][CPT / 2];
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
#pragma unroll
    for (int c = 0; c < CPT / 2; ++c) {
      ex[i][c] = i < nk && col_ok && !strip_zero
                     ? gauss_pair((float)(xc + 2 * c), P.uhi[i], P.ulo[i], P.chi[i], P.clo[i])
                     : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();  // Ey complete
  if (x0 >= ug.width) return;  // warp-uniform: this strip lies past the frame (no copies issued)
  if (strip_zero) {
    zero_strip(true, bulk);
    return;
  }

  // The lane's running maximum and the first row pair that holds it; the
  // pixel is found once per unit after the rows (ties: lower row, then
  // lower column, i.e. the lowest linear index).
  float best = -1.0f;
  int brow = -1;
  char* mrow = (MODE != kUnitMaxOnly && ug.M) ? ug.M + row0 * sizeof(TOut) : nullptr;
  char* grow = (MODE != kUnitMaxOnly && ug.G) ? ug.G + row0 * sizeof(TOut) : nullptr;
  // Scaled pass: divide by the maximum the first pass found (IEEE reciprocal
  // once per unit, then a product; the maximum itself maps to exactly 1)
  float mx = 0.0f, inv = 1.0f;
  bool scale = false;
  if (MODE == kUnitScaled) {
    const unsigned long long key = rec->argmax_key;
    mx = __uint_as_float((unsigned)(key >> 32));
    scale = n > 0 && key != 0ull && mx >= kNormFloor;
    inv = scale ? 1.0f / mx : 1.0f;
  }
  const size_t ostride = (size_t)ug.width * sizeof(TOut);
  // Sums of rows r and r+1 (r alone when !two): they start with the first
  // point's product; no kept point (nc = 0) gives zeros.
  auto sums = [&](int r, bool two, float2 (&a)[CPT / 2], float2 (&b)[CPT / 2]) {
    const float* ey0 = Ey + r * NMAX;
    const float* ey1 = Ey + (two ? r + 1 : r) * NMAX;
    if (nc == NMAX) {
      accum_two_rows<NMAX, CPT, NMAX, true>(ex, ey0, ey1, nc, a, b);
    } else if (nc > 0) {
      accum_two_rows<NMAX, CPT, 0, true>(ex, ey0, ey1, nc, a, b);
    } else {
#pragma unroll
      for (int c = 0; c < CPT / 2; ++c) a[c] = b[c] = make_float2(0.f, 0.f);
    }
  };
  // Rows r and r+1 per step: the ring slots of rows r-2 and r-1 were
  // consumed by the previous step, so rows r+S-2 and r+S-1 can be requested
  // before rows r, r+1 are read.  FAST: depth, M and G all present, every
  // lane's columns inside the frame and an even number of rows (the common
  // case), so a step carries no null, column or last-row checks.
  auto rows_loop = [&](auto fast_tag, auto nc_tag) {
    constexpr bool FAST = decltype(fast_tag)::value;
    constexpr int NCF = decltype(nc_tag)::value;  // > 0: the sums' trip count (padded)
    size_t off = 0;  // output rows advance by a stride: no per-row 64-bit multiply
    for (int r = 0; r < rows; r += 2, off += 2 * ostride) {
      const bool TWO = FAST || r + 1 < rows;
      issue(FAST);
      issue(FAST);
      cp_async_wait<S - 2>();
      float d0v[CPT], d1v[CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) d0v[c] = d1v[c] = 0.0f;
      if (FAST || dsrc) {
        Vec<TIn, CPT>::unpack(ring_row<kInBytes>(my_ring, (r & (S - 1)) * 32 + lane), d0v);
        if (TWO) Vec<TIn, CPT>::unpack(ring_row<kInBytes>(my_ring, ((r + 1) & (S - 1)) * 32 + lane), d1v);
      }
      float2 a[CPT / 2], b[CPT / 2];
      if constexpr (NCF > 0)
        accum_two_rows<NMAX, CPT, NCF, true>(ex, Ey + r * NMAX, Ey + (r + 1) * NMAX, NCF, a, b);
      else
        sums(r, TWO, a, b);
      if (!FAST && !col_ok) continue;
      if (MODE != kUnitMaxOnly) {
        const size_t o = off;
        auto emit = [&](const float2 (&acc)[CPT / 2], const float (&dv)[CPT], size_t oo, int ry) {
          float m[CPT];
#pragma unroll
          for (int c = 0; c < CPT / 2; ++c) {
            m[2 * c] = acc[c].x;
            m[2 * c + 1] = acc[c].y;
          }
          if (MODE == kUnitScaled && scale) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) m[c] = m[c] == mx ? 1.0f : m[c] * inv;
          }
          if (!in_plane(ug, ry, xc, CPT)) return;
          if (FAST || mrow) Vec<TOut, CPT>::store(mrow + oo, 0, m);
          if (FAST || grow) {
            float gv[CPT];
            guided<CPT>(m, dv, ug.d0, gv);
            Vec<TOut, CPT>::store(grow + oo, 0, gv);
          }
        };
        emit(a, d0v, o, y0 + r);
        if (TWO) emit(b, d1v, o + ostride, y0 + r + 1);
      }
      if (MODE != kUnitScaled) {
        const float mm = lane_max<CPT>(a, b, TWO);
        if (mm > best) {
          best = mm;
          brow = r;
        }
      }
    }
  };
  // FAST steps run the sums with a trip count fixed at compile time: the kept
  // count rounded up to a multiple of 4, and above 16 points of 8 when at
  // most 16 are kept.  The table and column factors past the kept points
  // are zeros, and a zero term leaves a sum of non-negative terms unchanged,
  // so the padded sums have the same bits.
  const bool inside = x0 + kStrip <= ug.width;  // warp-uniform: every lane's columns
  if (dsrc && mrow && grow && inside && (rows & 1) == 0 && nc > 0) {
    auto fast = [&](auto nc_tag) { rows_loop(std::true_type{}, nc_tag); };
    using std::integral_constant;
    switch (nc >> 2) {  // 1 .. NMAX / 4
      case 1: fast(integral_constant<int, padded_count(NMAX, 1)>{}); break;
      case 2: fast(integral_constant<int, padded_count(NMAX, 2)>{}); break;
      case 3: fast(integral_constant<int, padded_count(NMAX, 3)>{}); break;
      case 4: fast(integral_constant<int, padded_count(NMAX, 4)>{}); break;
      case 5: fast(integral_constant<int, padded_count(NMAX, 5)>{}); break;
      case 6: fast(integral_constant<int, padded_count(NMAX, 6)>{}); break;
      case 7: fast(integral_constant<int, padded_count(NMAX, 7)>{}); break;
      default: fast(integral_constant<int, NMAX>{}); break;
    }
  } else {
    rows_loop(std::false_type{}, std::integral_constant<int, 0>{});
  }
  cp_async_wait<0>();
  if (MODE != kUnitScaled) {
    unsigned long long key = 0ull;
    if (best >= 0.0f) {
      // the winning row pair again, with the same sums in the same order
      const bool two = brow + 1 < rows;
      float2 a[CPT / 2], b[CPT / 2];
      sums(brow, two, a, b);
      float ma = fmaxf(a[0].x, a[0].y);
#pragma unroll
      for (int c = 1; c < CPT / 2; ++c) ma = fmax3(ma, a[c].x, a[c].y);
      const bool first = ma == best;
      float m[CPT];
#pragma unroll
      for (int c = 0; c < CPT / 2; ++c) {
        m[2 * c] = first ? a[c].x : b[c].x;
        m[2 * c + 1] = first ? a[c].y : b[c].y;
      }
      unsigned off = CPT - 1;
#pragma unroll
      for (int c = CPT - 2; c >= 0; --c)
        if (m[c] == best) off = c;
      const unsigned bidx = (unsigned)((y0 + brow + (first ? 0 : 1)) * ug.width + xc) + off;
      key = ((unsigned long long)__float_as_uint(best) << 32) | (0xffffffffu - bidx);
    }
    publish_key(rec, key, n > 0);
  }
}

// Dynamic shared memory of a CTA running units of bucket NMAX with CPT
// pixels per lane and in_bytes-byte depth: the band's row factors, then
// every warp's depth ring.
__host__ __device__ constexpr size_t unit_smem_bytes(int nmax, int band_h, int cpt, int in_bytes) {
  return (size_t)band_h * nmax * 4 +
         (size_t)kGroupStrips * ring_stages(cpt, in_bytes, nmax) * 32 * cpt * in_bytes;
}

// Dynamic unit schedule of the persistent map kernels.  CTA c starts on
// unit c.  While the CTA works on a unit, its thread 0 holds a claim on the
// next one from a launch-wide counter (claims at or past the last unit end
// the CTA's loop), so CTAs that draw cheap units -- ones no point reaches --
// take more of them instead of idling at the end of the launch.  Every unit
// processed makes one claim, so a launch makes exactly `units` of them and
// the claim that returns units - 1 is its last: that thread puts the counter
// back to 0 for the next launch.  The counter must be 0 at launch, and no
// two launches in flight may share it; a launch holds fewer than 2^32 units.
__device__ __forceinline__ unsigned claim_unit(unsigned* ctr) {
  return threadIdx.x == 0 ? atomicAdd(ctr, 1u) : 0u;
}

// Called by every thread after the CTA's k-th unit with thread 0's claim:
// the CTA's next unit.  s_next is two shared slots, so a slow thread
// still reading slot k & 1 never sees the write of claim k + 1.
__device__ __forceinline__ long long next_unit(unsigned* ctr, unsigned claim, long long units,
                                               long long* s_next, int k) {
  if (threadIdx.x == 0) {
    s_next[k & 1] = (long long)gridDim.x + (long long)claim;
    if ((long long)claim == units - 1) *ctr = 0u;  // the launch's last claim
  }
  __syncthreads();
  return s_next[k & 1];
}

}  // namespace mf
