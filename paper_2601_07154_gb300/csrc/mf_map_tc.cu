// Tensor-core form of the map (Eq. 7) and the motion-guided depth, for the
// cases where the per-pixel FMA work, not HBM, bounds the CUDA-core kernel:
// 16-bit storage (6 B per pixel) and large windows.
//
// Over a tile of 128 columns x 128 rows the map is a rank-N product,
//     M[y][x] = sum_i Ey_i(y) Ex_i(x),   Ey_i(y) = exp(-(y-v_i)^2 c_i) / Z,
//                                        Ex_i(x) = exp(-(x-u_i)^2 c_i),
// a GEMM with K = N.  FP32 accuracy comes from three TF32 products:
// with e = e_hi + e_lo (e_hi = e truncated to TF32, e_lo exact),
//     Ex Ey ~= Ex_hi Ey_hi + Ex_hi Ey_lo + Ex_lo Ey_hi,
// the dropped Ex_lo Ey_lo and the TF32 reading of e_lo are below 2^-20
// relative.  The three products are stacked along K (K' = 3 Kp, Kp = N
// rounded up to 8), so one tcgen05.mma chain of K'/8 steps per tile computes
// the tile in TMEM with FP32 accumulation:
//     A (M = 128 columns x K') = [Ex_hi | Ex_hi | Ex_lo],
//     B (N = 64 rows     x K') = [Ey_hi | Ey_lo | Ey_hi],
//     D[x][y] = sum_k A[x][k] B[y][k]   (TMEM lane = column, TMEM column = row).
// With lane = column, each warp's epilogue reads one row of 32 adjacent
// columns per TMEM column, so depth loads and map stores are coalesced.
//
// Work item = one strip of 128 columns of one frame, all bands of 64 rows;
// CTAs take items from the map kernels' dynamic schedule.  A is built once
// per item (column factors of the points kept for the strip), B once per
// band.  One elected thread issues the MMAs and commits
// them to an mbarrier that the epilogue waits on (bounded; a wait that runs
// out poisons the band's maps with NaN rather than hang).  Operands live in
// shared memory in the no-swizzle K-major core-matrix layout (8 rows x 16 B
// per core matrix; K-adjacent core matrices 128 B apart, 8-row groups K'/4 *
// 128 B apart).  Each CTA holds 128 TMEM columns for its lifetime.
#include "mf_map_unit.cuh"

namespace mf {

namespace {

constexpr int kTcCols = 128;               // tile columns = MMA M = TMEM lanes
constexpr int kTcRows = 64;                // tile rows = MMA N = TMEM columns
constexpr int kTcKsMax = 2 * kMaxPts;      // stored K columns for 32 points
constexpr int kTcThreads = 256;
constexpr long long kTcWaitPolls = 1ll << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Word offset of element (r, k) in an operand with K' = kk (K-major, no swizzle).
__device__ __forceinline__ int operand_word(int r, int k, int kk) {
  return ((r >> 3) * (kk >> 2) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

// Shared-memory matrix descriptor: start address, K-direction core-matrix
// offset (LBO), 8-row-group offset (SBO), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t operand_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major,
// N = kTcRows, M = kTcCols.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                              ((uint32_t)(kTcRows >> 3) << 17) | ((uint32_t)(kTcCols >> 4) << 24);

__device__ __forceinline__ void split_tf32(float e, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(e) & 0xFFFFE000u);
  lo = e - hi;
}

template <typename T>
struct Scalar;
template <>
struct Scalar<float> {
  static __device__ __forceinline__ float load(const void* b, size_t i) {
    return __ldcs(static_cast<const float*>(b) + i);
  }
  static __device__ __forceinline__ void store(void* b, size_t i, float v) {
    __stcs(static_cast<float*>(b) + i, v);
  }
};
template <>
struct Scalar<__nv_bfloat16> {
  static __device__ __forceinline__ float load(const void* b, size_t i) {
    const unsigned short h = __ldcs(static_cast<const unsigned short*>(b) + i);
    return __uint_as_float((unsigned)h << 16);
  }
  static __device__ __forceinline__ void store(void* b, size_t i, float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    __stcs(static_cast<unsigned short*>(b) + i, *reinterpret_cast<const unsigned short*>(&h));
  }
};
template <>
struct Scalar<__half> {
  static __device__ __forceinline__ float load(const void* b, size_t i) {
    const unsigned short h = __ldcs(static_cast<const unsigned short*>(b) + i);
    return __half2float(*reinterpret_cast<const __half*>(&h));
  }
  static __device__ __forceinline__ void store(void* b, size_t i, float v) {
    const __half h = __float2half_rn(v);
    __stcs(static_cast<unsigned short*>(b) + i, *reinterpret_cast<const unsigned short*>(&h));
  }
};

__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_float(__half v) { return __half2float(v); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace

// Column factors of the kept points for one strip: A = [hi | lo], 2 kp
// stored K columns.  Consecutive threads fill one core matrix (8 rows x 4
// words), so a warp's stores are free of bank conflicts.
__device__ __forceinline__ void build_cols(float* sA, const PointsSmem<kMaxPts>& P, int nk, int kp,
                                           int gx0, int width) {
  const int ks = 2 * kp;
  for (int idx = threadIdx.x; idx < kTcCols * kp; idx += kTcThreads) {
    const int i_lo = idx & 3, r_lo = (idx >> 2) & 7, g = idx >> 5;
    const int kg = g % (kp >> 2), r_hi = g / (kp >> 2);
    const int m = 8 * r_hi + r_lo, i = 4 * kg + i_lo;
    const int x = gx0 + m;
    float e = 0.0f;
    if (i < nk && x < width) e = gauss_factor((float)x, P.uhi[i], P.ulo[i], P.chi[i], P.clo[i]);
    float hi, lo;
    split_tf32(e, hi, lo);
    sA[operand_word(m, i, ks)] = hi;
    sA[operand_word(m, kp + i, ks)] = lo;
  }
}

// Row factors times 1/Z for one band: B = [hi | lo].
__device__ __forceinline__ void build_rows(float* sB, const PointsSmem<kMaxPts>& P, int nk, int kp,
                                           int y0, int rows, float inv_n) {
  const int ks = 2 * kp;
  for (int idx = threadIdx.x; idx < kTcRows * kp; idx += kTcThreads) {
    const int i_lo = idx & 3, r_lo = (idx >> 2) & 7, g = idx >> 5;
    const int kg = g % (kp >> 2), r_hi = g / (kp >> 2);
    const int r = 8 * r_hi + r_lo, i = 4 * kg + i_lo;
    float e = 0.0f;
    if (i < nk && r < rows)
      e = gauss_factor((float)(y0 + r), P.vhi[i], P.vlo[i], P.chi[i], P.clo[i]) * inv_n;
    float hi, lo;
    split_tf32(e, hi, lo);
    sB[operand_word(r, i, ks)] = hi;
    sB[operand_word(r, kp + i, ks)] = lo;
  }
}

// One elected thread: D = A_hi B_hi + A_hi B_lo + A_lo B_hi into a TMEM
// accumulator, as 3 kp/8 MMAs of K = 8, then a commit to the mbarrier.
__device__ __forceinline__ void issue_mma(uint32_t d_tmem, const float* sA, const float* sB, int kp,
                                          uint64_t* bar) {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t lbo = 128, sbo = (uint32_t)(2 * kp >> 2) * 128;
  const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
  int step = 0;
  for (int j = 0; j < 3; ++j)
    for (int t = 0; t < kp / 8; ++t, ++step) {
      // blocks (A, B): (hi, hi), (hi, lo), (lo, hi)
      const uint32_t ka = (uint32_t)((j == 2 ? (kp >> 2) : 0) + 2 * t);
      const uint32_t kb = (uint32_t)((j == 1 ? (kp >> 2) : 0) + 2 * t);
      const uint64_t ad = operand_desc(a0 + ka * 128u, lbo, sbo);
      const uint64_t bd = operand_desc(b0 + kb * 128u, lbo, sbo);
      asm volatile(
          "{\n\t.reg .pred acc;\n\tsetp.ne.b32 acc, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, acc;\n\t}" ::"r"(d_tmem),
          "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(step)
          : "memory");
    }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// Requests a band's depth tile (64 rows x 128 columns) into shared memory.
template <typename TIn, bool VEC>
__device__ __forceinline__ void fetch_depth(TIn* sD, const TIn* dplane, int width, int gx0, int y0,
                                            int rows) {
  if (VEC) {
    constexpr int kPerCopy = 16 / (int)sizeof(TIn);
    constexpr int kCopiesPerRow = kTcCols / kPerCopy;
    for (int c = threadIdx.x; c < kTcRows * kCopiesPerRow; c += kTcThreads) {
      const int r = c / kCopiesPerRow, col = (c - r * kCopiesPerRow) * kPerCopy;
      if (r < rows && gx0 + col < width)
        cp_async<16>(sD + r * kTcCols + col, dplane + (size_t)(y0 + r) * width + gx0 + col);
    }
  } else {
    for (int c = threadIdx.x; c < kTcRows * kTcCols; c += kTcThreads) {
      const int r = c / kTcCols, col = c - r * kTcCols;
      if (r < rows && gx0 + col < width) sD[c] = dplane[(size_t)(y0 + r) * width + gx0 + col];
    }
  }
  cp_async_commit();
}

// A bounded wait that ran out: the frame's record is marked and the launch's
// fault word set, so the host reports MF_ERR_TIMEOUT instead of returning the
// NaN-filled bands silently.
__device__ __forceinline__ void report_wait_expired(const MapParams& p, const FrameRec* rec) {
  atomicExch(reinterpret_cast<int*>(const_cast<int32_t*>(&rec->status)), (int)MF_FRAME_TIMEOUT);
  if (p.fault) atomicExch_system(p.fault, kFaultWaitExpired);
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t phase) {
  uint32_t done = 0;
  for (long long it = 0; it < kTcWaitPolls && !done; ++it)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
  return done != 0;
}

// Software pipeline over the bands of a strip, two buffers deep: while the
// epilogue of band b reads TMEM accumulator b%2 and depth tile b%2, the
// depth copies and the MMAs of band b+1 run into the other buffers.
template <typename TIn, typename TOut, bool VEC>
__global__ void __launch_bounds__(kTcThreads, 2) map_tc_kernel(MapParams p, int strips, int ks_max) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  float* sA = reinterpret_cast<float*>(tc_smem);  // [128][ks_max]
  float* const sB0 = sA + (size_t)kTcCols * ks_max;
  float* const sB1 = sA + (size_t)(kTcCols + kTcRows) * ks_max;
  TIn* const sD0 = reinterpret_cast<TIn*>(sA + (size_t)(kTcCols + 2 * kTcRows) * ks_max);
  TIn* const sD1 = sD0 + kTcRows * kTcCols;
  __shared__ PointsSmem<kMaxPts> P;
  __shared__ __align__(8) uint64_t mma_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_kept;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    for (int k = 0; k < 2; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mma_bar[k])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(2 * kTcRows)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  uint32_t phase0 = 0u, phase1 = 0u;

  // epilogue role: TMEM lane quadrant q (32 columns), row half h (32 rows)
  const int q = warp & 3, h = warp >> 2;
  const size_t plane = (size_t)p.width * p.height;
  const int bands = (p.height + kTcRows - 1) / kTcRows;
  const int items = p.n_frames * strips;

  __shared__ long long s_next[2];
  long long next = blockIdx.x;
  for (int k = 0; next < items; ++k) {
    const int item = (int)next;
    const unsigned claim = claim_unit(p.sched);
    const int f = item / strips;
    const int gx0 = (item - f * strips) * kTcCols;
    const int gx1 = min(p.width, gx0 + kTcCols) - 1;
    const FrameRec* rec = p.recs + ((p.f0 + f) & p.rec_mask);
    const int n = rec->n_valid;
    const float inv_n = rec->inv_n;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // the previous item is done with every buffer
    if (warp == 0) {
      // points whose Gaussian can reach the strip (the CUDA-core kernel's
      // rule, over all rows of the frame); kept points keep their order
      bool keep = false;
      float uh = 0.f, ul = 0.f, vh = 0.f, vl = 0.f, ch = 0.f, cl = 0.f;
      if (lane < n) {
        uh = rec->ux_hi[lane];
        ul = rec->ux_lo[lane];
        vh = rec->vy_hi[lane];
        vl = rec->vy_lo[lane];
        ch = rec->c_hi[lane];
        cl = rec->c_lo[lane];
        const float xn = fminf(fmaxf(rintf(uh + ul), (float)gx0), (float)gx1);
        const float yn = fminf(fmaxf(rintf(vh + vl), 0.0f), (float)(p.height - 1));
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
    const int kp = (nk + 7) & ~7;

    const int x = gx0 + 32 * q + lane;
    const bool col_ok = x < p.width;
    float best = -1.0f;
    unsigned bidx = 0;
    const TIn* dplane = p.depth ? static_cast<const TIn*>(p.depth) + (size_t)f * plane : nullptr;
    char* mplane = p.M ? static_cast<char*>(p.M) + (size_t)f * plane * sizeof(TOut) : nullptr;
    char* gplane = p.G ? static_cast<char*>(p.G) + (size_t)f * plane * sizeof(TOut) : nullptr;
    const bool want_depth = dplane && gplane && nk > 0;

    if (nk > 0) {
      // prologue: band 0 into buffers 0
      build_cols(sA, P, nk, kp, gx0, p.width);
      if (want_depth) fetch_depth<TIn, VEC>(sD0, dplane, p.width, gx0, 0, min(kTcRows, p.height));
      build_rows(sB0, P, nk, kp, 0, min(kTcRows, p.height), inv_n);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) issue_mma(tmem, sA, sB0, kp, &mma_bar[0]);
    }

    for (int b = 0; b < bands; ++b) {
      const int cur = b & 1, nxt = cur ^ 1;
      const int y0 = b * kTcRows;
      const int rows = min(kTcRows, p.height - y0);
      bool ok = true;
      if (nk > 0) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // band b-1's epilogue is done with TMEM and depth buffers nxt
        const bool more = b + 1 < bands;
        if (more) {
          const int y1 = y0 + kTcRows, rows1 = min(kTcRows, p.height - y1);
          if (want_depth) fetch_depth<TIn, VEC>(nxt ? sD1 : sD0, dplane, p.width, gx0, y1, rows1);
          build_rows(nxt ? sB1 : sB0, P, nk, kp, y1, rows1, inv_n);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncthreads();  // B of band b+1 written
          if (tid == 0)
            issue_mma(tmem + (uint32_t)(nxt * kTcRows), sA, nxt ? sB1 : sB0, kp, &mma_bar[nxt]);
        }
        if (want_depth) {
          if (more)
            cp_async_wait<1>();
          else
            cp_async_wait<0>();
        }
        __syncthreads();  // every thread's part of depth tile b has landed
        ok = wait_bar(&mma_bar[cur], cur ? phase1 : phase0);
        if (!ok) report_wait_expired(p, rec);
        if (cur)
          phase1 ^= 1u;
        else
          phase0 ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      // epilogue: rows y0 + 32h + 16c + j of column x
      const TIn* dtile = cur ? sD1 : sD0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int r0 = 32 * h + 16 * c;
        float acc[16];
        if (nk > 0) {
          tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(cur * kTcRows + r0), acc);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] = 0.0f;
        }
        if (!col_ok || r0 >= rows) continue;
        float cmax = -1.0f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (r0 + j >= rows) break;
          const float m = ok ? acc[j] : __int_as_float(0x7fffffff);
          const size_t off = (size_t)(y0 + r0 + j) * p.width + x;
          if (mplane) Scalar<TOut>::store(mplane, off, m);
          if (gplane) {
            const float dv = want_depth ? to_float(dtile[(r0 + j) * kTcCols + 32 * q + lane]) : 0.0f;
            Scalar<TOut>::store(gplane, off, m * depth_weight(dv, rec->d0));
          }
          cmax = fmaxf(cmax, m);
        }
        if (cmax > best) {
          // first row of this chunk holding the new maximum
          int jb = 15;
#pragma unroll
          for (int j = 15; j >= 0; --j)
            if (r0 + j < rows && acc[j] == cmax) jb = j;
          best = cmax;
          bidx = (unsigned)((y0 + r0 + jb) * p.width + x);
        }
      }
    }
    unsigned long long key =
        best >= 0.0f ? ((unsigned long long)__float_as_uint(best) << 32) | (0xffffffffu - bidx) : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
      key = k2 > key ? k2 : key;
    }
    if (lane == 0 && n > 0 && key) atomicMax(const_cast<unsigned long long*>(&rec->argmax_key), key);
    next = next_unit(p.sched, claim, items, s_next, k);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * kTcRows)
                 : "memory");
}

namespace {

size_t tc_smem_bytes(int ks_max, size_t in_size) {
  return (size_t)(kTcCols + 2 * kTcRows) * ks_max * 4 + 2 * (size_t)kTcRows * kTcCols * in_size;
}

template <typename TIn, typename TOut, bool VEC>
cudaError_t launch_tc_typed(const MapParams& p, int kk_max, cudaStream_t st) {
  auto k = map_tc_kernel<TIn, TOut, VEC>;
  const size_t smem = tc_smem_bytes(kk_max, sizeof(TIn));
  // Shared-memory opt-in and carveout on this device (cached per device);
  // resident CTAs per SM from the kernel's own footprint -- shared memory
  // with the per-block reservation, registers -- at the full carveout it
  // asks for (the occupancy query does not assume that carveout), at most 4:
  // each CTA holds 128 TMEM columns, and four fill an SM's 512.
  const KernelFit f = host_kernel_fit(reinterpret_cast<const void*>(k), kTcThreads,
                                      tc_smem_bytes(kTcKsMax, sizeof(TIn)), smem, 100);
  int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, k);
  const size_t per_cta = smem + fa.sharedSizeBytes + (size_t)reserved;
  int fit = (int)((size_t)smem_sm / per_cta);
  if (fa.numRegs > 0) fit = std::min(fit, regs_sm / (fa.numRegs * kTcThreads));
  const int per_sm = std::max(1, std::min(fit, 4));
  const int sms = f.sms;
  const int strips = (p.width + kTcCols - 1) / kTcCols;
  const long long items = (long long)p.n_frames * strips;
  const long long grid = std::min<long long>(items, (long long)per_sm * sms);
  if (items > 0x7fffffffLL) return cudaErrorInvalidConfiguration;  // item indices are int
  k<<<(unsigned)grid, kTcThreads, smem, st>>>(p, strips, kk_max);
  return cudaGetLastError();
}

template <typename TIn, typename TOut>
cudaError_t launch_tc_vec(const MapParams& p, int kk_max, cudaStream_t st) {
  // 16-byte copies of depth rows need 16-byte aligned rows
  const bool vec = p.depth && ((uintptr_t)p.depth % 16) == 0 &&
                   ((size_t)p.width * sizeof(TIn)) % 16 == 0;
  return vec ? launch_tc_typed<TIn, TOut, true>(p, kk_max, st)
             : launch_tc_typed<TIn, TOut, false>(p, kk_max, st);
}

template <typename TIn>
cudaError_t launch_tc_out(const MapParams& p, int map_dtype, int kk_max, cudaStream_t st) {
  switch (map_dtype) {
    case MF_F32: return launch_tc_vec<TIn, float>(p, kk_max, st);
    case MF_BF16: return launch_tc_vec<TIn, __nv_bfloat16>(p, kk_max, st);
    case MF_F16: return launch_tc_vec<TIn, __half>(p, kk_max, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_map_tc(const MapParams& p, int window, int depth_dtype, int map_dtype,
                          cudaStream_t st, int64_t* launches) {
  if (p.n_frames <= 0) return cudaSuccess;
  if ((long long)p.n_frames * ((p.width + kTcCols - 1) / kTcCols) > 0x7fffffffLL)
    return cudaErrorInvalidConfiguration;
  const int kk_max = 2 * ((std::min(std::max(window, 1), kMaxPts) + 7) & ~7);  // stored K
  cudaError_t e;
  switch (depth_dtype) {
    case MF_F32: e = launch_tc_out<float>(p, map_dtype, kk_max, st); break;
    case MF_BF16: e = launch_tc_out<__nv_bfloat16>(p, map_dtype, kk_max, st); break;
    case MF_F16: e = launch_tc_out<__half>(p, map_dtype, kk_max, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) ++*launches;
  return e;
}

}  // namespace mf
