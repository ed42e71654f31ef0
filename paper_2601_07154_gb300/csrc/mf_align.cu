// Depth alignment across batches (Section 2.2, Fig. 3 "depth alignment"):
// the scale of a batch-local batch is the previous batch's scale times the
// lower median of the single-precision ratios D_prev / D_cur over the
// overlap frames' pixels where both depths are finite and > 0.
//
// The median is found by radix selection on the ratios' bit patterns
// (positive floats order like their bits): three histogram passes over the
// overlap planes (the top 11 bits, the next 11 bits of the ratios whose top
// bits match, the last 10 bits), each followed by a one-block kernel that
// finds the bin holding the wanted rank.  Everything stays on the device
// and in the stream's order; the counts use integer atomics only, so the
// result does not depend on the order in which pixels are counted.
#include <cfloat>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mf_internal.h"

namespace mf {
namespace {

constexpr int kAlignThreads = 256;
constexpr int kAlignPerThread = kAlignBins / kAlignThreads;  // bins scanned per thread
// state words after the three histograms
constexpr int kStN = 3 * kAlignBins;      // valid pairs
constexpr int kStRank = kStN + 1;         // wanted rank among the keys matching the prefix
constexpr int kStPrefix = kStN + 2;       // key bits selected so far
constexpr int kStEmpty = kStN + 3;        // 1: no valid pair (the scale stays)

__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_float(__half v) { return __half2float(v); }

// The ratio's bit pattern for pixel i, if both depths are finite and > 0.
template <typename T>
__device__ __forceinline__ bool ratio_key(const T* prev, const T* cur, int64_t i, unsigned* key) {
  const float a = to_float(prev[i]), b = to_float(cur[i]);
  if (!(a > 0.0f && a <= FLT_MAX && b > 0.0f && b <= FLT_MAX)) return false;  // NaN fails too
  *key = __float_as_uint(__fdiv_rn(a, b));  // IEEE single-precision quotient, >= 0
  return true;
}

// Histogram of one pass: pass 0 bins the top 11 bits of every key; pass 1
// the next 11 bits of the keys whose top 11 bits are the selected prefix;
// pass 2 the last 10 bits of the keys whose top 22 bits are.
template <typename T>
__global__ void __launch_bounds__(kAlignThreads) align_hist_kernel(const T* prev, const T* cur,
                                                                   int64_t count, unsigned* work,
                                                                   int pass) {
  __shared__ unsigned h[kAlignBins];
  for (int i = threadIdx.x; i < kAlignBins; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const bool skip = pass > 0 && work[kStEmpty] != 0u;
  const unsigned prefix = pass > 0 ? work[kStPrefix] : 0u;
  if (!skip) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
      unsigned key;
      if (!ratio_key(prev, cur, i, &key)) continue;
      unsigned bin;
      if (pass == 0) {
        bin = key >> 21;
      } else if (pass == 1) {
        if ((key >> 21) != prefix) continue;
        bin = (key >> 10) & 0x7ffu;
      } else {
        if ((key >> 10) != prefix) continue;
        bin = key & 0x3ffu;
      }
      atomicAdd(&h[bin], 1u);
    }
  }
  __syncthreads();
  unsigned* g = work + pass * kAlignBins;
  for (int i = threadIdx.x; i < kAlignBins; i += blockDim.x)
    if (h[i]) atomicAdd(&g[i], h[i]);
}

// One block: the bin of the pass's histogram that holds the wanted rank
// (pass 0 first counts the valid pairs n and sets the rank to (n-1)/2, the
// lower median); the prefix grows by that bin, and after the last pass the
// batch scale is multiplied by the selected ratio.
__global__ void __launch_bounds__(kAlignThreads) align_select_kernel(unsigned* work, int pass,
                                                                     double* scale) {
  __shared__ unsigned part[kAlignThreads];
  const unsigned* g = work + pass * kAlignBins;
  const int t = threadIdx.x;
  unsigned sum = 0u;
  for (int j = 0; j < kAlignPerThread; ++j) sum += g[t * kAlignPerThread + j];
  part[t] = sum;
  __syncthreads();
  if (t != 0) return;
  if (pass == 0) {
    unsigned n = 0u;
    for (int i = 0; i < kAlignThreads; ++i) n += part[i];
    work[kStN] = n;
    work[kStEmpty] = n == 0u ? 1u : 0u;
    work[kStRank] = n ? (n - 1u) / 2u : 0u;
  }
  if (work[kStEmpty]) return;
  const unsigned k = work[kStRank];
  unsigned acc = 0u;
  int tb = 0;
  while (tb < kAlignThreads - 1 && acc + part[tb] <= k) acc += part[tb++];
  int bin = tb * kAlignPerThread;
  for (int j = 0; j < kAlignPerThread; ++j) {
    const unsigned c = g[tb * kAlignPerThread + j];
    bin = tb * kAlignPerThread + j;
    if (acc + c > k) break;
    acc += c;
  }
  work[kStRank] = k - acc;
  const unsigned pre = pass == 0 ? (unsigned)bin
                                 : (work[kStPrefix] << (pass == 1 ? 11 : 10)) | (unsigned)bin;
  work[kStPrefix] = pre;
  if (pass == 2) *scale *= (double)__uint_as_float(pre);
}

template <typename T>
cudaError_t launch_typed(const AlignParams& p, cudaStream_t st, int64_t* launches) {
  const int64_t want = (p.count + kAlignThreads - 1) / kAlignThreads;
  const int blocks = (int)(want < 8 * 152 ? want : 8 * 152);
  for (int pass = 0; pass < 3; ++pass) {
    align_hist_kernel<T><<<blocks, kAlignThreads, 0, st>>>(static_cast<const T*>(p.prev),
                                                          static_cast<const T*>(p.cur), p.count,
                                                          p.work, pass);
    align_select_kernel<<<1, kAlignThreads, 0, st>>>(p.work, pass, p.scale);
  }
  *launches += 6;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_depth_align(const AlignParams& p, int depth_dtype, cudaStream_t st, int64_t* launches) {
  if (p.count <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(p.work, 0, kAlignWorkWords * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  switch (depth_dtype) {
    case MF_F32: return launch_typed<float>(p, st, launches);
    case MF_BF16: return launch_typed<__nv_bfloat16>(p, st, launches);
    case MF_F16: return launch_typed<__half>(p, st, launches);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mf
