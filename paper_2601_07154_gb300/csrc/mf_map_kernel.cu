// Motion-focus map launches (Eq. 7 and the motion-guided depth): the
// dispatch by window bucket and storage types, the in-place MF_NORM_MAX pass
// of the tiled fallback and the tensor-core kernel.  The per-pixel kernels
// and their launchers are templates in mf_map_kernel.cuh, instantiated one
// window bucket per translation unit (mf_map_n8.cu, mf_map_n16.cu,
// mf_map_n32.cu).
#include "mf_map_kernel.cuh"

namespace mf {

namespace mapk {
extern template cudaError_t launch_n<8>(const MapParams&, int, int, bool, cudaStream_t, int64_t*);
extern template cudaError_t launch_n<16>(const MapParams&, int, int, bool, cudaStream_t, int64_t*);
extern template cudaError_t launch_n<32>(const MapParams&, int, int, bool, cudaStream_t, int64_t*);
}  // namespace mapk

template <typename TOut, bool VEC>
__global__ void __launch_bounds__(256) normalize_kernel(NormalizeParams p) {
  const int f = blockIdx.y;
  const float z = norm_divisor(p.recs + ((p.f0 + f) & p.rec_mask));
  const size_t base = (size_t)f * p.plane;
  const size_t step = (size_t)gridDim.x * blockDim.x;
  if (VEC) {
    const size_t quads = p.plane / 4;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < quads; q += step) {
      const size_t i = base + 4 * q;
      float v[4];
      for (int c = 0; c < 2; ++c) {
        void* plane = c == 0 ? p.M : p.G;
        if (!plane) continue;
        const float4 x = Px<TOut>::load4(plane, i);
        v[0] = x.x / z;
        v[1] = x.y / z;
        v[2] = x.z / z;
        v[3] = x.w / z;
        Px<TOut>::store4(plane, i, make_float4(v[0], v[1], v[2], v[3]));
      }
    }
  } else {
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < (size_t)p.plane; j += step) {
      if (p.M) Px<TOut>::store1(p.M, base + j, Px<TOut>::load1(p.M, base + j) / z);
      if (p.G) Px<TOut>::store1(p.G, base + j, Px<TOut>::load1(p.G, base + j) / z);
    }
  }
}

namespace {
template <typename TOut>
cudaError_t launch_normalize_typed(const NormalizeParams& p, cudaStream_t st) {
  auto aligned = [](const void* q) { return q == nullptr || ((uintptr_t)q % (4 * sizeof(TOut))) == 0; };
  const bool vec = (p.plane % 4) == 0 && aligned(p.M) && aligned(p.G);
  const long long per = std::max<long long>(1, std::min<long long>(64, (p.plane / 4 + 255) / 256));
  const dim3 grid((unsigned)per, (unsigned)p.n_frames);
  if (vec)
    normalize_kernel<TOut, true><<<grid, 256, 0, st>>>(p);
  else
    normalize_kernel<TOut, false><<<grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_normalize(const NormalizeParams& p, int map_dtype, cudaStream_t st,
                             int64_t* launches) {
  if (p.n_frames <= 0 || (!p.M && !p.G)) return cudaSuccess;
  if (p.n_frames > 65535) return cudaErrorInvalidConfiguration;
  cudaError_t e;
  switch (map_dtype) {
    case MF_F32: e = launch_normalize_typed<float>(p, st); break;
    case MF_BF16: e = launch_normalize_typed<__nv_bfloat16>(p, st); break;
    case MF_F16: e = launch_normalize_typed<__half>(p, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) ++*launches;
  return e;
}

int map_tile_h(int width, int height, int window) {
  (void)width;
  (void)window;
  return height < 64 ? ((height + 7) / 8) * 8 : 64;
}

namespace mapk {

NormalizeParams normalize_params(const MapParams& p) {
  NormalizeParams np{};
  np.recs = p.recs;
  np.rec_mask = p.rec_mask;
  np.f0 = p.f0;
  np.n_frames = p.n_frames;
  np.plane = (int64_t)p.width * p.height;
  np.M = p.M;
  np.G = p.G;
  return np;
}
}  // namespace mapk


// The map is HBM-bound work (about N FMAs per 12 bytes), so the CUDA-core
// kernel is the default.  The tensor-core kernel runs only when forced: as
// a fraction of measured HBM bandwidth (algorithmic bytes, 1080p x 304
// frames, windows 8 / 16 / 32), CUDA vs tensor cores:
//   ACCEL   FP32   1.37 / 1.26 / 1.14  vs  1.25 / 1.16 / 0.69
//   ACCEL   16-bit 1.32 / 1.23 / 0.89  vs  0.65 / 0.60 / 0.54
//   HEADING FP32   1.03 / 1.02 / 0.89  vs  0.99 / 0.92 / 0.48
//   HEADING 16-bit 0.97 / 0.79 / 0.52  vs  0.51 / 0.45 / 0.39
bool map_uses_tensor_cores(int path) { return path == kMapTensorCores; }

cudaError_t launch_map(const MapParams& p, int window, int in_dtype, int out_dtype, int normalize,
                       cudaStream_t st, int64_t* launches) {
  if (p.n_frames <= 0) return cudaSuccess;
  const bool mx = normalize == MF_NORM_MAX;
  if (map_uses_tensor_cores(p.path)) {
    cudaError_t e = launch_map_tc(p, window, in_dtype, out_dtype, st, launches);
    if (e == cudaSuccess && mx) e = launch_normalize(mapk::normalize_params(p), out_dtype, st, launches);
    return e;
  }
  if (window <= 8) return mapk::launch_n<8>(p, in_dtype, out_dtype, mx, st, launches);
  if (window <= 16) return mapk::launch_n<16>(p, in_dtype, out_dtype, mx, st, launches);
  return mapk::launch_n<32>(p, in_dtype, out_dtype, mx, st, launches);
}

}  // namespace mf
