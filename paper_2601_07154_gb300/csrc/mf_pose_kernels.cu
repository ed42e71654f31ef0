// Pose-side kernels of one stream (FP64; bodies in mf_pose_device.cuh):
//   ingest_kernel    -- Section 2.2, one thread per emitted frame;
//   points_kernel    -- Section 2.3, Eqs. 1-6, one warp per frame;
//   finalize_kernel  -- per-frame result records (and motion points);
//   ring_copy_kernel -- carries the pose history over when it grows.
#include "mf_pose_device.cuh"

namespace mf {

__global__ void __launch_bounds__(128) ingest_kernel(IngestParams p) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p.n - p.first) return;
  ingest_frame(p.in, p.first, k, p.anchor, p.ring, p.ring_bad, p.ring_mask, p.e0,
               p.scale ? *p.scale : 1.0);
}

constexpr int kPtsWarps = 4;

__global__ void __launch_bounds__(kPtsWarps * 32) points_kernel(PointsParams p) {
  __shared__ PointsScratch S[kPtsWarps];
  const int wi = threadIdx.x >> 5;
  const int f = blockIdx.x * kPtsWarps + wi;
  if (f >= p.n_frames) return;  // warp-uniform
  const int64_t g = p.e0 + f;
  FrameParams fp;
  fp.window = p.window;
  fp.smooth_len = p.smooth_len;
  fp.width = p.width;
  fp.height = p.height;
  fp.calib_width = p.calib_width;
  fp.calib_height = p.calib_height;
  fp.sigma_rel = p.sigma_rel;
  fp.s_lo = p.s_lo;
  fp.s_hi = p.s_hi;
  // G's reference depth in the frame's depth scale: min(1, d0 / (s D)) =
  // min(1, (d0 / s) / D)
  fp.d0 = (float)(p.scale ? p.d0 / *p.scale : p.d0);
  fp.depth_scale = (float)(p.scale ? *p.scale : 1.0);
  frame_points(p.ring, p.ring_bad, p.ring_mask, g, fp, p.K, p.w, p.recs + (g & p.rec_mask), S[wi]);
}

__global__ void finalize_kernel(FinalizeParams p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (p.info && t < p.n_frames)
    finalize_frame(p.recs + ((p.f0 + t) & p.rec_mask), p.width, p.info + t, p.normalize);
  if (p.points) {
    const int total = p.n_frames * p.window;
    for (int e = t; e < total; e += gridDim.x * blockDim.x) {
      const int f = e / p.window, sl = e - f * p.window;
      motion_point(p.recs + ((p.f0 + f) & p.rec_mask), sl, p.points + e);
    }
  }
}

__global__ void ring_copy_kernel(const double* src, const int32_t* src_bad, int64_t src_mask,
                                 double* dst, int32_t* dst_bad, int64_t dst_mask, int64_t first,
                                 int count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const int64_t j = first + k;
  const double* s = src + (j & src_mask) * 12;
  double* t = dst + (j & dst_mask) * 12;
  for (int e = 0; e < 12; ++e) t[e] = s[e];
  dst_bad[j & dst_mask] = src_bad[j & src_mask];
}

// ------------------------------------------------------------ launchers --
cudaError_t launch_ingest(const IngestParams& p, cudaStream_t st, int64_t* launches) {
  const int n_emit = p.n - p.first;
  if (n_emit <= 0) return cudaSuccess;
  ingest_kernel<<<(n_emit + 127) / 128, 128, 0, st>>>(p);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_points(const PointsParams& p, cudaStream_t st, int64_t* launches) {
  if (p.n_frames <= 0) return cudaSuccess;
  points_kernel<<<(p.n_frames + kPtsWarps - 1) / kPtsWarps, kPtsWarps * 32, 0, st>>>(p);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeParams& p, cudaStream_t st, int64_t* launches) {
  if (p.n_frames <= 0 || (!p.info && !p.points)) return cudaSuccess;
  const int total = p.points ? p.n_frames * p.window : p.n_frames;
  int blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < (p.n_frames + 255) / 256) blocks = (p.n_frames + 255) / 256;
  finalize_kernel<<<blocks, 256, 0, st>>>(p);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_ring_copy(const double* src, const int32_t* src_bad, int64_t src_mask,
                             double* dst, int32_t* dst_bad, int64_t dst_mask, int64_t first,
                             int count, cudaStream_t st, int64_t* launches) {
  if (count <= 0) return cudaSuccess;
  ring_copy_kernel<<<(count + 127) / 128, 128, 0, st>>>(src, src_bad, src_mask, dst, dst_bad,
                                                         dst_mask, first, count);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace mf
