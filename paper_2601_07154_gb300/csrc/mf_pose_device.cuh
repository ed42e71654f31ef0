// Per-frame pose-side device code shared by the per-stream kernels
// (mf_pose_kernels.cu) and the batched engine kernels (mf_engine_kernels.cu),
// FP64 throughout:
//   ingest_frame   -- Section 2.2: rigidity check, gravity-locked incremental
//                     anchoring of a batch-local pose, append to the history;
//   frame_points   -- Section 2.3, Eqs. 1-6: one warp builds a frame's N
//                     motion points and its focus;
//   finalize_frame -- per-frame result record.
// FP64 stays here because the pose differences are ill-conditioned near zero
// translation; these run a few thousand operations per frame, so GB300's low
// FP64 rate never matters.
#pragma once

#include <math.h>

#include "mf_internal.h"

namespace mf {

__device__ __forceinline__ bool pose_is_rigid(const double* P) {
  for (int k = 0; k < 12; ++k)
    if (!isfinite(P[k])) return false;
  double err = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const double dot = P[4 * a + 0] * P[4 * b + 0] + P[4 * a + 1] * P[4 * b + 1] +
                         P[4 * a + 2] * P[4 * b + 2];
      err = fmax(err, fabs(dot - (a == b ? 1.0 : 0.0)));
    }
  return err <= kRigidTol;
}

// Camera centre of a world-to-camera pose [R | t]: c = -R^T t (Eq. 1 for a
// rigid transform).
__device__ __forceinline__ void pose_centre(const double* P, double c[3]) {
  for (int j = 0; j < 3; ++j)
    c[j] = -(P[0 * 4 + j] * P[3] + P[1 * 4 + j] * P[7] + P[2 * 4 + j] * P[11]);
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Splits a pixel coordinate u into float hi + lo with hi a multiple of 2^-8
// when |u| < 2^15, so that (integer pixel) - hi is exact in FP32.
__device__ __forceinline__ void split_coord(double u, float& hi, float& lo) {
  const double h = fabs(u) < 32768.0 ? rint(u * 256.0) * (1.0 / 256.0) : u;
  hi = (float)h;
  lo = (float)(u - (double)hi);
}

// Section 2.2 for push frame `first + k`: world pose into ring slot e0 + k.
// With `anchor`, the push is batch-local and its frame first-1 is the same
// camera as the history's last frame e0-1 (the transition frame): the
// local-to-world transform H = T_a^{-1} L_a is reduced to the rotation about
// the world y (gravity) axis closest to it, psi = atan2(R02 - R20, R00 + R22)
// (pitch and roll are not propagated), with the translation that puts the
// anchor's camera centre on its world position; T = L H^{-1}.
//
// scale: the batch's depth scale (depth alignment), multiplying every
// translation of the batch before anchoring (1: the poses as given).
__device__ __forceinline__ void ingest_frame(const double* in, int first, int k, int anchor,
                                             double* ring, int32_t* ring_bad, int64_t ring_mask,
                                             int64_t e0, double scale = 1.0) {
  double L[12], La[12];
  for (int e = 0; e < 12; ++e) L[e] = in[(size_t)(first + k) * 12 + e];
  for (int r = 0; r < 3; ++r) L[4 * r + 3] *= scale;
  double out[12];
  for (int e = 0; e < 12; ++e) out[e] = L[e];
  bool bad = !pose_is_rigid(L);
  if (anchor) {
    const int64_t aslot = (e0 - 1) & ring_mask;
    const double* Ta = ring + aslot * 12;
    for (int e = 0; e < 12; ++e) La[e] = in[(size_t)(first - 1) * 12 + e];
    for (int r = 0; r < 3; ++r) La[4 * r + 3] *= scale;
    if (ring_bad[aslot] || !pose_is_rigid(La)) {
      bad = true;
    } else {
      double rh[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
          rh[r][c] = Ta[0 * 4 + r] * La[0 * 4 + c] + Ta[1 * 4 + r] * La[1 * 4 + c] +
                     Ta[2 * 4 + r] * La[2 * 4 + c];
      const double ca = rh[0][0] + rh[2][2], sa = rh[0][2] - rh[2][0];
      const double rr = hypot(ca, sa);
      const double cs = rr > 0.0 ? ca / rr : 1.0;
      const double sn = rr > 0.0 ? sa / rr : 0.0;
      double cw[3], cl[3];
      pose_centre(Ta, cw);
      pose_centre(La, cl);
      const double tH[3] = {cw[0] - (cs * cl[0] + sn * cl[2]), cw[1] - cl[1],
                            cw[2] - (-sn * cl[0] + cs * cl[2])};
      for (int r = 0; r < 3; ++r) {
        const double l0 = L[4 * r + 0], l1 = L[4 * r + 1], l2 = L[4 * r + 2];
        const double r0 = l0 * cs + l2 * sn;
        const double r2 = -l0 * sn + l2 * cs;
        out[4 * r + 0] = r0;
        out[4 * r + 1] = l1;
        out[4 * r + 2] = r2;
        out[4 * r + 3] = L[4 * r + 3] - (r0 * tH[0] + l1 * tH[1] + r2 * tH[2]);
      }
    }
  }
  const int64_t slot = (e0 + k) & ring_mask;
  double* dst = ring + slot * 12;
  for (int e = 0; e < 12; ++e) dst[e] = out[e];
  ring_bad[slot] = bad ? 1 : 0;
}

// Per-warp scratch of frame_points (shared memory).
struct PointsScratch {
  double q[kMaxHist][3];
  int bad[kMaxHist];
  double Rg[9];
  double pg[3];
};

// Inputs of frame_points that describe the stream.
struct FrameParams {
  int window, smooth_len;
  int width, height, calib_width, calib_height;
  double sigma_rel, s_lo, s_hi;
  float d0;                // reference depth of G in the frame's depth scale
  float depth_scale;       // the batch's depth alignment scale (reported only)
};

// Eqs. 1-6 for emitted frame g of a stream, by one warp (all 32 lanes).
__device__ __forceinline__ void frame_points(const double* ring, const int32_t* ring_bad,
                                             int64_t ring_mask, int64_t g, const FrameParams& fp,
                                             const double* K, const double* w, FrameRec* rec,
                                             PointsScratch& S) {
  const int lane = threadIdx.x & 31;
  const int W = fp.window, Ks = fp.smooth_len, R = W + Ks - 1;
  const int64_t j0 = g - (R - 1);

  // Eq. 1: camera centres of the window's poses (two ring slots per lane).
  double pc[2][3];
  bool have[2];
  for (int h = 0; h < 2; ++h) {
    const int r = lane + 32 * h;
    const int64_t j = j0 + r;
    have[h] = false;
    if (r < R) {
      if (j >= 0) {
        const int64_t slot = j & ring_mask;
        const double* P = ring + slot * 12;
        pose_centre(P, pc[h]);
        have[h] = ring_bad[slot] == 0;
        if (r == R - 1) {
          for (int a = 0; a < 3; ++a) {
            S.pg[a] = pc[h][a];
            for (int b = 0; b < 3; ++b) S.Rg[3 * a + b] = P[4 * a + b];
          }
        }
      }
      S.bad[r] = have[h] ? 0 : 1;
    }
  }
  __syncwarp();
  double pg[3], Rg[9];
  for (int a = 0; a < 3; ++a) pg[a] = S.pg[a];
  for (int a = 0; a < 9; ++a) Rg[a] = S.Rg[a];
  const bool frame_bad = S.bad[R - 1] != 0;

  // Eq. 4 applied to relative positions: q_j = R_n (p_j - p_n).
  double rho = 0.0, pmax = 0.0;
  for (int h = 0; h < 2; ++h) {
    if (!have[h]) continue;
    const int r = lane + 32 * h;
    const double dx = pc[h][0] - pg[0], dy = pc[h][1] - pg[1], dz = pc[h][2] - pg[2];
    for (int a = 0; a < 3; ++a)
      S.q[r][a] = Rg[3 * a + 0] * dx + Rg[3 * a + 1] * dy + Rg[3 * a + 2] * dz;
    rho = fmax(rho, sqrt(dx * dx + dy * dy + dz * dz));
    pmax = fmax(pmax, sqrt(pc[h][0] * pc[h][0] + pc[h][1] * pc[h][1] + pc[h][2] * pc[h][2]));
  }
  rho = warp_max(rho);
  pmax = warp_max(pmax);
  __syncwarp();
  const bool moving = !frame_bad && rho > 0.0 && rho > kStaticRel * pmax;

  // Eqs. 2-3: motion vector of point i = g - W + 1 + lane by the K-sample
  // least-squares weights over ring entries lane .. lane + K - 1.
  bool valid = false;
  double d[3] = {0.0, 0.0, 0.0}, nd = 0.0;
  if (lane < W && moving) {
    const int ri = lane + Ks - 1;
    bool ok = true;
    for (int r = lane; r <= ri; ++r) ok = ok && S.bad[r] == 0;
    if (ok) {
      for (int k = 0; k < Ks; ++k) {
        const double wk = w[k];
        d[0] = fma(wk, S.q[ri - k][0], d[0]);
        d[1] = fma(wk, S.q[ri - k][1], d[1]);
        d[2] = fma(wk, S.q[ri - k][2], d[2]);
      }
      nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      valid = nd > kValidRelNorm * rho && fabs(d[2]) > kValidRelZ * nd;
    }
  }
  const unsigned mask = __ballot_sync(0xffffffffu, valid);
  const int nv = __popc(mask);
  const double sum = warp_sum(valid ? nd : 0.0);

  // Intrinsics compensation: K at the calibration resolution -> map pixels.
  double fx = K[0], fy = K[1], cx = K[2], cy = K[3];
  const int wc = fp.calib_width ? fp.calib_width : fp.width;
  const int hc = fp.calib_height ? fp.calib_height : fp.height;
  if (wc != fp.width) {
    const double sx = (double)fp.width / (double)wc;
    fx = fx * sx;
    cx = (cx + 0.5) * sx - 0.5;
  }
  if (hc != fp.height) {
    const double sy = (double)fp.height / (double)hc;
    fy = fy * sy;
    cy = (cy + 0.5) * sy - 0.5;
  }

  // Eq. 6 projection, magnitude s_i and spread sigma_i (Eq. 7).
  double u = 0.0, v = 0.0, sig = 0.0, sc = 0.0;
  if (valid) {
    const double mean = sum / nv;
    sc = fmin(fmax(nd / mean, fp.s_lo), fp.s_hi);
    sig = fp.sigma_rel * fx * sc;
    u = cx + fx * d[0] / d[2];
    v = cy + fy * d[1] / d[2];
  }
  rec->u[lane] = u;
  rec->v[lane] = v;
  rec->sigma[lane] = sig;
  rec->s[lane] = sc;
  rec->valid[lane] = valid ? 1 : 0;
  if (valid) {
    const int pos = __popc(mask & ((1u << lane) - 1u));
    float hi, lo;
    split_coord(u, hi, lo);
    rec->ux_hi[pos] = hi;
    rec->ux_lo[pos] = lo;
    split_coord(v, hi, lo);
    rec->vy_hi[pos] = hi;
    rec->vy_lo[pos] = lo;
    // log2(e) / (2 sigma^2): the map kernels evaluate the Gaussian as a
    // power of 2
    double c = 1.4426950408889634 / (2.0 * sig * sig);
    c = fmin(c, 1e30);
    const float chi = (float)c;
    rec->c_hi[pos] = chi;
    rec->c_lo[pos] = (float)(c - (double)chi);
  }
  if (lane == W - 1) {
    int px = -1, py = -1;
    if (valid) {
      const double xr = rint(u), yr = rint(v);
      if (xr >= 0.0 && xr < (double)fp.width && yr >= 0.0 && yr < (double)fp.height) {
        px = (int)xr;
        py = (int)yr;
      }
    }
    rec->focus_valid = valid ? 1 : 0;
    rec->focus_u = u;
    rec->focus_v = v;
    rec->focus_px_x = px;
    rec->focus_px_y = py;
  }
  if (lane == 0) {
    rec->n_valid = nv;
    rec->inv_n = nv ? (float)(1.0 / nv) : 0.0f;
    rec->valid_mask = mask;
    rec->status = frame_bad ? MF_FRAME_BAD_POSE : (nv ? MF_FRAME_OK : MF_FRAME_EMPTY);
    rec->frame_index = g;
    rec->argmax_key = 0ull;
    rec->d0 = fp.d0;
    rec->depth_scale = fp.depth_scale;
  }
}

// Divisor of a frame's maps under MF_NORM_MAX: the map maximum found by the
// fused argmax when it is at least kNormFloor, else 1 (a frame whose motion
// points all lie far outside the image keeps its near-zero count-normalised
// maps).  Dividing, rather than multiplying by a reciprocal, maps the
// maximum to exactly 1.
__device__ __forceinline__ float norm_divisor(const FrameRec* rec) {
  const unsigned long long key = rec->argmax_key;
  if (rec->n_valid <= 0 || key == 0ull) return 1.0f;
  const float mx = __uint_as_float((unsigned)(key >> 32));
  return mx >= kNormFloor ? mx : 1.0f;
}

__device__ __forceinline__ void finalize_frame(const FrameRec* rec, int width, mf_frame_info* out,
                                               int normalize = MF_NORM_COUNT) {
  mf_frame_info o;
  o.frame_index = rec->frame_index;
  o.status = rec->status;
  o.n_valid = rec->n_valid;
  o.valid_mask = rec->valid_mask;
  o.focus_valid = rec->focus_valid;
  o.focus_u = rec->focus_u;
  o.focus_v = rec->focus_v;
  o.focus_px_x = rec->focus_px_x;
  o.focus_px_y = rec->focus_px_y;
  const unsigned long long key = rec->argmax_key;
  if (rec->n_valid > 0 && key != 0ull) {
    const unsigned idx = 0xffffffffu - (unsigned)(key & 0xffffffffull);
    o.argmax_x = (int)(idx % (unsigned)width);
    o.argmax_y = (int)(idx / (unsigned)width);
    o.map_max = __uint_as_float((unsigned)(key >> 32));
    if (normalize == MF_NORM_MAX && o.map_max >= kNormFloor) o.map_max = 1.0f;
  } else {
    o.argmax_x = -1;
    o.argmax_y = -1;
    o.map_max = 0.0f;
  }
  o.depth_scale = rec->depth_scale;
  *out = o;
}

__device__ __forceinline__ void motion_point(const FrameRec* rec, int slot, mf_motion_point* out) {
  mf_motion_point q;
  q.u = rec->u[slot];
  q.v = rec->v[slot];
  q.sigma = rec->sigma[slot];
  q.s = rec->s[slot];
  q.valid = rec->valid[slot];
  q.reserved = 0;
  *out = q;
}

}  // namespace mf
