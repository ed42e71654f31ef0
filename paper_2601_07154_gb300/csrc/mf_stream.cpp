// Host engine behind the C ABI of include/mf.h: stream state, staging of
// host inputs and outputs, frame accounting of the sliding-batch ingestion
// (Section 2.2), and the launches of the pose and map kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mf_internal.h"

using mf::FrameRec;

namespace {

std::atomic<int64_t> g_launches{0};
thread_local std::string g_last_error;

int fail(int status, const char* what, cudaError_t e = cudaSuccess) {
  g_last_error = what;
  if (e != cudaSuccess) {
    g_last_error += ": ";
    g_last_error += cudaGetErrorString(e);
  }
  return status;
}

#define MF_CUDA(call, what)                                       \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return fail(MF_ERR_CUDA, what, e_);    \
  } while (0)

size_t dtype_size(int dt) { return dt == MF_F32 ? 4 : 2; }

// The first batch's depth scale (static storage: read by asynchronous copies).
const double kUnitScale = 1.0;

int map_path(uint32_t flags) {
  if (flags & MF_FLAG_MAP_TENSOR_CORES) return mf::kMapTensorCores;
  if (flags & MF_FLAG_MAP_CUDA_CORES) return mf::kMapCudaCores;
  return mf::kMapAuto;
}

int64_t pow2_at_least(int64_t v) {
  int64_t c = 1;
  while (c < v) c <<= 1;
  return c;
}

// Device that was current on entry, restored on exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int pointer_kind(const void* p, int dev) {
  if (!p) return mf::kPtrHost;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return mf::kPtrHost;
  }
  return mf::classify_pointer((int)a.type, a.device, dev);
}

// Exact least-squares derivative weights (Eqs. 2-3 generalised): the K
// newest samples sit at tau_k = -k; the fit p(tau) = c0 + c1 tau + c2 tau^2
// (a line when K = 2) gives d = 2 c2 (ACCEL) or c1 (HEADING) as
// sum_k w_k q_{i-k}.  Solved by Cramer's rule in 128-bit integers, so each
// weight is a reduced fraction and its double is correctly rounded.
using i128 = __int128;

i128 iabs128(i128 v) { return v < 0 ? -v : v; }
i128 gcd128(i128 a, i128 b) {
  a = iabs128(a);
  b = iabs128(b);
  while (b) {
    i128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

bool ls_weights(int K, int mode, double* w) {
  const int deg = K >= 3 ? 2 : 1;
  if (mode == MF_MODE_ACCEL && K < 3) return false;
  if (K < 2) return false;
  const int m = deg + 1;
  i128 S[5] = {0, 0, 0, 0, 0};  // S[e] = sum_k tau_k^e
  for (int k = 0; k < K; ++k) {
    i128 t = -k, pw = 1;
    for (int e = 0; e < 5; ++e) {
      S[e] += pw;
      pw *= t;
    }
  }
  i128 N[3][3];
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) N[a][b] = S[a + b];
  // adjugate row of the wanted coefficient, and the determinant
  const int want = mode == MF_MODE_ACCEL ? 2 : 1;
  const i128 factor = mode == MF_MODE_ACCEL ? 2 : 1;
  i128 adj[3] = {0, 0, 0}, det;
  if (m == 2) {
    det = N[0][0] * N[1][1] - N[0][1] * N[1][0];
    // inverse row `want`=1 of a 2x2: [-N10, N00] / det
    adj[0] = -N[1][0];
    adj[1] = N[0][0];
  } else {
    auto minor = [&](int r, int c) {
      int r0 = r == 0 ? 1 : 0, r1 = r == 2 ? 1 : 2;
      int c0 = c == 0 ? 1 : 0, c1 = c == 2 ? 1 : 2;
      return N[r0][c0] * N[r1][c1] - N[r0][c1] * N[r1][c0];
    };
    det = N[0][0] * minor(0, 0) - N[0][1] * minor(0, 1) + N[0][2] * minor(0, 2);
    // (N^{-1})[want][b] = cofactor(b, want) / det
    for (int b = 0; b < 3; ++b) adj[b] = (((b + want) & 1) ? -1 : 1) * minor(b, want);
  }
  for (int k = 0; k < K; ++k) {
    i128 t = -k, pw = 1, num = 0;
    for (int b = 0; b < m; ++b) {
      num += adj[b] * pw;
      pw *= t;
    }
    num *= factor;
    i128 den = det;
    if (den < 0) {
      den = -den;
      num = -num;
    }
    const i128 g = gcd128(num, den);
    if (g > 1) {
      num /= g;
      den /= g;
    }
    if (iabs128(num) >= ((i128)1 << 53) || den >= ((i128)1 << 53)) return false;
    w[k] = (double)(long long)num / (double)(long long)den;
  }
  return true;
}

struct Run {
  int64_t first;       // global index of the run's first frame
  int count;
  const char* depth;   // plane of frame `first`, or NULL
  int stage_slots;     // staging slots this run holds (0: caller memory)
  cudaEvent_t ready;   // upload of a staged run on the copy-in stream, or NULL
};

// Host-memory transfers are split into pieces of about this many bytes of
// traffic (depth in + both maps out) so that uploads, map launches and
// downloads of different pieces overlap.  Upload and download pieces hold
// the same number of frames, so each map launch covers one upload.
constexpr size_t kPieceBytes = 128u << 20;
constexpr int kMaxPieceFrames = 64;
constexpr int kOutSlots = 3;  // output staging pieces in flight

int piece_frames(size_t frame_bytes) {
  const size_t f = frame_bytes ? kPieceBytes / frame_bytes : kMaxPieceFrames;
  return (int)std::max<size_t>(1, std::min<size_t>(f, kMaxPieceFrames));
}

struct TimerPair {
  cudaEvent_t a, b;
};

// Adds the launches an entry point made to the process-wide counter.
struct LaunchTally {
  const int64_t* counter;
  int64_t start;
  explicit LaunchTally(const int64_t* c) : counter(c), start(*c) {}
  ~LaunchTally() { g_launches.fetch_add(*counter - start); }
};

}  // namespace

struct mf_stream {
  mf_stream_desc d{};
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  double w[mf::kMaxHist] = {};
  size_t plane_in = 0, plane_out = 0;  // bytes per depth plane / map plane
  int piece = 1;                       // frames per host-memory transfer piece

  double* ring = nullptr;
  int32_t* ring_bad = nullptr;
  int64_t ring_cap = 0;
  FrameRec* recs = nullptr;
  int64_t rec_cap = 0;
  unsigned int* sched = nullptr;  // map kernels' work counter
  // Fault word in mapped page-locked host memory: a map kernel whose bounded
  // device wait runs out sets it; the next completed wait reports it.
  unsigned int* fault_host = nullptr;
  unsigned int* fault_dev = nullptr;

  // Depth alignment across batches (MF_FLAG_DEPTH_ALIGN): the batch scale
  // (device double), the selection's work words, the previous batch's last
  // `overlap` depth planes and, for host depth, an upload of this batch's
  // first ones.
  bool align = false;
  double* scale_dev = nullptr;
  unsigned int* align_work = nullptr;
  char* ovl_prev = nullptr;
  char* ovl_cur = nullptr;
  bool ovl_valid = false;

  double* pose_dev = nullptr;      // device staging of host poses
  int64_t pose_dev_cap = 0;
  double* pose_host = nullptr;     // pinned bounce buffer for host poses
  int64_t pose_host_cap = 0;
  cudaEvent_t pose_ev = nullptr;   // last upload from pose_host

  char* stage = nullptr;           // device staging ring of depth planes
  int64_t stage_slots = 0, stage_head = 0, stage_used = 0;
  char* out_stage = nullptr;       // device staging of outputs bound for host
  size_t out_stage_bytes = 0;
  cudaEvent_t done_ev = nullptr;

  // Copy engines for host memory: uploads run on st_in and downloads on
  // st_out, so that both directions and the kernels on st overlap.
  cudaStream_t st_in = nullptr, st_out = nullptr;
  std::vector<cudaEvent_t> free_events;
  cudaEvent_t slot_ev[kOutSlots] = {};  // download of each output slot's piece
  bool slot_busy[kOutSlots] = {};

  int64_t emitted = 0, rendered = 0, pushes = 0, pushed_frames = 0;
  std::deque<Run> runs;
  int64_t launches = 0;
  std::vector<TimerPair> timers, free_timers;
  double map_ms = 0.0;
  int64_t map_timed = 0;
  int64_t device_bytes = 0;
  uint32_t last_map_kernel = 0;

  void* dalloc(size_t bytes) {
    void* p = nullptr;
    if (mf::fault_fires(mf::kFaultAllocFail)) return nullptr;
    if (d.dev_alloc) {
      p = d.dev_alloc(bytes, d.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) device_bytes += (int64_t)bytes;
    return p;
  }
  void dfree(void* p, size_t bytes) {
    if (!p) return;
    if (d.dev_free)
      d.dev_free(p, d.alloc_ctx);
    else
      cudaFree(p);
    device_bytes -= (int64_t)bytes;
  }
};

namespace {

int grow_ring(mf_stream* s, int64_t need) {
  if (need <= s->ring_cap) return MF_OK;
  const int64_t cap = pow2_at_least(std::max<int64_t>(need, 128));
  double* ring = (double*)s->dalloc((size_t)cap * 12 * sizeof(double));
  int32_t* bad = (int32_t*)s->dalloc((size_t)cap * sizeof(int32_t));
  if (!ring || !bad) {
    s->dfree(ring, (size_t)cap * 12 * sizeof(double));
    s->dfree(bad, (size_t)cap * sizeof(int32_t));
    return fail(MF_ERR_OOM, "pose history allocation failed");
  }
  if (s->ring && s->emitted > 0) {
    const int64_t keep = std::min<int64_t>(s->emitted, s->d.window + s->d.smooth_len - 1);
    MF_CUDA(mf::launch_ring_copy(s->ring, s->ring_bad, s->ring_cap - 1, ring, bad, cap - 1,
                                 s->emitted - keep, (int)keep, s->st, &s->launches),
            "history copy launch");
  }
  if (s->ring) {
    MF_CUDA(cudaStreamSynchronize(s->st), "stream sync before freeing history");
    s->dfree(s->ring, (size_t)s->ring_cap * 12 * sizeof(double));
    s->dfree(s->ring_bad, (size_t)s->ring_cap * sizeof(int32_t));
  }
  s->ring = ring;
  s->ring_bad = bad;
  s->ring_cap = cap;
  return MF_OK;
}

int take_event(mf_stream* s, cudaEvent_t* ev) {
  if (!s->free_events.empty()) {
    *ev = s->free_events.back();
    s->free_events.pop_back();
    return MF_OK;
  }
  MF_CUDA(cudaEventCreateWithFlags(ev, cudaEventDisableTiming), "event create");
  return MF_OK;
}

// Makes `st` wait for a run's upload; the event goes back to the pool (a
// wait enqueued on a stream keeps the state the event had at that time).
int consume_ready(mf_stream* s, Run& r, cudaStream_t st) {
  if (!r.ready) return MF_OK;
  MF_CUDA(cudaStreamWaitEvent(st, r.ready, 0), "wait for upload");
  s->free_events.push_back(r.ready);
  r.ready = nullptr;
  return MF_OK;
}

// st_b waits for all work enqueued so far on st_a.
int order_after(mf_stream* s, cudaStream_t st_b, cudaStream_t st_a) {
  cudaEvent_t ev;
  int rc = take_event(s, &ev);
  if (rc) return rc;
  MF_CUDA(cudaEventRecord(ev, st_a), "event record");
  MF_CUDA(cudaStreamWaitEvent(st_b, ev, 0), "stream wait");
  s->free_events.push_back(ev);
  return MF_OK;
}

int ensure_copy_streams(mf_stream* s) {
  if (s->st_in) return MF_OK;
  MF_CUDA(cudaStreamCreateWithFlags(&s->st_in, cudaStreamNonBlocking), "copy stream creation");
  MF_CUDA(cudaStreamCreateWithFlags(&s->st_out, cudaStreamNonBlocking), "copy stream creation");
  for (int k = 0; k < kOutSlots; ++k)
    MF_CUDA(cudaEventCreateWithFlags(&s->slot_ev[k], cudaEventDisableTiming), "event create");
  return MF_OK;
}

// Staging ring of depth planes for host-memory depth.  Grows (copying the
// pending planes in order) when the pending planes plus `need` do not fit.
int ensure_stage(mf_stream* s, int64_t need) {
  if (s->stage_used + need <= s->stage_slots) return MF_OK;
  const int64_t slots = std::max<int64_t>(s->stage_used + need, 2 * s->stage_slots);
  char* buf = (char*)s->dalloc((size_t)slots * s->plane_in);
  if (!buf) return fail(MF_ERR_OOM, "depth staging allocation failed");
  // move pending planes to slots 0..used-1 (after their uploads) and
  // repoint their runs
  int64_t moved = 0;
  for (Run& r : s->runs) {
    if (r.stage_slots == 0) continue;
    int rc = consume_ready(s, r, s->st);
    if (rc) return rc;
    MF_CUDA(cudaMemcpyAsync(buf + (size_t)moved * s->plane_in, r.depth,
                            (size_t)r.count * s->plane_in, cudaMemcpyDeviceToDevice, s->st),
            "staging move");
    r.depth = buf + (size_t)moved * s->plane_in;
    moved += r.count;
  }
  if (s->stage) {
    // uploads of runs dropped by mf_reset_stream may still be in flight
    if (s->st_in) MF_CUDA(cudaStreamSynchronize(s->st_in), "copy stream sync");
    MF_CUDA(cudaStreamSynchronize(s->st), "stream sync before freeing staging");
    s->dfree(s->stage, (size_t)s->stage_slots * s->plane_in);
  }
  s->stage = buf;
  s->stage_slots = slots;
  s->stage_head = 0;
  s->stage_used = moved;
  return MF_OK;
}

int ensure_out_stage(mf_stream* s, size_t bytes) {
  if (bytes <= s->out_stage_bytes) return MF_OK;
  if (s->out_stage) {
    if (s->st_out) MF_CUDA(cudaStreamSynchronize(s->st_out), "copy stream sync");
    MF_CUDA(cudaStreamSynchronize(s->st), "stream sync before freeing output staging");
    s->dfree(s->out_stage, s->out_stage_bytes);
    s->out_stage = nullptr;
    s->out_stage_bytes = 0;
  }
  s->out_stage = (char*)s->dalloc(bytes);
  if (!s->out_stage) return fail(MF_ERR_OOM, "output staging allocation failed");
  s->out_stage_bytes = bytes;
  return MF_OK;
}

// A completed wait on the stream reports a device wait that ran out in a map
// kernel since the last report (the fault word), or one injected on the host.
int check_fault(mf_stream* s) {
  if (mf::fault_fires(mf::kFaultWaitTimeout)) *reinterpret_cast<volatile unsigned int*>(s->fault_host) = 1u;
  const unsigned int f = __atomic_exchange_n(s->fault_host, 0u, __ATOMIC_ACQ_REL);
  if (f == 0u) return MF_OK;
  if (f == mf::kFaultOutOfRange)
    return fail(MF_ERR_CUDA, "checked build: an index outside its plane was caught (access skipped)");
  return fail(MF_ERR_TIMEOUT,
              "a bounded device wait of the tensor-core map kernel ran out: the frames concerned are "
              "marked MF_FRAME_TIMEOUT and bands of their maps hold NaN");
}

int wait_event(cudaEvent_t ev, int64_t timeout_ns) {
  const auto t0 = std::chrono::steady_clock::now();
  int spins = 0;
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return MF_OK;
    if (e != cudaErrorNotReady) return fail(MF_ERR_CUDA, "event query", e);
    if (timeout_ns >= 0) {
      const auto ns = std::chrono::duration_cast<std::chrono::nanoseconds>(
                          std::chrono::steady_clock::now() - t0)
                          .count();
      if (ns > timeout_ns) return fail(MF_ERR_TIMEOUT, "wait timed out");
    }
    if (++spins > 64)
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    else
      std::this_thread::yield();
  }
}

int collect_timers(mf_stream* s) {
  for (TimerPair& t : s->timers) {
    MF_CUDA(cudaEventSynchronize(t.b), "timer sync");
    float ms = 0.0f;
    MF_CUDA(cudaEventElapsedTime(&ms, t.a, t.b), "timer elapsed");
    s->map_ms += ms;
    ++s->map_timed;
    s->free_timers.push_back(t);
  }
  s->timers.clear();
  return MF_OK;
}

int timer_pair(mf_stream* s, TimerPair* out) {
  if (!s->free_timers.empty()) {
    *out = s->free_timers.back();
    s->free_timers.pop_back();
    return MF_OK;
  }
  MF_CUDA(cudaEventCreate(&out->a), "event create");
  MF_CUDA(cudaEventCreate(&out->b), "event create");
  return MF_OK;
}

void destroy(mf_stream* s) {
  if (s->st) cudaStreamSynchronize(s->st);
  if (s->st_in) cudaStreamSynchronize(s->st_in);
  if (s->st_out) cudaStreamSynchronize(s->st_out);
  for (Run& r : s->runs)
    if (r.ready) cudaEventDestroy(r.ready);
  for (cudaEvent_t ev : s->free_events) cudaEventDestroy(ev);
  for (int k = 0; k < kOutSlots; ++k)
    if (s->slot_ev[k]) cudaEventDestroy(s->slot_ev[k]);
  if (s->st_in) cudaStreamDestroy(s->st_in);
  if (s->st_out) cudaStreamDestroy(s->st_out);
  collect_timers(s);
  for (TimerPair& t : s->free_timers) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  s->dfree(s->ring, (size_t)s->ring_cap * 12 * sizeof(double));
  s->dfree(s->ring_bad, (size_t)s->ring_cap * sizeof(int32_t));
  s->dfree(s->recs, (size_t)s->rec_cap * sizeof(FrameRec));
  s->dfree(s->sched, sizeof(unsigned int));
  s->dfree(s->scale_dev, sizeof(double));
  s->dfree(s->align_work, mf::kAlignWorkWords * sizeof(unsigned int));
  s->dfree(s->ovl_prev, (size_t)s->d.overlap * s->plane_in);
  s->dfree(s->ovl_cur, (size_t)s->d.overlap * s->plane_in);
  s->dfree(s->pose_dev, (size_t)s->pose_dev_cap * 12 * sizeof(double));
  s->dfree(s->stage, (size_t)s->stage_slots * s->plane_in);
  s->dfree(s->out_stage, s->out_stage_bytes);
  if (s->pose_host) cudaFreeHost(s->pose_host);
  if (s->fault_host) cudaFreeHost(s->fault_host);
  if (s->pose_ev) cudaEventDestroy(s->pose_ev);
  if (s->done_ev) cudaEventDestroy(s->done_ev);
  if (s->own_stream && s->st) cudaStreamDestroy(s->st);
  delete s;
}

int validate_desc(const mf_stream_desc* d) {
  if (!d) return fail(MF_ERR_INVALID_ARG, "NULL descriptor");
  if (d->width < 1 || d->height < 1 || d->width > MF_MAX_DIM || d->height > MF_MAX_DIM)
    return fail(MF_ERR_INVALID_ARG, "width/height out of range");
  if ((int64_t)d->width * d->height > 0x7fffffffLL)
    return fail(MF_ERR_INVALID_ARG, "frame too large");
  if (d->calib_width < 0 || d->calib_height < 0)
    return fail(MF_ERR_INVALID_ARG, "negative calibration size");
  if (d->window < 1 || d->window > MF_MAX_WINDOW)
    return fail(MF_ERR_INVALID_ARG, "window must be 1..32");
  if (d->mode != MF_MODE_ACCEL && d->mode != MF_MODE_HEADING)
    return fail(MF_ERR_INVALID_ARG, "unknown mode");
  if (d->smooth_len < (d->mode == MF_MODE_ACCEL ? 3 : 2))
    return fail(MF_ERR_INVALID_ARG, "smooth_len too small for the mode");
  if (d->window + d->smooth_len - 1 > MF_MAX_HISTORY)
    return fail(MF_ERR_INVALID_ARG, "window + smooth_len - 1 exceeds 64");
  if (d->pose_frame == MF_POSES_WORLD) {
    if (d->overlap != 0) return fail(MF_ERR_INVALID_ARG, "overlap must be 0 for world poses");
  } else if (d->pose_frame == MF_POSES_BATCH_LOCAL) {
    if (d->overlap < 1) return fail(MF_ERR_INVALID_ARG, "batch-local poses need overlap >= 1");
  } else {
    return fail(MF_ERR_INVALID_ARG, "unknown pose frame");
  }
  for (int dt : {d->depth_dtype, d->map_dtype})
    if (dt != MF_F32 && dt != MF_BF16 && dt != MF_F16)
      return fail(MF_ERR_INVALID_ARG, "unknown dtype");
  if (d->max_pending < 1 || d->max_pending > (1 << 24))
    return fail(MF_ERR_INVALID_ARG, "max_pending out of range");
  if (d->normalize != MF_NORM_COUNT && d->normalize != MF_NORM_MAX)
    return fail(MF_ERR_INVALID_ARG, "unknown normalisation");
  if ((d->flags & MF_FLAG_MAP_CUDA_CORES) && (d->flags & MF_FLAG_MAP_TENSOR_CORES))
    return fail(MF_ERR_INVALID_ARG, "choose one map kernel");
  if ((d->flags & MF_FLAG_DEPTH_ALIGN) && d->pose_frame != MF_POSES_BATCH_LOCAL)
    return fail(MF_ERR_INVALID_ARG, "depth alignment needs batch-local poses");
  if (!(d->sigma_rel > 0.0) || !(d->s_lo > 0.0) || !(d->s_hi >= d->s_lo) ||
      !(d->depth_ref_m > 0.0) || !std::isfinite(d->sigma_rel) || !std::isfinite(d->s_hi) ||
      !std::isfinite(d->depth_ref_m))
    return fail(MF_ERR_INVALID_ARG, "sigma_rel, s_lo, s_hi or depth_ref_m invalid");
  if ((d->dev_alloc == nullptr) != (d->dev_free == nullptr))
    return fail(MF_ERR_INVALID_ARG, "dev_alloc and dev_free must be given together");
  return MF_OK;
}

}  // namespace

namespace mf {
// Host helpers shared with the allocation-free entry point (mf_noalloc.cu).
bool host_ls_weights(int K, int mode, double* w) { return ls_weights(K, mode, w); }
int host_validate_desc(const mf_stream_desc* d) { return validate_desc(d); }
int host_map_path(uint32_t flags) { return map_path(flags); }
int host_fail(int status, const char* what, cudaError_t e) { return fail(status, what, e); }
void host_count_launches(int64_t n) { g_launches.fetch_add(n); }
int host_pointer_kind(const void* p, int dev) { return pointer_kind(p, dev); }

KernelFit host_kernel_fit(const void* kernel, int threads, size_t smem_limit, size_t smem_launch,
                          int carveout) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t, size_t>, KernelFit> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(kernel, dev, smem_limit, smem_launch);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  KernelFit f;
  cudaDeviceGetAttribute(&f.sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit);
  if (carveout >= 0) cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem_launch) != cudaSuccess) {
    cudaGetLastError();
    per = 1;
  }
  f.per_sm = per < 1 ? 1 : per;
  if (f.sms < 1) f.sms = 1;
  cache.emplace(key, f);
  return f;
}
}  // namespace mf

extern "C" {

void mf_stream_desc_init(mf_stream_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->window = 8;
  d->smooth_len = 15;
  d->mode = MF_MODE_ACCEL;
  d->pose_frame = MF_POSES_WORLD;
  d->depth_dtype = MF_F32;
  d->map_dtype = MF_F32;
  d->max_pending = 1024;
  d->sigma_rel = 0.1;
  d->s_lo = 0.25;
  d->s_hi = 4.0;
  d->depth_ref_m = 1.0;
}

int mf_open_stream(const mf_stream_desc* d, mf_stream** out) {
  if (!out) return fail(MF_ERR_INVALID_ARG, "NULL output handle");
  *out = nullptr;
  int rc = validate_desc(d);
  if (rc) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(MF_ERR_NO_DEVICE, "no CUDA device");
  }
  mf_stream* s = new (std::nothrow) mf_stream();
  if (!s) return fail(MF_ERR_OOM, "host allocation failed");
  s->d = *d;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return fail(MF_ERR_NO_DEVICE, "cudaGetDevice failed");
  }
  if (!ls_weights(d->smooth_len, d->mode, s->w)) {
    delete s;
    return fail(MF_ERR_INVALID_ARG, "least-squares weights not representable");
  }
  s->plane_in = (size_t)d->width * d->height * dtype_size(d->depth_dtype);
  s->plane_out = (size_t)d->width * d->height * dtype_size(d->map_dtype);
  s->piece = piece_frames(s->plane_in + 2 * s->plane_out);
  if (d->cuda_stream) {
    s->st = (cudaStream_t)d->cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return fail(MF_ERR_CUDA, "stream creation failed");
    }
    s->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&s->pose_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->done_ev, cudaEventDisableTiming) != cudaSuccess) {
    destroy(s);
    return fail(MF_ERR_CUDA, "event creation failed");
  }
  s->rec_cap = pow2_at_least(d->max_pending);
  s->recs = (FrameRec*)s->dalloc((size_t)s->rec_cap * sizeof(FrameRec));
  s->sched = (unsigned int*)s->dalloc(sizeof(unsigned int));
  if (!s->recs || !s->sched) {
    destroy(s);
    return fail(MF_ERR_OOM, "frame record or work counter allocation failed");
  }
  if (cudaHostAlloc((void**)&s->fault_host, sizeof(unsigned int), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&s->fault_dev, s->fault_host, 0) != cudaSuccess) {
    cudaGetLastError();
    destroy(s);
    return fail(MF_ERR_OOM, "fault word allocation failed");
  }
  *s->fault_host = 0u;
  if (d->flags & MF_FLAG_DEPTH_ALIGN) {
    s->align = true;
    s->scale_dev = (double*)s->dalloc(sizeof(double));
    s->align_work = (unsigned int*)s->dalloc(mf::kAlignWorkWords * sizeof(unsigned int));
    s->ovl_prev = (char*)s->dalloc((size_t)d->overlap * s->plane_in);
    s->ovl_cur = (char*)s->dalloc((size_t)d->overlap * s->plane_in);
    if (!s->scale_dev || !s->align_work || !s->ovl_prev || !s->ovl_cur) {
      destroy(s);
      return fail(MF_ERR_OOM, "depth alignment buffers");
    }
    if (cudaMemcpyAsync(s->scale_dev, &kUnitScale, sizeof(double), cudaMemcpyHostToDevice, s->st) !=
        cudaSuccess) {
      cudaGetLastError();
      destroy(s);
      return fail(MF_ERR_CUDA, "depth scale initialisation failed");
    }
  }
  // every map launch of the stream leaves its counter at 0 again
  if (cudaMemsetAsync(s->sched, 0, sizeof(unsigned int), s->st) != cudaSuccess) {
    cudaGetLastError();
    destroy(s);
    return fail(MF_ERR_CUDA, "work counter initialisation failed");
  }
  rc = grow_ring(s, d->window + d->smooth_len + 64);
  if (rc) {
    destroy(s);
    return rc;
  }
  *out = s;
  return MF_OK;
}

int mf_push_frames(mf_stream* s, int32_t n, const double* poses, const void* depth,
                   const double* K) {
  mf::NvtxRange range("mf_push_frames");
  if (!s) return fail(MF_ERR_INVALID_ARG, "NULL stream");
  if (n < 1 || !poses || !K) return fail(MF_ERR_INVALID_ARG, "n < 1 or NULL poses/K");
  const bool local = s->d.pose_frame == MF_POSES_BATCH_LOCAL;
  const int O = (local && s->pushes > 0) ? s->d.overlap : 0;
  if (n <= O) return fail(MF_ERR_INVALID_ARG, "batch must hold more frames than the overlap");
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(K[k])) return fail(MF_ERR_INVALID_ARG, "non-finite intrinsics");
  if (!(K[0] > 0.0) || !(K[1] > 0.0)) return fail(MF_ERR_INVALID_ARG, "fx, fy must be > 0");
  const int n_emit = n - O;
  if (s->emitted - s->rendered + n_emit > s->rec_cap || s->emitted - s->rendered + n_emit > s->d.max_pending)
    return fail(MF_ERR_NOT_READY, "too many pending frames: call mf_get_maps first");
  DeviceGuard guard(s->device);
  LaunchTally tally(&s->launches);

  const int hist = s->d.window + s->d.smooth_len - 1;
  int rc = grow_ring(s, (int64_t)hist + n_emit + 1);
  if (rc) return rc;

  // Poses: device pointers are read in place; host poses go through a pinned
  // bounce buffer so the caller may reuse its memory at once.
  const double* pdev = poses;
  const int pose_kind = pointer_kind(poses, s->device);
  const int depth_kind = pointer_kind(depth, s->device);
  if (pose_kind == mf::kPtrOtherDevice || depth_kind == mf::kPtrOtherDevice)
    return fail(MF_ERR_INVALID_ARG, "poses or depth live on another GPU than the stream's device");
  if (pose_kind != mf::kPtrDevice) {
    if ((int64_t)n > s->pose_dev_cap) {
      const int64_t cap = pow2_at_least(std::max<int64_t>(n, 256));
      double* nd = (double*)s->dalloc((size_t)cap * 12 * sizeof(double));
      if (!nd) return fail(MF_ERR_OOM, "pose staging allocation failed");
      if (s->pose_dev) {
        MF_CUDA(cudaStreamSynchronize(s->st), "stream sync");
        s->dfree(s->pose_dev, (size_t)s->pose_dev_cap * 12 * sizeof(double));
      }
      s->pose_dev = nd;
      s->pose_dev_cap = cap;
    }
    MF_CUDA(cudaEventSynchronize(s->pose_ev), "pose upload wait");
    if ((int64_t)n > s->pose_host_cap) {
      if (s->pose_host) cudaFreeHost(s->pose_host);
      s->pose_host = nullptr;
      const int64_t cap = pow2_at_least(std::max<int64_t>(n, 256));
      MF_CUDA(cudaMallocHost(&s->pose_host, (size_t)cap * 12 * sizeof(double)), "pinned alloc");
      s->pose_host_cap = cap;
    }
    std::memcpy(s->pose_host, poses, (size_t)n * 12 * sizeof(double));
    for (int32_t k = 0; k < n; ++k)  // injected fault: a pose that is no rotation
      if (mf::fault_fires(mf::kFaultBadPose)) s->pose_host[(size_t)k * 12] *= 2.0;
    MF_CUDA(cudaMemcpyAsync(s->pose_dev, s->pose_host, (size_t)n * 12 * sizeof(double),
                            cudaMemcpyHostToDevice, s->st),
            "pose upload");
    MF_CUDA(cudaEventRecord(s->pose_ev, s->st), "event record");
    pdev = s->pose_dev;
  }

  // Depth: device planes are referenced; host planes are copied to staging.
  std::vector<Run> new_runs;
  if (depth) {
    const char* dsrc = static_cast<const char*>(depth) + (size_t)O * s->plane_in;
    if (depth_kind == mf::kPtrDevice) {
      new_runs.push_back(Run{s->emitted, n_emit, dsrc, 0, nullptr});
    } else {
      rc = ensure_stage(s, n_emit);
      if (rc) return rc;
      rc = ensure_copy_streams(s);
      if (rc) return rc;
      // A staging slot is reused only after the map kernels that read its
      // previous plane: the uploads start after the work already on st.
      rc = order_after(s, s->st_in, s->st);
      if (rc) return rc;
      const int piece = s->piece;
      int64_t done = 0;
      while (done < n_emit) {
        const int64_t slot = (s->stage_head + s->stage_used) % s->stage_slots;
        const int64_t chunk = std::min<int64_t>({n_emit - done, s->stage_slots - slot, (int64_t)piece});
        char* dst = s->stage + (size_t)slot * s->plane_in;
        MF_CUDA(cudaMemcpyAsync(dst, dsrc + (size_t)done * s->plane_in,
                                (size_t)chunk * s->plane_in, cudaMemcpyHostToDevice, s->st_in),
                "depth upload");
        cudaEvent_t ev;
        rc = take_event(s, &ev);
        if (rc) return rc;
        MF_CUDA(cudaEventRecord(ev, s->st_in), "event record");
        new_runs.push_back(Run{s->emitted + done, (int)chunk, dst, (int)chunk, ev});
        s->stage_used += chunk;
        done += chunk;
      }
    }
  } else {
    new_runs.push_back(Run{s->emitted, n_emit, nullptr, 0, nullptr});
  }

  // Depth alignment: this batch's scale from the overlap frames' depth ratios
  // against the previous batch (Section 2.2), before any pose is anchored.
  if (s->align && depth && n < s->d.overlap)
    return fail(MF_ERR_INVALID_ARG, "depth alignment needs batches of at least `overlap` frames");
  if (s->align && O > 0 && depth && s->ovl_valid) {
    const void* cur = depth;
    if (depth_kind != mf::kPtrDevice) {
      MF_CUDA(cudaMemcpyAsync(s->ovl_cur, depth, (size_t)O * s->plane_in, cudaMemcpyHostToDevice, s->st),
              "overlap depth upload");
      cur = s->ovl_cur;
    }
    mf::AlignParams ap{};
    ap.prev = s->ovl_prev;
    ap.cur = cur;
    ap.count = (int64_t)O * s->d.width * s->d.height;
    ap.work = s->align_work;
    ap.scale = s->scale_dev;
    MF_CUDA(mf::launch_depth_align(ap, s->d.depth_dtype, s->st, &s->launches), "depth alignment launch");
  }

  mf::IngestParams ip{};
  ip.scale = s->align ? s->scale_dev : nullptr;
  ip.in = pdev;
  ip.n = n;
  ip.first = O;
  ip.anchor = O > 0 ? 1 : 0;
  ip.ring = s->ring;
  ip.ring_bad = s->ring_bad;
  ip.ring_mask = s->ring_cap - 1;
  ip.e0 = s->emitted;
  MF_CUDA(mf::launch_ingest(ip, s->st, &s->launches), "ingest launch");

  mf::PointsParams pp{};
  pp.ring = s->ring;
  pp.ring_bad = s->ring_bad;
  pp.ring_mask = s->ring_cap - 1;
  pp.recs = s->recs;
  pp.rec_mask = s->rec_cap - 1;
  pp.e0 = s->emitted;
  pp.n_frames = n_emit;
  pp.window = s->d.window;
  pp.smooth_len = s->d.smooth_len;
  pp.width = s->d.width;
  pp.height = s->d.height;
  pp.calib_width = s->d.calib_width;
  pp.calib_height = s->d.calib_height;
  for (int k = 0; k < 4; ++k) pp.K[k] = K[k];
  pp.sigma_rel = s->d.sigma_rel;
  pp.s_lo = s->d.s_lo;
  pp.s_hi = s->d.s_hi;
  for (int k = 0; k < mf::kMaxHist; ++k) pp.w[k] = k < s->d.smooth_len ? s->w[k] : 0.0;
  pp.d0 = s->d.depth_ref_m;
  pp.scale = s->align ? s->scale_dev : nullptr;
  MF_CUDA(mf::launch_points(pp, s->st, &s->launches), "points launch");

  // the last `overlap` depth planes, for the next batch's alignment (after
  // the selection above has read the previous ones)
  if (s->align) {
    s->ovl_valid = depth != nullptr;
    if (depth) {
      const size_t bytes = (size_t)s->d.overlap * s->plane_in;
      const char* src = static_cast<const char*>(depth) + (size_t)(n - s->d.overlap) * s->plane_in;
      MF_CUDA(cudaMemcpyAsync(s->ovl_prev, src, bytes,
                              depth_kind == mf::kPtrDevice ? cudaMemcpyDeviceToDevice
                                                           : cudaMemcpyHostToDevice,
                              s->st),
              "overlap depth copy");
    }
  }

  for (const Run& r : new_runs) s->runs.push_back(r);
  s->emitted += n_emit;
  s->pushed_frames += n;
  ++s->pushes;
  return MF_OK;
}

int mf_get_maps(mf_stream* s, int32_t max_frames, void* focus_map, void* guided_depth,
                mf_frame_info* info, mf_motion_point* points, int32_t* n_out,
                int64_t timeout_ns) {
  mf::NvtxRange range("mf_get_maps");
  if (!s || !n_out) return fail(MF_ERR_INVALID_ARG, "NULL stream or n_out");
  *n_out = 0;
  if (max_frames < 0) return fail(MF_ERR_INVALID_ARG, "max_frames < 0");
  const int64_t take = std::min<int64_t>(max_frames, s->emitted - s->rendered);
  if (take <= 0) return MF_OK;
  DeviceGuard guard(s->device);
  LaunchTally tally(&s->launches);

  const int kinds[4] = {pointer_kind(focus_map, s->device), pointer_kind(guided_depth, s->device),
                        pointer_kind(info, s->device), pointer_kind(points, s->device)};
  for (int k : kinds)
    if (k == mf::kPtrOtherDevice)
      return fail(MF_ERR_INVALID_ARG, "an output lives on another GPU than the stream's device");
  const bool m_host = focus_map && kinds[0] != mf::kPtrDevice;
  const bool g_host = guided_depth && kinds[1] != mf::kPtrDevice;
  const bool i_host = info && kinds[2] != mf::kPtrDevice;
  const bool p_host = points && kinds[3] != mf::kPtrDevice;
  const bool maps_host = m_host || g_host;
  // Maps bound for host memory are rendered in pieces into a ring of
  // kOutSlots staging pieces; each piece's download on st_out overlaps the
  // next pieces' kernels and the uploads on st_in.
  const int piece = maps_host ? s->piece : (int)take;
  const size_t map_stage_bytes = maps_host ? (size_t)kOutSlots * piece * s->plane_out : 0;
  const size_t info_bytes = (size_t)take * sizeof(mf_frame_info);
  const size_t pts_bytes = (size_t)take * s->d.window * sizeof(mf_motion_point);
  auto round256 = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t need = 0;
  if (m_host) need += round256(map_stage_bytes);
  if (g_host) need += round256(map_stage_bytes);
  if (i_host) need += round256(info_bytes);
  if (p_host) need += round256(pts_bytes);
  int rc = ensure_out_stage(s, need);
  if (rc) return rc;
  if (maps_host || i_host || p_host) {
    rc = ensure_copy_streams(s);
    if (rc) return rc;
  }
  char* cur = s->out_stage;
  auto place = [&](bool host, void* user, size_t bytes) -> char* {
    if (!user) return nullptr;
    if (!host) return static_cast<char*>(user);
    char* p = cur;
    cur += round256(bytes);
    return p;
  };
  char* Mst = place(m_host, focus_map, map_stage_bytes);
  char* Gst = place(g_host, guided_depth, map_stage_bytes);
  char* Id = place(i_host, info, info_bytes);
  char* Pd = place(p_host, points, pts_bytes);

  // Download of one rendered piece (host maps only), issued one piece late
  // so that a synchronous copy into pageable memory still overlaps the next
  // piece's kernel.
  struct Piece {
    int slot;
    int64_t done;
    int cnt;
  };
  Piece pending{-1, 0, 0};
  auto download = [&](const Piece& q) -> int {
    cudaEvent_t ev;
    int r2 = take_event(s, &ev);
    if (r2) return r2;
    MF_CUDA(cudaEventRecord(ev, s->st), "event record");
    MF_CUDA(cudaStreamWaitEvent(s->st_out, ev, 0), "stream wait");
    s->free_events.push_back(ev);
    const size_t off = (size_t)q.slot * piece * s->plane_out;
    const size_t bytes = (size_t)q.cnt * s->plane_out;
    if (m_host)
      MF_CUDA(cudaMemcpyAsync(static_cast<char*>(focus_map) + (size_t)q.done * s->plane_out,
                              Mst + off, bytes, cudaMemcpyDeviceToHost, s->st_out), "D2H");
    if (g_host)
      MF_CUDA(cudaMemcpyAsync(static_cast<char*>(guided_depth) + (size_t)q.done * s->plane_out,
                              Gst + off, bytes, cudaMemcpyDeviceToHost, s->st_out), "D2H");
    MF_CUDA(cudaEventRecord(s->slot_ev[q.slot], s->st_out), "event record");
    s->slot_busy[q.slot] = true;
    return MF_OK;
  };

  // one map launch per contiguous depth run (per piece for host maps)
  int64_t f = s->rendered;
  int64_t done = 0;
  int pieces = 0;
  const bool timed = (s->d.flags & MF_FLAG_TIME_KERNELS) != 0;
  while (done < take) {
    Run& r = s->runs.front();
    const int64_t skip = f - r.first;
    const int cnt = (int)std::min<int64_t>({r.count - skip, take - done, (int64_t)piece});
    rc = consume_ready(s, r, s->st);
    if (rc) return rc;
    const int slot = pieces % kOutSlots;
    if (maps_host && s->slot_busy[slot])
      MF_CUDA(cudaStreamWaitEvent(s->st, s->slot_ev[slot], 0), "wait for output slot");
    auto target = [&](bool host, char* stage, void* user) -> char* {
      if (!user) return nullptr;
      if (host) return stage + (size_t)slot * piece * s->plane_out;
      return static_cast<char*>(user) + (size_t)done * s->plane_out;
    };
    char* Mp = target(m_host, Mst, focus_map);
    char* Gp = target(g_host, Gst, guided_depth);
    mf::MapParams mp{};
    mp.recs = s->recs;
    mp.rec_mask = s->rec_cap - 1;
    mp.f0 = f;
    mp.n_frames = cnt;
    mp.width = s->d.width;
    mp.height = s->d.height;
    mp.tile_h = mf::map_tile_h(s->d.width, s->d.height, s->d.window);
    mp.tiles_x = (s->d.width + mf::kTileW - 1) / mf::kTileW;
    mp.tiles_y = (s->d.height + mp.tile_h - 1) / mp.tile_h;
    mp.depth = r.depth ? r.depth + (size_t)skip * s->plane_in : nullptr;
    mp.M = Mp;
    mp.G = Gp;
    mp.path = map_path(s->d.flags);
    mp.sched = s->sched;
    mp.fault = s->fault_dev;
    TimerPair tp{};
    if (timed) {
      rc = timer_pair(s, &tp);
      if (rc) return rc;
      MF_CUDA(cudaEventRecord(tp.a, s->st), "event record");
    }
    MF_CUDA(mf::launch_map(mp, s->d.window, s->d.depth_dtype, s->d.map_dtype, s->d.normalize, s->st,
                           &s->launches),
            "map launch");
    s->last_map_kernel = mf::map_uses_tensor_cores(mp.path)
                             ? MF_FLAG_MAP_TENSOR_CORES
                             : MF_FLAG_MAP_CUDA_CORES;
    if (timed) {
      MF_CUDA(cudaEventRecord(tp.b, s->st), "event record");
      s->timers.push_back(tp);
    }
    if (maps_host) {
      if (pending.slot >= 0) {
        rc = download(pending);
        if (rc) return rc;
      }
      pending = Piece{slot, done, cnt};
    }
    ++pieces;
    f += cnt;
    done += cnt;
    if (skip + cnt == r.count) {
      if (r.stage_slots) {
        s->stage_head = (s->stage_head + r.stage_slots) % s->stage_slots;
        s->stage_used -= r.stage_slots;
      }
      s->runs.pop_front();
    }
  }
  if (pending.slot >= 0) {
    rc = download(pending);
    if (rc) return rc;
  }
  mf::FinalizeParams fp{};
  fp.recs = s->recs;
  fp.rec_mask = s->rec_cap - 1;
  fp.f0 = s->rendered;
  fp.n_frames = (int)take;
  fp.width = s->d.width;
  fp.window = s->d.window;
  fp.normalize = s->d.normalize;
  fp.info = reinterpret_cast<mf_frame_info*>(Id);
  fp.points = reinterpret_cast<mf_motion_point*>(Pd);
  MF_CUDA(mf::launch_finalize(fp, s->st, &s->launches), "finalize launch");
  s->rendered += take;
  *n_out = (int32_t)take;

  if (maps_host || i_host || p_host) {
    if (i_host || p_host) {
      rc = order_after(s, s->st_out, s->st);
      if (rc) return rc;
      if (i_host)
        MF_CUDA(cudaMemcpyAsync(info, Id, info_bytes, cudaMemcpyDeviceToHost, s->st_out), "D2H");
      if (p_host)
        MF_CUDA(cudaMemcpyAsync(points, Pd, pts_bytes, cudaMemcpyDeviceToHost, s->st_out), "D2H");
    }
    // Later work on st (and mf_sync) comes after the downloads.
    rc = order_after(s, s->st, s->st_out);
    if (rc) return rc;
    for (int k = 0; k < kOutSlots; ++k) s->slot_busy[k] = false;
    MF_CUDA(cudaEventRecord(s->done_ev, s->st), "event record");
    rc = wait_event(s->done_ev, timeout_ns);
    return rc ? rc : check_fault(s);
  }
  return MF_OK;
}

int mf_sync(mf_stream* s, int64_t timeout_ns) {
  if (!s) return fail(MF_ERR_INVALID_ARG, "NULL stream");
  DeviceGuard guard(s->device);
  MF_CUDA(cudaEventRecord(s->done_ev, s->st), "event record");
  const int rc = wait_event(s->done_ev, timeout_ns);
  return rc ? rc : check_fault(s);
}

int mf_pending_frames(const mf_stream* s, int32_t* n) {
  if (!s || !n) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  *n = (int32_t)(s->emitted - s->rendered);
  return MF_OK;
}

int mf_reset_stream(mf_stream* s) {
  if (!s) return fail(MF_ERR_INVALID_ARG, "NULL stream");
  // Host bookkeeping only: every kernel and copy already enqueued reads and
  // writes library memory in stream order before anything enqueued later.
  s->emitted = s->rendered = s->pushes = 0;
  for (Run& r : s->runs)
    if (r.ready) s->free_events.push_back(r.ready);
  s->runs.clear();
  s->stage_head = s->stage_used = 0;
  if (s->align) {  // the next batch is a first batch again: scale 1
    DeviceGuard guard(s->device);
    s->ovl_valid = false;
    MF_CUDA(cudaMemcpyAsync(s->scale_dev, &kUnitScale, sizeof(double), cudaMemcpyHostToDevice, s->st),
            "depth scale reset");
  }
  return MF_OK;
}

int mf_stream_stats(mf_stream* s, mf_stats* out) {
  if (!s || !out) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard guard(s->device);
  int rc = collect_timers(s);
  if (rc) return rc;
  out->frames_pushed = s->pushed_frames;
  out->frames_emitted = s->emitted;
  out->frames_rendered = s->rendered;
  out->kernel_launches = s->launches;
  out->map_launches = s->map_timed;
  out->map_kernel_ms = s->map_ms;
  out->device_bytes = s->device_bytes;
  out->last_map_kernel = s->last_map_kernel;
  out->reserved = 0;
  return MF_OK;
}

namespace {

// Layout of a stream snapshot: this header, then `hist` world poses (12
// doubles each, oldest first), their bad flags (int32), then, with depth
// alignment and a valid overlap, `overlap` depth planes.
struct SnapHeader {
  char magic[4];
  int32_t version;
  int64_t bytes;
  // the descriptor fields the state depends on (must match on restore)
  int32_t width, height, calib_width, calib_height, window, smooth_len, mode, pose_frame, overlap,
      depth_dtype, map_dtype, normalize, align;
  int32_t hist, ovl_valid, pad;
  double sigma_rel, s_lo, s_hi, depth_ref_m;
  int64_t emitted, pushes, pushed_frames;
  double scale;
};

void snap_fill_desc(const mf_stream* s, SnapHeader* h) {
  std::memset(h, 0, sizeof(*h));
  std::memcpy(h->magic, "MFSN", 4);
  h->version = 1;
  h->width = s->d.width;
  h->height = s->d.height;
  h->calib_width = s->d.calib_width;
  h->calib_height = s->d.calib_height;
  h->window = s->d.window;
  h->smooth_len = s->d.smooth_len;
  h->mode = s->d.mode;
  h->pose_frame = s->d.pose_frame;
  h->overlap = s->d.overlap;
  h->depth_dtype = s->d.depth_dtype;
  h->map_dtype = s->d.map_dtype;
  h->normalize = s->d.normalize;
  h->align = s->align ? 1 : 0;
  h->sigma_rel = s->d.sigma_rel;
  h->s_lo = s->d.s_lo;
  h->s_hi = s->d.s_hi;
  h->depth_ref_m = s->d.depth_ref_m;
}

// Copies `count` ring entries starting at emitted-frame index `first`
// between the device ring and host arrays (the ring wraps at its capacity).
int ring_transfer(mf_stream* s, int64_t first, int64_t count, double* poses, int32_t* bad, bool to_host) {
  int64_t done = 0;
  while (done < count) {
    const int64_t slot = (first + done) & (s->ring_cap - 1);
    const int64_t run = std::min<int64_t>(count - done, s->ring_cap - slot);
    double* dp = s->ring + slot * 12;
    int32_t* db = s->ring_bad + slot;
    if (to_host) {
      MF_CUDA(cudaMemcpy(poses + done * 12, dp, (size_t)run * 12 * sizeof(double), cudaMemcpyDeviceToHost),
              "snapshot copy");
      MF_CUDA(cudaMemcpy(bad + done, db, (size_t)run * sizeof(int32_t), cudaMemcpyDeviceToHost), "snapshot copy");
    } else {
      MF_CUDA(cudaMemcpy(dp, poses + done * 12, (size_t)run * 12 * sizeof(double), cudaMemcpyHostToDevice),
              "restore copy");
      MF_CUDA(cudaMemcpy(db, bad + done, (size_t)run * sizeof(int32_t), cudaMemcpyHostToDevice), "restore copy");
    }
    done += run;
  }
  return MF_OK;
}

}  // namespace

int mf_stream_snapshot(mf_stream* s, void* buf, int64_t cap, int64_t* bytes) {
  if (!s || !bytes) return fail(MF_ERR_INVALID_ARG, "NULL stream or size");
  if (s->emitted != s->rendered) return fail(MF_ERR_NOT_READY, "frames pending: call mf_get_maps first");
  const int64_t hist = std::min<int64_t>(s->emitted, s->d.window + s->d.smooth_len - 1);
  const bool ovl = s->align && s->ovl_valid;
  const int64_t need = (int64_t)sizeof(SnapHeader) + hist * (12 * (int64_t)sizeof(double) + 4) +
                       (ovl ? (int64_t)s->d.overlap * (int64_t)s->plane_in : 0);
  *bytes = need;
  if (!buf) return MF_OK;
  if (cap < need) return fail(MF_ERR_INVALID_ARG, "snapshot buffer too small");
  DeviceGuard guard(s->device);
  MF_CUDA(cudaStreamSynchronize(s->st), "stream sync");
  SnapHeader h;
  snap_fill_desc(s, &h);
  h.bytes = need;
  h.hist = (int32_t)hist;
  h.ovl_valid = ovl ? 1 : 0;
  h.emitted = s->emitted;
  h.pushes = s->pushes;
  h.pushed_frames = s->pushed_frames;
  h.scale = 1.0;
  if (s->align) MF_CUDA(cudaMemcpy(&h.scale, s->scale_dev, sizeof(double), cudaMemcpyDeviceToHost), "snapshot copy");
  char* p = static_cast<char*>(buf);
  std::memcpy(p, &h, sizeof(h));
  double* poses = reinterpret_cast<double*>(p + sizeof(h));
  int32_t* bad = reinterpret_cast<int32_t*>(poses + hist * 12);
  int rc = ring_transfer(s, s->emitted - hist, hist, poses, bad, true);
  if (rc) return rc;
  if (ovl)
    MF_CUDA(cudaMemcpy(reinterpret_cast<char*>(bad + hist), s->ovl_prev, (size_t)s->d.overlap * s->plane_in,
                       cudaMemcpyDeviceToHost),
            "snapshot copy");
  return MF_OK;
}

int mf_stream_restore(mf_stream* s, const void* buf, int64_t bytes) {
  if (!s || !buf) return fail(MF_ERR_INVALID_ARG, "NULL stream or snapshot");
  if (s->emitted != 0 || s->pushes != 0)
    return fail(MF_ERR_NOT_READY, "restore into a stream that has taken no push (or was reset)");
  if (bytes < (int64_t)sizeof(SnapHeader)) return fail(MF_ERR_INVALID_ARG, "not a stream snapshot");
  SnapHeader h;
  std::memcpy(&h, buf, sizeof(h));
  SnapHeader mine;
  snap_fill_desc(s, &mine);
  if (std::memcmp(h.magic, "MFSN", 4) != 0 || h.version != 1 || h.bytes != bytes)
    return fail(MF_ERR_INVALID_ARG, "not a stream snapshot of this version");
  // every descriptor field the state depends on must match
  const size_t fields = offsetof(SnapHeader, hist) - offsetof(SnapHeader, width);
  if (std::memcmp(&h.width, &mine.width, fields) != 0 || h.sigma_rel != mine.sigma_rel ||
      h.s_lo != mine.s_lo || h.s_hi != mine.s_hi || h.depth_ref_m != mine.depth_ref_m)
    return fail(MF_ERR_INVALID_ARG, "the snapshot's stream descriptor differs from this stream's");
  const int64_t max_hist = s->d.window + s->d.smooth_len - 1;
  if (h.hist < 0 || h.hist > max_hist || h.hist > h.emitted || h.emitted < 0 ||
      (h.ovl_valid && !s->align))
    return fail(MF_ERR_INVALID_ARG, "inconsistent stream snapshot");
  const int64_t need = (int64_t)sizeof(SnapHeader) + (int64_t)h.hist * (12 * (int64_t)sizeof(double) + 4) +
                       (h.ovl_valid ? (int64_t)s->d.overlap * (int64_t)s->plane_in : 0);
  if (need != bytes) return fail(MF_ERR_INVALID_ARG, "stream snapshot size mismatch");
  DeviceGuard guard(s->device);
  int rc = grow_ring(s, max_hist + 64);
  if (rc) return rc;
  MF_CUDA(cudaStreamSynchronize(s->st), "stream sync");
  const char* p = static_cast<const char*>(buf);
  const double* poses = reinterpret_cast<const double*>(p + sizeof(h));
  const int32_t* bad = reinterpret_cast<const int32_t*>(poses + (int64_t)h.hist * 12);
  rc = ring_transfer(s, h.emitted - h.hist, h.hist, const_cast<double*>(poses), const_cast<int32_t*>(bad),
                     false);
  if (rc) return rc;
  if (s->align) {
    MF_CUDA(cudaMemcpy(s->scale_dev, &h.scale, sizeof(double), cudaMemcpyHostToDevice), "restore copy");
    s->ovl_valid = h.ovl_valid != 0;
    if (s->ovl_valid)
      MF_CUDA(cudaMemcpy(s->ovl_prev, reinterpret_cast<const char*>(bad + h.hist),
                         (size_t)s->d.overlap * s->plane_in, cudaMemcpyHostToDevice),
              "restore copy");
  }
  s->emitted = s->rendered = h.emitted;
  s->pushes = h.pushes;
  s->pushed_frames = h.pushed_frames;
  return MF_OK;
}

int mf_close_stream(mf_stream* s) {
  if (!s) return MF_OK;
  DeviceGuard guard(s->device);
  destroy(s);
  return MF_OK;
}

const char* mf_status_string(int status) {
  switch (status) {
    case MF_OK: return "ok";
    case MF_ERR_INVALID_ARG: return "invalid argument";
    case MF_ERR_INVALID_POSE: return "invalid pose";
    case MF_ERR_OOM: return "out of memory";
    case MF_ERR_NOT_READY: return "not ready: too many pending frames";
    case MF_ERR_TIMEOUT: return "timeout";
    case MF_ERR_CUDA: return "CUDA error";
    case MF_ERR_ADMISSION: return "admission refused";
    case MF_ERR_NO_DEVICE: return "no CUDA device";
  }
  return "unknown status";
}

int mf_version(void) { return MF_VERSION; }

int64_t mf_total_kernel_launches(void) { return g_launches.load(); }

const char* mf_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
