// Batched engine (include/mf.h, "Batched engine"): stream slots with
// resident pose histories, admission against a device-memory budget, ticks
// that process every submitted push as one batch (a CUDA graph of the tick
// table upload and four kernels), and the tile-height autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <deque>
#include <memory>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "mf_engine_internal.h"

using mf::FrameRec;
using mf::SlotParams;
using mf::TickFrame;
using mf::TickHeader;
using mf::TickPush;

namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }
size_t dtype_bytes(int dt) { return dt == MF_F32 ? 4 : 2; }
int64_t pow2_at_least(int64_t v) {
  int64_t c = 1;
  while (c < v) c <<= 1;
  return c;
}

int fail(int st, const char* what, cudaError_t e = cudaSuccess) { return mf::host_fail(st, what, e); }

#define ENG_CUDA(call, what)                                   \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return fail(MF_ERR_CUDA, what, e_); \
  } while (0)


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

// Plain-path tile height (used without tuning).
int default_band(int height) {
  const int bands = (height + mf::kBandMax - 1) / mf::kBandMax;
  return (height + bands - 1) / bands;
}

}  // namespace

void mf::latency_summary(const std::vector<double>& v, mf_latency_stats* out) {
  std::memset(out, 0, sizeof(*out));
  out->frames = (int64_t)v.size();
  if (v.empty()) return;
  std::vector<double> s(v);
  std::sort(s.begin(), s.end());
  // nearest-rank percentile: the smallest value with at least p of the samples at or below it
  auto q = [&](double p) {
    const size_t i = std::min(s.size() - 1, (size_t)std::ceil(p * s.size()) - (p > 0 ? 1 : 0));
    return s[i];
  };
  out->p50_ms = q(0.50);
  out->p90_ms = q(0.90);
  out->p99_ms = q(0.99);
  out->max_ms = s.back();
  double sum = 0.0;
  for (double x : s) sum += x;
  out->mean_ms = sum / s.size();
}

int64_t mf::engine_now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Submit times of one tick's frames and the time its work finished on the
// GPU (written by a host function the driver runs behind the tick).
struct TickRecord {
  std::vector<int64_t> submit_ns;  // one per frame
  std::atomic<int64_t> done_ns{0};
};

void CUDART_CB stamp_tick_done(void* p) {
  static_cast<TickRecord*>(p)->done_ns.store(now_ns(), std::memory_order_release);
}

struct Slot {
  bool used = false;
  mf_stream_desc d{};
  double* ring = nullptr;
  int32_t* ring_bad = nullptr;
  int64_t ring_cap = 0;
  int64_t emitted = 0, pushes = 0;
  int64_t reserve = 0;
  int64_t pending_tick = -1;  // tick id of the slot's queued push
  int64_t last_tick = -1;     // last tick that used the slot
  size_t plane_in = 0, plane_out = 0;
  int path = 0;                        // map path (mf::kEnginePaths)
  int band_h = 0, bands = 0, groups_x = 0;
};

// Columns per lane and per map unit of a path, for maps of map_dtype.
int path_cpt(int path, int map_dtype) {
  return path ? mf::engine_wide_cpt((int)dtype_bytes(map_dtype)) : mf::kEngineCPT;
}
int path_group_w(int path, int map_dtype) { return mf::kGroupStrips * 32 * path_cpt(path, map_dtype); }

// The 16-point path serves windows up to 16 points on widths divisible by
// its columns per lane; every other stream takes the 32-point path.
int stream_path(int width, int window, int map_dtype) {
  return window <= mf::kEngineWideNMAX && width % path_cpt(1, map_dtype) == 0 ? 1 : 0;
}

}  // namespace

struct mf_engine {
  mf_engine_desc d{};
  int device = 0;
  cudaStream_t st = nullptr, cap_st = nullptr;
  mf::EngineFork fork{};  // side stream and events of the concurrent map paths
  bool own_stream = false;
  std::vector<Slot> slots;
  SlotParams* slots_dev = nullptr;  // max_streams + 1 entries (the last: tuner)
  SlotParams* slots_pinned = nullptr;  // host staging of slot uploads (pinned)
  double* ring_pool = nullptr;       // pose histories of all slots (allocated at open)
  int32_t* bad_pool = nullptr;
  int64_t ring_cap = 0;              // poses per slot history
  FrameRec* recs = nullptr;
  unsigned int* sched = nullptr;  // map paths' work counters (kEnginePaths)
  size_t tab_bytes = 0;
  char* host_tab[2] = {nullptr, nullptr};
  char* dev_tab[2] = {nullptr, nullptr};
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraphNode_t copy_node[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  cudaEvent_t t0[2] = {nullptr, nullptr};
  int64_t buf_tick[2] = {-1, -1};
  mf::EngineGrids grids{};
  // the tick being assembled
  std::vector<TickPush> pushes;
  std::vector<TickFrame> frames;
  std::vector<double> poses;
  int64_t next_tick = 0;
  std::map<std::tuple<int, int, int>, int> tuned;  // (width, height, window bucket) -> band_h
  // statistics
  int64_t ticks = 0, frames_done = 0, units_done = 0, launches = 0, graph_launches = 0;
  int64_t frames_path_done[mf::kEnginePaths] = {};
  int64_t device_bytes = 0;
  double tick_ms = 0.0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending_timers;
  // latency accounting
  std::vector<int64_t> frame_submit_ns;          // the tick being assembled
  std::deque<std::unique_ptr<TickRecord>> in_flight;
  std::vector<double> latencies_ms;

  void* dalloc(size_t n) {
    void* p = nullptr;
    if (mf::fault_fires(mf::kFaultAllocFail)) return nullptr;
    if (cudaMalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    device_bytes += (int64_t)n;
    return p;
  }
  void dfree(void* p, size_t n) {
    if (!p) return;
    cudaFree(p);
    device_bytes -= (int64_t)n;
  }
  size_t poses_cap() const {
    return (size_t)d.max_tick_frames + (size_t)d.max_streams * (MF_MAX_HISTORY - 1);
  }
  int64_t accounted() const {
    int64_t a = device_bytes;
    for (const Slot& s : slots)
      if (s.used) a += s.reserve;
    return a;
  }
};

namespace {

size_t table_bytes(size_t frames, size_t pushes, size_t poses) {
  size_t off = align256(sizeof(TickHeader));
  off = align256(off + frames * sizeof(TickFrame));
  off = align256(off + frames * sizeof(int32_t));
  off = align256(off + pushes * sizeof(TickPush));
  return off + poses * 12 * sizeof(double);
}

// Numbers every frame's units within its map path and writes the tick (or a
// given frame list) into table `tab`; returns the bytes used.
size_t write_table(char* tab, std::vector<TickFrame>& frames, const std::vector<TickPush>& pushes,
                   const std::vector<double>& poses, int64_t* units_out) {
  TickHeader h{};
  std::vector<int32_t> order;
  order.reserve(frames.size());
  for (int p = 0; p < mf::kEnginePaths; ++p) {
    int64_t u = 0;
    int32_t nf = 0;
    for (size_t t = 0; t < frames.size(); ++t) {
      TickFrame& f = frames[t];
      if (f.path != p) continue;
      f.unit_begin = u;
      u += (int64_t)f.bands * f.groups_x;
      order.push_back((int32_t)t);
      ++nf;
    }
    h.n_units_path[p] = u;
    h.n_frames_path[p] = nf;
    h.n_units += u;
  }
  h.n_frames = (int32_t)frames.size();
  h.n_pushes = (int32_t)pushes.size();
  h.frames_off = (int64_t)align256(sizeof(TickHeader));
  h.order_off = (int64_t)align256(h.frames_off + frames.size() * sizeof(TickFrame));
  h.pushes_off = (int64_t)align256(h.order_off + frames.size() * sizeof(int32_t));
  h.poses_off = (int64_t)align256(h.pushes_off + pushes.size() * sizeof(TickPush));
  std::memcpy(tab, &h, sizeof(h));
  if (!frames.empty()) {
    std::memcpy(tab + h.frames_off, frames.data(), frames.size() * sizeof(TickFrame));
    std::memcpy(tab + h.order_off, order.data(), order.size() * sizeof(int32_t));
  }
  if (!pushes.empty()) std::memcpy(tab + h.pushes_off, pushes.data(), pushes.size() * sizeof(TickPush));
  if (!poses.empty()) std::memcpy(tab + h.poses_off, poses.data(), poses.size() * sizeof(double));
  if (units_out) *units_out = h.n_units;
  return (size_t)h.poses_off + poses.size() * sizeof(double);
}

mf::EngineKernelArgs kernel_args(mf_engine* e, int b) {
  mf::EngineKernelArgs a{};
  a.table = reinterpret_cast<const TickHeader*>(e->dev_tab[b]);
  a.slots = e->slots_dev;
  a.recs = e->recs;
  a.max_frames = e->d.max_tick_frames;
  a.sched = e->sched;
  a.fault = e->sched + mf::kEnginePaths;
  return a;
}

int build_graphs(mf_engine* e) {
  for (int b = 0; b < 2; ++b) {
    ENG_CUDA(cudaStreamBeginCapture(e->cap_st, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t c1 = cudaMemcpyAsync(e->dev_tab[b], e->host_tab[b], e->tab_bytes,
                                     cudaMemcpyHostToDevice, e->cap_st);
    int64_t dummy = 0;
    cudaError_t c2 = mf::launch_engine_tick(kernel_args(e, b), e->d.depth_dtype, e->d.map_dtype,
                                            e->grids, e->cap_st, e->fork, &dummy);
    cudaGraph_t g = nullptr;
    cudaError_t c3 = cudaStreamEndCapture(e->cap_st, &g);
    if (c1 != cudaSuccess || c2 != cudaSuccess || c3 != cudaSuccess)
      return fail(MF_ERR_CUDA, "tick graph capture", c1 != cudaSuccess ? c1 : (c2 != cudaSuccess ? c2 : c3));
    e->graph[b] = g;
    size_t n = 0;
    ENG_CUDA(cudaGraphGetNodes(g, nullptr, &n), "graph nodes");
    std::vector<cudaGraphNode_t> nodes(n);
    ENG_CUDA(cudaGraphGetNodes(g, nodes.data(), &n), "graph nodes");
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType t;
      ENG_CUDA(cudaGraphNodeGetType(nd, &t), "graph node type");
      if (t == cudaGraphNodeTypeMemcpy) e->copy_node[b] = nd;
    }
    if (!e->copy_node[b]) return fail(MF_ERR_CUDA, "tick graph has no copy node");
    ENG_CUDA(cudaGraphInstantiate(&e->exec[b], g, 0), "graph instantiate");
  }
  return MF_OK;
}

void destroy(mf_engine* e) {
  if (e->st) cudaStreamSynchronize(e->st);
  for (auto& t : e->pending_timers) {
    cudaEventDestroy(t.first);
    cudaEventDestroy(t.second);
  }
  e->dfree(e->ring_pool, (size_t)e->d.max_streams * e->ring_cap * 12 * sizeof(double));
  e->dfree(e->bad_pool, (size_t)e->d.max_streams * e->ring_cap * sizeof(int32_t));
  if (e->slots_pinned) cudaFreeHost(e->slots_pinned);
  for (int b = 0; b < 2; ++b) {
    if (e->exec[b]) cudaGraphExecDestroy(e->exec[b]);
    if (e->graph[b]) cudaGraphDestroy(e->graph[b]);
    if (e->host_tab[b]) cudaFreeHost(e->host_tab[b]);
    e->dfree(e->dev_tab[b], e->tab_bytes);
    if (e->done[b]) cudaEventDestroy(e->done[b]);
    if (e->t0[b]) cudaEventDestroy(e->t0[b]);
  }
  e->dfree(e->recs, (size_t)e->d.max_tick_frames * sizeof(FrameRec));
  e->dfree(e->sched, (mf::kEnginePaths + 1) * sizeof(unsigned int));
  e->dfree(e->slots_dev, (size_t)(e->d.max_streams + 1) * sizeof(SlotParams));
  if (e->cap_st) cudaStreamDestroy(e->cap_st);
  if (e->fork.side) {
    cudaStreamSynchronize(e->fork.side);
    cudaStreamDestroy(e->fork.side);
  }
  if (e->fork.fork) cudaEventDestroy(e->fork.fork);
  if (e->fork.join) cudaEventDestroy(e->fork.join);
  if (e->own_stream && e->st) cudaStreamDestroy(e->st);
  delete e;
}

int wait_event(cudaEvent_t ev, int64_t timeout_ns) {
  const auto t0 = std::chrono::steady_clock::now();
  int spins = 0;
  for (;;) {
    const cudaError_t q = cudaEventQuery(ev);
    if (q == cudaSuccess) return MF_OK;
    if (q != cudaErrorNotReady) return fail(MF_ERR_CUDA, "event query", q);
    if (timeout_ns >= 0 &&
        std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0)
                .count() > timeout_ns)
      return fail(MF_ERR_TIMEOUT, "tick wait timed out");
    if (++spins > 64)
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    else
      std::this_thread::yield();
  }
}

// Waits until tick `t` and every earlier tick finished (ticks run in order).
int wait_tick(mf_engine* e, int64_t t, int64_t timeout_ns) {
  if (t < 0 || t >= e->next_tick) return MF_OK;
  const int b = (int)(t & 1);
  if (e->buf_tick[b] != t) return MF_OK;  // buffer reused: tick t finished earlier
  const int rc = wait_event(e->done[b], timeout_ns);
  if (rc || !mf::kChecked) return rc;
  // checked builds: an access outside a plane was caught and skipped
  unsigned int f = 0u;
  ENG_CUDA(cudaMemcpy(&f, e->sched + mf::kEnginePaths, sizeof(f), cudaMemcpyDeviceToHost), "fault word");
  if (f == 0u) return MF_OK;
  ENG_CUDA(cudaMemset(e->sched + mf::kEnginePaths, 0, sizeof(f)), "fault word");
  return fail(MF_ERR_CUDA, "checked build: an index outside its plane was caught (access skipped)");
}

int collect_timers(mf_engine* e) {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> keep;
  for (auto& t : e->pending_timers) {
    ENG_CUDA(cudaEventSynchronize(t.second), "timer sync");
    float ms = 0.0f;
    ENG_CUDA(cudaEventElapsedTime(&ms, t.first, t.second), "timer elapsed");
    e->tick_ms += ms;
    cudaEventDestroy(t.first);
    cudaEventDestroy(t.second);
  }
  e->pending_timers.clear();
  return MF_OK;
}

void fill_slot_params(const Slot& s, const double* w, SlotParams* out) {
  std::memset(out, 0, sizeof(*out));
  out->ring = s.ring;
  out->ring_bad = s.ring_bad;
  out->ring_mask = s.ring_cap - 1;
  out->fp.window = s.d.window;
  out->fp.smooth_len = s.d.smooth_len;
  out->fp.width = s.d.width;
  out->fp.height = s.d.height;
  out->fp.calib_width = s.d.calib_width;
  out->fp.calib_height = s.d.calib_height;
  out->fp.sigma_rel = s.d.sigma_rel;
  out->fp.s_lo = s.d.s_lo;
  out->fp.s_hi = s.d.s_hi;
  out->d0 = (float)s.d.depth_ref_m;
  out->fp.d0 = out->d0;
  out->fp.depth_scale = 1.0f;
  for (int k = 0; k < mf::kMaxHist; ++k) out->w[k] = k < s.d.smooth_len ? w[k] : 0.0;
}

// Candidate tile heights for a frame height: divisions of the height into
// equal bands no taller than each nominal value.
std::vector<int> band_candidates(int height) {
  std::vector<int> out;
  for (int nominal : {32, 64, 96, 128, 192, 256}) {
    const int bands = (height + nominal - 1) / nominal;
    const int bh = (height + bands - 1) / bands;
    if (std::find(out.begin(), out.end(), bh) == out.end()) out.push_back(bh);
  }
  return out;
}

// Tuning classes: resolution and the window rounded up to 8, 16 or 32 points.
int window_bucket(int window) { return window <= 8 ? 8 : (window <= 16 ? 16 : 32); }

int tune_class(mf_engine* e, int width, int height, int window, int* band_out) {
  window = window_bucket(window);
  const auto key = std::make_tuple(width, height, window);
  auto it = e->tuned.find(key);
  if (it != e->tuned.end()) {
    *band_out = it->second;
    return MF_OK;
  }
  ENG_CUDA(cudaStreamSynchronize(e->st), "stream sync before tuning");
  const size_t px = (size_t)width * height;
  const size_t per_frame = px * (dtype_bytes(e->d.depth_dtype) + 2 * dtype_bytes(e->d.map_dtype));
  int frames = (int)std::max<size_t>(2, std::min<size_t>(64, ((size_t)4 << 30) / per_frame));
  frames = std::min(frames, e->d.max_tick_frames);
  char* buf = (char*)e->dalloc(per_frame * frames);
  if (!buf) return fail(MF_ERR_OOM, "tuning buffers");
  ENG_CUDA(cudaMemsetAsync(buf, 0, per_frame * frames, e->st), "tuning memset");
  // synthetic worst case: `window` points spread inside the frame
  std::vector<FrameRec> recs(frames);
  const double fx = 0.9 * width;
  for (int f = 0; f < frames; ++f) {
    FrameRec& r = recs[f];
    std::memset(&r, 0, sizeof(r));
    const int n = std::min(window, (int)mf::kMaxPts);
    r.n_valid = n;
    r.inv_n = (float)(1.0 / n);
    for (int i = 0; i < n; ++i) {
      const double fu = std::fmod(0.1 + 0.618034 * (i + 3 * f), 1.0);
      const double fv = std::fmod(0.2 + 0.414214 * (i + 5 * f), 1.0);
      const double sig = 0.1 * fx * (0.5 + fu);
      r.ux_hi[i] = (float)(width * (0.1 + 0.8 * fu));
      r.vy_hi[i] = (float)(height * (0.1 + 0.8 * fv));
      const double c = 1.4426950408889634 / (2.0 * sig * sig);  // log2(e) / (2 sigma^2)
      r.c_hi[i] = (float)c;
      r.c_lo[i] = (float)(c - (double)(float)c);
    }
  }
  ENG_CUDA(cudaMemcpyAsync(e->recs, recs.data(), sizeof(FrameRec) * frames, cudaMemcpyHostToDevice, e->st),
           "tuning records");
  Slot tmp;
  tmp.d.width = width;
  tmp.d.height = height;
  tmp.d.window = window;
  tmp.d.depth_ref_m = 1.0;
  SlotParams sp;
  double w[mf::kMaxHist] = {};
  fill_slot_params(tmp, w, &sp);
  ENG_CUDA(cudaMemcpyAsync(e->slots_dev + e->d.max_streams, &sp, sizeof(sp), cudaMemcpyHostToDevice, e->st),
           "tuning slot");
  const size_t pin = per_frame / (dtype_bytes(e->d.depth_dtype) + 2 * dtype_bytes(e->d.map_dtype));
  cudaEvent_t a, b2;
  ENG_CUDA(cudaEventCreate(&a), "event");
  ENG_CUDA(cudaEventCreate(&b2), "event");
  int best_band = default_band(height);
  float best_ms = 1e30f;
  std::vector<TickPush> pushes(1);
  pushes[0].slot = e->d.max_streams;
  std::vector<double> no_poses;
  const int path = stream_path(width, window, e->d.map_dtype);
  // A candidate's cost is the time of all `frames` synthetic frames minus
  // the time of the first half: the marginal time of a frame, without the
  // launch's partly filled last wave of units (with few frames of one class
  // that tail makes tall bands look slower than in a tick of many streams).
  auto time_frames = [&](int bh, int nf, float* ms) -> int {
    std::vector<TickFrame> frs(nf);
    for (int f = 0; f < nf; ++f) {
      TickFrame& t = frs[f];
      std::memset(&t, 0, sizeof(t));
      t.push = 0;
      t.k = f;
      t.bucket = window;
      t.path = path;
      t.band_h = bh;
      t.bands = (height + bh - 1) / bh;
      t.groups_x = (width + path_group_w(path, e->d.map_dtype) - 1) / path_group_w(path, e->d.map_dtype);
      char* base = buf + (size_t)f * per_frame;
      t.depth = base;
      t.M = base + pin * dtype_bytes(e->d.depth_dtype);
      t.G = t.M + pin * dtype_bytes(e->d.map_dtype);
      t.info = nullptr;
    }
    const size_t used = write_table(e->host_tab[0], frs, pushes, no_poses, nullptr);
    ENG_CUDA(cudaMemcpyAsync(e->dev_tab[0], e->host_tab[0], used, cudaMemcpyHostToDevice, e->st), "table");
    const mf::EngineKernelArgs args = kernel_args(e, 0);
    ENG_CUDA(mf::launch_engine_map_only(args, e->d.depth_dtype, e->d.map_dtype, e->grids, e->st), "tune");
    ENG_CUDA(cudaEventRecord(a, e->st), "event");
    for (int rep = 0; rep < 3; ++rep)
      ENG_CUDA(mf::launch_engine_map_only(args, e->d.depth_dtype, e->d.map_dtype, e->grids, e->st), "tune");
    ENG_CUDA(cudaEventRecord(b2, e->st), "event");
    ENG_CUDA(cudaEventSynchronize(b2), "event");
    ENG_CUDA(cudaEventElapsedTime(ms, a, b2), "elapsed");
    e->launches += 4 * mf::kEnginePaths;
    return MF_OK;
  };
  for (int bh : band_candidates(height)) {
    float all = 0.0f, half = 0.0f;
    int rc2 = time_frames(bh, frames, &all);
    if (rc2 == MF_OK) rc2 = time_frames(bh, frames / 2, &half);
    if (rc2 != MF_OK) {
      cudaEventDestroy(a);
      cudaEventDestroy(b2);
      e->dfree(buf, per_frame * frames);
      return rc2;
    }
    const float ms = all - half;
    if (ms < best_ms) {
      best_ms = ms;
      best_band = bh;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b2);
  ENG_CUDA(cudaStreamSynchronize(e->st), "stream sync after tuning");
  e->dfree(buf, per_frame * frames);
  e->buf_tick[0] = -1;  // the table buffer held tuning data
  e->tuned[key] = best_band;
  *band_out = best_band;
  return MF_OK;
}

// Moves the latencies of finished ticks (in order) into the window.
void collect_latencies(mf_engine* e) {
  while (!e->in_flight.empty()) {
    TickRecord* r = e->in_flight.front().get();
    const int64_t done = r->done_ns.load(std::memory_order_acquire);
    if (!done) break;
    for (int64_t t : r->submit_ns) e->latencies_ms.push_back((double)(done - t) * 1e-6);
    e->in_flight.pop_front();
  }
}

}  // namespace

extern "C" {

void mf_engine_desc_init(mf_engine_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->max_streams = 256;
  d->max_tick_frames = 4096;
  d->max_stream_frames = 64;
  d->depth_dtype = MF_F32;
  d->map_dtype = MF_F32;
}

int mf_engine_open(const mf_engine_desc* d, mf_engine** out) {
  if (!out || !d) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (d->max_streams < 1 || d->max_streams > 65536 || d->max_tick_frames < 1 ||
      d->max_tick_frames > (1 << 20) || d->max_stream_frames < 1 ||
      d->max_stream_frames > d->max_tick_frames || d->memory_budget < 0)
    return fail(MF_ERR_INVALID_ARG, "engine limits out of range");
  for (int dt : {d->depth_dtype, d->map_dtype})
    if (dt != MF_F32 && dt != MF_BF16 && dt != MF_F16) return fail(MF_ERR_INVALID_ARG, "unknown dtype");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(MF_ERR_NO_DEVICE, "no CUDA device");
  }
  mf_engine* e = new (std::nothrow) mf_engine();
  if (!e) return fail(MF_ERR_OOM, "host allocation");
  e->d = *d;
  cudaGetDevice(&e->device);
  e->slots.resize(d->max_streams);
  if (d->cuda_stream) {
    e->st = (cudaStream_t)d->cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete e;
      return fail(MF_ERR_CUDA, "stream creation");
    }
    e->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&e->cap_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&e->fork.side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->fork.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->fork.join, cudaEventDisableTiming) != cudaSuccess) {
    destroy(e);
    return fail(MF_ERR_CUDA, "stream or event creation");
  }
  e->slots_dev = (SlotParams*)e->dalloc((size_t)(d->max_streams + 1) * sizeof(SlotParams));
  // every slot's pose history is allocated now, so admission never allocates
  e->ring_cap = pow2_at_least(std::max<int64_t>(128, MF_MAX_HISTORY - 1 + d->max_stream_frames));
  e->ring_pool = (double*)e->dalloc((size_t)d->max_streams * e->ring_cap * 12 * sizeof(double));
  e->bad_pool = (int32_t*)e->dalloc((size_t)d->max_streams * e->ring_cap * sizeof(int32_t));
  if (cudaMallocHost(&e->slots_pinned, (size_t)(d->max_streams + 1) * sizeof(SlotParams)) != cudaSuccess) {
    cudaGetLastError();
    e->slots_pinned = nullptr;
  }
  e->recs = (FrameRec*)e->dalloc((size_t)d->max_tick_frames * sizeof(FrameRec));
  // the map paths' work counters, then the fault word of checked builds
  e->sched = (unsigned int*)e->dalloc((mf::kEnginePaths + 1) * sizeof(unsigned int));
  if (e->sched &&
      cudaMemsetAsync(e->sched, 0, (mf::kEnginePaths + 1) * sizeof(unsigned int), e->st) != cudaSuccess) {
    cudaGetLastError();
    e->dfree(e->sched, (mf::kEnginePaths + 1) * sizeof(unsigned int));
    e->sched = nullptr;
  }
  e->tab_bytes = table_bytes(d->max_tick_frames, d->max_streams, e->poses_cap());
  for (int b = 0; b < 2; ++b) {
    e->dev_tab[b] = (char*)e->dalloc(e->tab_bytes);
    if (cudaMallocHost(&e->host_tab[b], e->tab_bytes) != cudaSuccess) {
      cudaGetLastError();
      e->host_tab[b] = nullptr;
    }
    if (cudaEventCreateWithFlags(&e->done[b], cudaEventDisableTiming) != cudaSuccess) e->done[b] = nullptr;
  }
  if (!e->slots_dev || !e->ring_pool || !e->bad_pool || !e->slots_pinned || !e->recs || !e->sched ||
      !e->dev_tab[0] || !e->dev_tab[1] || !e->host_tab[0] ||
      !e->host_tab[1] || !e->done[0] || !e->done[1]) {
    destroy(e);
    return fail(MF_ERR_OOM, "engine allocation");
  }
  if (d->memory_budget > 0 && e->device_bytes > d->memory_budget) {
    destroy(e);
    return fail(MF_ERR_ADMISSION, "engine tables exceed the memory budget");
  }
  e->grids = mf::engine_map_grids(d->depth_dtype, d->map_dtype);
  // an empty table in both buffers, so a graph replay with nothing to do is harmless
  for (int b = 0; b < 2; ++b) {
    std::vector<TickFrame> nf;
    std::vector<TickPush> np;
    std::vector<double> npo;
    const size_t used = write_table(e->host_tab[b], nf, np, npo, nullptr);
    if (cudaMemcpy(e->dev_tab[b], e->host_tab[b], used, cudaMemcpyHostToDevice) != cudaSuccess) {
      destroy(e);
      return fail(MF_ERR_CUDA, "table init");
    }
  }
  if (!(d->flags & MF_ENGINE_NO_GRAPH)) {
    const int rc = build_graphs(e);
    if (rc) {
      destroy(e);
      return rc;
    }
  }
  *out = e;
  return MF_OK;
}

int mf_engine_add_stream(mf_engine* e, const mf_stream_desc* d, int64_t reserve_bytes, int32_t* slot) {
  if (!e || !d || !slot) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  *slot = -1;
  int rc = mf::host_validate_desc(d);
  if (rc) return rc;
  if (d->depth_dtype != e->d.depth_dtype || d->map_dtype != e->d.map_dtype)
    return fail(MF_ERR_INVALID_ARG, "stream dtypes differ from the engine's");
  if (reserve_bytes < 0) return fail(MF_ERR_INVALID_ARG, "negative reservation");
  if (d->width % mf::kEngineCPT) return fail(MF_ERR_INVALID_ARG, "engine streams need an even width");
  if (d->normalize != MF_NORM_COUNT)
    return fail(MF_ERR_INVALID_ARG, "engine streams use Z = number of valid points");
  int free_slot = -1;
  for (int i = 0; i < e->d.max_streams; ++i)
    if (!e->slots[i].used) {
      free_slot = i;
      break;
    }
  if (d->flags & MF_FLAG_DEPTH_ALIGN)
    return fail(MF_ERR_INVALID_ARG, "depth alignment runs on mf_stream only, not in the engine");
  if (free_slot < 0) return fail(MF_ERR_ADMISSION, "every stream slot is taken");
  if (mf::fault_fires(mf::kFaultAdmissionFull))
    return fail(MF_ERR_ADMISSION, "admission refused (injected fault)");
  // the slot's history is part of the engine's memory already; the budget
  // admits the caller's reservation on top of it
  if (e->d.memory_budget > 0 && e->accounted() + reserve_bytes > e->d.memory_budget)
    return fail(MF_ERR_ADMISSION, "device memory budget exhausted");
  double w[mf::kMaxHist] = {};
  if (!mf::host_ls_weights(d->smooth_len, d->mode, w))
    return fail(MF_ERR_INVALID_ARG, "least-squares weights not representable");
  DeviceGuard guard(e->device);
  int band = default_band(d->height);
  if (!(e->d.flags & MF_ENGINE_NO_TUNE)) {
    rc = tune_class(e, d->width, d->height, std::min(d->window, (int)mf::kMaxPts), &band);
    if (rc) return rc;
  }
  Slot& s = e->slots[free_slot];
  s = Slot();
  s.d = *d;
  s.ring_cap = e->ring_cap;
  s.ring = e->ring_pool + (size_t)free_slot * e->ring_cap * 12;
  s.ring_bad = e->bad_pool + (size_t)free_slot * e->ring_cap;
  s.reserve = reserve_bytes;
  s.plane_in = (size_t)d->width * d->height * dtype_bytes(d->depth_dtype);
  s.plane_out = (size_t)d->width * d->height * dtype_bytes(d->map_dtype);
  s.path = stream_path(d->width, std::min(d->window, (int)mf::kMaxPts), e->d.map_dtype);
  s.band_h = band;
  s.bands = (d->height + band - 1) / band;
  s.groups_x = (d->width + path_group_w(s.path, e->d.map_dtype) - 1) / path_group_w(s.path, e->d.map_dtype);
  // stream-ordered upload from pinned staging: earlier ticks never read this
  // slot (it was free), later ticks see it; nothing waits
  fill_slot_params(s, w, e->slots_pinned + free_slot);
  ENG_CUDA(cudaMemcpyAsync(e->slots_dev + free_slot, e->slots_pinned + free_slot, sizeof(SlotParams),
                           cudaMemcpyHostToDevice, e->st),
           "slot upload");
  s.used = true;
  *slot = free_slot;
  return MF_OK;
}

int mf_engine_remove_stream(mf_engine* e, int32_t slot) {
  if (!e || slot < 0 || slot >= e->d.max_streams || !e->slots[slot].used)
    return fail(MF_ERR_INVALID_ARG, "no such stream");
  Slot& s = e->slots[slot];
  if (s.pending_tick == e->next_tick) return fail(MF_ERR_INVALID_ARG, "the stream has a queued push");
  DeviceGuard guard(e->device);
  // the slot's pinned staging and history may be reused by the next
  // admission only once the ticks that used them are done
  int rc = wait_tick(e, s.last_tick, -1);
  if (rc) return rc;
  s = Slot();
  return MF_OK;
}

int mf_engine_submit(mf_engine* e, int32_t slot, int32_t n, const double* poses, const void* depth,
                     const double* K, void* focus_map, void* guided_depth, mf_frame_info* info) {
  return mf::engine_submit_at(e, slot, n, poses, depth, K, focus_map, guided_depth, info, now_ns());
}

}  // extern "C"

int mf::engine_submit_at(mf_engine* e, int32_t slot, int32_t n, const double* poses,
                         const void* depth, const double* K, void* focus_map, void* guided_depth,
                         mf_frame_info* info, int64_t t_sub) {
  if (!e || slot < 0 || slot >= e->d.max_streams || !e->slots[slot].used)
    return fail(MF_ERR_INVALID_ARG, "no such stream");
  Slot& s = e->slots[slot];
  if (n < 1 || !poses || !K) return fail(MF_ERR_INVALID_ARG, "n < 1 or NULL poses/K");
  if (s.pending_tick == e->next_tick) return fail(MF_ERR_NOT_READY, "the stream already has a push in this tick");
  const bool local = s.d.pose_frame == MF_POSES_BATCH_LOCAL;
  const int O = (local && s.pushes > 0) ? s.d.overlap : 0;
  if (n <= O) return fail(MF_ERR_INVALID_ARG, "batch must hold more frames than the overlap");
  const int n_emit = n - O;
  if (n_emit > e->d.max_stream_frames) return fail(MF_ERR_INVALID_ARG, "push exceeds max_stream_frames");
  if ((int64_t)e->frames.size() + n_emit > e->d.max_tick_frames)
    return fail(MF_ERR_NOT_READY, "the tick is full: call mf_engine_tick");
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(K[k])) return fail(MF_ERR_INVALID_ARG, "non-finite intrinsics");
  if (!(K[0] > 0.0) || !(K[1] > 0.0)) return fail(MF_ERR_INVALID_ARG, "fx, fy must be > 0");
  DeviceGuard guard(e->device);
  if (mf::host_pointer_kind(poses, e->device) != mf::kPtrHost)
    return fail(MF_ERR_INVALID_ARG, "engine poses must be host memory");
  for (const void* p : {depth, (const void*)focus_map, (const void*)guided_depth, (const void*)info})
    if (p && mf::host_pointer_kind(p, e->device) != mf::kPtrDevice)
      return fail(MF_ERR_INVALID_ARG, "engine planes and records must be device memory of the engine's GPU");
  // two pixels per lane access: planes aligned to two elements
  if ((depth && (uintptr_t)depth % (2 * dtype_bytes(e->d.depth_dtype))) ||
      (focus_map && (uintptr_t)focus_map % (2 * dtype_bytes(e->d.map_dtype))) ||
      (guided_depth && (uintptr_t)guided_depth % (2 * dtype_bytes(e->d.map_dtype))) ||
      (info && (uintptr_t)info % 8))
    return fail(MF_ERR_INVALID_ARG, "misaligned plane or record pointer");
  // the 16-point path reads and writes path_cpt(1) elements at a time; a
  // push whose planes are not aligned to that runs on the 32-point path
  int path = s.path, band_h = s.band_h, bands = s.bands, groups_x = s.groups_x;
  const size_t wc = (size_t)path_cpt(1, e->d.map_dtype);
  if (path == 1 &&
      ((depth && (uintptr_t)depth % (wc * dtype_bytes(e->d.depth_dtype))) ||
       (focus_map && (uintptr_t)focus_map % (wc * dtype_bytes(e->d.map_dtype))) ||
       (guided_depth && (uintptr_t)guided_depth % (wc * dtype_bytes(e->d.map_dtype))))) {
    path = 0;
    band_h = default_band(s.d.height);
    bands = (s.d.height + band_h - 1) / band_h;
    groups_x = (s.d.width + path_group_w(0, e->d.map_dtype) - 1) / path_group_w(0, e->d.map_dtype);
  }
  TickPush ps{};
  ps.slot = slot;
  ps.n = n;
  ps.first = O;
  ps.anchor = O > 0 ? 1 : 0;
  ps.e0 = s.emitted;
  ps.pose_off = (int64_t)(e->poses.size() / 12);
  for (int k = 0; k < 4; ++k) ps.K[k] = K[k];
  const int push_idx = (int)e->pushes.size();
  e->pushes.push_back(ps);
  e->poses.insert(e->poses.end(), poses, poses + (size_t)n * 12);
  for (int k = 0; k < n_emit; ++k) {
    TickFrame t{};
    t.push = push_idx;
    t.k = k;
    t.bucket = s.d.window;
    t.path = path;
    t.band_h = band_h;
    t.bands = bands;
    t.groups_x = groups_x;
    t.depth = depth ? static_cast<const char*>(depth) + (size_t)(O + k) * s.plane_in : nullptr;
    t.M = focus_map ? static_cast<char*>(focus_map) + (size_t)k * s.plane_out : nullptr;
    t.G = guided_depth ? static_cast<char*>(guided_depth) + (size_t)k * s.plane_out : nullptr;
    t.info = info ? info + k : nullptr;
    e->frames.push_back(t);
  }
  e->frame_submit_ns.insert(e->frame_submit_ns.end(), (size_t)n_emit, t_sub);
  s.emitted += n_emit;
  ++s.pushes;
  s.pending_tick = e->next_tick;
  s.last_tick = e->next_tick;
  return MF_OK;
}

extern "C" {

int64_t mf_clock_ns(void) { return now_ns(); }

int mf_engine_submit_batch(mf_engine* e, int32_t n, const mf_push* pushes, int32_t* accepted) {
  if (!e || (n > 0 && !pushes) || !accepted || n < 0) return fail(MF_ERR_INVALID_ARG, "bad batch");
  *accepted = 0;
  for (int32_t i = 0; i < n; ++i) {
    const mf_push& p = pushes[i];
    const int rc = mf::engine_submit_at(e, p.slot, p.n, p.poses_w2c_3x4, p.depth, p.K, p.focus_map,
                                        p.guided_depth, p.info, p.arrival_ns ? p.arrival_ns : now_ns());
    if (rc) return rc;
    ++*accepted;
  }
  return MF_OK;
}

int mf_engine_tick(mf_engine* e, int64_t* tick) {
  mf::NvtxRange range("mf_engine_tick");
  if (!e || !tick) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  *tick = -1;
  if (e->frames.empty()) return MF_OK;
  DeviceGuard guard(e->device);
  const int64_t t = e->next_tick;
  const int b = (int)(t & 1);
  // the buffer's previous tick must have consumed its table
  if (e->buf_tick[b] >= 0) {
    const int rc = wait_event(e->done[b], -1);
    if (rc) return rc;
  }
  int64_t units = 0;
  const size_t used = write_table(e->host_tab[b], e->frames, e->pushes, e->poses, &units);
  cudaEvent_t ta = nullptr, tb = nullptr;
  if (e->d.flags & MF_FLAG_TIME_KERNELS) {
    ENG_CUDA(cudaEventCreate(&ta), "event");
    ENG_CUDA(cudaEventCreate(&tb), "event");
    ENG_CUDA(cudaEventRecord(ta, e->st), "event");
  }
  if (e->exec[b]) {
    ENG_CUDA(cudaGraphExecMemcpyNodeSetParams1D(e->exec[b], e->copy_node[b], e->dev_tab[b],
                                                e->host_tab[b], used, cudaMemcpyHostToDevice),
             "graph copy update");
    ENG_CUDA(cudaGraphLaunch(e->exec[b], e->st), "graph launch");
    ++e->graph_launches;
    e->launches += mf::kEngineTickLaunches;
  } else {
    ENG_CUDA(cudaMemcpyAsync(e->dev_tab[b], e->host_tab[b], used, cudaMemcpyHostToDevice, e->st), "table");
    ENG_CUDA(mf::launch_engine_tick(kernel_args(e, b), e->d.depth_dtype, e->d.map_dtype, e->grids,
                                    e->st, e->fork, &e->launches),
             "tick launch");
  }
  mf::host_count_launches(mf::kEngineTickLaunches);
  if (ta) {
    ENG_CUDA(cudaEventRecord(tb, e->st), "event");
    e->pending_timers.emplace_back(ta, tb);
  }
  {
    std::unique_ptr<TickRecord> rec(new TickRecord());
    rec->submit_ns.swap(e->frame_submit_ns);
    ENG_CUDA(cudaLaunchHostFunc(e->st, stamp_tick_done, rec.get()), "tick completion stamp");
    e->in_flight.push_back(std::move(rec));
  }
  // recorded after the stamp: a tick that waits report as done has its
  // completion time stamped too
  ENG_CUDA(cudaEventRecord(e->done[b], e->st), "event");
  e->frame_submit_ns.clear();
  e->buf_tick[b] = t;
  ++e->ticks;
  e->frames_done += (int64_t)e->frames.size();
  for (const TickFrame& f : e->frames) ++e->frames_path_done[f.path];
  e->units_done += units;
  e->frames.clear();
  e->pushes.clear();
  e->poses.clear();
  e->next_tick = t + 1;
  *tick = t;
  return MF_OK;
}

int mf_engine_query(mf_engine* e, int64_t tick, int32_t* done) {
  if (!e || !done) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  *done = 1;
  if (tick < 0 || tick >= e->next_tick) return MF_OK;
  const int b = (int)(tick & 1);
  if (e->buf_tick[b] != tick) return MF_OK;
  DeviceGuard guard(e->device);
  const cudaError_t q = cudaEventQuery(e->done[b]);
  if (q == cudaErrorNotReady) {
    *done = 0;
    return MF_OK;
  }
  if (q != cudaSuccess) return fail(MF_ERR_CUDA, "event query", q);
  return MF_OK;
}

int mf_engine_wait(mf_engine* e, int64_t tick, int64_t timeout_ns) {
  if (!e) return fail(MF_ERR_INVALID_ARG, "NULL engine");
  DeviceGuard guard(e->device);
  return wait_tick(e, tick, timeout_ns);
}

int mf_engine_tune(mf_engine* e, int32_t width, int32_t height, int32_t window, int32_t* band_h) {
  if (!e || !band_h || width < 1 || height < 1 || width > MF_MAX_DIM || height > MF_MAX_DIM ||
      window < 1 || window > MF_MAX_WINDOW)
    return fail(MF_ERR_INVALID_ARG, "bad tuning request");
  if (!e->frames.empty()) return fail(MF_ERR_NOT_READY, "a tick is being assembled");
  DeviceGuard guard(e->device);
  e->tuned.erase(std::make_tuple(width, height, window_bucket(window)));
  return tune_class(e, width, height, window, band_h);
}

int mf_engine_get_stats(mf_engine* e, mf_engine_stats* out) {
  if (!e || !out) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard guard(e->device);
  int rc = collect_timers(e);
  if (rc) return rc;
  std::memset(out, 0, sizeof(*out));
  out->ticks = e->ticks;
  out->frames = e->frames_done;
  out->units = e->units_done;
  out->kernel_launches = e->launches;
  out->graph_launches = e->graph_launches;
  int n = 0;
  for (const Slot& s : e->slots) n += s.used ? 1 : 0;
  out->streams = n;
  out->device_bytes = e->device_bytes;
  out->accounted_bytes = e->accounted();
  out->tick_gpu_ms = e->tick_ms;
  for (int p = 0; p < mf::kEnginePaths; ++p) out->frames_path[p] = e->frames_path_done[p];
  return MF_OK;
}

int mf_engine_latency(mf_engine* e, mf_latency_stats* out, int32_t reset) {
  if (!e || !out) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  collect_latencies(e);
  mf::latency_summary(e->latencies_ms, out);
  if (reset) e->latencies_ms.clear();
  return MF_OK;
}

int mf_engine_close(mf_engine* e) {
  if (!e) return MF_OK;
  DeviceGuard guard(e->device);
  destroy(e);
  return MF_OK;
}

}  // extern "C"
