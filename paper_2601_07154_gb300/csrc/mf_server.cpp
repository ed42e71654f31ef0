// Serving loop (include/mf.h, "Serving loop"): continuous batching of the
// pushes of many live streams over one engine.  Clients queue pushes from any
// thread; one background thread owns the engine's tick path: it gathers the
// oldest queued push of every stream (waiting at most tick_us for more work),
// submits them with their clients' submit times, launches the tick and
// retires finished ticks, without waiting for a tick to finish before the
// next one is assembled (the engine keeps two in flight).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "mf_engine_internal.h"

namespace {

int fail(int st, const char* what) { return mf::host_fail(st, what, cudaSuccess); }

struct QueuedPush {
  int32_t n = 0, n_emit = 0;
  std::vector<double> poses;
  const void* depth = nullptr;
  double K[4] = {0, 0, 0, 0};
  void* M = nullptr;
  void* G = nullptr;
  mf_frame_info* info = nullptr;
  int64_t t_submit = 0;
};

struct ServerSlot {
  bool used = false;
  bool local = false;
  int32_t overlap = 0;
  int64_t pushes = 0;             // pushes accepted (for the overlap rule)
  std::deque<QueuedPush> queue;
  int64_t frames_submitted = 0;   // frames accepted
  int64_t frames_done = 0;        // frames whose tick finished
};

struct InFlight {
  int64_t tick;
  std::vector<std::pair<int32_t, int32_t>> frames;  // (slot, frames)
};

}  // namespace

struct mf_server {
  mf_server_desc d{};
  mf_engine* eng = nullptr;
  std::mutex mu;                 // queues, counters
  std::mutex emu;                // engine calls
  std::condition_variable cv;
  std::thread th;
  bool stop = false;
  int err = MF_OK;
  std::vector<ServerSlot> slots;
  std::deque<InFlight> flight;
  int64_t queued = 0;            // pushes waiting in queues
  int32_t rr = 0;                // first slot scanned by the next tick
};

namespace {

void retire(mf_server* s) {  // caller holds mu and emu
  while (!s->flight.empty()) {
    int32_t done = 0;
    if (mf_engine_query(s->eng, s->flight.front().tick, &done) != MF_OK || !done) break;
    for (auto& sf : s->flight.front().frames) s->slots[sf.first].frames_done += sf.second;
    s->flight.pop_front();
  }
}

void run(mf_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  std::vector<std::pair<int32_t, QueuedPush>> batch;
  while (!s->stop) {
    {
      std::lock_guard<std::mutex> eg(s->emu);
      retire(s);
    }
    s->cv.notify_all();
    if (s->queued == 0) {
      s->cv.wait_for(lk, std::chrono::microseconds(s->flight.empty() ? 2000 : 50));
      continue;
    }
    // gather for at most tick_us after the oldest queued push arrived
    int64_t oldest = INT64_MAX;
    for (const ServerSlot& sl : s->slots)
      if (sl.used && !sl.queue.empty()) oldest = std::min(oldest, sl.queue.front().t_submit);
    const int64_t waited = mf::engine_now_ns() - oldest;
    const int64_t limit = (int64_t)s->d.tick_us * 1000;
    if (waited < limit) {
      s->cv.wait_for(lk, std::chrono::nanoseconds(limit - waited));
      continue;
    }
    // one push per stream per tick, within the tick's frame capacity
    batch.clear();
    int64_t frames = 0;
    const int32_t ns = (int32_t)s->slots.size();
    for (int32_t j = 0; j < ns; ++j) {  // round robin, so a full tick favours no slot
      const int32_t i = (s->rr + j) % ns;
      ServerSlot& sl = s->slots[i];
      if (!sl.used || sl.queue.empty()) continue;
      if (frames + sl.queue.front().n_emit > s->d.engine.max_tick_frames) continue;
      frames += sl.queue.front().n_emit;
      batch.emplace_back(i, std::move(sl.queue.front()));
      sl.queue.pop_front();
      --s->queued;
    }
    s->rr = (s->rr + 1) % ns;
    lk.unlock();
    InFlight fl;
    {
      std::lock_guard<std::mutex> eg(s->emu);
      for (auto& bp : batch) {
        QueuedPush& q = bp.second;
        const int rc = mf::engine_submit_at(s->eng, bp.first, q.n, q.poses.data(), q.depth, q.K, q.M,
                                            q.G, q.info, q.t_submit);
        if (rc == MF_OK)
          fl.frames.emplace_back(bp.first, q.n_emit);
        else
          s->err = rc;
      }
      int64_t tick = -1;
      const int rc = mf_engine_tick(s->eng, &tick);
      if (rc != MF_OK) s->err = rc;
      fl.tick = tick;
    }
    lk.lock();
    if (fl.tick >= 0) s->flight.push_back(std::move(fl));
  }
}

}  // namespace

extern "C" {

void mf_server_desc_init(mf_server_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  mf_engine_desc_init(&d->engine);
  d->tick_us = 200;
  d->queue_limit = 64;
}

int mf_server_open(const mf_server_desc* d, mf_server** out) {
  if (!d || !out) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (d->tick_us < 0 || d->queue_limit < 1) return fail(MF_ERR_INVALID_ARG, "bad serving limits");
  mf_server* s = new (std::nothrow) mf_server();
  if (!s) return fail(MF_ERR_OOM, "host allocation");
  s->d = *d;
  const int rc = mf_engine_open(&d->engine, &s->eng);
  if (rc) {
    delete s;
    return rc;
  }
  s->slots.resize(d->engine.max_streams);
  s->th = std::thread(run, s);
  *out = s;
  return MF_OK;
}

int mf_server_add_stream(mf_server* s, const mf_stream_desc* d, int64_t reserve_bytes, int32_t* slot) {
  if (!s || !d || !slot) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  int rc;
  {
    std::lock_guard<std::mutex> eg(s->emu);
    rc = mf_engine_add_stream(s->eng, d, reserve_bytes, slot);
  }
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(s->mu);
  ServerSlot& sl = s->slots[*slot];
  sl = ServerSlot();
  sl.used = true;
  sl.local = d->pose_frame == MF_POSES_BATCH_LOCAL;
  sl.overlap = d->overlap;
  return MF_OK;
}

namespace {

// Queues one push; the caller holds s->mu.
int enqueue(mf_server* s, const mf_push& p, int64_t t_now) {
  if (p.slot < 0 || p.slot >= (int32_t)s->slots.size()) return fail(MF_ERR_INVALID_ARG, "no such stream");
  if (p.n < 1 || !p.poses_w2c_3x4 || !p.K) return fail(MF_ERR_INVALID_ARG, "n < 1 or NULL poses/K");
  if (s->err) return s->err;
  ServerSlot& sl = s->slots[p.slot];
  if (!sl.used) return fail(MF_ERR_INVALID_ARG, "no such stream");
  if ((int32_t)sl.queue.size() >= s->d.queue_limit) return fail(MF_ERR_NOT_READY, "stream queue full");
  const int O = (sl.local && sl.pushes > 0) ? sl.overlap : 0;
  if (p.n <= O) return fail(MF_ERR_INVALID_ARG, "batch must hold more frames than the overlap");
  if (p.n - O > s->d.engine.max_stream_frames)
    return fail(MF_ERR_INVALID_ARG, "push exceeds max_stream_frames");
  if (mf::fault_fires(mf::kFaultDropPush)) {
    // injected fault: the push is accepted and lost, so its frames never
    // complete (drain with a timeout and frames_done detect it)
    ++sl.pushes;
    sl.frames_submitted += p.n - O;
    return MF_OK;
  }
  QueuedPush q;
  q.t_submit = p.arrival_ns ? p.arrival_ns : t_now;
  q.n = p.n;
  q.n_emit = p.n - O;
  q.poses.assign(p.poses_w2c_3x4, p.poses_w2c_3x4 + (size_t)p.n * 12);
  q.depth = p.depth;
  for (int k = 0; k < 4; ++k) q.K[k] = p.K[k];
  q.M = p.focus_map;
  q.G = p.guided_depth;
  q.info = p.info;
  ++sl.pushes;
  sl.frames_submitted += q.n_emit;
  sl.queue.push_back(std::move(q));
  ++s->queued;
  return MF_OK;
}

}  // namespace

int mf_server_submit(mf_server* s, int32_t slot, int32_t n, const double* poses, const void* depth,
                     const double* K, void* focus_map, void* guided_depth, mf_frame_info* info) {
  if (!s) return fail(MF_ERR_INVALID_ARG, "NULL server");
  mf_push p{};
  p.slot = slot;
  p.n = n;
  p.poses_w2c_3x4 = poses;
  p.depth = depth;
  p.K = K;
  p.focus_map = focus_map;
  p.guided_depth = guided_depth;
  p.info = info;
  int rc;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    rc = enqueue(s, p, mf::engine_now_ns());
  }
  if (rc == MF_OK) s->cv.notify_all();
  return rc;
}

int mf_server_submit_batch(mf_server* s, int32_t n, const mf_push* pushes, int32_t* accepted) {
  if (!s || !accepted || n < 0 || (n > 0 && !pushes)) return fail(MF_ERR_INVALID_ARG, "bad batch");
  *accepted = 0;
  int rc = MF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t t = mf::engine_now_ns();
    for (int32_t i = 0; i < n && rc == MF_OK; ++i) {
      rc = enqueue(s, pushes[i], t);
      if (rc == MF_OK) ++*accepted;
    }
  }
  if (*accepted) s->cv.notify_all();
  return rc;
}

int mf_server_frames_done(mf_server* s, int32_t slot, int64_t* frames) {
  if (!s || !frames || slot < 0 || slot >= (int32_t)s->slots.size())
    return fail(MF_ERR_INVALID_ARG, "bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *frames = s->slots[slot].frames_done;
  return s->err;
}

int mf_server_remove_stream(mf_server* s, int32_t slot) {
  if (!s || slot < 0 || slot >= (int32_t)s->slots.size()) return fail(MF_ERR_INVALID_ARG, "no such stream");
  {
    std::unique_lock<std::mutex> lk(s->mu);
    ServerSlot& sl = s->slots[slot];
    if (!sl.used) return fail(MF_ERR_INVALID_ARG, "no such stream");
    s->cv.wait(lk, [&] { return s->err || (sl.queue.empty() && sl.frames_done >= sl.frames_submitted); });
    sl.used = false;
  }
  std::lock_guard<std::mutex> eg(s->emu);
  return mf_engine_remove_stream(s->eng, slot);
}

int mf_server_drain(mf_server* s, int64_t timeout_ns) {
  if (!s) return fail(MF_ERR_INVALID_ARG, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [&] {
    if (s->err) return true;
    if (s->queued || !s->flight.empty()) return false;
    for (const ServerSlot& sl : s->slots)
      if (sl.used && sl.frames_done < sl.frames_submitted) return false;
    return true;
  };
  if (timeout_ns < 0) {
    s->cv.wait(lk, idle);
  } else if (!s->cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), idle)) {
    return fail(MF_ERR_TIMEOUT, "drain timed out");
  }
  return s->err;
}

int mf_server_latency(mf_server* s, mf_latency_stats* out, int32_t reset) {
  if (!s) return fail(MF_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> eg(s->emu);
  return mf_engine_latency(s->eng, out, reset);
}

int mf_server_tune(mf_server* s, int32_t width, int32_t height, int32_t window, int32_t* band_h) {
  if (!s) return fail(MF_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> eg(s->emu);
  return mf_engine_tune(s->eng, width, height, window, band_h);
}

int mf_server_get_stats(mf_server* s, mf_engine_stats* out) {
  if (!s) return fail(MF_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> eg(s->emu);
  return mf_engine_get_stats(s->eng, out);
}

int mf_server_close(mf_server* s) {
  if (!s) return MF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  const int rc = mf_engine_close(s->eng);
  delete s;
  return rc;
}

}  // extern "C"
