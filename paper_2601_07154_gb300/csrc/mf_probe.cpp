// Latency probe (include/mf.h): completion stamps for work queued on any
// CUDA stream, by the engine's own mechanism -- a host function enqueued
// behind the work records the steady clock when the stream reaches it.
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "mf_engine_internal.h"

namespace {

struct Stamp {
  std::vector<int64_t> arrival_ns;
  std::atomic<int64_t> done_ns{0};
};

void CUDART_CB stamp_done(void* p) {
  static_cast<Stamp*>(p)->done_ns.store(mf::engine_now_ns(), std::memory_order_release);
}

int fail(int st, const char* what, cudaError_t e = cudaSuccess) { return mf::host_fail(st, what, e); }

}  // namespace

struct mf_latency_probe {
  std::deque<std::unique_ptr<Stamp>> in_flight;
  std::vector<double> latencies_ms;
};

namespace {

void collect(mf_latency_probe* p) {
  while (!p->in_flight.empty()) {
    Stamp* s = p->in_flight.front().get();
    const int64_t done = s->done_ns.load(std::memory_order_acquire);
    if (!done) break;
    for (int64_t t : s->arrival_ns) p->latencies_ms.push_back((double)(done - t) * 1e-6);
    p->in_flight.pop_front();
  }
}

}  // namespace

extern "C" {

int mf_probe_open(mf_latency_probe** out) {
  if (!out) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  *out = new (std::nothrow) mf_latency_probe();
  return *out ? MF_OK : fail(MF_ERR_OOM, "host allocation");
}

int mf_probe_stamp(mf_latency_probe* p, void* cuda_stream, int32_t n, const int64_t* arrival_ns) {
  if (!p || n < 0 || (n > 0 && !arrival_ns)) return fail(MF_ERR_INVALID_ARG, "bad probe stamp");
  if (n == 0) return MF_OK;
  std::unique_ptr<Stamp> s(new (std::nothrow) Stamp());
  if (!s) return fail(MF_ERR_OOM, "host allocation");
  s->arrival_ns.assign(arrival_ns, arrival_ns + n);
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : cudaStreamLegacy;
  const cudaError_t e = cudaLaunchHostFunc(st, stamp_done, s.get());
  if (e != cudaSuccess) return fail(MF_ERR_CUDA, "probe stamp", e);
  p->in_flight.push_back(std::move(s));
  collect(p);
  return MF_OK;
}

int mf_probe_latency(mf_latency_probe* p, mf_latency_stats* out, int32_t reset) {
  if (!p || !out) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  collect(p);
  mf::latency_summary(p->latencies_ms, out);
  if (reset) p->latencies_ms.clear();
  return MF_OK;
}

int mf_probe_close(mf_latency_probe* p) {
  if (!p) return MF_OK;
  // The host functions still queued write into their stamps: wait for them
  // (at most 30 s; a stream that never gets there keeps its stamps, which
  // are then left allocated rather than freed under a pending writer).
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::seconds(30);
  while (!p->in_flight.empty()) {
    if (p->in_flight.front()->done_ns.load(std::memory_order_acquire)) {
      p->in_flight.pop_front();
    } else if (std::chrono::steady_clock::now() > deadline) {
      for (auto& s : p->in_flight) s.release();
      p->in_flight.clear();
      delete p;
      return fail(MF_ERR_TIMEOUT, "probe stamps still in flight at close");
    } else {
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  delete p;
  return MF_OK;
}

}  // extern "C"
