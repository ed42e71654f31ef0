// Host-side fault injection (include/mf.h, mf_set_fault).  Every fault is
// made on the host, at a chosen call: an allocation that fails, a pose made
// non-rigid on its way to the device, a serving push that is accepted and
// then dropped, an admission that is refused, a device wait that is
// reported as run out.  Nothing here makes a GPU fault, trap or hang; the
// library's own detection (status codes, per-frame flags, bounded waits on
// the host) is what the injected faults exercise.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "mf_internal.h"

namespace {

struct FaultRule {
  std::atomic<bool> on{false};
  std::atomic<int64_t> at{0};  // 1-based occurrence that fires (0: every one)
  std::atomic<int64_t> seen{0};
};

FaultRule g_rules[mf::kFaultKinds];
std::mutex g_mu;
std::once_flag g_env_once;

const char* kNames[mf::kFaultKinds] = {"alloc_fail", "bad_pose", "drop_push", "admission_full",
                                       "wait_timeout"};

// Parses "name[@n],name[@n],..." into rules; false on a malformed spec.
bool parse(const char* spec, bool (&on)[mf::kFaultKinds], int64_t (&at)[mf::kFaultKinds]) {
  for (int k = 0; k < mf::kFaultKinds; ++k) {
    on[k] = false;
    at[k] = 0;
  }
  if (!spec) return true;
  std::string s(spec);
  size_t pos = 0;
  while (pos < s.size()) {
    size_t end = s.find(',', pos);
    if (end == std::string::npos) end = s.size();
    std::string item = s.substr(pos, end - pos);
    pos = end + 1;
    if (item.empty()) continue;
    std::string name = item;
    int64_t n = 0;
    const size_t a = item.find('@');
    if (a != std::string::npos) {
      name = item.substr(0, a);
      const std::string num = item.substr(a + 1);
      if (num.empty() || num.find_first_not_of("0123456789") != std::string::npos) return false;
      n = std::strtoll(num.c_str(), nullptr, 10);
      if (n < 1) return false;
    }
    int kind = -1;
    for (int k = 0; k < mf::kFaultKinds; ++k)
      if (name == kNames[k]) kind = k;
    if (kind < 0) return false;
    on[kind] = true;
    at[kind] = n;
  }
  return true;
}

void install(const bool (&on)[mf::kFaultKinds], const int64_t (&at)[mf::kFaultKinds]) {
  for (int k = 0; k < mf::kFaultKinds; ++k) {
    g_rules[k].on.store(false);
    g_rules[k].seen.store(0);
    g_rules[k].at.store(at[k]);
    g_rules[k].on.store(on[k]);
  }
}

void load_env() {
  bool on[mf::kFaultKinds];
  int64_t at[mf::kFaultKinds];
  if (parse(std::getenv("MF_FAULT"), on, at)) install(on, at);
}

}  // namespace

bool mf::fault_fires(int kind) {
  std::call_once(g_env_once, load_env);
  FaultRule& r = g_rules[kind];
  if (!r.on.load(std::memory_order_acquire)) return false;
  const int64_t n = r.seen.fetch_add(1) + 1;
  const int64_t at = r.at.load();
  return at == 0 || n == at;
}

extern "C" int mf_set_fault(const char* spec) {
  std::call_once(g_env_once, load_env);
  bool on[mf::kFaultKinds];
  int64_t at[mf::kFaultKinds];
  if (!parse(spec, on, at)) return mf::host_fail(MF_ERR_INVALID_ARG, "malformed fault spec", cudaSuccess);
  std::lock_guard<std::mutex> lk(g_mu);
  install(on, at);
  return MF_OK;
}
