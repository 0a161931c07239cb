// Per-kernel tracing: launch counter and optional CUDA-event timing.
//
// Every kernel of the library is launched through spf::launch(), which counts
// the launch and, while profiling is on, records a start and a stop event on
// the launching stream. spf_profile_read() waits for those events and returns
// per-kernel launch counts and summed device time, so a caller can measure a
// kernel's average duration inside a timed region without a profiler.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.h"

namespace spf {

std::atomic<long long> g_launches{0};

namespace {

struct Pending {
  int kernel;
  cudaEvent_t a, b;
};

struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<std::string> names;
  std::vector<long long> count;
  std::vector<double> ms;
  std::vector<double> bytes;
  std::vector<Pending> pending;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
  size_t pool_used = 0;
  long long dropped = 0;
  std::vector<std::string> selected;   // empty: every kernel
};

Prof& prof() {
  static Prof* p = new Prof();   // never destroyed: events may outlive static teardown
  return *p;
}

int kernel_id(Prof& P, const char* name) {
  for (size_t i = 0; i < P.names.size(); ++i)
    if (P.names[i] == name) return (int)i;
  P.names.emplace_back(name);
  P.count.push_back(0);
  P.ms.push_back(0.0);
  P.bytes.push_back(0.0);
  return (int)P.names.size() - 1;
}

void drain(Prof& P) {
  for (auto& q : P.pending) {
    float t = 0.f;
    if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess)
      P.ms[q.kernel] += t;
    P.count[q.kernel] += 1;
  }
  P.pending.clear();
  P.pool_used = 0;
}

}  // namespace

bool prof_on() { return prof().on; }

int prof_begin(const char* name, cudaStream_t s, double bytes) {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  if (!P.on) return -1;
  if (!P.selected.empty()) {
    bool hit = false;
    for (const auto& n : P.selected) hit = hit || n == name;
    if (!hit) return -1;
  }
  if (P.pool_used == P.pool.size()) {
    if (P.pool.size() >= 8192) {
      ++P.dropped;
      return -1;
    }
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return -1;
    }
    P.pool.emplace_back(a, b);
  }
  auto ev = P.pool[P.pool_used++];
  cudaEventRecord(ev.first, s);
  const int id = kernel_id(P, name);
  P.bytes[id] += bytes;
  P.pending.push_back({id, ev.first, ev.second});
  return (int)P.pending.size() - 1;
}

void prof_end(int slot, cudaStream_t s) {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  if (slot >= 0 && slot < (int)P.pending.size()) cudaEventRecord(P.pending[slot].b, s);
}

}  // namespace spf

using namespace spf;

extern "C" {

int spf_profile_enable(int on) {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  drain(P);
  if (on) {
    for (size_t i = 0; i < P.count.size(); ++i) {
      P.count[i] = 0;
      P.ms[i] = 0.0;
      P.bytes[i] = 0.0;
    }
    P.dropped = 0;
  }
  P.on = on != 0;
  return SPF_OK;
}

int spf_profile_select(const char* names) {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  P.selected.clear();
  if (!names) return SPF_OK;
  std::string cur;
  for (const char* c = names;; ++c) {
    if (*c == ',' || *c == 0) {
      if (!cur.empty()) P.selected.push_back(cur);
      cur.clear();
      if (*c == 0) break;
    } else if (*c != ' ') {
      cur.push_back(*c);
    }
  }
  return SPF_OK;
}

int spf_profile_read(int index, char* name, int name_len, long long* launches, double* total_ms) {
  clear_error();
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  drain(P);
  if (index < 0 || index >= (int)P.names.size()) {
    set_error("no profiled kernel at index %d", index);
    return SPF_ERR_ARG;
  }
  if (name && name_len > 0) {
    strncpy(name, P.names[index].c_str(), name_len - 1);
    name[name_len - 1] = 0;
  }
  if (launches) *launches = P.count[index];
  if (total_ms) *total_ms = P.ms[index];
  return SPF_OK;
}

int spf_profile_bytes(int index, double* bytes) {
  clear_error();
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  if (index < 0 || index >= (int)P.names.size()) {
    set_error("no profiled kernel at index %d", index);
    return SPF_ERR_ARG;
  }
  if (bytes) *bytes = P.bytes[index];
  return SPF_OK;
}

long long spf_launch_count(void) { return g_launches.load(); }

}  // extern "C"
