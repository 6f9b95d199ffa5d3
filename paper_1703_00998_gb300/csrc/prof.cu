// Launch counting and optional per-kernel-class timing with CUDA events.
//
// Every kernel launch of the library calls note_launch(); when profiling is
// on, the launch sites of each kernel class bracket their launches with a
// pair of events on the launching stream and record the algorithmic flops
// and bytes of the launch.  Elapsed times are collected after the stream has
// been synchronised (prof_flush), so profiling adds no host synchronisation.
#include <atomic>
#include <mutex>
#include <vector>
#include "common.cuh"
#include "internal.h"

namespace rutv {

static std::atomic<unsigned long long> g_launches{0};
static bool g_prof_on = false;

struct Pending { cudaEvent_t a, b; int cls; double flops, bytes; };
static std::mutex g_mu;
static std::vector<cudaEvent_t> g_free_events;
static std::vector<Pending> g_pending;
static ProfTotals g_tot[kProfClasses];

void note_launch(int n) { g_launches.fetch_add(static_cast<unsigned long long>(n)); }
unsigned long long launch_count() { return g_launches.load(); }
bool prof_enabled() { return g_prof_on; }

static cudaEvent_t get_event() {
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfToken prof_begin(cudaStream_t s, int cls) {
  ProfToken t{-1};
  if (!g_prof_on) return t;
  std::lock_guard<std::mutex> lk(g_mu);
  Pending p{get_event(), get_event(), cls, 0.0, 0.0};
  cudaEventRecord(p.a, s);
  g_pending.push_back(p);
  t.idx = static_cast<int>(g_pending.size()) - 1;
  return t;
}

void prof_end(cudaStream_t s, ProfToken t, double flops, double bytes) {
  if (t.idx < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Pending& p = g_pending[t.idx];
  p.flops = flops;
  p.bytes = bytes;
  cudaEventRecord(p.b, s);
}

void prof_flush() {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      ProfTotals& T = g_tot[p.cls];
      T.ms += ms;
      T.launches += 1;
      T.flops += p.flops;
      T.bytes += p.bytes;
    }
    g_free_events.push_back(p.a);
    g_free_events.push_back(p.b);
  }
  g_pending.clear();
}

void prof_set(bool on) {
  prof_flush();
  g_prof_on = on;
}

ProfTotals prof_read(int cls) {
  prof_flush();
  std::lock_guard<std::mutex> lk(g_mu);
  return g_tot[cls];
}

void prof_reset() {
  prof_flush();
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& t : g_tot) t = ProfTotals{};
}

}  // namespace rutv

extern "C" {

int randutv_profile_enable(int on) {
  rutv::prof_set(on != 0);
  return RANDUTV_OK;
}

int randutv_profile_reset(void) {
  rutv::prof_reset();
  return RANDUTV_OK;
}

int randutv_profile_read(int cls, double* ms, int64_t* launches, double* flops, double* bytes) {
  if (cls < 0 || cls >= rutv::kProfClasses) return -1;
  rutv::ProfTotals t = rutv::prof_read(cls);
  if (ms) *ms = t.ms;
  if (launches) *launches = t.launches;
  if (flops) *flops = t.flops;
  if (bytes) *bytes = t.bytes;
  return RANDUTV_OK;
}

uint64_t randutv_launch_count(void) { return rutv::launch_count(); }

}  // extern "C"
