// prof.h - per-kernel-class launch counters and optional CUDA-event timing.
//
// Every launch site calls prof_pre / prof_post around the launch with its
// kernel class. Counting is always on; with profiling enabled on the handle
// each launch is bracketed by two events from a preallocated pool on the
// launch stream, and the elapsed times are summed per class after the solve.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/gkb.h"

namespace gkb {

struct Profiler {
  bool timing = false;
  long long launches[GKB_KC_COUNT] = {};
  long long units[GKB_KC_COUNT] = {};   // unknowns (or elements) processed
  double ms[GKB_KC_COUNT] = {};
  // timed launches of each class's largest work per launch (its finest
  // level): count, that work, summed time
  long long top_launches[GKB_KC_COUNT] = {};
  long long top_units[GKB_KC_COUNT] = {};
  double top_ms[GKB_KC_COUNT] = {};
  std::vector<cudaEvent_t> pool;
  std::vector<int> rec_class;
  std::vector<long long> rec_work;
  long long cur_work = 0;
  size_t used = 0;  // events used (pairs)
  int cur = -1;
  int phase = -1;   // >= 0 while a graph is captured: launches go to cap[phase]
  long long cap_l[5][GKB_KC_COUNT] = {};
  long long cap_u[5][GKB_KC_COUNT] = {};

  void enable(size_t pairs) {
    timing = true;
    if (pool.size() < 2 * pairs) {
      size_t old = pool.size();
      pool.resize(2 * pairs);
      for (size_t i = old; i < pool.size(); ++i) cudaEventCreate(&pool[i]);
    }
  }
  void reset() {
    for (int k = 0; k < GKB_KC_COUNT; ++k) {
      launches[k] = 0; ms[k] = 0; units[k] = 0;
      top_launches[k] = 0; top_units[k] = 0; top_ms[k] = 0;
    }
    used = 0;
    rec_class.clear();
    rec_work.clear();
  }
  void pre(int kc, cudaStream_t s, long long work) {
    if (phase >= 0) {
      cap_l[phase][kc] += 1;
      cap_u[phase][kc] += work;
      cur = -1;
      return;
    }
    launches[kc] += 1;
    units[kc] += work;
    cur = -1;
    if (timing && 2 * used + 1 < pool.size()) {
      cudaEventRecord(pool[2 * used], s);
      cur = kc;
      cur_work = work;
    }
  }
  void post(int kc, cudaStream_t s) {
    if (cur == kc && timing) {
      cudaEventRecord(pool[2 * used + 1], s);
      rec_class.push_back(kc);
      rec_work.push_back(cur_work);
      used += 1;
    }
    cur = -1;
  }
  // after a stream synchronisation
  void collect() {
    for (size_t i = 0; i < used; ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) != cudaSuccess) continue;
      const int kc = rec_class[i];
      const long long w = rec_work[i];
      ms[kc] += t;
      if (w > top_units[kc]) {   // a larger level than seen so far: restart its sums
        top_units[kc] = w;
        top_launches[kc] = 0;
        top_ms[kc] = 0;
      }
      if (w == top_units[kc]) {
        top_launches[kc] += 1;
        top_ms[kc] += t;
      }
    }
    (void)cudaGetLastError();
    used = 0;
    rec_class.clear();
    rec_work.clear();
  }
  ~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

// the profiler of the handle whose call is running on this thread
extern thread_local Profiler* g_prof;

inline void prof_pre(int kc, cudaStream_t s, long long work = 0) {
  if (g_prof) g_prof->pre(kc, s, work);
}
inline void prof_post(int kc, cudaStream_t s) {
  if (g_prof) g_prof->post(kc, s);
}

struct ProfScope {
  int kc;
  cudaStream_t s;
  ProfScope(int k, cudaStream_t st, long long work = 0) : kc(k), s(st) { prof_pre(kc, s, work); }
  ~ProfScope() { prof_post(kc, s); }
};

}  // namespace gkb
