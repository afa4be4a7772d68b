// Optional per-pass device timing with CUDA events recorded on the
// launching stream (used by benchmarks to time the dominant kernel inside
// a longer timed region).  Events come from a pre-created pool; when the
// pool is exhausted further launches are simply not timed.
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace rve {

enum PassId : int {
  PASS_XFWD = 0,
  PASS_YFWD = 1,
  PASS_ZPROJ = 2,
  PASS_YINV = 3,
  PASS_XINV = 4,
  PASS_YPROJ2D = 5,
  PASS_TRIAL = 6,
  PASS_CGVEC = 7,
  PASS_COUNT = 8,
};

struct PassTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> ids;  // pass id of each (begin, end) pair
  int used = 0;          // events used
  long long counts[PASS_COUNT] = {};
  double ms[PASS_COUNT] = {};

  cudaError_t enable(int npairs) {
    reset();
    if ((int)pool.size() < 2 * npairs) {
      const int have = (int)pool.size();
      pool.resize(2 * npairs);
      for (int i = have; i < 2 * npairs; ++i) {
        cudaError_t e = cudaEventCreate(&pool[i]);
        if (e != cudaSuccess) {
          pool.resize(i);
          return e;
        }
      }
    }
    on = true;
    return cudaSuccess;
  }
  void reset() {
    used = 0;
    ids.clear();
    for (int i = 0; i < PASS_COUNT; ++i) { counts[i] = 0; ms[i] = 0.0; }
  }
  // record the start of a launch; returns false when not timing
  bool begin(cudaStream_t st, int id) {
    if (!on || used + 2 > (int)pool.size()) return false;
    cudaEventRecord(pool[used], st);
    ids.push_back(id);
    ++used;
    return true;
  }
  void end(cudaStream_t st) {
    cudaEventRecord(pool[used], st);
    ++used;
  }
  // fold recorded pairs into the totals (synchronises on the last event)
  cudaError_t flush() {
    if (used == 0) return cudaSuccess;
    cudaError_t e = cudaEventSynchronize(pool[used - 1]);
    if (e != cudaSuccess) return e;
    for (int p = 0; p < (int)ids.size(); ++p) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, pool[2 * p], pool[2 * p + 1]);
      if (e != cudaSuccess) return e;
      counts[ids[p]] += 1;
      ms[ids[p]] += t;
    }
    used = 0;
    ids.clear();
    return cudaSuccess;
  }
  void destroy() {
    for (cudaEvent_t ev : pool) cudaEventDestroy(ev);
    pool.clear();
    on = false;
  }
};

// RAII helper around one launch.
struct PassScope {
  PassTimer* t;
  cudaStream_t st;
  bool rec;
  PassScope(PassTimer* t_, cudaStream_t st_, int id) : t(t_), st(st_), rec(t_ ? t_->begin(st_, id) : false) {}
  ~PassScope() {
    if (rec) t->end(st);
  }
};

}  // namespace rve
