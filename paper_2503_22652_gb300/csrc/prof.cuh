// Opt-in per-kernel-class device timers (rchfsi_profile / rchfsi_profile_read).
//
// When enabled on a handle, each instrumented launch is bracketed by two CUDA events recorded on
// the launching stream, and the launch's algorithmic flops and bytes are recorded with it.  The
// totals give each kernel class's achieved rate without a profiler attached.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace rchfsi {
namespace prof {

struct Rec {
  int cls;
  cudaEvent_t a, b;
  double flops, bytes;
};

struct Profiler {
  bool on = false;
  int64_t launch_base = 0;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    cudaEvent_t e;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  }
  void clear() {
    for (auto& r : recs) {
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
  }
  ~Profiler() {
    clear();
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// Profiler of the handle the current host thread is executing (null when disabled).
Profiler*& current();

struct Scope {
  Profiler* p;
  cudaStream_t s;
  size_t idx;
  Scope(cudaStream_t s_, int cls, double flops, double bytes) : p(current()), s(s_), idx(0) {
    if (!p || !p->on) {
      p = nullptr;
      return;
    }
    Rec r{cls, p->get(), p->get(), flops, bytes};
    cudaEventRecord(r.a, s);
    p->recs.push_back(r);
    idx = p->recs.size() - 1;
  }
  ~Scope() {
    if (p) cudaEventRecord(p->recs[idx].b, s);
  }
};

}  // namespace prof
}  // namespace rchfsi
