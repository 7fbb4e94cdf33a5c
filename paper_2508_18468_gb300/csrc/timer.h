// Per-phase CUDA-event timing of the step (tracing), host side.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace fm {

constexpr int kNumPhases = 6;  // FM_NPHASES

class PhaseTimer {
 public:
  bool on = false;
  cudaStream_t st = nullptr;

  ~PhaseTimer() {
    for (auto& p : pending_) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : pool_) cudaEventDestroy(e);
  }
  void begin(int phase) {
    if (!on) return;
    cur_a_ = take();
    cur_phase_ = phase;
    cudaEventRecord(cur_a_, st);
  }
  void end(int phase) {
    if (!on || phase != cur_phase_ || !cur_a_) return;
    cudaEvent_t b = take();
    cudaEventRecord(b, st);
    pending_.push_back({cur_a_, b, phase});
    cur_a_ = nullptr;
  }
  // synchronise, accumulate and reset; returns false if an event query failed
  bool collect(double* ms, int64_t* counts) {
    if (ms) for (int i = 0; i < kNumPhases; ++i) ms[i] = 0.0;
    if (counts) for (int i = 0; i < kNumPhases; ++i) counts[i] = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess) return false;
    bool ok = true;
    for (auto& p : pending_) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.a, p.b) != cudaSuccess) ok = false;
      if (ms) ms[p.phase] += t;
      if (counts) counts[p.phase] += 1;
      pool_.push_back(p.a);
      pool_.push_back(p.b);
    }
    pending_.clear();
    return ok;
  }

 private:
  struct Pair { cudaEvent_t a, b; int phase; };
  std::vector<Pair> pending_;
  std::vector<cudaEvent_t> pool_;
  cudaEvent_t cur_a_ = nullptr;
  int cur_phase_ = -1;
  cudaEvent_t take() {
    if (!pool_.empty()) { cudaEvent_t e = pool_.back(); pool_.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};

}  // namespace fm
