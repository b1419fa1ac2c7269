// Kernel-class timing with CUDA events recorded on the launching stream.  Off by
// default; when on, every launch site records an event pair around its kernel and
// fn_profile_read() sums the elapsed times per class.  Event pairs come from a pool
// that grows on demand and is reused after every read.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace fn {

enum ProfClass {
  kProfPrep = 0, kProfFeatures, kProfPair, kProfPairFull, kProfOrbFix, kProfMeanGemm, kProfLayerValue, kProfLayerFull, kProfOrbValue,
  kProfOrbFull, kProfDetValue, kProfDetFull, kProfSampler, kProfInit, kProfBwdOrb, kProfBwdGemm, kProfBwdPair,
  kProfBwdMisc, kProfSpinMeans, kProfOptim, kProfCount
};

inline const char* prof_name(int c) {
  static const char* names[kProfCount] = {
      "prep_params", "features", "pair_value", "pair_full", "orbital_fixup", "mean_field_gemm", "layer_value", "layer_full",
      "orbitals_value", "orbitals_full", "det_value", "det_full", "sampler", "init",
      "bwd_orbitals", "bwd_gemm", "bwd_pair", "bwd_misc", "spin_means", "optimizer"};
  return names[c];
}

struct Profiler {
  bool on = false;
  struct Rec { int cls; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
  size_t used = 0;
  int64_t launches[kProfCount] = {};
  double ms[kProfCount] = {};

  void begin(int cls, cudaStream_t st, cudaEvent_t* b_out) {
    if (used == pool.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      pool.push_back({a, b});
    }
    auto pr = pool[used++];
    cudaEventRecord(pr.first, st);
    pending.push_back({cls, pr.first, pr.second});
    *b_out = pr.second;
  }
  void collect() {
    for (auto& r : pending) {
      float t = 0.f;
      cudaEventSynchronize(r.b);
      cudaEventElapsedTime(&t, r.a, r.b);
      ms[r.cls] += t;
      launches[r.cls] += 1;
    }
    pending.clear();
    used = 0;
  }
  void reset() {
    collect();
    for (int c = 0; c < kProfCount; ++c) { launches[c] = 0; ms[c] = 0.0; }
  }
  ~Profiler() {
    for (auto& p : pool) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
  }
};

// RAII scope around one kernel launch.
struct ProfScope {
  Profiler* p;
  cudaStream_t st;
  cudaEvent_t b = nullptr;
  ProfScope(Profiler* prof, int cls, cudaStream_t s) : p(prof && prof->on ? prof : nullptr), st(s) {
    if (p) p->begin(cls, st, &b);
  }
  ~ProfScope() {
    if (p) cudaEventRecord(b, st);
  }
};

}  // namespace fn
