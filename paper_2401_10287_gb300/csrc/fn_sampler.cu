// Electron sampler ("Electron Sampler" section): walker initialisation around the
// nuclei chosen by Algorithm 1, Gaussian all-electron proposals and the Metropolis
// acceptance on |psi|^2, plus the Gaussian parameter initialisation.
//
// All random numbers come from fn_rng.cuh (Philox4x32-10 + Box-Muller).  The
// position arithmetic r + s z is done in FP64 with separately rounded multiply and
// add (no fused multiply-add) and then rounded to the walker dtype, so that the
// result is reproducible bit for bit.
#include <algorithm>
#include <vector>

#include "fn_internal.cuh"
#include "fn_rng.cuh"

namespace fn {

template <typename Wlk>
__global__ void k_init_walkers(int B, int N, const int* __restrict__ atom, const double* __restrict__ nuc,
                               double init_std, uint64_t seed, uint64_t walker_offset, Wlk* __restrict__ out) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)B * N * 3) return;
  const int64_t w = gid / (3 * N);
  const int j = (int)(gid % (3 * N));
  const int e = j / 3, c = j % 3;
  const double z = normal_at((uint64_t)j, (uint32_t)(walker_offset + w), 0u, kStreamInit, seed);
  out[gid] = (Wlk)__dadd_rn(nuc[3 * atom[e] + c], __dmul_rn(z, init_std));
}

template <typename Wlk>
__global__ void k_propose(int B, int N, const Wlk* __restrict__ r, Wlk* __restrict__ out, double step,
                          uint64_t seed, uint32_t step_idx, uint64_t walker_offset) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)B * N * 3) return;
  const int64_t w = gid / (3 * N);
  const int j = (int)(gid % (3 * N));
  const double z = normal_at((uint64_t)j, (uint32_t)(walker_offset + w), step_idx, kStreamProposal, seed);
  out[gid] = (Wlk)__dadd_rn((double)r[gid], __dmul_rn(z, step));
}

template <typename Wlk>
__global__ void k_accept(int B, int N, Wlk* __restrict__ r, const Wlk* __restrict__ prop, double* __restrict__ lp,
                         const double* __restrict__ lp_new, uint64_t seed, uint32_t step_idx,
                         uint64_t walker_offset, unsigned long long* __restrict__ accepted) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  bool acc = false;
  if (w < B) {
    const double log_u = log_uniform_accept((uint32_t)(walker_offset + w), step_idx, seed);
    const double a = __dmul_rn(2.0, __dadd_rn(lp_new[w], -lp[w]));
    acc = log_u <= a;          // ties accept; NaN proposals are rejected
    if (acc) {
      for (int k = 0; k < 3 * N; ++k) r[(int64_t)w * 3 * N + k] = prop[(int64_t)w * 3 * N + k];
      lp[w] = lp_new[w];
    }
  }
  if (accepted) {
    const unsigned ballot = __ballot_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(accepted, (unsigned long long)__popc(ballot));
  }
}

// Parameter initialisation: segment table of (start, end, kind, fan_in)
struct InitSegs {
  int64_t start[4 * kMaxLayers + 8];
  int64_t end[4 * kMaxLayers + 8];
  int kind[4 * kMaxLayers + 8];      // 0 normal / sqrt(fan_in), 1 ones, 2 identity 3x3 blocks
  int fan_in[4 * kMaxLayers + 8];
  int n;
};

template <typename Par>
__global__ void k_init_params(int64_t P, InitSegs segs, uint64_t seed, Par* __restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  int s = 0;
  while (s < segs.n - 1 && p >= segs.end[s]) ++s;
  double v;
  if (segs.kind[s] == 0) {
    const double z = normal_at((uint64_t)p, 0u, 0u, kStreamParams, seed);
    v = __dmul_rn(z, __ddiv_rn(1.0, __dsqrt_rn((double)segs.fan_in[s])));
  } else if (segs.kind[s] == 1) {
    v = 1.0;
  } else {
    const int64_t q = (p - segs.start[s]) % 9;
    v = (q == 0 || q == 4 || q == 8) ? 1.0 : 0.0;
  }
  out[p] = (Par)v;
}

template <class Mode>
void launch_init_walkers(const fn_system* s, int B, uint64_t seed, double std_, void* walkers, cudaStream_t st) {
  using Wlk = typename Mode::Wlk;
  const int64_t n = (int64_t)B * s->N * 3;
  ProfScope ps(s->prof, kProfInit, st);
  k_init_walkers<Wlk><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(B, s->N, s->d_elec_atom, s->d_nuclei, std_, seed,
                                                                     s->walker_offset, (Wlk*)walkers);
}

template <class Mode>
void launch_propose(const fn_system* s, int B, const void* walkers, void* out, double step, uint64_t seed,
                    uint32_t step_idx, cudaStream_t st) {
  using Wlk = typename Mode::Wlk;
  const int64_t n = (int64_t)B * s->N * 3;
  ProfScope ps(s->prof, kProfSampler, st);
  k_propose<Wlk><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(B, s->N, (const Wlk*)walkers, (Wlk*)out, step, seed,
                                                                step_idx, s->walker_offset);
}

template <class Mode>
void launch_accept(const fn_system* s, int B, void* walkers, const void* prop, double* lp, const double* lp_new,
                   uint64_t seed, uint32_t step_idx, int64_t* accept_count, cudaStream_t st) {
  using Wlk = typename Mode::Wlk;
  ProfScope ps(s->prof, kProfSampler, st);
  k_accept<Wlk><<<(B + 127) / 128, 128, 0, st>>>(B, s->N, (Wlk*)walkers, (const Wlk*)prop, lp, lp_new, seed, step_idx,
                                                  s->walker_offset, (unsigned long long*)accept_count);
}

template <class Mode>
void launch_init_params(const fn_system* s, uint64_t seed, void* params, cudaStream_t st) {
  using Par = typename Mode::Par;
  InitSegs g{};
  auto add = [&](int64_t a, int64_t b, int kind, int fan) {
    g.start[g.n] = a; g.end[g.n] = b; g.kind[g.n] = kind; g.fan_in[g.n] = fan; ++g.n;
  };
  const int L = s->cfg.n_layers, h1 = s->cfg.h1, h2 = s->cfg.h2, K = s->cfg.n_dets;
  for (int l = 0; l < L; ++l) {
    const LayerDims& d = s->layer[l];
    const int f_in = 3 * d.d_h + 2 * d.d_g;
    add(d.off_V, d.off_V + (int64_t)h1 * f_in, 0, f_in);
    add(d.off_b, d.off_b + h1, 0, f_in);
    if (l < L - 1) {
      add(d.off_W, d.off_W + (int64_t)h2 * d.d_g, 0, d.d_g);
      add(d.off_c, d.off_c + h2, 0, d.d_g);
    }
  }
  const int ns[2] = {s->n_up, s->n_dn};
  for (int a = 0; a < 2; ++a)
    if (ns[a]) {
      add(s->off_w[a], s->off_w[a] + (int64_t)K * ns[a] * h1, 0, h1);
      add(s->off_g[a], s->off_g[a] + (int64_t)K * ns[a], 0, h1);
    }
  for (int a = 0; a < 2; ++a)
    if (ns[a]) {
      add(s->off_pi[a], s->off_sig[a], 1, 1);
      const int64_t end = (a == 0 && ns[1]) ? s->off_pi[1] : s->P;
      add(s->off_sig[a], end, s->cfg.envelope == FN_ENV_ANISOTROPIC ? 2 : 1, 1);
    }
  ProfScope ps(s->prof, kProfInit, st);
  k_init_params<Par><<<(unsigned)((s->P + 255) / 256), 256, 0, st>>>(s->P, g, seed, (Par*)params);
}

#define FN_INST(M)                                                                                          \
  template void launch_init_walkers<M>(const fn_system*, int, uint64_t, double, void*, cudaStream_t);        \
  template void launch_propose<M>(const fn_system*, int, const void*, void*, double, uint64_t, uint32_t,     \
                                  cudaStream_t);                                                             \
  template void launch_accept<M>(const fn_system*, int, void*, const void*, double*, const double*, uint64_t, \
                                 uint32_t, int64_t*, cudaStream_t);                                          \
  template void launch_init_params<M>(const fn_system*, uint64_t, void*, cudaStream_t);
FN_INST(ModeF64)
FN_INST(ModeF32)
FN_INST(ModeBF16)

}  // namespace fn
