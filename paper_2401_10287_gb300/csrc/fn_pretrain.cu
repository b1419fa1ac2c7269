// Pretraining loss of Eq. 5 and its seed for the parameter gradient.
//
// Eq. 5 compares the network's orbital matrices with Hartree-Fock orbitals at the sampled
// electron positions: L = (1/B) sum_w sum_spin sum_{k,i,j} (Phi_kij - Phi^HF_ij)^2, with k the
// determinant, i the orbital and j the electron of that spin; B is the number of walkers, and
// the same occupied UHF orbital i (STO-6G, in order of orbital energy) is the target of every
// determinant.  The value-only forward pass leaves Phi in the workspace; k_pretrain_seed
// evaluates the HF orbitals at the walker's electrons, writes dL/dPhi (up to the factor 2/B,
// which goes into the per-walker weight) where the backward pass reads its seed, and the
// per-walker loss; k_pretrain_loss sums those in a fixed order.
#include "fn_device.cuh"
#include "fn_internal.cuh"

namespace fn {

constexpr int kHfMaxBasis = 20;
constexpr int kHfPerFunction = 18;   // centre[3], powers[3], exponents[6], weights[6]

// One warp per walker, one lane per electron (N <= 32).
template <typename Det, typename PhiT, typename Wlk>
__global__ void k_pretrain_seed(const Wlk* __restrict__ r, Shape sh, const double* __restrict__ hf, int nbf,
                                const PhiT* __restrict__ Phi, int64_t PW, int K, Det* __restrict__ dPhi,
                                double* __restrict__ cw, double* __restrict__ wloss) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + warp;
  if (w >= sh.B) return;                                   // warp-uniform
  const int N = sh.N;
  Det loss = 0;
  if (lane < N) {
    const int spin = lane < sh.n_up ? 0 : 1;
    const int n = spin ? sh.n_dn : sh.n_up;
    const int jj = lane - (spin ? sh.n_up : 0);
    const Det x = (Det)r[((int64_t)w * N + lane) * 3], y = (Det)r[((int64_t)w * N + lane) * 3 + 1],
              z = (Det)r[((int64_t)w * N + lane) * 3 + 2];
    Det chi[kHfMaxBasis];
#pragma unroll
    for (int mu = 0; mu < kHfMaxBasis; ++mu) {
      chi[mu] = 0;
      if (mu < nbf) {
        const double* f = hf + mu * kHfPerFunction;
        const Det dx = x - (Det)f[0], dy = y - (Det)f[1], dz = z - (Det)f[2];
        const Det r2 = dx * dx + dy * dy + dz * dz;
        Det poly = 1;
        if (f[3] > 0.5) poly *= dx;
        if (f[4] > 0.5) poly *= dy;
        if (f[5] > 0.5) poly *= dz;
        Det v = 0;
        for (int k = 0; k < 6; ++k) v += (Det)f[12 + k] * f_exp(-(Det)f[6 + k] * r2);
        chi[mu] = poly * v;
      }
    }
    const double* C = hf + nbf * kHfPerFunction + (spin ? (int64_t)nbf * sh.n_up : 0);
    const int64_t blk = spin ? (int64_t)K * sh.n_up * sh.n_up : 0;
    for (int i = 0; i < n; ++i) {
      Det target = 0;
#pragma unroll
      for (int mu = 0; mu < kHfMaxBasis; ++mu)
        if (mu < nbf) target += (Det)C[mu * n + i] * chi[mu];
      for (int k = 0; k < K; ++k) {
        const int64_t e = blk + (int64_t)k * n * n + (int64_t)i * n + jj;
        const Det diff = (Det)Phi[(int64_t)w * PW + e] - target;
        dPhi[(int64_t)w * PW + e] = diff;
        loss += diff * diff;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, off);
  if (lane == 0) {
    wloss[w] = (double)loss;
    cw[w] = 2.0 / (double)sh.B;                            // dL/dPhi = (2 / B) (Phi - Phi^HF)
  }
}

__global__ void k_pretrain_loss(int B, const double* __restrict__ wloss, double* __restrict__ out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int w = threadIdx.x; w < B; w += blockDim.x) s += wloss[w];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / (double)B;
}

template <class Mode>
void launch_pretrain_seed(const fn_system* s, const void* walkers, const Shape& sh, double* loss, cudaStream_t st) {
  using Det = typename Mode::Det; using PhiT = typename Mode::PhiT; using Wlk = typename Mode::Wlk;
  const Workspace& ws = s->ws;
  ProfScope ps(s->prof, kProfBwdOrb, st);
  const int warps = 4;
  k_pretrain_seed<Det, PhiT, Wlk><<<(unsigned)((sh.B + warps - 1) / warps), 32 * warps, 0, st>>>(
      (const Wlk*)walkers, sh, s->d_hf, s->hf_nbf, (const PhiT*)ws.Phi, phi_walker_stride(s, 1), s->cfg.n_dets,
      (Det*)ws.dPhi, ws.scratch_d, ws.scratch_d + sh.B);
  if (loss) k_pretrain_loss<<<1, 1024, 0, st>>>(sh.B, ws.scratch_d + sh.B, loss);
}

template void launch_pretrain_seed<ModeF64>(const fn_system*, const void*, const Shape&, double*, cudaStream_t);
template void launch_pretrain_seed<ModeF32>(const fn_system*, const void*, const Shape&, double*, cudaStream_t);
template void launch_pretrain_seed<ModeBF16>(const fn_system*, const void*, const Shape&, double*, cudaStream_t);

}  // namespace fn
