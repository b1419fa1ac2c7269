// Determinant stage and local-energy assembly (one CTA per walker).
//
// For every determinant k and spin block of n x n orbitals A (psi = sum_k
// det A_k,up det A_k,down, empty blocks have determinant 1):
//   * LU with partial pivoting in shared memory, one warp per spin block, lane =
//     matrix row, warp shuffles pick the first maximal |pivot|;
//   * C = A^{-1} by substitution, lane = right-hand-side column;
//   * for every coordinate t (one thread per (block, t) item):
//       g_t = tr(C d_t A),   q_t = tr((C d_t A)^2) = sum_i B_ii^2 + 2 sum_{i<j} B_ij B_ji,
//     and tr(C lap A) for the Laplacian slab, so that
//       d_t log|det A| = g_t,   lap log|det A| = tr(C lap A) - sum_t q_t;
//   * the K terms combine by a signed log-sum-exp with rho_k = D_k / psi:
//       grad log|psi| = sum_k rho_k g_k,
//       lap log|psi| = sum_k rho_k (lap_k + |g_k|^2) - |grad log|psi||^2,
//   * E_L = -1/2 (|grad|^2 + lap) + V_ee + V_ne + V_nn (Eqs. 2-3).
// All of it runs in the Det type (FP64 in the FP64 and BF16-mixed modes).
#include <algorithm>

#include "fn_device.cuh"
#include "fn_internal.cuh"

namespace fn {

struct DetArgs {
  const void* Phi;
  int64_t PW;
  int K;
  double* e_local;
  double* log_psi;
  int8_t* sign;
  void* inv_out;      // value-pass backward seed rho_k A^{-T}, [B][K (nu^2 + nd^2)], or null
  const double* charges;
  double v_nn;
  int* status;
};

// LU with partial pivoting of the n x n row-major matrix A (in place) by one warp,
// then C = A^{-1}.  Returns log|det| and sign (0 when a pivot is exactly zero).
template <typename Det>
__device__ void warp_lu_inverse(Det* A, Det* C, int n, Det* ld_out, Det* sign_out) {
  const int lane = threadIdx.x & 31;
  int perm = lane;
  Det sgn = 1;
  bool singular = false;
  for (int c = 0; c < n; ++c) {
    Det v = (lane >= c && lane < n) ? f_abs(A[lane * n + c]) : (Det)-1;
    int idx = lane;
    for (int off = 16; off > 0; off >>= 1) {
      const Det ov = __shfl_down_sync(0xffffffffu, v, off);
      const int oi = __shfl_down_sync(0xffffffffu, idx, off);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    const int piv = __shfl_sync(0xffffffffu, idx, 0);
    const Det pv = __shfl_sync(0xffffffffu, v, 0);
    if (!(pv > (Det)0)) { singular = true; break; }
    if (piv != c) {
      if (lane < n) {
        const Det tmp = A[c * n + lane];
        A[c * n + lane] = A[piv * n + lane];
        A[piv * n + lane] = tmp;
      }
      const int pc = __shfl_sync(0xffffffffu, perm, c);
      const int pp = __shfl_sync(0xffffffffu, perm, piv);
      if (lane == c) perm = pp;
      if (lane == piv) perm = pc;
      sgn = -sgn;
    }
    __syncwarp();
    if (lane > c && lane < n) {
      const Det f = A[lane * n + c] / A[c * n + c];
      A[lane * n + c] = f;
      for (int j = c + 1; j < n; ++j) A[lane * n + j] -= f * A[c * n + j];
    }
    __syncwarp();
  }
  // log|det| = sum of log|pivot|; sign = permutation sign (warp-uniform) * pivot signs
  Det ld = 0;
  int neg = 0;
  if (!singular && lane < n) {
    const Det d = A[lane * n + lane];
    ld = f_log(f_abs(d));
    neg = d < 0 ? 1 : 0;
  }
  for (int off = 16; off > 0; off >>= 1) {
    ld += __shfl_down_sync(0xffffffffu, ld, off);
    neg += __shfl_down_sync(0xffffffffu, neg, off);
  }
  if (lane == 0) {
    *ld_out = singular ? (Det)0 : ld;
    *sign_out = singular ? (Det)0 : ((neg & 1) ? -sgn : sgn);
  }
  // inverse: lane j solves A x = e_j with P A = L U
  for (int i = 0; i < n; ++i) {
    const int pi = __shfl_sync(0xffffffffu, perm, i);
    if (lane < n) {
      if (singular) { C[i * n + lane] = 0; continue; }
      Det y = (pi == lane) ? (Det)1 : (Det)0;
      for (int k = 0; k < i; ++k) y -= A[i * n + k] * C[k * n + lane];
      C[i * n + lane] = y;
    }
  }
  __syncwarp();
  if (lane < n && !singular)
    for (int i = n - 1; i >= 0; --i) {
      Det x = C[i * n + lane];
      for (int k = i + 1; k < n; ++k) x -= A[i * n + k] * C[k * n + lane];
      C[i * n + lane] = x / A[i * n + i];
    }
  __syncwarp();
}

template <typename Det, typename Wlk, bool FULL>
__global__ void __launch_bounds__(128) k_det_energy(const Wlk* __restrict__ r, const double* __restrict__ nuc,
                                                    Shape sh, DetArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = sh.N, T = sh.T, K = a.K, NC = 3 * N;
  const int ns[2] = {sh.n_up, sh.n_dn};
  const int nmax = max(ns[0], ns[1]);
  Det* lu = (Det*)smem_raw;                  // [2][nmax^2]
  Det* inv = lu + 2 * nmax * nmax;           // [2][nmax^2]
  Det* ldk = inv + 2 * nmax * nmax;          // [K]
  Det* sk = ldk + K;                         // [K]
  Det* lapk = sk + K;                        // [K]
  Det* rho = lapk + K;                       // [K]
  Det* gradk = rho + K;                      // [K][NC]   (FULL)
  Det* gt = gradk + (FULL ? K * NC : 0);     // [2][NC]
  Det* qt = gt + (FULL ? 2 * NC : 0);        // [2][NC]
  Det* misc = qt + (FULL ? 2 * NC : 0);      // [8]
  Det* red = misc + 8;                       // [128]
  const Det* Phi = (const Det*)a.Phi + (int64_t)w * a.PW;
  const int64_t blk_off[2] = {0, (int64_t)K * T * ns[0] * ns[0]};
  const int64_t inv_off[2] = {0, (int64_t)K * ns[0] * ns[0]};

  for (int k = 0; k < K; ++k) {
    for (int e = tid; e < ns[0] * ns[0] + ns[1] * ns[1]; e += blockDim.x) {
      const int s = e < ns[0] * ns[0] ? 0 : 1;
      const int idx = s ? e - ns[0] * ns[0] : e;
      lu[s * nmax * nmax + idx] = Phi[blk_off[s] + (int64_t)k * T * ns[s] * ns[s] + idx];
    }
    __syncthreads();
    if (warp < 2) {
      if (ns[warp] > 0) {
        warp_lu_inverse<Det>(lu + warp * nmax * nmax, inv + warp * nmax * nmax, ns[warp], misc + warp,
                             misc + 2 + warp);
      } else if ((tid & 31) == 0) {
        misc[warp] = 0;
        misc[2 + warp] = 1;
      }
    }
    __syncthreads();
    if (FULL) {
      // items: (spin, t) for the 3N gradient slabs, then (spin) for the Laplacian slab
      const int per = NC + 1;
      for (int it = tid; it < 2 * per; it += blockDim.x) {
        const int s = it / per, tr = it % per;
        const int n = ns[s];
        if (n == 0) {
          if (tr < NC) { gt[s * NC + tr] = 0; qt[s * NC + tr] = 0; } else { misc[4 + s] = 0; }
          continue;
        }
        const Det* Cm = inv + s * nmax * nmax;
        const int t = tr < NC ? 1 + tr : T - 1;
        const Det* D = Phi + blk_off[s] + (int64_t)k * T * n * n + (int64_t)t * n * n;
        if (tr < NC) {
          Det g = 0, q = 0;
          for (int i = 0; i < n; ++i) {
            for (int j = i; j < n; ++j) {
              Det bij = 0;
              for (int m = 0; m < n; ++m) bij += Cm[i * n + m] * D[m * n + j];
              if (j == i) {
                g += bij;
                q += bij * bij;
              } else {
                Det bji = 0;
                for (int m = 0; m < n; ++m) bji += Cm[j * n + m] * D[m * n + i];
                q += (Det)2 * bij * bji;
              }
            }
          }
          gt[s * NC + tr] = g;
          qt[s * NC + tr] = q;
        } else {
          Det l = 0;
          for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) l += Cm[j * n + i] * D[i * n + j];
          misc[4 + s] = l;
        }
      }
      __syncthreads();
      for (int t = tid; t < NC; t += blockDim.x) gradk[k * NC + t] = gt[t] + gt[NC + t];
      if (warp == 0) {
        Det qs = 0;
        for (int t = tid; t < 2 * NC; t += 32) qs += qt[t];
        for (int off = 16; off > 0; off >>= 1) qs += __shfl_down_sync(0xffffffffu, qs, off);
        if (tid == 0) lapk[k] = misc[4] + misc[5] - qs;
      }
    }
    if (tid == 0) {
      ldk[k] = misc[0] + misc[1];
      sk[k] = misc[2] * misc[3];
    }
    if (a.inv_out) {
      Det* io = (Det*)a.inv_out + (int64_t)w * K * (ns[0] * ns[0] + ns[1] * ns[1]);
      for (int e = tid; e < ns[0] * ns[0] + ns[1] * ns[1]; e += blockDim.x) {
        const int s = e < ns[0] * ns[0] ? 0 : 1;
        const int idx = s ? e - ns[0] * ns[0] : e;
        const int n = ns[s], i = idx / n, j = idx % n;
        io[inv_off[s] + (int64_t)k * n * n + idx] = inv[s * nmax * nmax + j * n + i];   // A^{-T}
      }
    }
    __syncthreads();
  }
  // signed log-sum-exp over determinants
  if (tid == 0) {
    Det m = -INFINITY;
    for (int k = 0; k < K; ++k)
      if (sk[k] != 0 && ldk[k] > m) m = ldk[k];
    Det S = 0;
    for (int k = 0; k < K; ++k) {
      rho[k] = sk[k] != 0 ? sk[k] * f_exp(ldk[k] - m) : (Det)0;
      S += rho[k];
    }
    for (int k = 0; k < K; ++k) rho[k] = S != 0 ? rho[k] / S : (Det)0;
    misc[6] = m + f_log(f_abs(S));
    misc[7] = S > 0 ? 1 : (S < 0 ? -1 : 0);
  }
  __syncthreads();
  const double lpsi = (double)misc[6];
  const int sgn = (int)misc[7];
  if (a.inv_out) {
    Det* io = (Det*)a.inv_out + (int64_t)w * K * (ns[0] * ns[0] + ns[1] * ns[1]);
    // scale each determinant's block by rho_k
    for (int s = 0; s < 2; ++s) {
      const int nn = ns[s] * ns[s];
      for (int e = tid; e < K * nn; e += blockDim.x) io[inv_off[s] + e] *= rho[e / nn];
    }
  }
  if (FULL) {
    // E_kin = -1/2 (|grad log psi|^2 + lap log psi) = -1/2 sum_k rho_k (lap_k + |g_k|^2)
    Det kin = 0;
    for (int k = tid; k < K; k += blockDim.x) {
      Det g2 = 0;
      for (int t = 0; t < NC; ++t) g2 += gradk[k * NC + t] * gradk[k * NC + t];
      kin += rho[k] * (lapk[k] + g2);
    }
    double pot = 0.0;
    const Wlk* rw = r + (int64_t)w * N * 3;
    for (int p = tid; p < N * N; p += blockDim.x) {
      const int i = p / N, j = p % N;
      if (j <= i) continue;
      const double dx = (double)rw[3 * i] - (double)rw[3 * j], dy = (double)rw[3 * i + 1] - (double)rw[3 * j + 1],
                   dz = (double)rw[3 * i + 2] - (double)rw[3 * j + 2];
      pot += 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
    }
    for (int p = tid; p < N * sh.M; p += blockDim.x) {
      const int i = p / sh.M, m = p % sh.M;
      const double dx = (double)rw[3 * i] - nuc[3 * m], dy = (double)rw[3 * i + 1] - nuc[3 * m + 1],
                   dz = (double)rw[3 * i + 2] - nuc[3 * m + 2];
      pot -= a.charges[m] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    red[tid] = (Det)(-0.5) * kin + (Det)pot;
    __syncthreads();
    for (int off = 64; off > 0; off >>= 1) {
      if (tid < off) red[tid] += red[tid + off];
      __syncthreads();
    }
    if (tid == 0) {
      const double e = (double)red[0] + a.v_nn;
      a.e_local[w] = e;
      if (!isfinite(e) || !isfinite(lpsi)) atomicOr(a.status, kStatusNonFinite);
    }
  }
  if (tid == 0) {
    if (a.log_psi) a.log_psi[w] = lpsi;
    if (a.sign) a.sign[w] = (int8_t)sgn;
    if (sgn == 0) atomicOr(a.status, kStatusSingular);
  }
}

template <class Mode>
void launch_det_energy(const fn_system* s, const void* walkers, const Shape& sh, double* e_local, double* log_psi,
                       int8_t* sign, bool keep_inverse, cudaStream_t st) {
  using Det = typename Mode::Det; using Wlk = typename Mode::Wlk;
  DetArgs a{};
  a.Phi = s->ws.Phi;
  a.PW = phi_walker_stride(s, sh.T);
  a.K = s->cfg.n_dets;
  a.e_local = e_local;
  a.log_psi = log_psi;
  a.sign = sign;
  a.inv_out = keep_inverse ? s->ws.dPhi : nullptr;
  a.charges = s->d_charges;
  a.v_nn = s->v_nn;
  a.status = s->ws.status;
  const bool full = sh.T > 1 && e_local != nullptr;
  const int nmax = std::max(s->n_up, s->n_dn), NC = 3 * s->N, K = s->cfg.n_dets;
  const size_t smem = sizeof(Det) * (4 * nmax * nmax + 4 * K + (full ? K * NC + 4 * NC : 0) + 8 + 128);
  ProfScope ps(s->prof, full ? kProfDetFull : kProfDetValue, st);
  if (full) {
    cudaFuncSetAttribute(k_det_energy<Det, Wlk, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_det_energy<Det, Wlk, true><<<sh.B, 128, smem, st>>>((const Wlk*)walkers, s->d_nuclei, sh, a);
  } else {
    cudaFuncSetAttribute(k_det_energy<Det, Wlk, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_det_energy<Det, Wlk, false><<<sh.B, 128, smem, st>>>((const Wlk*)walkers, s->d_nuclei, sh, a);
  }
}

template void launch_det_energy<ModeF64>(const fn_system*, const void*, const Shape&, double*, double*, int8_t*,
                                         bool, cudaStream_t);
template void launch_det_energy<ModeF32>(const fn_system*, const void*, const Shape&, double*, double*, int8_t*,
                                         bool, cudaStream_t);
template void launch_det_energy<ModeBF16>(const fn_system*, const void*, const Shape&, double*, double*, int8_t*,
                                          bool, cudaStream_t);

}  // namespace fn
