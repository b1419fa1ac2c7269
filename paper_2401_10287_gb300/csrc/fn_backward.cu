// VMC energy gradient (Eq. 6): grad = sum_w c_w d log|psi_w| / d theta with
// c_w = 2 (E_L,w - mean E_L) / B, E_L held fixed.  A reverse pass over the
// value-only forward (recomputed by the caller with keep_for_backward; no tangent
// slab is stored):
//   determinants   d log|psi| / d A_k = rho_k A_k^{-T}   (written by the det kernel)
//   orbitals       phi = P env:  dP = dphi env,  d env = dphi P;
//                  d pi, d sigma accumulated per thread, flushed once per CTA
//   projection     dW_orb = dP^T h_L, dg = column sums of dP, dh_L = dP W_orb
//   stream layer   dz = dh (1 - a^2); dV_self = X^T dz, db = sum dz,
//                  dU = Hbar^T (walker sums of dz); dX = dz V_self;
//                  dh_l = dX_h + dh_{l+1} (residual) + dHbar / n_spin
//   pair layer     one warp per pair, lane = channel; dW, dc reduced in registers,
//                  then per CTA, then one atomic per element (BF16 mode: warp-level
//                  BF16 MMAs over all pairs of a walker)
// In BF16 mode the large GEMMs run on the tensor cores (fn_layer_tc.cu): row-major
// products directly, weight gradients as split-K products over the electron rows on
// transposed BF16 copies.  Parameter gradients accumulate in the internal layout and
// are scattered back to the blob order at the end.
#include <algorithm>

#include "fn_device.cuh"
#include "fn_gemm.cuh"
#include "fn_internal.cuh"

namespace fn {

// ---- weights c_w = 2 (E_w - mean) / B -------------------------------------------------
// e and c may be the same buffer: each thread reads e[w] before writing c[w], and only
// after the barrier that ends the sum.
__global__ void k_energy_weights(int B, const double* e, double* c, double* __restrict__ mean_out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int w = threadIdx.x; w < B; w += blockDim.x) s += e[w];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  const double mean = red[0] / B;
  for (int w = threadIdx.x; w < B; w += blockDim.x) c[w] = 2.0 * (e[w] - mean) / B;
  if (threadIdx.x == 0 && mean_out) *mean_out = mean;
}

template <class Mode>
void launch_energy_weights(const fn_system* s, int B, const double* e_local, double* weights, double* e_mean,
                           cudaStream_t st) {
  ProfScope ps(s->prof, kProfBwdMisc, st);
  k_energy_weights<<<1, 1024, 0, st>>>(B, e_local, weights, e_mean);
}

// ---- column sums (atomic) -------------------------------------------------------------
template <typename T, typename Cmp>
__global__ void k_colsum(const T* __restrict__ src, int64_t rows, int64_t lds, int cols, Cmp* __restrict__ dst) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const int64_t chunk = (rows + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
  Cmp acc = 0;
  for (int64_t r = r0; r < r1; ++r) acc += (Cmp)ld(src + r * lds + c);
  atomicAdd(dst + c, acc);
}

template <typename T, typename Cmp>
static void colsum(const fn_system* s, cudaStream_t st, const T* src, int64_t rows, int64_t ld, int cols, Cmp* dst) {
  ProfScope ps(s->prof, kProfBwdMisc, st);
  dim3 grid((cols + 127) / 128, (unsigned)std::min<int64_t>(64, std::max<int64_t>(1, rows / 256)));
  k_colsum<T, Cmp><<<grid, 128, 0, st>>>(src, rows, ld, cols, dst);
}

// ---- BF16 operands of the tensor-core backward GEMMs (BF16 mode) ---------------------
// out[r][c] = bf16(in[r][c]) (when out is given) and outT[c][r] = bf16(in[r][c]) (when outT
// is given) over the R tile rows and `cols` columns; rows that hold no electron are written
// as zero.  32 x 32 tiles pass through shared memory, so the row-major reads and the
// transposed writes are both coalesced.
template <typename Tin>
__global__ void k_bf16_copy_T(Shape sh, const Tin* __restrict__ in, int64_t ld_in, int cols,
                              __nv_bfloat16* __restrict__ out, int64_t ld_out, __nv_bfloat16* __restrict__ outT) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32;
  const int64_t r0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int k = ty; k < 32; k += 8) {
    const int64_t r = r0 + k;
    const int c = c0 + tx;
    const int rr = (int)(r % kTileRows), q = (int)(r / kTileRows);
    const bool valid = rr / sh.N < sh.wpt && q * sh.wpt + rr / sh.N < sh.B;
    const float v = (c < cols && valid) ? (float)ld(in + r * ld_in + c) : 0.f;
    tile[k][tx] = v;
    if (out && c < cols) out[r * ld_out + c] = __float2bfloat16_rn(v);
  }
  if (!outT) return;
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int c = c0 + k;
    if (c < cols) outT[(int64_t)c * sh.R + r0 + tx] = __float2bfloat16_rn(tile[tx][k]);
  }
}

template <typename Tin>
static void bf16_copy_T(const fn_system* s, cudaStream_t st, const Shape& sh, const Tin* in, int64_t ld_in, int cols,
                        __nv_bfloat16* out, int64_t ld_out, __nv_bfloat16* outT) {
  ProfScope ps(s->prof, kProfBwdMisc, st);
  dim3 grid((cols + 31) / 32, (unsigned)(sh.R / 32));
  k_bf16_copy_T<Tin><<<grid, dim3(32, 8), 0, st>>>(sh, in, ld_in, cols, out, ld_out, outT);
}

// K splits of a weight-gradient GEMM (K = all rows): about two CTAs per SM, >= 4 k-blocks each.
static int ksplit_for(const fn_system* s, int rows, int ncols, int64_t k) {
  const int tiles = (rows + 127) / 128, ctiles = (ncols + 127) / 128;
  const int64_t nkb = (k + 63) / 64;
  const int want = std::max(1, 2 * s->sm_count / std::max(1, tiles * ctiles));
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, nkb / 4));
}

static void tc_or_flag(const fn_system* s, bool ok) {
  if (!ok) const_cast<fn_system*>(s)->host_error = FN_ERR_CUDA;
}

// ---- orbitals and envelopes ----------------------------------------------------------
struct OrbBwdArgs {
  const void* HL;            // [R][h1] value slab
  const void* wT[2]; const void* g[2]; const void* pi[2]; const void* sig[2];
  const void* dPhi;          // [B][K (nu^2 + nd^2)] rho_k A^{-T}
  const double* cw;          // [B]
  void* dP;                  // [R][K N]
  void* gpi[2]; void* gsig[2];
  int h1, K, aniso, chunk;
};

// Thread per orbital (k, i) of one spin, looping over a chunk of walkers and that spin's
// electrons j.  dP holds the projections P = h_L w + g on entry (written by a GEMM over
// all rows); the kernel replaces P by dphi env in the spin's own columns of row (w, j),
// zeroes the other spin's columns there, and accumulates the envelope gradients in
// registers (MM >= the number of nuclei bounds the unrolled per-nucleus arrays).
template <typename Cmp, typename Det, typename Wlk, int MM>
__global__ void k_orb_bwd(const Wlk* __restrict__ r, const double* __restrict__ nuc, Shape sh, OrbBwdArgs a) {
  const int spin = blockIdx.y;
  const int n = spin ? sh.n_dn : sh.n_up, n_o = spin ? sh.n_up : sh.n_dn;
  if (n == 0) return;
  const int n_ko = a.K * n, ko = threadIdx.x;
  const bool active = ko < n_ko;
  const int k = active ? ko / n : 0, i = active ? ko % n : 0;
  const Cmp* pi = (const Cmp*)a.pi[spin] + (int64_t)(active ? ko : 0) * sh.M;
  const Cmp* sg = (const Cmp*)a.sig[spin] + (int64_t)(active ? ko : 0) * sh.M * (a.aniso ? 9 : 1);
  Cmp pim[MM], S[MM][9], acc_pi[MM], acc_sig[MM][9];
#pragma unroll
  for (int m = 0; m < MM; ++m) {
    pim[m] = m < sh.M ? pi[m] : (Cmp)0;
    acc_pi[m] = 0;
#pragma unroll
    for (int x = 0; x < 9; ++x) {
      S[m][x] = m < sh.M ? (a.aniso ? sg[m * 9 + x] : (x == 0 ? sg[m] : (Cmp)0)) : (Cmp)0;
      acc_sig[m][x] = 0;
    }
  }
  const int64_t PW1 = (int64_t)a.K * (sh.n_up * sh.n_up + sh.n_dn * sh.n_dn);
  const int64_t inv_off = spin ? (int64_t)a.K * sh.n_up * sh.n_up : 0;
  const int ldp = a.K * sh.N, poff = spin ? a.K * sh.n_up : 0, poff_o = spin ? 0 : a.K * sh.n_up;
  const int w0 = blockIdx.x * a.chunk, w1 = min(sh.B, w0 + a.chunk);
  Cmp* dP = (Cmp*)a.dP;
  for (int w = w0; w < w1; ++w) {
    const Cmp cw = (Cmp)a.cw[w];
    for (int jj = 0; jj < n; ++jj) {
      const int j = jj + (spin ? sh.n_up : 0);
      const int64_t row = tile_row(w, j, sh.N, sh.wpt);
      if (ko < a.K * n_o) dP[row * ldp + poff_o + ko] = (Cmp)0;
      if (!active) continue;
      const Cmp P = dP[row * ldp + poff + ko] + ((const Cmp*)a.g[spin])[ko];
      const Wlk* rj = r + ((int64_t)w * sh.N + j) * 3;
      Cmp dv[MM][3], sv[MM], em[MM];
      Cmp env = 0;
#pragma unroll
      for (int m = 0; m < MM; ++m) {
        if (m >= sh.M) break;
#pragma unroll
        for (int c = 0; c < 3; ++c) dv[m][c] = (Cmp)((double)rj[c] - nuc[3 * m + c]);
        if (!a.aniso) {
          sv[m] = S[m][0] * f_sqrt(dv[m][0] * dv[m][0] + dv[m][1] * dv[m][1] + dv[m][2] * dv[m][2]);
        } else {
          Cmp u2 = 0;
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            const Cmp u = S[m][3 * x] * dv[m][0] + S[m][3 * x + 1] * dv[m][1] + S[m][3 * x + 2] * dv[m][2];
            u2 += u * u;
          }
          sv[m] = f_sqrt(u2);
        }
        em[m] = f_exp(-sv[m]);
        env += pim[m] * em[m];
      }
      const Cmp dphi = cw * (Cmp)((const Det*)a.dPhi)[(int64_t)w * PW1 + inv_off + (int64_t)k * n * n + i * n + jj];
      const Cmp denv = dphi * P;
      dP[row * ldp + poff + ko] = dphi * env;
#pragma unroll
      for (int m = 0; m < MM; ++m) {
        if (m >= sh.M) break;
        acc_pi[m] += denv * em[m];
        const Cmp f = -denv * pim[m] * em[m];
        if (!a.aniso) {
          acc_sig[m][0] += f * f_sqrt(dv[m][0] * dv[m][0] + dv[m][1] * dv[m][1] + dv[m][2] * dv[m][2]);
        } else {
          const Cmp inv_s = (Cmp)1 / sv[m];
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            const Cmp u = S[m][3 * x] * dv[m][0] + S[m][3 * x + 1] * dv[m][1] + S[m][3 * x + 2] * dv[m][2];
#pragma unroll
            for (int y = 0; y < 3; ++y) acc_sig[m][3 * x + y] += f * u * dv[m][y] * inv_s;
          }
        }
      }
    }
  }
  if (active) {
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      if (m >= sh.M) break;
      atomicAdd((Cmp*)a.gpi[spin] + (int64_t)ko * sh.M + m, acc_pi[m]);
      if (!a.aniso) atomicAdd((Cmp*)a.gsig[spin] + (int64_t)ko * sh.M + m, acc_sig[m][0]);
      else
#pragma unroll
        for (int x = 0; x < 9; ++x) atomicAdd((Cmp*)a.gsig[spin] + ((int64_t)ko * sh.M + m) * 9 + x, acc_sig[m][x]);
    }
  }
}

// ---- stream layers -------------------------------------------------------------------
template <typename Cmp>
__global__ void k_bwd_tanh(Shape sh, int h1, const Cmp* __restrict__ dH, const Cmp* __restrict__ act,
                           Cmp* __restrict__ dZ, Cmp* __restrict__ dZw) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)sh.B * h1) return;
  const int w = (int)(gid / h1), c = (int)(gid % h1);
  Cmp sum = 0;
  for (int i = 0; i < sh.N; ++i) {
    const int64_t row = tile_row(w, i, sh.N, sh.wpt);
    const Cmp a = act[row * h1 + c];
    const Cmp dz = dH[row * h1 + c] * ((Cmp)1 - a * a);
    dZ[row * h1 + c] = dz;
    sum += dz;
  }
  dZw[(int64_t)w * h1 + c] = sum;
}

template <typename Cmp>
__global__ void k_bwd_dh(Shape sh, int h1, int ldx, int d_h, const Cmp* __restrict__ dX,
                         const Cmp* __restrict__ dHbar, Cmp* __restrict__ dH) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)sh.B * sh.N * h1) return;
  const int c = (int)(gid % h1);
  const int64_t wi = gid / h1;
  const int w = (int)(wi / sh.N), i = (int)(wi % sh.N);
  const int s = i < sh.n_up ? 0 : 1;
  const int ns = s ? sh.n_dn : sh.n_up;
  const int64_t row = tile_row(w, i, sh.N, sh.wpt);
  dH[row * h1 + c] = dX[row * ldx + c] + dH[row * h1 + c] + dHbar[(int64_t)w * 2 * d_h + s * d_h + c] / (Cmp)ns;
}

// ---- two-electron stream, level l ----------------------------------------------------
struct PairBwdArgs {
  int l, L, h2, d_g;          // level, layers, pair width, input width of level l
  const void* g_in;           // g^l values [B][N][N][h2] (l >= 1), null: recompute features
  const void* g_out;          // g^{l+1} values (l < L-1)
  const void* W; const void* c;   // pair layer l weights [h2][d_g], [h2] (l < L-1)
  void* gW; void* gc;         // gradients of W_l, c_l
  void* dG;                   // [B][N][N][h2]: in dg^{l+1}, out dg^l
  const void* dX; int ldx; int col0;   // mean-g columns of the one-electron layer-l input gradient
};

template <typename Cmp, typename Wlk>
__global__ void __launch_bounds__(128) k_pair_bwd(const Wlk* __restrict__ r, Shape sh, PairBwdArgs a) {
  __shared__ Cmp red[4][32][33];
  __shared__ Cmp sW[32][33];                                   // W_l[q][c], zero outside [h2][d_g]
  const int w = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = sh.N;
  const bool has_layer = a.l < a.L - 1;
  if (has_layer)
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      const int q = e >> 5, c = e & 31;
      sW[q][c] = (q < a.h2 && c < a.d_g) ? ((const Cmp*)a.W)[q * a.d_g + c] : (Cmp)0;
    }
  __syncthreads();
  // dW[q][lane] and dc[lane] of this warp's pairs, in registers (the q loop is unrolled)
  Cmp accW[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) accW[q] = 0;
  Cmp accc = 0;
  const Wlk* rw = r + (int64_t)w * N * 3;
  // The loads of a warp's next pair are issued before the current pair's products, so
  // their latency overlaps the 32 x 32 accumulation.
  struct PairIn { Cmp gin, dgn, gout, dxv; };
  auto load = [&](int p) {
    PairIn v{(Cmp)0, (Cmp)0, (Cmp)0, (Cmp)0};
    if (p >= N * N) return v;
    const int i = p / N, j = p - i * N;
    const int64_t pidx = ((int64_t)w * N + i) * N + j;
    if (a.g_in) {
      v.gin = lane < a.d_g ? ((const Cmp*)a.g_in)[pidx * a.h2 + lane] : (Cmp)0;
    } else if (i != j && lane < 4) {
      const double d[3] = {(double)rw[3 * i] - (double)rw[3 * j], (double)rw[3 * i + 1] - (double)rw[3 * j + 1],
                           (double)rw[3 * i + 2] - (double)rw[3 * j + 2]};
      v.gin = lane == 0 ? (Cmp)d[0] : lane == 1 ? (Cmp)d[1] : lane == 2 ? (Cmp)d[2]
                                                  : (Cmp)sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
    if (has_layer && lane < a.h2) {
      v.dgn = ((const Cmp*)a.dG)[pidx * a.h2 + lane];
      v.gout = ((const Cmp*)a.g_out)[pidx * a.h2 + lane];
    }
    if (lane < a.d_g) {
      const int sj = j < sh.n_up ? 0 : 1;
      const int nsj = sj ? sh.n_dn : sh.n_up;
      const int64_t row = tile_row(w, i, N, sh.wpt);
      v.dxv = ((const Cmp*)a.dX)[row * a.ldx + a.col0 + sj * a.d_g + lane] / (Cmp)nsj;
    }
    return v;
  };
  PairIn cur = load(warp);
  for (int p = warp; p < N * N; p += 4) {
    const PairIn nxt = load(p + 4);
    const int i = p / N, j = p - (p / N) * N;
    const int64_t pidx = ((int64_t)w * N + i) * N + j;
    const Cmp gin = cur.gin;
    Cmp dgl = 0;
    if (has_layer) {
      const Cmp dgn = cur.dgn;
      const Cmp t = a.l >= 1 ? cur.gout - gin : cur.gout;
      const Cmp dz = lane < a.h2 ? dgn * ((Cmp)1 - t * t) : (Cmp)0;
      accc += dz;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const Cmp dzq = __shfl_sync(0xffffffffu, dz, q);      // zero for q >= h2
        accW[q] += dzq * gin;                                  // dW[q][lane]
        dgl += sW[q][lane] * dzq;
      }
      if (a.l >= 1) dgl += dgn;
    }
    dgl += cur.dxv;
    if (a.l >= 1 && lane < a.h2) ((Cmp*)a.dG)[pidx * a.h2 + lane] = dgl;
    cur = nxt;
  }
  if (!has_layer) return;
  // block reduction of dW (lane = column, q = row) and dc
#pragma unroll
  for (int q = 0; q < 32; ++q) red[warp][q][lane] = accW[q];
  __syncthreads();
  for (int e = threadIdx.x; e < a.h2 * a.d_g; e += blockDim.x) {
    const int q = e / a.d_g, c = e % a.d_g;
    const Cmp v = red[0][q][c] + red[1][q][c] + red[2][q][c] + red[3][q][c];
    atomicAdd((Cmp*)a.gW + e, v);
  }
  __syncthreads();
  red[warp][0][lane] = accc;
  __syncthreads();
  if (threadIdx.x < a.h2)
    atomicAdd((Cmp*)a.gc + threadIdx.x, red[0][0][threadIdx.x] + red[1][0][threadIdx.x] + red[2][0][threadIdx.x] +
                                             red[3][0][threadIdx.x]);
}

// BF16 mode: the same level on warp-level BF16 MMAs (hi/lo splits, three products, FP32
// accumulation).  Per walker, with dz = dG^{l+1} (1 - t^2) for all N^2 pairs in shared memory:
// the weight gradient dW = dz^T g^l (pairs as the contraction dimension; the four warps split
// the 32 x 32 output) and the input gradient dz W (pairs as rows), then one coalesced pass adds
// dG^{l+1} (residual, l >= 1) and the layer input's spin-mean gradient, as k_pair_bwd does.

template <typename Wlk>
__global__ void __launch_bounds__(128) k_pair_bwd_mma(const Wlk* __restrict__ r, Shape sh, PairBwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = lane >> 2, tig = lane & 3;
  const int N = sh.N, NP = N * N, NPp = (NP + 15) & ~15;
  const bool has_layer = a.l < a.L - 1;
  __nv_bfloat16* wth = (__nv_bfloat16*)smem_raw;                 // [32 c][kBwdWLd]: bf16(W[q][c]) at [c][q]
  __nv_bfloat16* wtl = wth + 32 * kBwdWLd;
  float* gin_s = (float*)(wtl + 32 * kBwdWLd);                   // [NPp][33] g^l, later dz W
  float* dz_s = gin_s + NPp * 33;                                // [NPp][33]
  const float* dG = (const float*)a.dG + (int64_t)w * NP * a.h2;
  if (has_layer) {
    const float* W = (const float*)a.W;                          // [h2][d_g]
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
      const int c = e >> 5, q = e & 31;
      const float v = (q < a.h2 && c < a.d_g) ? W[q * a.d_g + c] : 0.f;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      wth[c * kBwdWLd + q] = h;
      wtl[c * kBwdWLd + q] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
    for (int e = tid; e < NPp * 33; e += blockDim.x) { gin_s[e] = 0.f; dz_s[e] = 0.f; }
    __syncthreads();
    const Wlk* rw = r + (int64_t)w * N * 3;
    const float* gin_g = a.g_in ? (const float*)a.g_in + (int64_t)w * NP * a.h2 : nullptr;
    const float* gout_g = (const float*)a.g_out + (int64_t)w * NP * a.h2;
    // four elements per thread and round: all their global loads are issued before any use
    for (int e0 = tid; e0 < NP * 32; e0 += 4 * blockDim.x) {
      float gin[4], gout[4], dg[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * blockDim.x;
        const int p = e >> 5, c = e & 31;
        gin[u] = 0.f; gout[u] = 0.f; dg[u] = 0.f;
        if (e >= NP * 32) continue;
        if (gin_g) {
          if (c < a.d_g) gin[u] = gin_g[p * a.h2 + c];
        } else if (c < 4) {
          const int i = p / N, j = p - (p / N) * N;
          if (i != j) {
            const float d0 = (float)rw[3 * i] - (float)rw[3 * j], d1 = (float)rw[3 * i + 1] - (float)rw[3 * j + 1],
                        d2 = (float)rw[3 * i + 2] - (float)rw[3 * j + 2];
            gin[u] = c == 0 ? d0 : c == 1 ? d1 : c == 2 ? d2 : sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
          }
        }
        if (c < a.h2) {
          gout[u] = gout_g[p * a.h2 + c];
          dg[u] = dG[p * a.h2 + c];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e >= NP * 32) continue;
        const int p = e >> 5, c = e & 31;
        gin_s[p * 33 + c] = gin[u];
        if (c < a.h2) {
          const float t = a.l >= 1 ? gout[u] - gin[u] : gout[u];
          dz_s[p * 33 + c] = dg[u] * (1.f - t * t);
        }
      }
    }
    __syncthreads();
    // dc = column sums of dz: four partial sums per column, one atomic per column
    {
      __shared__ float dcs[4][32];
      const int q = tid & 31, k = tid >> 5;
      float sum = 0.f;
      for (int p = k; p < NP; p += 4) sum += dz_s[p * 33 + q];
      dcs[k][q] = sum;
      __syncthreads();
      if (tid < a.h2) atomicAdd((float*)a.gc + tid, dcs[0][tid] + dcs[1][tid] + dcs[2][tid] + dcs[3][tid]);
    }
    // dW[q][c] = sum_p dz[p][q] g[p][c]: warp -> rows q0 .. q0 + 15, column blocks nb0, nb0 + 1
    {
      const int q0 = (warp >> 1) * 16, nb0 = (warp & 1) * 2;
      float c2[2][4] = {};
      for (int p0 = 0; p0 < NPp; p0 += 16) {
        uint32_t ah[4], al[4];
        const float* zc0 = dz_s + (p0 + 2 * tig) * 33 + q0 + grp;      // A[m = q][k = p] = dz[p][q]
        split_pack(zc0[0], zc0[33], ah[0], al[0]);
        split_pack(zc0[8], zc0[33 + 8], ah[1], al[1]);
        split_pack(zc0[8 * 33], zc0[9 * 33], ah[2], al[2]);
        split_pack(zc0[8 * 33 + 8], zc0[9 * 33 + 8], ah[3], al[3]);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int n = 8 * (nb0 + u) + grp;                          // B[k = p][n = c] = g[p][c]
          const float* gc0 = gin_s + (p0 + 2 * tig) * 33 + n;
          uint32_t bh0, bl0, bh1, bl1;
          split_pack(gc0[0], gc0[33], bh0, bl0);
          split_pack(gc0[8 * 33], gc0[9 * 33], bh1, bl1);
          mma_16816(c2[u], ah, bh0, bh1);
          mma_16816(c2[u], ah, bl0, bl1);
          mma_16816(c2[u], al, bh0, bh1);
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const int qq = q0 + grp + (q4 >= 2 ? 8 : 0), cc = 8 * (nb0 + u) + 2 * tig + (q4 & 1);
          if (qq < a.h2 && cc < a.d_g) atomicAdd((float*)a.gW + qq * a.d_g + cc, c2[u][q4]);
        }
    }
    __syncthreads();                                               // gin_s is overwritten below
    // dz W -> gin_s (rows = pairs)
    for (int mt = warp; mt < NPp / 16; mt += (int)(blockDim.x >> 5)) {
      const int p0 = mt * 16;
      float c[4][4] = {};
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const int k0 = ks * 16;
        const float* r0 = dz_s + (p0 + grp) * 33 + k0 + 2 * tig;
        const float* r1 = dz_s + (p0 + grp + 8) * 33 + k0 + 2 * tig;
        uint32_t ah[4], al[4];
        split_pack(r0[0], r0[1], ah[0], al[0]);
        split_pack(r1[0], r1[1], ah[1], al[1]);
        split_pack(r0[8], r0[9], ah[2], al[2]);
        split_pack(r1[8], r1[9], ah[3], al[3]);
#pragma unroll
        for (int nb = 0; nb < 4; ++nb) {
          const int off = (8 * nb + grp) * kBwdWLd + k0 + 2 * tig;
          const uint32_t bh0 = *(const uint32_t*)(wth + off), bh1 = *(const uint32_t*)(wth + off + 8);
          const uint32_t bl0 = *(const uint32_t*)(wtl + off), bl1 = *(const uint32_t*)(wtl + off + 8);
          mma_16816(c[nb], ah, bh0, bh1);
          mma_16816(c[nb], ah, bl0, bl1);
          mma_16816(c[nb], al, bh0, bh1);
        }
      }
#pragma unroll
      for (int nb = 0; nb < 4; ++nb)
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4)
          gin_s[(p0 + grp + (q4 >= 2 ? 8 : 0)) * 33 + 8 * nb + 2 * tig + (q4 & 1)] = c[nb][q4];
    }
    __syncthreads();
  }
  if (a.l < 1) return;                                             // no gradient below the input features
  // dG^l = (dz W) + dG^{l+1} (residual) + the spin-mean gradient of the layer input
  float* dGo = (float*)a.dG + (int64_t)w * NP * a.h2;
  for (int e = tid; e < NP * a.h2; e += blockDim.x) {
    const int p = e / a.h2, c = e - (e / a.h2) * a.h2;
    const int i = p / N, j = p - (p / N) * N;
    float v = 0.f;
    if (has_layer) v = gin_s[p * 33 + c] + dGo[e];
    if (c < a.d_g) {
      const int sj = j < sh.n_up ? 0 : 1;
      const int nsj = sj ? sh.n_dn : sh.n_up;
      v += ((const float*)a.dX)[tile_row(w, i, N, sh.wpt) * a.ldx + a.col0 + sj * a.d_g + c] / (float)nsj;
    }
    dGo[e] = v;
  }
}

// ---- internal layout -> blob order ---------------------------------------------------
template <typename Par, typename Cmp>
__global__ void k_unprep(Par* __restrict__ blob, const CopyDesc* __restrict__ descs, const Cmp* __restrict__ gradc) {
  const CopyDesc d = descs[blockIdx.y];
  if (d.to16) return;
  const int64_t n = (int64_t)d.rows * d.cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rr = e / d.cols, cc = e % d.cols;
    blob[d.src + rr * d.s_rs + cc * d.s_cs] = (Par)gradc[d.dst + rr * d.d_rs + cc * d.d_cs];
  }
}

template <class Mode>
void launch_backward(const fn_system* s, const void* walkers, const Shape& sh, const double* weights, void* grad,
                     cudaStream_t st) {
  using Act = typename Mode::Act; using Cmp = typename Mode::Cmp; using Det = typename Mode::Det;
  using Wlk = typename Mode::Wlk; using Par = typename Mode::Par;
  const Workspace& ws = s->ws;
  const int L = s->cfg.n_layers, h1 = s->cfg.h1, h2 = s->cfg.h2, K = s->cfg.n_dets, N = s->N;
  const Cmp* prep = (const Cmp*)ws.prep;
  Cmp* gradc = (Cmp*)ws.gradc;
  const PrepLayout& pl = s->prep;
  const Wlk* r = (const Wlk*)walkers;
  const int64_t R = sh.R;
  const int ldp = K * N;
  const int split = (int)std::max<int64_t>(1, std::min<int64_t>(64, R / 1024));
  cudaMemsetAsync(gradc, 0, sizeof(Cmp) * pl.total, st);
  cudaMemsetAsync(ws.dH, 0, sizeof(Cmp) * R * h1, st);
  // orbitals + envelopes: P = h_L w (both spins, every row), then the envelope kernel turns
  // it into dP in place; rows that hold no electron are zeroed for the weight GEMMs below
  constexpr bool kTc = Mode::kMode == FN_BF16_MIXED;
  const __nv_bfloat16* prep16 = (const __nv_bfloat16*)ws.prep16;
  {
    ProfScope ps(s->prof, kProfBwdGemm, st);
    if (kTc) {
      tc_or_flag(s, launch_gemm_tc((int)R, h1, ws.HL, h1, prep16 + pl.W16, 2 * h1, h1, ldp, (float*)ws.dP, ldp, nullptr,
                                   0, 1, false, ws.status, st));
    } else {
      for (int q = 0; q < 2; ++q) {
        const int n_q = q ? s->n_dn : s->n_up;
        if (!n_q) continue;
        gemm<Act, Cmp, Cmp, Cmp>(st, (int)R, K * n_q, h1, (const Act*)ws.HL, h1, 1, prep + pl.wT[q], K * n_q, 1,
                                 (Cmp*)ws.dP + (q ? K * s->n_up : 0), ldp, 1, (const Cmp*)nullptr, 0, 1, false);
      }
    }
  }
  {
    const size_t row_bytes = sizeof(Cmp) * ldp;
    const int used = sh.wpt * N;
    if (used < kTileRows)
      cudaMemset2DAsync((char*)ws.dP + used * row_bytes, kTileRows * row_bytes, 0, (kTileRows - used) * row_bytes,
                        sh.tiles, st);
    const int last = sh.B - (sh.tiles - 1) * sh.wpt;
    if (last < sh.wpt)
      cudaMemsetAsync((char*)ws.dP + ((int64_t)(sh.tiles - 1) * kTileRows + (int64_t)last * N) * row_bytes, 0,
                      (size_t)(sh.wpt - last) * N * row_bytes, st);
  }
  {
    OrbBwdArgs a{};
    a.HL = ws.HL;
    for (int q = 0; q < 2; ++q) {
      a.wT[q] = prep + pl.wT[q]; a.g[q] = prep + pl.g[q]; a.pi[q] = prep + pl.pi[q]; a.sig[q] = prep + pl.sig[q];
      a.gpi[q] = gradc + pl.pi[q]; a.gsig[q] = gradc + pl.sig[q];
    }
    a.dPhi = ws.dPhi; a.cw = weights; a.dP = ws.dP;
    a.h1 = h1; a.K = K; a.aniso = s->cfg.envelope == FN_ENV_ANISOTROPIC;
    a.chunk = std::max(1, sh.B / (4 * s->sm_count));
    const int threads = (int)std::min<int64_t>(1024, round_up((int64_t)K * std::max(s->n_up, s->n_dn), 32));
    dim3 grid((sh.B + a.chunk - 1) / a.chunk, 2);
    ProfScope ps(s->prof, kProfBwdOrb, st);
    if (s->M <= 2) k_orb_bwd<Cmp, Det, Wlk, 2><<<grid, threads, 0, st>>>(r, s->d_nuclei, sh, a);
    else if (s->M <= 4) k_orb_bwd<Cmp, Det, Wlk, 4><<<grid, threads, 0, st>>>(r, s->d_nuclei, sh, a);
    else if (s->M <= 8) k_orb_bwd<Cmp, Det, Wlk, 8><<<grid, threads, 0, st>>>(r, s->d_nuclei, sh, a);
    else k_orb_bwd<Cmp, Det, Wlk, kMaxNuclei><<<grid, threads, 0, st>>>(r, s->d_nuclei, sh, a);
  }
  const int ns[2] = {s->n_up, s->n_dn};
  __nv_bfloat16* g16 = (__nv_bfloat16*)ws.g16;
  __nv_bfloat16* t16a = (__nv_bfloat16*)ws.t16a;
  __nv_bfloat16* t16b = (__nv_bfloat16*)ws.t16b;
  if (kTc) {
    // dP as a bf16 row-major copy and transposed; h_L transposed
    bf16_copy_T<Cmp>(s, st, sh, (const Cmp*)ws.dP, ldp, ldp, g16, pl.ldWT, t16b);
    bf16_copy_T<Act>(s, st, sh, (const Act*)ws.HL, h1, h1, nullptr, 0, t16a);
    for (int q = 0; q < 2; ++q) {
      if (!ns[q]) continue;
      const int n_ko = K * ns[q];
      // dW_orb^T [h1][K n] += h_L^T dP (K = all rows, split)
      {
        ProfScope ps(s->prof, kProfBwdGemm, st);
        tc_or_flag(s, launch_gemm_tc(h1, (int)R, t16a, (int)R, t16b + (int64_t)(q ? K * s->n_up : 0) * R, (int)R, 0,
                                     n_ko, (float*)(gradc + pl.wT[q]), n_ko, nullptr, 0,
                                     ksplit_for(s, h1, n_ko, R), true, ws.status, st));
      }
      colsum<Cmp, Cmp>(s, st, (const Cmp*)ws.dP + (q ? K * s->n_up : 0), R, ldp, n_ko, gradc + pl.g[q]);
    }
    // dh_L = dP W (both spins: the other spin's columns of a row are zero)
    ProfScope ps(s->prof, kProfBwdGemm, st);
    tc_or_flag(s, launch_gemm_tc((int)R, ldp, g16, pl.ldWT, prep16 + pl.W16T, 2 * pl.ldWT, pl.ldWT, h1, (float*)ws.dH,
                                 h1, nullptr, 0, 1, false, ws.status, st));
  }
  for (int q = 0; q < 2 && !kTc; ++q) {
    if (!ns[q]) continue;
    const int n_ko = K * ns[q];
    const Cmp* dPq = (const Cmp*)ws.dP + (q ? K * s->n_up : 0);
    // dW_orb^T [h1][K n]: sum over rows of h_L[row][c] dP[row][ko]
    {
      ProfScope ps(s->prof, kProfBwdGemm, st);
      gemm<Act, Cmp, Cmp, Cmp>(st, h1, n_ko, (int)R, (const Act*)ws.HL, 1, h1, dPq, ldp, 1, gradc + pl.wT[q], n_ko, 1,
                               (const Cmp*)nullptr, 0, split, true);
    }
    colsum<Cmp, Cmp>(s, st, dPq, R, ldp, n_ko, gradc + pl.g[q]);
    // dh_L[row][c] += sum_ko dP[row][ko] w[ko][c]
    {
      ProfScope ps(s->prof, kProfBwdGemm, st);
      gemm<Cmp, Cmp, Cmp, Cmp>(st, (int)R, h1, n_ko, dPq, ldp, 1, prep + pl.wT[q], 1, n_ko, (Cmp*)ws.dH, h1, 1,
                               (const Cmp*)nullptr, 0, 1, true);
    }
  }
  Cmp* dH = (Cmp*)ws.dH;
  Cmp* dZ = (Cmp*)ws.dZ;
  Cmp* dZw = (Cmp*)ws.dZw;
  Cmp* dX = (Cmp*)ws.dX;
  Cmp* dHbar = (Cmp*)ws.dHbar;
  for (int l = L - 1; l >= 0; --l) {
    const LayerDims& d = s->layer[l];
    cudaMemsetAsync(dZ, 0, sizeof(Cmp) * R * h1, st);
    {
      const int64_t n = (int64_t)sh.B * h1;
      ProfScope ps(s->prof, kProfBwdMisc, st);
      k_bwd_tanh<Cmp><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sh, h1, dH, (const Cmp*)ws.act[l], dZ, dZw);
    }
    const Act* X = (const Act*)ws.X[l];
    if (kTc) {
      // bf16 operands: dZ row-major and transposed, X_l transposed
      bf16_copy_T<Cmp>(s, st, sh, dZ, h1, h1, g16, h1, t16b);
      bf16_copy_T<Act>(s, st, sh, X, d.ldx, d.k_self, nullptr, 0, t16a);
    }
    // dV_self (internal [k_self][h1]) += X^T dZ
    {
      ProfScope ps(s->prof, kProfBwdGemm, st);
      if (kTc)
        tc_or_flag(s, launch_gemm_tc(d.k_self, (int)R, t16a, (int)R, t16b, (int)R, 0, h1, (float*)(gradc + pl.VsT[l]),
                                     h1, nullptr, 0, ksplit_for(s, d.k_self, h1, R), true, ws.status, st));
      else
        gemm<Act, Cmp, Cmp, Cmp>(st, d.k_self, h1, (int)R, X, 1, d.ldx, dZ, h1, 1, gradc + pl.VsT[l], h1, 1,
                                 (const Cmp*)nullptr, 0, split, true);
    }
    colsum<Cmp, Cmp>(s, st, dZw, sh.B, h1, h1, gradc + pl.b[l]);
    // dU (internal [2 d_h][h1]) += Hbar^T dZw
    const int splitB = (int)std::max(1, std::min(32, sh.B / 256));
    {
      ProfScope ps(s->prof, kProfBwdGemm, st);
      gemm<Act, Cmp, Cmp, Cmp>(st, 2 * d.d_h, h1, sh.B, (const Act*)ws.Hbar[l], 1, 2 * d.d_h, dZw, h1, 1,
                               gradc + pl.UT[l], h1, 1, (const Cmp*)nullptr, 0, splitB, true);
    }
    // dX = dZ V_self^T  ([R][k_self], row stride ldx)
    {
      ProfScope ps(s->prof, kProfBwdGemm, st);
      if (kTc)
        tc_or_flag(s, launch_gemm_tc((int)R, h1, g16, h1, prep16 + pl.VsT16[l], 2 * h1, h1, d.k_self, (float*)dX, d.ldx,
                                     nullptr, 0, 1, false, ws.status, st));
      else
        gemm<Cmp, Cmp, Cmp, Cmp>(st, (int)R, d.k_self, h1, dZ, h1, 1, prep + pl.VsT[l], 1, h1, dX, d.ldx, 1,
                                 (const Cmp*)nullptr, 0, 1, false);
    }
    if (l >= 1) {
      {
        ProfScope ps(s->prof, kProfBwdGemm, st);
        gemm<Cmp, Cmp, Cmp, Cmp>(st, sh.B, 2 * d.d_h, h1, dZw, h1, 1, prep + pl.UT[l], 1, h1, dHbar, 2 * d.d_h, 1,
                                 (const Cmp*)nullptr, 0, 1, false);
      }
      const int64_t n = (int64_t)sh.B * N * h1;
      ProfScope ps(s->prof, kProfBwdMisc, st);
      k_bwd_dh<Cmp><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sh, h1, d.ldx, d.d_h, dX, dHbar, dH);
    }
    // two-electron stream level l
    if (L > 1) {
      PairBwdArgs a{};
      a.l = l; a.L = L; a.h2 = h2; a.d_g = d.d_g;
      a.g_in = l >= 1 ? ws.gpair[l] : nullptr;
      a.g_out = l < L - 1 ? ws.gpair[l + 1] : nullptr;
      if (l < L - 1) {
        a.W = prep + pl.W[l]; a.c = prep + pl.c[l];
        a.gW = gradc + pl.W[l]; a.gc = gradc + pl.c[l];
      }
      a.dG = ws.dG; a.dX = dX; a.ldx = d.ldx; a.col0 = d.d_h;
      ProfScope ps(s->prof, kProfBwdPair, st);
      if (Mode::kMode == FN_BF16_MIXED) {
        const size_t smem = smem_pair_bwd_mma(N);
        cudaFuncSetAttribute(k_pair_bwd_mma<Wlk>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_pair_bwd_mma<Wlk><<<sh.B, 128, smem, st>>>(r, sh, a);
      } else {
        k_pair_bwd<Cmp, Wlk><<<sh.B, 128, 0, st>>>(r, sh, a);
      }
    }
  }
  dim3 grid(32, s->n_descs);
  ProfScope ps(s->prof, kProfBwdMisc, st);
  k_unprep<Par, Cmp><<<grid, 256, 0, st>>>((Par*)grad, (const CopyDesc*)s->d_descs, gradc);
}

#define FN_INST(M)                                                                                           \
  template void launch_energy_weights<M>(const fn_system*, int, const double*, double*, double*, cudaStream_t); \
  template void launch_backward<M>(const fn_system*, const void*, const Shape&, const double*, void*, cudaStream_t);
FN_INST(ModeF64)
FN_INST(ModeF32)
FN_INST(ModeBF16)

}  // namespace fn
