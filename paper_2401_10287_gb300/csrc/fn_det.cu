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
#include <climits>
#include <cstdlib>
#include <cstring>
#include <type_traits>

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

// One thread factorises one small matrix held in shared memory with element (i, j) at
// A[(i n + j) ST] (ST = number of matrices interleaved, so neighbouring threads touch
// neighbouring words).  Partial pivoting picks the first maximal |pivot|; the
// determinant is tracked as mantissa * 2^exponent so that a single log per matrix is
// needed; the pivot reciprocals are kept for the inverse.
// Widening of a stored orbital entry to the determinant type.  FP32 -> FP64 goes through
// integer bit operations (sign, exponent re-biased by 1023 - 127, mantissa shifted into the
// top of the 52-bit field): exact for every normal FP32 value, FP32 subnormals become signed
// zero, infinities and NaNs keep their class.  It keeps the conversions off the FP64 pipe,
// which sets the pace of this stage.
template <typename Det, typename PhiT> __device__ __forceinline__ Det widen(PhiT v) { return (Det)v; }
template <> __device__ __forceinline__ double widen<double, float>(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xFFu, sign = u & 0x80000000u, man = u & 0x7FFFFFu;
  const uint32_t ex64 = ex == 0 ? 0u : (ex == 0xFFu ? 0x7FFu : ex + 896u);
  const uint32_t hi = sign | (ex64 << 20) | (ex == 0 ? 0u : (man >> 3));
  const uint32_t lo = ex == 0 ? 0u : (man << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// Pivot search key: |v| as an unsigned integer (the bit patterns of non-negative IEEE
// numbers order like their values), so the comparisons leave the FP64 pipe alone.
__device__ __forceinline__ unsigned long long abs_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned int abs_key(float v) { return __float_as_uint(v) & 0x7FFFFFFFu; }

template <typename Det>
__device__ void thread_lu(Det* A, int n, int ST, int* perm, Det* rcp, Det* ld_out, Det* sign_out) {
  Det sgn = 1, mant = 1;
  int expo = 0;
  bool singular = false;
  for (int i = 0; i < n; ++i) perm[i * ST] = i;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    auto best = abs_key(A[(c * n + c) * ST]);
    for (int r = c + 1; r < n; ++r) {
      const auto v = abs_key(A[(r * n + c) * ST]);
      if (v > best) { best = v; piv = r; }
    }
    if (best == 0) { singular = true; break; }
    if (piv != c) {
      for (int j = 0; j < n; ++j) {
        const Det t = A[(c * n + j) * ST];
        A[(c * n + j) * ST] = A[(piv * n + j) * ST];
        A[(piv * n + j) * ST] = t;
      }
      const int tp = perm[c * ST]; perm[c * ST] = perm[piv * ST]; perm[piv * ST] = tp;
      sgn = -sgn;
    }
    const Det p = A[(c * n + c) * ST];
    const Det rp = (Det)1 / p;
    rcp[c * ST] = rp;
    int e;
    mant *= frexp(p, &e);
    expo += e;
    int e2;
    mant = frexp(mant, &e2);
    expo += e2;
    for (int r = c + 1; r < n; ++r) {
      const Det f = A[(r * n + c) * ST] * rp;
      A[(r * n + c) * ST] = f;
      for (int j = c + 1; j < n; ++j) A[(r * n + j) * ST] -= f * A[(c * n + j) * ST];
    }
  }
  if (singular) {
    *ld_out = 0;
    *sign_out = 0;
    return;
  }
  *sign_out = mant < 0 ? -sgn : sgn;
  *ld_out = f_log(f_abs(mant)) + (Det)expo * (Det)0.6931471805599453;
}

// C = A^{-1} from the factors of thread_lu (same interleaving): column j of C solves
// L U x = e_{perm^-1(j)}.
template <typename Det>
__device__ void thread_inverse(const Det* A, const int* perm, const Det* rcp, int n, int ST, Det* C) {
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) {
      Det y = perm[i * ST] == j ? (Det)1 : (Det)0;
      for (int k = 0; k < i; ++k) y -= A[(i * n + k) * ST] * C[(k * n + j) * ST];
      C[(i * n + j) * ST] = y;
    }
    for (int i = n - 1; i >= 0; --i) {
      Det x = C[(i * n + j) * ST];
      for (int k = i + 1; k < n; ++k) x -= A[(i * n + k) * ST] * C[(k * n + j) * ST];
      C[(i * n + j) * ST] = x * rcp[i * ST];
    }
  }
}

// Tangent item for an n x n block with n known at compile time: B = C D row by row with n
// independent accumulators (no serial dot-product chains), then g = tr B and q = tr(B^2)
// from the registers.  C is interleaved with stride ST; D is the slab in global memory.
template <int NN, typename Det, typename PhiT>
__device__ __forceinline__ void tangent_item_fixed(const Det* __restrict__ Cm, int ST, const PhiT* __restrict__ D,
                                                   Det* g_out, Det* q_out) {
  Det B[NN][NN];
  Det d[NN][NN];
#pragma unroll
  for (int m = 0; m < NN; ++m)
#pragma unroll
    for (int j = 0; j < NN; ++j) d[m][j] = widen<Det, PhiT>(D[m * NN + j]);
#pragma unroll
  for (int i = 0; i < NN; ++i) {
#pragma unroll
    for (int j = 0; j < NN; ++j) B[i][j] = 0;
#pragma unroll
    for (int m = 0; m < NN; ++m) {
      const Det c = Cm[(int64_t)(i * NN + m) * ST];
#pragma unroll
      for (int j = 0; j < NN; ++j) B[i][j] += c * d[m][j];
    }
  }
  Det g = 0, q = 0;
#pragma unroll
  for (int i = 0; i < NN; ++i) {
    g += B[i][i];
    q += B[i][i] * B[i][i];
#pragma unroll
    for (int j = i + 1; j < NN; ++j) q += (Det)2 * B[i][j] * B[j][i];
  }
  *g_out = g;
  *q_out = q;
}

// Same for any n (serial dots; used for blocks larger than 8).
template <typename Det, typename PhiT>
__device__ void tangent_item_any(const Det* __restrict__ Cm, int ST, const PhiT* __restrict__ D, int n, Det* g_out,
                                 Det* q_out) {
  Det g = 0, q = 0;
  for (int i = 0; i < n; ++i) {
    for (int j = i; j < n; ++j) {
      Det bij = 0;
      for (int m = 0; m < n; ++m) bij += Cm[(int64_t)(i * n + m) * ST] * widen<Det, PhiT>(D[m * n + j]);
      if (j == i) {
        g += bij;
        q += bij * bij;
      } else {
        Det bji = 0;
        for (int m = 0; m < n; ++m) bji += Cm[(int64_t)(j * n + m) * ST] * widen<Det, PhiT>(D[m * n + i]);
        q += (Det)2 * bij * bji;
      }
    }
  }
  *g_out = g;
  *q_out = q;
}

template <typename Det, typename PhiT>
__device__ __forceinline__ void tangent_item(const Det* Cm, int ST, const PhiT* D, int n, Det* g, Det* q) {
  switch (n) {
    case 1: tangent_item_fixed<1>(Cm, ST, D, g, q); break;
    case 2: tangent_item_fixed<2>(Cm, ST, D, g, q); break;
    case 3: tangent_item_fixed<3>(Cm, ST, D, g, q); break;
    case 4: tangent_item_fixed<4>(Cm, ST, D, g, q); break;
    case 5: tangent_item_fixed<5>(Cm, ST, D, g, q); break;
    case 6: tangent_item_fixed<6>(Cm, ST, D, g, q); break;
    case 7: tangent_item_fixed<7>(Cm, ST, D, g, q); break;
    case 8: tangent_item_fixed<8>(Cm, ST, D, g, q); break;
    default: tangent_item_any(Cm, ST, D, n, g, q); break;
  }
}

// ---- double-FP32 tangent products (BF16-mixed mode) -------------------------------------
// In the BF16-mixed mode the orbital tangents D are FP32 values and C = A^-1 is FP64.  The
// products B = C D, g = tr B and q = tr(B^2) are evaluated in double-FP32 arithmetic on the
// FP32 pipe, which on this part runs 64 times as many operations per clock as the FP64
// pipe: C = c_hi + c_lo (two FP32 values, 48 significant bits), every D entry is exact in
// FP32, each product c_hi d is split exactly by an FMA (Dekker's two-product), sums are
// accumulated with Knuth's error-free two-sum and the small terms (c_lo d, the rounding
// errors) in a second FP32 word.  The result carries about 46 significant bits, converted to
// FP64 at the end; the LU, the inverse and every later step stay FP64.
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (sh, sl) += (xh, xl) * (yh, yl) * scale, scale = 1 or 2 (exact)
__device__ __forceinline__ void ff_fma_acc(float xh, float xl, float yh, float yl, float scale, float& sh,
                                           float& sl) {
  const float p = __fmul_rn(xh, yh);
  float pe = __fmaf_rn(xh, yh, -p);
  pe = __fmaf_rn(xh, yl, __fmaf_rn(xl, yh, pe));
  float s, e;
  ff_two_sum(sh, __fmul_rn(p, scale), s, e);
  sh = s;
  sl = __fadd_rn(sl, __fmaf_rn(pe, scale, e));
}

template <int NN>
__device__ __forceinline__ void tangent_item_ff(const float* __restrict__ Ch, const float* __restrict__ Cl, int ST,
                                                const float* __restrict__ D, double* g_out, double* q_out) {
  float bh[NN][NN], bl[NN][NN];
#pragma unroll
  for (int i = 0; i < NN; ++i)
#pragma unroll
    for (int j = 0; j < NN; ++j) { bh[i][j] = 0.f; bl[i][j] = 0.f; }
#pragma unroll
  for (int m = 0; m < NN; ++m) {
    float d[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) d[j] = D[m * NN + j];
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      const float ch = Ch[(i * NN + m) * ST], cl = Cl[(i * NN + m) * ST];
#pragma unroll
      for (int j = 0; j < NN; ++j) {
        const float p = __fmul_rn(ch, d[j]);
        const float pe = __fmaf_rn(ch, d[j], -p);
        float s, e;
        ff_two_sum(bh[i][j], p, s, e);
        bh[i][j] = s;
        bl[i][j] = __fmaf_rn(cl, d[j], __fadd_rn(bl[i][j], __fadd_rn(e, pe)));
      }
    }
  }
  float gh = 0.f, gl = 0.f, qh = 0.f, ql = 0.f;
#pragma unroll
  for (int i = 0; i < NN; ++i) {
    float s, e;
    ff_two_sum(gh, bh[i][i], s, e);
    gh = s;
    gl = __fadd_rn(gl, __fadd_rn(e, bl[i][i]));
    ff_fma_acc(bh[i][i], bl[i][i], bh[i][i], bl[i][i], 1.f, qh, ql);
#pragma unroll
    for (int j = i + 1; j < NN; ++j) ff_fma_acc(bh[i][j], bl[i][j], bh[j][i], bl[j][i], 2.f, qh, ql);
  }
  *g_out = (double)gh + (double)gl;
  *q_out = (double)qh + (double)ql;
}

template <typename Det, typename PhiT>
__device__ __forceinline__ bool tangent_item_split(const float* Ch, const float* Cl, int ST, const PhiT* D, int n,
                                                   Det* g, Det* q) {
  if constexpr (std::is_same<Det, double>::value && std::is_same<PhiT, float>::value) {
    switch (n) {
      case 1: tangent_item_ff<1>(Ch, Cl, ST, D, g, q); return true;
      case 2: tangent_item_ff<2>(Ch, Cl, ST, D, g, q); return true;
      case 3: tangent_item_ff<3>(Ch, Cl, ST, D, g, q); return true;
      case 4: tangent_item_ff<4>(Ch, Cl, ST, D, g, q); return true;
      case 5: tangent_item_ff<5>(Ch, Cl, ST, D, g, q); return true;
      case 6: tangent_item_ff<6>(Ch, Cl, ST, D, g, q); return true;
      case 7: tangent_item_ff<7>(Ch, Cl, ST, D, g, q); return true;
      case 8: tangent_item_ff<8>(Ch, Cl, ST, D, g, q); return true;
      default: return false;
    }
  }
  return false;
}

// Local-energy pass: one CTA per walker.  Threads 0..2K-1 factorise and invert the
// (determinant, spin) blocks; then every thread takes (block, coordinate) items
// g_t = tr(C d_t A), q_t = tr((C d_t A)^2) and tr(C lap A); then the determinant terms
// are combined and E_L assembled.
template <typename Det, typename Wlk, typename PhiT>
__global__ void __launch_bounds__(128) k_det_energy(const Wlk* __restrict__ r, const double* __restrict__ nuc,
                                                    Shape sh, DetArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = blockIdx.x, tid = threadIdx.x;
  const int N = sh.N, T = sh.T, K = a.K, NC = 3 * N, NM = 2 * K;
  const int ST = (int)round_up(NM, 32);
  const int ns[2] = {sh.n_up, sh.n_dn};
  const int nmax = max(ns[0], ns[1]);
  Det* A = (Det*)smem_raw;                                // [nmax^2][ST]
  Det* C = A + (int64_t)nmax * nmax * ST;                 // [nmax^2][ST]
  Det* rcp = C + (int64_t)nmax * nmax * ST;               // [nmax][ST]
  Det* ld2 = rcp + (int64_t)nmax * ST;                   // [NM]
  Det* sg2 = ld2 + NM;                                   // [NM]
  Det* gt = sg2 + NM;                                    // [NM][NC]
  Det* qt = gt + NM * NC;                                // [NM][NC]
  Det* lt = qt + NM * NC;                                // [NM]
  Det* gradk = lt + NM;                                  // [K][NC]
  Det* lapk = gradk + K * NC;                            // [K]
  Det* rho = lapk + K;                                   // [K]
  Det* red = rho + K;                                    // [128]
  int* perm = (int*)(red + 128);                         // [nmax][ST]
  // double-FP32 copies of C (BF16-mixed mode): [nmax^2][ST] high words, then low words
  constexpr bool kSplit = std::is_same<Det, double>::value && std::is_same<PhiT, float>::value;
  float* Ch = (float*)(perm + (int64_t)nmax * ST);
  float* Cl = Ch + (int64_t)nmax * nmax * ST;
  const PhiT* Phi = (const PhiT*)a.Phi + (int64_t)w * a.PW;
  const int64_t blk_off[2] = {0, (int64_t)K * T * ns[0] * ns[0]};
  // value slabs of every block, interleaved by block (thread 2k + spin)
  for (int sp = 0; sp < 2; ++sp) {
    const int nn = ns[sp] * ns[sp];
    for (int e = tid; e < K * nn; e += blockDim.x) {
      const int k = e / nn, idx = e % nn;
      A[(int64_t)idx * ST + 2 * k + sp] = widen<Det, PhiT>(Phi[blk_off[sp] + (int64_t)k * T * nn + idx]);
    }
  }
  __syncthreads();
  if (tid < NM) {
    const int n = ns[tid & 1];
    if (n == 0) {
      ld2[tid] = 0;
      sg2[tid] = 1;
    } else {
      thread_lu<Det>(A + tid, n, ST, perm + tid, rcp + tid, ld2 + tid, sg2 + tid);
      if (sg2[tid] != 0) thread_inverse<Det>(A + tid, perm + tid, rcp + tid, n, ST, C + tid);
      else for (int e = 0; e < n * n; ++e) C[(int64_t)e * ST + tid] = 0;
      if (kSplit && n <= 8) {
        for (int e = 0; e < n * n; ++e) {
          const double c = (double)C[(int64_t)e * ST + tid];
          const float ch = __double2float_rn(c);
          Ch[(int64_t)e * ST + tid] = ch;
          Cl[(int64_t)e * ST + tid] = __double2float_rn(c - (double)ch);
        }
      }
    }
  }
  __syncthreads();
  // items: (block p, coordinate t < NC) and (block p, Laplacian)
  const int per = NC + 1;
  for (int it = tid; it < NM * per; it += blockDim.x) {
    const int p = it / per, tr = it % per;
    const int k = p >> 1, sp = p & 1, n = ns[sp];
    if (n == 0) {
      if (tr < NC) { gt[p * NC + tr] = 0; qt[p * NC + tr] = 0; } else { lt[p] = 0; }
      continue;
    }
    const Det* Cm = C + p;
    const int t = tr < NC ? 1 + tr : T - 1;
    const PhiT* D = Phi + blk_off[sp] + (int64_t)k * T * n * n + (int64_t)t * n * n;
    if (tr < NC) {
      Det g, q;
      if (!tangent_item_split<Det, PhiT>(Ch + p, Cl + p, ST, D, n, &g, &q)) tangent_item<Det, PhiT>(Cm, ST, D, n, &g, &q);
      gt[p * NC + tr] = g;
      qt[p * NC + tr] = q;
    } else {
      Det l = 0;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) l += Cm[(int64_t)(j * n + i) * ST] * widen<Det, PhiT>(D[i * n + j]);
      lt[p] = l;
    }
  }
  __syncthreads();
  for (int e = tid; e < K * NC; e += blockDim.x) {
    const int k = e / NC, t = e % NC;
    gradk[e] = gt[(2 * k) * NC + t] + gt[(2 * k + 1) * NC + t];
  }
  for (int k = tid; k < K; k += blockDim.x) {
    Det qs = 0;
    for (int t = 0; t < NC; ++t) qs += qt[(2 * k) * NC + t] + qt[(2 * k + 1) * NC + t];
    lapk[k] = lt[2 * k] + lt[2 * k + 1] - qs;
  }
  __syncthreads();
  if (tid == 0) {
    Det m = -INFINITY;
    for (int k = 0; k < K; ++k) {
      const Det sk = sg2[2 * k] * sg2[2 * k + 1];
      if (sk != 0 && ld2[2 * k] + ld2[2 * k + 1] > m) m = ld2[2 * k] + ld2[2 * k + 1];
    }
    Det S = 0;
    for (int k = 0; k < K; ++k) {
      const Det sk = sg2[2 * k] * sg2[2 * k + 1];
      rho[k] = sk != 0 ? sk * f_exp(ld2[2 * k] + ld2[2 * k + 1] - m) : (Det)0;
      S += rho[k];
    }
    for (int k = 0; k < K; ++k) rho[k] = S != 0 ? rho[k] / S : (Det)0;
    red[0] = m + f_log(f_abs(S));
    red[1] = S > 0 ? 1 : (S < 0 ? -1 : 0);
  }
  __syncthreads();
  const double lpsi = (double)red[0];
  const int sgn = (int)red[1];
  __syncthreads();
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
    if (a.log_psi) a.log_psi[w] = lpsi;
    if (a.sign) a.sign[w] = (int8_t)sgn;
    if (sgn == 0) atomicOr(a.status, kStatusSingular);
    else if (!isfinite(e) || !isfinite(lpsi)) atomicOr(a.status, kStatusNonFinite);
  }
}

// ---- local-energy pass on 8-lane groups (BF16-mixed mode, blocks of up to 8 electrons) ----
// One CTA of 128 threads per walker, in 16 groups of 8 lanes; lane r of a group holds row r
// of one (determinant, spin) block.  Every lane works in every phase, so no thread waits on
// a barrier while a few others factorise, and no thread holds a whole matrix in registers:
//   1. Gauss-Jordan elimination with partial pivoting on [A | I] in FP64 registers, the pivot
//      row found by a group reduction and broadcast by shuffles.  The rows are not swapped:
//      the lane that supplies column c's pivot ends with row c of C = A^-1.  The unused rows
//      receive the updates of an LU factorisation, so the pivots are those of the one-thread
//      LU (log|det| agrees with it to rounding, 1e-14 in log|psi| measured).  The same lanes
//      form the Laplacian trace tr(C lap A) in FP64 and store C as double-FP32 rows.
//   2. Tangent items (block, coordinate): lane r forms row r of B = C d_t A in double-FP32
//      arithmetic (the operations of the one-thread items: from the same C they give the
//      same entries), then g = tr B and q = tr(B^2) from the rows staged in shared memory
//      and a double-FP32 reduction over the group.
//   3. The determinant terms are combined and E_L assembled as in k_det_energy.
constexpr int kGrpN = 8;                 // rows per group (largest block of this kernel)
constexpr int kGrpCP = kGrpN + 1;        // padded row of a staged C copy (floats)
constexpr int kGrpBS = 2 * kGrpN + 1;    // padded row of a staged B row (high, low words)

__host__ __device__ inline size_t smem_det_energy_grp(int N, int K) {
  const int NM = 2 * K, NC = 3 * N;
  return sizeof(double) * ((size_t)2 * NM * NC + 3 * NM + (size_t)K * NC + 2 * K + 128) +
         sizeof(float) * ((size_t)NM * 2 * kGrpN * kGrpCP + 16 * 8 * kGrpBS);
}

// (h, l) += the (h, l) of the lane `off` away (double-FP32 sum, error-free on the high words)
__device__ __forceinline__ void ff_add_xor(float& h, float& l, int off) {
  const float oh = __shfl_xor_sync(0xffffffffu, h, off), ol = __shfl_xor_sync(0xffffffffu, l, off);
  float s, e;
  ff_two_sum(h, oh, s, e);
  h = s;
  l = __fadd_rn(__fadd_rn(l, ol), e);
}

// Row r of B = C D for an M x M block: M double-FP32 accumulators (the operations of
// tangent_item_ff's inner loop, in the same order).
template <int M>
__device__ __forceinline__ void ff_row(const float* __restrict__ chr, const float* __restrict__ clr,
                                       const float* __restrict__ D, float (&bh)[kGrpN], float (&bl)[kGrpN]) {
#pragma unroll
  for (int j = 0; j < M; ++j) { bh[j] = 0.f; bl[j] = 0.f; }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const float ch = chr[m], cl = clr[m];
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const float d = __ldg(D + m * M + j);
      const float p = __fmul_rn(ch, d);
      const float pe = __fmaf_rn(ch, d, -p);
      float s, e;
      ff_two_sum(bh[j], p, s, e);
      bh[j] = s;
      bl[j] = __fmaf_rn(cl, d, __fadd_rn(bl[j], __fadd_rn(e, pe)));
    }
  }
}

// The same row for two consecutive tangent slabs of a block (D1 = D0 + M^2): the C row is
// read once and the two sets of accumulators are independent (twice the instruction-level
// parallelism of ff_row).
template <int M>
__device__ __forceinline__ void ff_row2(const float* __restrict__ chr, const float* __restrict__ clr,
                                        const float* __restrict__ D0, float (&bh0)[kGrpN], float (&bl0)[kGrpN],
                                        float (&bh1)[kGrpN], float (&bl1)[kGrpN]) {
  const float* D1 = D0 + M * M;
#pragma unroll
  for (int j = 0; j < M; ++j) { bh0[j] = 0.f; bl0[j] = 0.f; bh1[j] = 0.f; bl1[j] = 0.f; }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const float ch = chr[m], cl = clr[m];
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const float d0 = __ldg(D0 + m * M + j), d1 = __ldg(D1 + m * M + j);
      const float p0 = __fmul_rn(ch, d0), p1 = __fmul_rn(ch, d1);
      const float pe0 = __fmaf_rn(ch, d0, -p0), pe1 = __fmaf_rn(ch, d1, -p1);
      float s0, e0, s1, e1;
      ff_two_sum(bh0[j], p0, s0, e0);
      ff_two_sum(bh1[j], p1, s1, e1);
      bh0[j] = s0;
      bh1[j] = s1;
      bl0[j] = __fmaf_rn(cl, d0, __fadd_rn(bl0[j], __fadd_rn(e0, pe0)));
      bl1[j] = __fmaf_rn(cl, d1, __fadd_rn(bl1[j], __fadd_rn(e1, pe1)));
    }
  }
}

template <typename Wlk>
__global__ void __launch_bounds__(128, 4) k_det_energy_grp(const Wlk* __restrict__ r, const double* __restrict__ nuc,
                                                           Shape sh, DetArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = blockIdx.x, tid = threadIdx.x;
  const int N = sh.N, T = sh.T, K = a.K, NC = 3 * N, NM = 2 * K;
  const int ns[2] = {sh.n_up, sh.n_dn};
  // g and q of every item as double-FP32 pairs (converted to FP64 in the reductions, where
  // every lane of a warp has work: an FP64 instruction costs the same warp slot with one
  // active lane as with 32)
  float2* gt = (float2*)smem_raw;                         // [NM][NC]
  float2* qt = gt + NM * NC;                              // [NM][NC]
  double* lt = (double*)(qt + NM * NC);                   // [NM]
  double* ld2 = lt + NM;                                  // [NM]
  double* sg2 = ld2 + NM;                                 // [NM]
  double* gradk = sg2 + NM;                               // [K][NC]
  double* lapk = gradk + K * NC;                          // [K]
  double* rho = lapk + K;                                 // [K]
  double* red = rho + K;                                  // [128]
  float* Cs = (float*)(red + 128);                        // [NM][2][8][9]: rows of C, high then low words
  float* Bs = Cs + NM * 2 * kGrpN * kGrpCP;               // [16 groups][8 rows][17]: B rows of an item
  const float* Phi = (const float*)a.Phi + (int64_t)w * a.PW;
  const int64_t blk_off[2] = {0, (int64_t)K * T * ns[0] * ns[0]};
  const int lane = tid & 31, gid = tid >> 3, rr = tid & 7;
  const int gbase = lane & ~7;                            // the group's first lane in the warp

  // 1. factorisation, 16 blocks at a time (every lane runs every shuffle)
  for (int p0 = 0; p0 < NM; p0 += 16) {
    const int p = p0 + gid;
    const bool live = p < NM;
    const int n = live ? ns[p & 1] : 0;
    const float* Ab = Phi + blk_off[p & 1] + (int64_t)(p >> 1) * T * n * n;     // value slab of the block
    double av[kGrpN], vv[kGrpN];
#pragma unroll
    for (int j = 0; j < kGrpN; ++j) {
      av[j] = (rr < n && j < n) ? widen<double, float>(Ab[rr * n + j]) : 0.0;
      vv[j] = j == rr ? 1.0 : 0.0;
    }
    bool used = rr >= n, singular = false;
    int mycol = -1, pc[kGrpN];
    double mant = 1.0;
    int expo = 0;
#pragma unroll
    for (int c = 0; c < kGrpN; ++c) {
      const bool col = c < n;
      // pivot: the unused row of largest |a_c| (the first such row on ties)
      unsigned long long key = (!used && col) ? abs_key(av[c]) : 0ull;
      int li = rr;
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, off);
        const int ol = __shfl_xor_sync(0xffffffffu, li, off);
        if (ok > key || (ok == key && ol < li)) { key = ok; li = ol; }
      }
      pc[c] = li;
      if (col && key == 0ull) singular = true;
      double pa[kGrpN], pv[kGrpN];
#pragma unroll
      for (int j = 0; j < kGrpN; ++j) {
        pa[j] = j >= c ? __shfl_sync(0xffffffffu, av[j], gbase + li) : 0.0;
        pv[j] = __shfl_sync(0xffffffffu, vv[j], gbase + li);
      }
      if (col && !singular) {
        const double piv = pa[c];
        const double rp = 1.0 / piv;
        int e;
        mant *= frexp(piv, &e);
        expo += e;
        int e2;
        mant = frexp(mant, &e2);
        expo += e2;
        // (only the columns right of c of the A part are read again)
        if (rr == li) {
#pragma unroll
          for (int j = c + 1; j < kGrpN; ++j) av[j] = pa[j] * rp;
#pragma unroll
          for (int j = 0; j < kGrpN; ++j) vv[j] = pv[j] * rp;
          used = true;
          mycol = c;
        } else {
          const double f = av[c] * rp;
#pragma unroll
          for (int j = c + 1; j < kGrpN; ++j) av[j] -= f * pa[j];
#pragma unroll
          for (int j = 0; j < kGrpN; ++j) vv[j] -= f * pv[j];
        }
      }
    }
    // log|det| and its sign: the pivots' product (mantissa x 2^exponent) and the parity of
    // the permutation column c -> pivot row pc[c]
    int par = 0;
#pragma unroll
    for (int i = 0; i < kGrpN; ++i)
#pragma unroll
      for (int j = i + 1; j < kGrpN; ++j)
        if (j < n && pc[i] > pc[j]) par ^= 1;
    if (live && rr == 0) {
      if (n == 0) {
        ld2[p] = 0;
        sg2[p] = 1;
      } else if (singular) {
        ld2[p] = 0;
        sg2[p] = 0;
      } else {
        const double sgn = par ? -1.0 : 1.0;
        sg2[p] = mant < 0 ? -sgn : sgn;
        ld2[p] = log(fabs(mant)) + (double)expo * 0.6931471805599453;
      }
    }
    // row `row` of C (zero for a singular block) as double-FP32 words, and this row's part of
    // tr(C lap A) = sum_i C[row][i] lap A[i][row]
    const int row = singular ? rr : mycol;
    double lpart = 0.0;
    if (live && rr < n && row >= 0 && row < n) {
      float* ch = Cs + ((int64_t)(p * 2) * kGrpN + row) * kGrpCP;
      float* cl = ch + kGrpN * kGrpCP;
      const float* Dl = Phi + blk_off[p & 1] + (int64_t)(p >> 1) * T * n * n + (int64_t)(T - 1) * n * n;
#pragma unroll
      for (int m = 0; m < kGrpN; ++m) {
        if (m < n) {
          const double c = singular ? 0.0 : vv[m];
          const float h = __double2float_rn(c);
          ch[m] = h;
          cl[m] = __double2float_rn(c - (double)h);
          lpart += c * widen<double, float>(Dl[m * n + row]);
        }
      }
    }
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) lpart += __shfl_xor_sync(0xffffffffu, lpart, off);
    if (live && rr == 0) lt[p] = lpart;
  }
  __syncthreads();

  // 2. tangent items: each group takes two coordinates (tr0, tr0 + 1) of a block per step,
  // four groups per warp
  const int NP2 = (NC + 1) / 2;                           // coordinate pairs per block
  for (int base = (tid >> 5) * 4; base < NM * NP2; base += 16) {
    const int it = base + ((tid >> 3) & 3);
    const bool live = it < NM * NP2;
    const int p = live ? it / NP2 : 0;
    const int tr0 = live ? 2 * (it - p * NP2) : 0;
    const bool two = tr0 + 1 < NC;
    const int n = live ? ns[p & 1] : 0;
    float bh0[kGrpN], bl0[kGrpN], bh1[kGrpN], bl1[kGrpN];
#pragma unroll
    for (int j = 0; j < kGrpN; ++j) { bh0[j] = 0.f; bl0[j] = 0.f; bh1[j] = 0.f; bl1[j] = 0.f; }
    float* brow = Bs + (gid * 8 + rr) * kGrpBS;
    {
      // the orbital tangents are read once, from DRAM: start the pair of blocks this group
      // takes two steps later on its way into L2 (up to four 128-byte lines)
      const int it2 = it + 32;
      if (rr < 4 && it2 < NM * NP2) {
        const int p2 = it2 / NP2, n2 = ns[p2 & 1];
        const float* D2 = Phi + blk_off[p2 & 1] + (int64_t)(p2 >> 1) * T * n2 * n2 +
                          (int64_t)(1 + 2 * (it2 - p2 * NP2)) * n2 * n2;
        if (rr * 32 < 2 * n2 * n2) asm volatile("prefetch.L2 [%0];" ::"l"(D2 + rr * 32));
      }
    }
    if (rr < n) {
      // (a block's last odd coordinate runs its pair on the same slab twice and keeps one)
      const float* D = Phi + blk_off[p & 1] + (int64_t)(p >> 1) * T * n * n + (int64_t)(1 + tr0 - (two ? 0 : 1)) * n * n;
      const float* chr = Cs + ((int64_t)(p * 2) * kGrpN + rr) * kGrpCP;
      const float* clr = chr + kGrpN * kGrpCP;
      switch (n) {
        case 1: ff_row2<1>(chr, clr, D, bh0, bl0, bh1, bl1); break;
        case 2: ff_row2<2>(chr, clr, D, bh0, bl0, bh1, bl1); break;
        case 3: ff_row2<3>(chr, clr, D, bh0, bl0, bh1, bl1); break;
        case 4: ff_row2<4>(chr, clr, D, bh0, bl0, bh1, bl1); break;
        case 5: ff_row2<5>(chr, clr, D, bh0, bl0, bh1, bl1); break;
        case 6: ff_row2<6>(chr, clr, D, bh0, bl0, bh1, bl1); break;
        case 7: ff_row2<7>(chr, clr, D, bh0, bl0, bh1, bl1); break;
        default: ff_row2<8>(chr, clr, D, bh0, bl0, bh1, bl1); break;
      }
      if (!two) {
#pragma unroll
        for (int j = 0; j < kGrpN; ++j) { bh0[j] = bh1[j]; bl0[j] = bl1[j]; }
      }
    }
    // g: this row's diagonal entry; q: sum_j B[rr][j] B[j][rr]; the rows of the first slab,
    // then of the second, pass through the group's staging rows
    float g0h = 0.f, g0l = 0.f, q0h = 0.f, q0l = 0.f, g1h = 0.f, g1l = 0.f, q1h = 0.f, q1l = 0.f;
    const float* bcol = Bs + (gid * 8) * kGrpBS + 2 * rr;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float(&bh)[kGrpN] = half ? bh1 : bh0;
      float(&bl)[kGrpN] = half ? bl1 : bl0;
      if (rr < n) {
#pragma unroll
        for (int j = 0; j < kGrpN; ++j) {
          brow[2 * j] = bh[j];
          brow[2 * j + 1] = bl[j];
        }
      }
      __syncwarp();
      float gh = 0.f, gl = 0.f, qh = 0.f, ql = 0.f;
      if (rr < n) {
        gh = bcol[rr * kGrpBS];
        gl = bcol[rr * kGrpBS + 1];
#pragma unroll
        for (int j = 0; j < kGrpN; ++j)
          if (j < n) ff_fma_acc(bh[j], bl[j], bcol[j * kGrpBS], bcol[j * kGrpBS + 1], 1.f, qh, ql);
      }
      __syncwarp();
      if (half) { g1h = gh; g1l = gl; q1h = qh; q1l = ql; } else { g0h = gh; g0l = gl; q0h = qh; q0l = ql; }
    }
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
      ff_add_xor(g0h, g0l, off);
      ff_add_xor(q0h, q0l, off);
      ff_add_xor(g1h, g1l, off);
      ff_add_xor(q1h, q1l, off);
    }
    if (live && rr == 0) {
      gt[p * NC + tr0] = make_float2(g0h, g0l);
      qt[p * NC + tr0] = make_float2(q0h, q0l);
      if (two) {
        gt[p * NC + tr0 + 1] = make_float2(g1h, g1l);
        qt[p * NC + tr0 + 1] = make_float2(q1h, q1l);
      }
    }
  }
  __syncthreads();
  // 3. the determinant terms and E_L (as in k_det_energy)
  for (int e = tid; e < K * NC; e += blockDim.x) {
    const int k = e / NC, t = e % NC;
    const float2 g0 = gt[(2 * k) * NC + t], g1 = gt[(2 * k + 1) * NC + t];
    gradk[e] = ((double)g0.x + (double)g0.y) + ((double)g1.x + (double)g1.y);
  }
  for (int k = tid; k < K; k += blockDim.x) {
    double qs = 0;
    for (int t = 0; t < NC; ++t) {
      const float2 q0 = qt[(2 * k) * NC + t], q1 = qt[(2 * k + 1) * NC + t];
      qs += ((double)q0.x + (double)q0.y) + ((double)q1.x + (double)q1.y);
    }
    lapk[k] = lt[2 * k] + lt[2 * k + 1] - qs;
  }
  __syncthreads();
  if (tid == 0) {
    double m = -INFINITY;
    for (int k = 0; k < K; ++k) {
      const double sk = sg2[2 * k] * sg2[2 * k + 1];
      if (sk != 0 && ld2[2 * k] + ld2[2 * k + 1] > m) m = ld2[2 * k] + ld2[2 * k + 1];
    }
    double S = 0;
    for (int k = 0; k < K; ++k) {
      const double sk = sg2[2 * k] * sg2[2 * k + 1];
      rho[k] = sk != 0 ? sk * f_exp(ld2[2 * k] + ld2[2 * k + 1] - m) : (double)0;
      S += rho[k];
    }
    for (int k = 0; k < K; ++k) rho[k] = S != 0 ? rho[k] / S : (double)0;
    red[0] = m + f_log(f_abs(S));
    red[1] = S > 0 ? 1 : (S < 0 ? -1 : 0);
  }
  __syncthreads();
  const double lpsi = (double)red[0];
  const int sgn = (int)red[1];
  __syncthreads();
  // E_kin = -1/2 (|grad log psi|^2 + lap log psi) = -1/2 sum_k rho_k (lap_k + |g_k|^2)
  double kin = 0;
  for (int k = tid; k < K; k += blockDim.x) {
    double g2 = 0;
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
  red[tid] = (double)(-0.5) * kin + (double)pot;
  __syncthreads();
  for (int off = 64; off > 0; off >>= 1) {
    if (tid < off) red[tid] += red[tid + off];
    __syncthreads();
  }
  if (tid == 0) {
    const double e = (double)red[0] + a.v_nn;
    a.e_local[w] = e;
    if (a.log_psi) a.log_psi[w] = lpsi;
    if (a.sign) a.sign[w] = (int8_t)sgn;
    if (sgn == 0) atomicOr(a.status, kStatusSingular);
    else if (!isfinite(e) || !isfinite(lpsi)) atomicOr(a.status, kStatusNonFinite);
  }
}


// Value pass (log|psi|, plus the backward seed rho_k A^{-T} when requested): one CTA per
// walker, one thread per (determinant, spin) block.
template <typename Det, typename PhiT>
__global__ void k_det_value(Shape sh, DetArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = blockIdx.x, tid = threadIdx.x;
  const int K = a.K, NM = 2 * K, ST = blockDim.x;
  const int ns[2] = {sh.n_up, sh.n_dn};
  const int nmax = max(ns[0], ns[1]);
  const bool want_inv = a.inv_out != nullptr;
  Det* A = (Det*)smem_raw;                                // [nmax^2][ST]
  Det* C = A + (int64_t)nmax * nmax * ST;                 // [nmax^2][ST] (inverse)
  Det* rcp = C + (want_inv ? (int64_t)nmax * nmax * ST : 0);   // [nmax][ST]
  Det* ld2 = rcp + (int64_t)nmax * ST;                   // [NM]
  Det* sg2 = ld2 + NM;
  Det* rho = sg2 + NM;                                   // [K]
  int* perm = (int*)(rho + K);                           // [nmax][ST]
  const PhiT* Phi = (const PhiT*)a.Phi + (int64_t)w * a.PW;
  const int64_t blk_off[2] = {0, (int64_t)K * ns[0] * ns[0]};
  const int64_t per = (int64_t)K * (ns[0] * ns[0] + ns[1] * ns[1]);
  Det* io = want_inv ? (Det*)a.inv_out + (int64_t)w * per : nullptr;
  // coalesced staging: block (k, spin) -> thread 2k + spin
  for (int e = tid; e < per; e += blockDim.x) {
    const int sp = e < blk_off[1] ? 0 : 1;
    const int n = ns[sp];
    const int64_t q = e - blk_off[sp];
    const int k = (int)(q / (n * n)), idx = (int)(q % (n * n));
    A[(int64_t)idx * ST + 2 * k + sp] = widen<Det, PhiT>(Phi[e]);
  }
  __syncthreads();
  if (tid < NM) {
    const int k = tid >> 1, sp = tid & 1, n = ns[sp];
    if (n == 0) {
      ld2[tid] = 0;
      sg2[tid] = 1;
    } else {
      thread_lu<Det>(A + tid, n, ST, perm + tid, rcp + tid, ld2 + tid, sg2 + tid);
      if (want_inv) {
        if (sg2[tid] != 0) thread_inverse<Det>(A + tid, perm + tid, rcp + tid, n, ST, C + tid);
        else for (int e = 0; e < n * n; ++e) C[(int64_t)e * ST + tid] = 0;
      }
    }
    (void)k;
  }
  __syncthreads();
  if (tid == 0) {
    Det m = -INFINITY;
    for (int k = 0; k < K; ++k) {
      const Det sk = sg2[2 * k] * sg2[2 * k + 1];
      if (sk != 0 && ld2[2 * k] + ld2[2 * k + 1] > m) m = ld2[2 * k] + ld2[2 * k + 1];
    }
    Det S = 0;
    for (int k = 0; k < K; ++k) {
      const Det sk = sg2[2 * k] * sg2[2 * k + 1];
      rho[k] = sk != 0 ? sk * f_exp(ld2[2 * k] + ld2[2 * k + 1] - m) : (Det)0;
      S += rho[k];
    }
    for (int k = 0; k < K; ++k) rho[k] = S != 0 ? rho[k] / S : (Det)0;
    const double lpsi = (double)(m + f_log(f_abs(S)));
    const int sgn = S > 0 ? 1 : (S < 0 ? -1 : 0);
    if (a.log_psi) a.log_psi[w] = lpsi;
    if (a.sign) a.sign[w] = (int8_t)sgn;
    if (sgn == 0) atomicOr(a.status, kStatusSingular);
    else if (!isfinite(lpsi)) atomicOr(a.status, kStatusNonFinite);
  }
  if (want_inv) {
    __syncthreads();
    for (int e = tid; e < per; e += blockDim.x) {
      const int sp = e < blk_off[1] ? 0 : 1;
      const int n = ns[sp];
      const int64_t q = e - blk_off[sp];
      const int k = (int)(q / (n * n)), idx = (int)(q % (n * n));
      const int i = idx / n, j = idx % n;
      io[e] = rho[k] * C[(int64_t)(j * n + i) * ST + 2 * k + sp];        // rho_k A^{-T}
    }
  }
}

// Register-resident LU of one n x n block (n <= 8 known at compile time): one elimination
// step per template instance, so every matrix index is a compile-time constant and the block
// stays in registers; partial pivoting by predicated row swaps; log|det| and sign by
// mantissa/exponent tracking.
template <int NN, int C, typename Det>
struct LuStep {
  static __device__ __forceinline__ void run(Det (&a)[NN][NN], Det& sgn, Det& mant, int& expo, bool& singular) {
    auto best = abs_key(a[C][C]);
    int piv = C;
#pragma unroll
    for (int r = C + 1; r < NN; ++r) {
      const auto v = abs_key(a[r][C]);
      if (v > best) { best = v; piv = r; }
    }
    if (best == 0) singular = true;
#pragma unroll
    for (int r = C + 1; r < NN; ++r) {
      const bool sw = r == piv;
#pragma unroll
      for (int j = 0; j < NN; ++j) {
        const Det t = a[C][j];
        a[C][j] = sw ? a[r][j] : t;
        a[r][j] = sw ? t : a[r][j];
      }
    }
    if (piv != C) sgn = -sgn;
    const Det p = a[C][C];
    const Det rp = (Det)1 / p;
    int e;
    mant *= frexp(p, &e);
    expo += e;
    int e2;
    mant = frexp(mant, &e2);
    expo += e2;
#pragma unroll
    for (int r = C + 1; r < NN; ++r) {
      const Det f = a[r][C] * rp;
#pragma unroll
      for (int j = C + 1; j < NN; ++j) a[r][j] -= f * a[C][j];
    }
    LuStep<NN, C + 1, Det>::run(a, sgn, mant, expo, singular);
  }
};
template <int NN, typename Det>
struct LuStep<NN, NN, Det> {
  static __device__ __forceinline__ void run(Det (&)[NN][NN], Det&, Det&, int&, bool&) {}
};

template <int NN, typename Det, typename PhiT>
__device__ __forceinline__ void lu_regs(const PhiT* __restrict__ Ag, Det* mant_out, int* expo_out) {
  Det a[NN][NN];
#pragma unroll
  for (int i = 0; i < NN; ++i)
#pragma unroll
    for (int j = 0; j < NN; ++j) a[i][j] = widen<Det, PhiT>(Ag[i * NN + j]);
  Det sgn = 1, mant = 1;
  int expo = 0;
  bool singular = false;
  LuStep<NN, 0, Det>::run(a, sgn, mant, expo, singular);
  *mant_out = singular ? (Det)0 : sgn * mant;
  *expo_out = singular ? 0 : expo;
}

// det A = mant 2^expo with |mant| in [1/2, 1) (mant = 0 for a singular block)
template <typename Det, typename PhiT>
__device__ __forceinline__ void lu_regs_any(const PhiT* Ag, int n, Det* mant, int* expo) {
  switch (n) {
    case 1: lu_regs<1, Det, PhiT>(Ag, mant, expo); break;
    case 2: lu_regs<2, Det, PhiT>(Ag, mant, expo); break;
    case 3: lu_regs<3, Det, PhiT>(Ag, mant, expo); break;
    case 4: lu_regs<4, Det, PhiT>(Ag, mant, expo); break;
    case 5: lu_regs<5, Det, PhiT>(Ag, mant, expo); break;
    case 6: lu_regs<6, Det, PhiT>(Ag, mant, expo); break;
    case 7: lu_regs<7, Det, PhiT>(Ag, mant, expo); break;
    default: lu_regs<8, Det, PhiT>(Ag, mant, expo); break;
  }
}

// Value pass without the backward seed, blocks of at most 8 x 8: one thread per
// (determinant, spin) block, 128 / (2K) walkers per CTA, no shared-memory staging.  Each
// block's determinant is kept as mantissa x 2^exponent; a walker's K terms
// D_k = det A_k,up det A_k,down are summed after scaling by 2^(e_k - max e), so that
// log|psi| = log|S| + (max e) ln 2 takes one logarithm per walker and no exponential
// (the same signed log-sum-exp, without forming log|D_k|).
template <typename Det, typename PhiT>
__global__ void __launch_bounds__(128, 3) k_det_value_small(Shape sh, DetArgs a) {
  __shared__ Det mt2[128];
  __shared__ int ex2[128];
  const int K = a.K, NM = 2 * K;
  const int per_cta = 128 / NM;
  const int wl = threadIdx.x / NM, p = threadIdx.x % NM;
  const int w = blockIdx.x * per_cta + wl;
  const int ns[2] = {sh.n_up, sh.n_dn};
  if (wl < per_cta && w < sh.B) {
    const int k = p >> 1, sp = p & 1, n = ns[sp];
    if (n == 0) {
      mt2[threadIdx.x] = (Det)1;
      ex2[threadIdx.x] = 0;
    } else {
      const PhiT* A = (const PhiT*)a.Phi + (int64_t)w * a.PW + (sp ? (int64_t)K * ns[0] * ns[0] : 0) +
                      (int64_t)k * n * n;
      lu_regs_any<Det, PhiT>(A, n, mt2 + threadIdx.x, ex2 + threadIdx.x);
    }
  }
  __syncthreads();
  if (threadIdx.x < per_cta) {
    const int w2 = blockIdx.x * per_cta + threadIdx.x;
    if (w2 < sh.B) {
      const Det* mt = mt2 + threadIdx.x * NM;
      const int* ex = ex2 + threadIdx.x * NM;
      int emax = INT_MIN;
      for (int k = 0; k < K; ++k)
        if (mt[2 * k] * mt[2 * k + 1] != 0 && ex[2 * k] + ex[2 * k + 1] > emax) emax = ex[2 * k] + ex[2 * k + 1];
      Det S = 0;
      for (int k = 0; k < K; ++k) {
        const Det mk = mt[2 * k] * mt[2 * k + 1];
        if (mk != 0) S += ldexp(mk, ex[2 * k] + ex[2 * k + 1] - emax);
      }
      const int sgn = S > 0 ? 1 : (S < 0 ? -1 : 0);
      const double lpsi = sgn == 0 ? (double)f_log(f_abs(S)) : (double)(f_log(f_abs(S)) + (Det)emax * (Det)0.6931471805599453);
      if (a.log_psi) a.log_psi[w2] = lpsi;
      if (a.sign) a.sign[w2] = (int8_t)sgn;
      if (sgn == 0) atomicOr(a.status, kStatusSingular);
      else if (!isfinite(lpsi)) atomicOr(a.status, kStatusNonFinite);
    }
  }
}

// ---- local-energy pass for small blocks --------------------------------------------------
// Blocks of at most 4 x 4 and at most 8 electrons (hydrogen, lithium hydride and its ions,
// atoms up to oxygen): one thread per (walker, determinant, spin) block does the
// Gauss-Jordan inversion with partial pivoting (first maximal |pivot|), the determinant as
// mantissa x 2^exponent, every tangent trace g_t = tr(C d_t A), the sum over t of
// q_t = tr((C d_t A)^2) and tr(C lap A), all in registers; one thread per walker then combines
// the K terms and assembles E_L.  128 / (2K) walkers share a CTA, so a small walker does not
// occupy a CTA of idle threads.
template <int NMAX, typename Det, typename Wlk, typename PhiT>
__global__ void __launch_bounds__(128) k_det_energy_small(const Wlk* __restrict__ r, const double* __restrict__ nuc,
                                                          Shape sh, DetArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = a.K, NM = 2 * K, NC = 3 * sh.N, T = sh.T;
  const int per_cta = 128 / NM;
  const int wl = threadIdx.x / NM, p = threadIdx.x % NM;
  const int w = blockIdx.x * per_cta + wl;
  const int ns[2] = {sh.n_up, sh.n_dn};
  // per walker of the CTA: gt [NM][NC], lt [NM], qs [NM], mant [NM]; then expo [NM] ints
  const int stride = NM * (NC + 3);
  Det* sd = (Det*)smem_raw;
  int* sexp = (int*)(sd + (int64_t)per_cta * stride);
  if (wl < per_cta && w < sh.B) {
    Det* gt = sd + (int64_t)wl * stride + p * NC;
    Det* lt = sd + (int64_t)wl * stride + NM * NC + p;
    Det* qs = lt + NM;
    Det* mt = qs + NM;
    const int k = p >> 1, sp = p & 1, n = ns[sp];
    if (n == 0) {
      for (int t = 0; t < NC; ++t) gt[t] = 0;
      *lt = 0; *qs = 0; *mt = 1;
      sexp[wl * NM + p] = 0;
    } else {
      const PhiT* blk = (const PhiT*)a.Phi + (int64_t)w * a.PW + (sp ? (int64_t)K * T * ns[0] * ns[0] : 0) +
                        (int64_t)k * T * n * n;
      // [A | I] -> [I | A^-1]
      Det M[NMAX][2 * NMAX];
#pragma unroll
      for (int i = 0; i < NMAX; ++i)
#pragma unroll
        for (int j = 0; j < 2 * NMAX; ++j) M[i][j] = 0;
#pragma unroll
      for (int i = 0; i < NMAX; ++i)
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
          if (i < n && j < n) M[i][j] = widen<Det, PhiT>(blk[i * n + j]);
#pragma unroll
      for (int i = 0; i < NMAX; ++i) M[i][NMAX + i] = (i < n) ? (Det)1 : (Det)0;
      Det sgn = 1, mant = 1;
      int expo = 0;
      bool singular = false;
#pragma unroll
      for (int c = 0; c < NMAX; ++c) {
        if (c < n) {
          int piv = c;
          auto best = abs_key(M[c][c]);
#pragma unroll
          for (int i = c + 1; i < NMAX; ++i)
            if (i < n && abs_key(M[i][c]) > best) { best = abs_key(M[i][c]); piv = i; }
          if (best == 0) singular = true;
#pragma unroll
          for (int i = c + 1; i < NMAX; ++i)
            if (i == piv) {
#pragma unroll
              for (int j = 0; j < 2 * NMAX; ++j) { const Det tmp = M[c][j]; M[c][j] = M[i][j]; M[i][j] = tmp; }
            }
          if (piv != c) sgn = -sgn;
          const Det pv = M[c][c];
          int e;
          mant *= frexp(pv, &e);
          expo += e;
          int e2;
          mant = frexp(mant, &e2);
          expo += e2;
          const Det rp = (Det)1 / pv;
#pragma unroll
          for (int j = 0; j < 2 * NMAX; ++j) M[c][j] *= rp;
#pragma unroll
          for (int i = 0; i < NMAX; ++i)
            if (i != c && i < n) {
              const Det f = M[i][c];
#pragma unroll
              for (int j = 0; j < 2 * NMAX; ++j) M[i][j] -= f * M[c][j];
            }
        }
      }
      *mt = singular ? (Det)0 : sgn * mant;
      sexp[wl * NM + p] = singular ? 0 : expo;
      // C = A^-1 in M[.][NMAX ..]; tangent items
      Det qsum = 0;
      for (int t = 0; t < NC; ++t) {
        const PhiT* D = blk + (int64_t)(1 + t) * n * n;
        Det Bm[NMAX][NMAX];
#pragma unroll
        for (int i = 0; i < NMAX; ++i)
#pragma unroll
          for (int j = 0; j < NMAX; ++j) {
            Det s = 0;
#pragma unroll
            for (int m = 0; m < NMAX; ++m)
              if (m < n && j < n) s += M[i][NMAX + m] * widen<Det, PhiT>(D[m * n + j]);
            Bm[i][j] = s;
          }
        Det g = 0, q = 0;
#pragma unroll
        for (int i = 0; i < NMAX; ++i) {
          if (i < n) {
            g += Bm[i][i];
            q += Bm[i][i] * Bm[i][i];
#pragma unroll
            for (int j = i + 1; j < NMAX; ++j)
              if (j < n) q += (Det)2 * Bm[i][j] * Bm[j][i];
          }
        }
        gt[t] = singular ? (Det)0 : g;
        qsum += q;
      }
      const PhiT* DL = blk + (int64_t)(T - 1) * n * n;
      Det l = 0;
#pragma unroll
      for (int i = 0; i < NMAX; ++i)
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
          if (i < n && j < n) l += M[j][NMAX + i] * widen<Det, PhiT>(DL[i * n + j]);
      *lt = singular ? (Det)0 : l;
      *qs = singular ? (Det)0 : qsum;
    }
  }
  __syncthreads();
  if (threadIdx.x < per_cta) {
    const int wc = threadIdx.x;
    const int w2 = blockIdx.x * per_cta + wc;
    if (w2 < sh.B) {
      const Det* gtw = sd + (int64_t)wc * stride;
      const Det* ltw = gtw + NM * NC;
      const Det* qsw = ltw + NM;
      const Det* mtw = qsw + NM;
      const int* ew = sexp + wc * NM;
      int emax = INT_MIN;
      for (int kk = 0; kk < K; ++kk)
        if (mtw[2 * kk] * mtw[2 * kk + 1] != 0 && ew[2 * kk] + ew[2 * kk + 1] > emax) emax = ew[2 * kk] + ew[2 * kk + 1];
      Det S = 0;
      for (int kk = 0; kk < K; ++kk) {
        const Det mk = mtw[2 * kk] * mtw[2 * kk + 1];
        if (mk != 0) S += ldexp(mk, ew[2 * kk] + ew[2 * kk + 1] - emax);
      }
      // E_kin = -1/2 sum_k rho_k (lap_k + |g_k|^2), rho_k = D_k / psi
      Det kin = 0;
      for (int kk = 0; kk < K; ++kk) {
        const Det mk = mtw[2 * kk] * mtw[2 * kk + 1];
        if (mk == 0 || S == 0) continue;
        const Det rho = ldexp(mk, ew[2 * kk] + ew[2 * kk + 1] - emax) / S;
        Det g2 = 0;
        for (int t = 0; t < NC; ++t) {
          const Det g = gtw[(2 * kk) * NC + t] + gtw[(2 * kk + 1) * NC + t];
          g2 += g * g;
        }
        kin += rho * (ltw[2 * kk] + ltw[2 * kk + 1] - qsw[2 * kk] - qsw[2 * kk + 1] + g2);
      }
      double pot = 0.0;
      const Wlk* rw = r + (int64_t)w2 * sh.N * 3;
      for (int i = 0; i < sh.N; ++i)
        for (int j = i + 1; j < sh.N; ++j) {
          const double dx = (double)rw[3 * i] - (double)rw[3 * j], dy = (double)rw[3 * i + 1] - (double)rw[3 * j + 1],
                       dz = (double)rw[3 * i + 2] - (double)rw[3 * j + 2];
          pot += 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
        }
      for (int i = 0; i < sh.N; ++i)
        for (int m = 0; m < sh.M; ++m) {
          const double dx = (double)rw[3 * i] - nuc[3 * m], dy = (double)rw[3 * i + 1] - nuc[3 * m + 1],
                       dz = (double)rw[3 * i + 2] - nuc[3 * m + 2];
          pot -= a.charges[m] / sqrt(dx * dx + dy * dy + dz * dz);
        }
      const int sgn = S > 0 ? 1 : (S < 0 ? -1 : 0);
      const double lpsi = sgn == 0 ? (double)f_log(f_abs(S)) : (double)(f_log(f_abs(S)) + (Det)emax * (Det)0.6931471805599453);
      const double e = (double)((Det)(-0.5) * kin) + pot + a.v_nn;
      a.e_local[w2] = e;
      if (a.log_psi) a.log_psi[w2] = lpsi;
      if (a.sign) a.sign[w2] = (int8_t)sgn;
      if (sgn == 0) atomicOr(a.status, kStatusSingular);
      else if (!isfinite(e) || !isfinite(lpsi)) atomicOr(a.status, kStatusNonFinite);
    }
  }
}

inline size_t smem_det_energy_small(int det_bytes, int N, int K) {
  const int NM = 2 * K, per_cta = 128 / NM;
  return (size_t)per_cta * ((size_t)det_bytes * NM * (3 * N + 3) + sizeof(int) * NM);
}

// The BF16-mixed local-energy pass uses the 8-lane-group kernel for blocks of up to 8
// electrons; FN_DET_KERNEL=thread selects the one-thread-per-block kernel instead (the same
// pivots; C = A^-1 by forward and back substitution instead of Gauss-Jordan; the results
// agree to rounding).
static bool det_grp_enabled() {
  const char* v = getenv("FN_DET_KERNEL");
  return !(v && strcmp(v, "thread") == 0);
}

template <class Mode>
void launch_det_energy(const fn_system* s, const void* walkers, const Shape& sh, double* e_local, double* log_psi,
                       int8_t* sign, bool keep_inverse, cudaStream_t st) {
  using Det = typename Mode::Det; using Wlk = typename Mode::Wlk; using PhiT = typename Mode::PhiT;
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
  const int nmax = std::max(s->n_up, s->n_dn), K = s->cfg.n_dets;
  ProfScope ps(s->prof, full ? kProfDetFull : kProfDetValue, st);
  if (full && nmax <= 4 && s->N <= 8) {
    const int per_cta = 128 / (2 * K);
    const size_t smem = smem_det_energy_small(sizeof(Det), s->N, K);
    cudaFuncSetAttribute(k_det_energy_small<4, Det, Wlk, PhiT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_det_energy_small<4, Det, Wlk, PhiT><<<(unsigned)((sh.B + per_cta - 1) / per_cta), 128, smem, st>>>(
        (const Wlk*)walkers, s->d_nuclei, sh, a);
  } else if (full && std::is_same<Det, double>::value && std::is_same<PhiT, float>::value && nmax <= kGrpN &&
             det_grp_enabled()) {
    const size_t smem = smem_det_energy_grp(s->N, K);
    cudaFuncSetAttribute(k_det_energy_grp<Wlk>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_det_energy_grp<Wlk><<<sh.B, 128, smem, st>>>((const Wlk*)walkers, s->d_nuclei, sh, a);
  } else if (full) {
    const size_t smem = smem_det_energy(sizeof(Det), nmax, s->N, K,
                                        std::is_same<Det, double>::value && std::is_same<PhiT, float>::value);
    cudaFuncSetAttribute(k_det_energy<Det, Wlk, PhiT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_det_energy<Det, Wlk, PhiT><<<sh.B, 128, smem, st>>>((const Wlk*)walkers, s->d_nuclei, sh, a);
  } else if (!keep_inverse && nmax <= 8) {
    const int per_cta = 128 / (2 * K);
    k_det_value_small<Det, PhiT><<<(unsigned)((sh.B + per_cta - 1) / per_cta), 128, 0, st>>>(sh, a);
  } else {
    const int threads = (int)round_up(2 * K, 32);
    const size_t vsmem = smem_det_value(sizeof(Det), nmax, K, keep_inverse);
    cudaFuncSetAttribute(k_det_value<Det, PhiT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsmem);
    k_det_value<Det, PhiT><<<sh.B, threads, vsmem, st>>>(sh, a);
  }
}

template void launch_det_energy<ModeF64>(const fn_system*, const void*, const Shape&, double*, double*, int8_t*,
                                         bool, cudaStream_t);
template void launch_det_energy<ModeF32>(const fn_system*, const void*, const Shape&, double*, double*, int8_t*,
                                         bool, cudaStream_t);
template void launch_det_energy<ModeBF16>(const fn_system*, const void*, const Shape&, double*, double*, int8_t*,
                                          bool, cudaStream_t);

}  // namespace fn
