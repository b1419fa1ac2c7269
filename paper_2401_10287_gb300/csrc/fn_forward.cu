// Forward pass of the wavefunction with forward-mode Laplacian tangents
// ("FermiNet Model" section; Eq. 4 envelope): SIMT kernels for FP64/FP32, the BF16-mode
// kernels around the tensor-core ones of fn_layer_tc.cu, and the launch sequence:
//   k_prep             parameter blob -> internal layouts (one launch, descriptor table)
//   k_features_en      one-electron stream input [r_i - R_m, |r_i - R_m|] with tangents
//   k_features_mean    spin means of the one-electron input
//   k_pair_full/value  two-electron stream, SIMT (a pair depends on r_i - r_j only: 5 jet
//                      rows) and its spin means for every layer
//   k_pair_*_mma       the same on warp-level BF16 MMAs with hi/lo splits (BF16 mode)
//   k_spin_means_bf16  spin means of a BF16 stream-layer output (next mean-field input)
//   k_gemm             tiled SIMT GEMM (mean-field term U [hbar_up, hbar_dn] + b)
//   k_layer            one-electron layer GEMM over all tangent slabs with the fused
//                      tanh forward-Laplacian epilogue, residual and next spin means
//   k_envelope_values  envelope values per (electron, orbital) for the tensor-core orbitals
//   k_orbital_fixup    envelope-derivative terms of the tensor-core orbitals
//   k_orbitals         orbital projection x envelope with the product rule (SIMT)
#include <algorithm>
#include <vector>

#include "fn_device.cuh"
#include "fn_gemm.cuh"
#include "fn_internal.cuh"

namespace fn {

// ---------------------------------------------------------------------------------------
// parameter preparation
// ---------------------------------------------------------------------------------------

template <typename Par, typename Cmp>
__global__ void k_prep(const Par* __restrict__ blob, const CopyDesc* __restrict__ descs, int n_desc,
                       Cmp* __restrict__ prep, __nv_bfloat16* __restrict__ prep16) {
  const CopyDesc d = descs[blockIdx.y];
  const int64_t n = (int64_t)d.rows * d.cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / d.cols, c = e % d.cols;
    if (d.to16 == 3) {
      prep16[d.dst + r * d.d_rs + c * d.d_cs] = __float2bfloat16_rn(0.f);
      continue;
    }
    const Par v = blob[d.src + r * d.s_rs + c * d.s_cs];
    if (d.to16) {
      const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
      prep16[d.dst + r * d.d_rs + c * d.d_cs] =
          d.to16 == 1 ? hi : __float2bfloat16_rn((float)v - __bfloat162float(hi));
    }
    else prep[d.dst + r * d.d_rs + c * d.d_cs] = (Cmp)v;
  }
}

static std::vector<CopyDesc> build_descs(const fn_system* s, bool with16) {
  std::vector<CopyDesc> v;
  const int L = s->cfg.n_layers, h1 = s->cfg.h1, h2 = s->cfg.h2, K = s->cfg.n_dets, M = s->M;
  const PrepLayout& p = s->prep;
  for (int l = 0; l < L; ++l) {
    const LayerDims& d = s->layer[l];
    const int f_in = 3 * d.d_h + 2 * d.d_g;
    // VsT[k][n] = V[n][k] for k < d_h, V[n][3 d_h + (k - d_h)] for the pair-mean columns
    v.push_back({d.off_V, 1, f_in, p.VsT[l], h1, 1, d.d_h, h1, 0});
    v.push_back({d.off_V + 3 * d.d_h, 1, f_in, p.VsT[l] + (int64_t)d.d_h * h1, h1, 1, 2 * d.d_g, h1, 0});
    v.push_back({d.off_V + d.d_h, 1, f_in, p.UT[l], h1, 1, 2 * d.d_h, h1, 0});
    v.push_back({d.off_b, 0, 1, p.b[l], 0, 1, 1, h1, 0});
    if (l < L - 1) {
      v.push_back({d.off_W, d.d_g, 1, p.W[l], d.d_g, 1, h2, d.d_g, 0});
      v.push_back({d.off_c, 0, 1, p.c[l], 0, 1, 1, h2, 0});
    }
    if (with16) {
      // hi part in columns [0, k), residual lo part in [ld, ld + k) of a [rows][2 ld] matrix
      for (int part = 1; part <= 2; ++part) {
        const int ox = part == 2 ? d.ldx : 0, ou = part == 2 ? 2 * d.d_h : 0;
        v.push_back({d.off_V, f_in, 1, p.Vs16[l] + ox, 2 * d.ldx, 1, h1, d.d_h, part});
        v.push_back({d.off_V + 3 * d.d_h, f_in, 1, p.Vs16[l] + d.d_h + ox, 2 * d.ldx, 1, h1, 2 * d.d_g, part});
        v.push_back({d.off_V + d.d_h, f_in, 1, p.U16[l] + ou, 4 * d.d_h, 1, h1, 2 * d.d_h, part});
      }
      // zero padding between k_self and ldx of both parts: the tensor-core B tiles read these
      // columns against zero-filled A columns, so they must hold finite values
      if (d.ldx > d.k_self)
        for (int part = 0; part < 2; ++part)
          v.push_back({0, 0, 0, p.Vs16[l] + part * d.ldx + d.k_self, 2 * d.ldx, 1, h1, d.ldx - d.k_self, 3});
    }
  }
  const int ns[2] = {s->n_up, s->n_dn};
  const int sig_sz = s->cfg.envelope == FN_ENV_ANISOTROPIC ? 9 : 1;
  if (with16)
    for (int a = 0; a < 2; ++a)
      if (ns[a])
        for (int part = 1; part <= 2; ++part) {
          v.push_back({s->off_w[a], h1, 1, p.W16 + (a ? (int64_t)K * ns[0] * 2 * h1 : 0) + (part == 2 ? h1 : 0),
                       2 * h1, 1, K * ns[a], h1, part});
          // transposed: row c, column ko (up block first)
          v.push_back({s->off_w[a], 1, h1, p.W16T + (a ? (int64_t)K * ns[0] : 0) + (part == 2 ? p.ldWT : 0),
                       2 * p.ldWT, 1, h1, K * ns[a], part});
        }
  if (with16 && p.ldWT > K * (ns[0] + ns[1]))
    for (int part = 0; part < 2; ++part)
      v.push_back({0, 0, 0, p.W16T + part * p.ldWT + K * (ns[0] + ns[1]), 2 * p.ldWT, 1, h1,
                   p.ldWT - K * (ns[0] + ns[1]), 3});
  if (with16)
    for (int l = 0; l < L; ++l) {
      const LayerDims& d = s->layer[l];
      const int f_in = 3 * d.d_h + 2 * d.d_g;
      // VsT16[k][n] = V[n][k] for k < d_h, V[n][3 d_h + (k - d_h)] for the pair-mean columns
      for (int part = 1; part <= 2; ++part) {
        const int oh = part == 2 ? h1 : 0;
        v.push_back({d.off_V, 1, f_in, p.VsT16[l] + oh, 2 * h1, 1, d.d_h, h1, part});
        v.push_back({d.off_V + 3 * d.d_h, 1, f_in, p.VsT16[l] + (int64_t)d.d_h * 2 * h1 + oh, 2 * h1, 1, 2 * d.d_g,
                     h1, part});
      }
    }
  for (int a = 0; a < 2; ++a) {
    if (!ns[a]) continue;
    const int ko = K * ns[a];
    v.push_back({s->off_w[a], 1, h1, p.wT[a], ko, 1, h1, ko, 0});
    v.push_back({s->off_g[a], 0, 1, p.g[a], 0, 1, 1, ko, 0});
    v.push_back({s->off_pi[a], 0, 1, p.pi[a], 0, 1, 1, ko * M, 0});
    v.push_back({s->off_sig[a], 0, 1, p.sig[a], 0, 1, 1, ko * M * sig_sz, 0});
  }
  return v;
}

fn_status upload_prep_descs(fn_system* s) {
  std::vector<CopyDesc> v = build_descs(s, s->cfg.precision == FN_BF16_MIXED);
  cudaError_t e = cudaMallocAsync(&s->d_descs, sizeof(CopyDesc) * v.size(), cudaStreamPerThread);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_descs, v.data(), sizeof(CopyDesc) * v.size(), cudaMemcpyHostToDevice, cudaStreamPerThread);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamPerThread);
  if (e != cudaSuccess) return cuda_status(e, "parameter descriptor upload");
  s->n_descs = (int)v.size();
  return FN_OK;
}

template <class Mode>
void launch_prep_params(const fn_system* s, const void* params, cudaStream_t st) {
  using Par = typename Mode::Par; using Cmp = typename Mode::Cmp;
  dim3 grid(32, s->n_descs);
  ProfScope ps(s->prof, kProfPrep, st);
  k_prep<Par, Cmp><<<grid, 256, 0, st>>>((const Par*)params, (const CopyDesc*)s->d_descs, s->n_descs,
                                         (Cmp*)s->ws.prep,
                                         (__nv_bfloat16*)s->ws.prep16);
}

// ---------------------------------------------------------------------------------------
// input features
// ---------------------------------------------------------------------------------------
template <typename Act, typename Wlk>
__global__ void k_features_en(const Wlk* __restrict__ r, const double* __restrict__ nuc, Shape sh,
                              Act* __restrict__ X0, int ldx) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)sh.B * sh.N) return;
  const int w = (int)(gid / sh.N), i = (int)(gid % sh.N);
  const int64_t row = tile_row(w, i, sh.N, sh.wpt);
  const int64_t slab = sh.R * ldx;
  const double rx = (double)r[gid * 3], ry = (double)r[gid * 3 + 1], rz = (double)r[gid * 3 + 2];
  for (int m = 0; m < sh.M; ++m) {
    const double d[3] = {rx - nuc[3 * m], ry - nuc[3 * m + 1], rz - nuc[3 * m + 2]};
    const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    Act* base = X0 + row * ldx + 4 * m;
    for (int a = 0; a < 3; ++a) st(base + a, d[a]);
    st(base + 3, dist);
    if (SplitValue<Act>::value) {
      Act* lo = base + sh.T * slab;
      for (int a = 0; a < 3; ++a) st_lo(lo + a, d[a]);
      st_lo(lo + 3, dist);
    }
    if (sh.T == 1) continue;
    for (int t = 1; t < sh.T; ++t) {
      Act* o = base + t * slab;
      const int e = (t - 1) / 3, c = (t - 1) % 3;
      if (t == sh.T - 1) {
        st(o, 0.0); st(o + 1, 0.0); st(o + 2, 0.0); st(o + 3, 2.0 / dist);
      } else if (e == i) {
        for (int a = 0; a < 3; ++a) st(o + a, a == c ? 1.0 : 0.0);
        st(o + 3, d[c] / dist);
      } else {
        for (int a = 0; a < 4; ++a) st(o + a, 0.0);
      }
    }
  }
}

// Hbar0[t][w][spin * 4M + 4m + a]: mean over the electrons of one spin of h0.
template <typename Act, typename Wlk>
__global__ void k_features_mean(const Wlk* __restrict__ r, const double* __restrict__ nuc, Shape sh,
                                Act* __restrict__ Hbar) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)sh.B * 2 * sh.M) return;
  const int w = (int)(gid / (2 * sh.M)), spin = (int)((gid / sh.M) % 2), m = (int)(gid % sh.M);
  const int lo = spin ? sh.n_up : 0, hi = spin ? sh.N : sh.n_up;
  const int n_s = hi - lo;
  const int width = 2 * 4 * sh.M;
  const int64_t slab = (int64_t)sh.B * width;
  Act* base = Hbar + (int64_t)w * width + spin * 4 * sh.M + 4 * m;
  const double inv = n_s ? 1.0 / n_s : 0.0;
  double v[4] = {0, 0, 0, 0}, lap = 0.0;
  for (int e = lo; e < hi; ++e) {
    const Wlk* re = r + ((int64_t)w * sh.N + e) * 3;
    const double d[3] = {(double)re[0] - nuc[3 * m], (double)re[1] - nuc[3 * m + 1], (double)re[2] - nuc[3 * m + 2]};
    const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    v[0] += d[0]; v[1] += d[1]; v[2] += d[2]; v[3] += dist;
    lap += 2.0 / dist;
    if (sh.T > 1)
      for (int c = 0; c < 3; ++c) {
        Act* o = base + (1 + 3 * e + c) * slab;
        for (int a = 0; a < 3; ++a) st(o + a, a == c ? inv : 0.0);
        st(o + 3, d[c] / dist * inv);
        if (SplitValue<Act>::value) {
          Act* ol = o + sh.T * slab;
          for (int a = 0; a < 3; ++a) st_lo(ol + a, a == c ? inv : 0.0);
          st_lo(ol + 3, d[c] / dist * inv);
        }
      }
  }
  for (int a = 0; a < 4; ++a) st(base + a, v[a] * inv);
  if (SplitValue<Act>::value)
    for (int a = 0; a < 4; ++a) st_lo(base + sh.T * slab + a, v[a] * inv);
  if (sh.T == 1) return;
  Act* o = base + (sh.T - 1) * slab;
  st(o, 0.0); st(o + 1, 0.0); st(o + 2, 0.0); st(o + 3, lap * inv);
  if (SplitValue<Act>::value) {
    Act* ol = o + sh.T * slab;
    st_lo(ol, 0.0); st_lo(ol + 1, 0.0); st_lo(ol + 2, 0.0); st_lo(ol + 3, lap * inv);
  }
  // slabs of the other spin's electrons are zero
  const int olo = spin ? 0 : sh.n_up, ohi = spin ? sh.n_up : sh.N;
  for (int e = olo; e < ohi; ++e)
    for (int c = 0; c < 3; ++c) {
      Act* q = base + (1 + 3 * e + c) * slab;
      st(q, 0.0); st(q + 1, 0.0); st(q + 2, 0.0); st(q + 3, 0.0);
      if (SplitValue<Act>::value) {
        Act* ql = q + sh.T * slab;
        st_lo(ql, 0.0); st_lo(ql + 1, 0.0); st_lo(ql + 2, 0.0); st_lo(ql + 3, 0.0);
      }
    }
}

// ---------------------------------------------------------------------------------------
// two-electron stream.  A pair (i, j) depends only on r_i - r_j, so d/dr_j = -d/dr_i and
// its jet reduces to 5 rows: value, d/dr_i (3), Laplacian.  Pairs never interact across
// layers, so a thread carries its pair (and, in the full pass, one jet row) through every
// layer; the channels live in registers and the layer weights, transposed, in shared memory
// (every thread reads the same weight at the same time: broadcast).
//   full pass : a CTA per (walker, run of electrons i), 5 lanes per pair (one per jet row);
//               the value row's tanh and the tangent rows' squares are exchanged with
//               shuffles inside the group;
//   value pass: one CTA per walker, one thread per pair.
// The spin means over j are reduced in shared memory and written to the mean-g columns of
// every layer's input X_l; the derivative of mean_j g_ij along r_j (j != i) is
// (1/n_spin) d g_ij / d r_j, written directly.
// ---------------------------------------------------------------------------------------
struct PairArgs {
  void* X[kMaxLayers];
  int ldx[kMaxLayers];
  int col0[kMaxLayers];       // first mean-g column of X_l (= d_h of layer l)
  int d_g[kMaxLayers];
  const void* W[kMaxLayers];  // prepared pair weights [h2][d_g]
  const void* c[kMaxLayers];
  void* gstore[kMaxLayers];   // value of g^l for l >= 1, [B][N][N][h2] (backward), or null
  int L, h2;
};

// Stage W_l^T [d_g][h2] and c_l of every pair layer in shared memory.
template <typename Cmp>
__device__ void stage_pair_weights(const PairArgs& a, Cmp* sW, Cmp* sc) {
  for (int l = 0; l + 1 < a.L; ++l) {
    const Cmp* W = (const Cmp*)a.W[l];
    const int dg = a.d_g[l];
    for (int e = threadIdx.x; e < kMaxH2 * kMaxH2; e += blockDim.x) {
      const int k = e / kMaxH2, c = e % kMaxH2;
      sW[l * kMaxH2 * kMaxH2 + e] = (k < dg && c < a.h2) ? W[c * dg + k] : (Cmp)0;
    }
    for (int c = threadIdx.x; c < kMaxH2; c += blockDim.x) sc[l * kMaxH2 + c] = c < a.h2 ? ((const Cmp*)a.c[l])[c] : (Cmp)0;
  }
}

// z[c] = sum_k W^T[k][c] g[k] (+ bias); the weight row is read as 16-byte vectors that
// every thread of the block reads at the same time (broadcast).
__device__ __forceinline__ void load_row(const float* p, float (&w)[kMaxH2]) {
  const float4* q = (const float4*)p;
#pragma unroll
  for (int v = 0; v < kMaxH2 / 4; ++v) {
    const float4 f = q[v];
    w[4 * v] = f.x; w[4 * v + 1] = f.y; w[4 * v + 2] = f.z; w[4 * v + 3] = f.w;
  }
}
__device__ __forceinline__ void load_row(const double* p, double (&w)[kMaxH2]) {
  const double2* q = (const double2*)p;
#pragma unroll
  for (int v = 0; v < kMaxH2 / 2; ++v) {
    const double2 f = q[v];
    w[2 * v] = f.x; w[2 * v + 1] = f.y;
  }
}

template <typename Cmp>
__device__ __forceinline__ void pair_matvec(const Cmp* __restrict__ sWl, const Cmp* __restrict__ scl, bool bias,
                                            int dg, const Cmp (&g)[kMaxH2], Cmp (&z)[kMaxH2]) {
  if (bias) load_row(scl, z);
  else {
#pragma unroll
    for (int c = 0; c < kMaxH2; ++c) z[c] = 0;
  }
#pragma unroll
  for (int k = 0; k < kMaxH2; ++k) {
    if (k < dg) {
      Cmp row[kMaxH2];
      load_row(sWl + k * kMaxH2, row);
      const Cmp gk = g[k];
#pragma unroll
      for (int c = 0; c < kMaxH2; ++c) z[c] += row[c] * gk;
    }
  }
}

// Full pass.  The pair features depend only on r_i - r_j, so at every layer
// d g / d r_j = -d g / d r_i and the Laplacian over both electrons is 2 d^2 g / d r_i^2: a
// pair's jet has 5 rows (value, d/dr_i along x, y, z, Laplacian), carried by a group of 5
// lanes, 6 groups per warp.  A CTA covers walker w and `ib` consecutive electrons i, all
// their partners j.  Per layer every pair's rows are staged in shared memory; from there
// the CTA writes the spin means over j (value, Laplacian, d/dr_i) and the d/dr_j slabs
// (-d/dr_i / n_spin) to the layer input, adjacent columns from adjacent threads.

template <typename Act, typename Cmp, typename Wlk>
__global__ void __launch_bounds__(256) k_pair_full(const Wlk* __restrict__ r, Shape sh, PairArgs a, int ib) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cmp* sW = (Cmp*)smem_raw;                                  // [L-1][32][32]
  Cmp* sc = sW + (a.L - 1) * kMaxH2 * kMaxH2;               // [L-1][32]
  Cmp* gs = sc + (a.L - 1) * kMaxH2;                        // [ib][N][5][33]: value, lap, d/dr_i x, y, z
  const int blocks_per_walker = (sh.N + ib - 1) / ib;
  const int w = blockIdx.x / blocks_per_walker, i0 = (blockIdx.x % blocks_per_walker) * ib;
  const int n_i = min(ib, sh.N - i0);
  const int lane = threadIdx.x & 31, grp = lane / kPairLanes;
  const int q = lane - grp * kPairLanes;
  const int p = (threadIdx.x >> 5) * kPairGroups + grp;      // pair index within the CTA
  const bool live = grp < kPairGroups && p < n_i * sh.N;
  const int ii = live ? p / sh.N : 0, j = live ? p % sh.N : 0, i = i0 + ii;
  const int base = grp < kPairGroups ? grp * kPairLanes : 0;  // value lane of this group
  stage_pair_weights(a, sW, sc);
  const int srow = q == 0 ? 0 : (q == 4 ? 1 : q + 1);       // this lane's row in the staging area
  Cmp g[kMaxH2];
#pragma unroll
  for (int c = 0; c < kMaxH2; ++c) g[c] = 0;
  if (live && j != i) {
    const Wlk* rw = r + (int64_t)w * sh.N * 3;
    double d[3];
    for (int c = 0; c < 3; ++c) d[c] = (double)rw[3 * i + c] - (double)rw[3 * j + c];
    const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (q == 0) {
      g[0] = (Cmp)d[0]; g[1] = (Cmp)d[1]; g[2] = (Cmp)d[2]; g[3] = (Cmp)dist;
    } else if (q == 4) {
      g[3] = (Cmp)(4.0 / dist);                              // Laplacian of |r_i - r_j| over both electrons
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c)                            // static indices keep g and d in registers
        if (c == q - 1) {
          g[c] = (Cmp)1;
          g[3] = (Cmp)(d[c] / dist);
        }
    }
  }
  for (int l = 0; l < a.L; ++l) {
    const int dg = a.d_g[l];
    Act* X = (Act*)a.X[l];
    const int64_t slab = sh.R * a.ldx[l];
    if (live) {
      Cmp* gr = gs + (p * 5 + srow) * 33;
#pragma unroll
      for (int c = 0; c < kMaxH2; ++c)
        if (c < dg) gr[c] = g[c];
    }
    __syncthreads();
    // The layer input row of electron i holds [mean over up partners, mean over down
    // partners], 2 d_g columns from col0.  A warp writes one row at a time, lane c the
    // column pair (2c, 2c + 1); all loop bounds and row indices are warp-uniform.
    const int64_t ldx = a.ldx[l];
    Act* Xc = X + a.col0[l];
    const int warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    const int col = 2 * lane, half0 = col < dg ? 0 : 1, half1 = col + 1 < dg ? 0 : 1;
    const int c0 = col - half0 * dg, c1 = col + 1 - half1 * dg;
    // d/dr_j slabs (j != i): -d g_ij / d r_i / n_spin(j) in j's spin half, 0 in the other
    for (int pp = warp; pp < n_i * sh.N; pp += n_warps) {
      const int e_i = pp / sh.N, jj = pp - e_i * sh.N;
      if (jj == i0 + e_i || lane >= dg) continue;
      const int sjj = jj < sh.n_up ? 0 : 1;
      const Cmp scale = -(Cmp)1 / (Cmp)(sjj ? sh.n_dn : sh.n_up);
      const int64_t row = tile_row(w, i0 + e_i, sh.N, sh.wpt) * ldx;
#pragma unroll
      for (int axis = 0; axis < 3; ++axis) {
        const Cmp* src = gs + (pp * 5 + 2 + axis) * 33;
        const Cmp v0 = half0 == sjj ? src[c0] * scale : (Cmp)0, v1 = half1 == sjj ? src[c1] * scale : (Cmp)0;
        st2(Xc + (1 + 3 * jj + axis) * slab + row + col, v0, v1);
        if (SplitValue<Act>::value) st2_lo(Xc + (sh.T + 1 + 3 * jj + axis) * slab + row + col, v0, v1);
      }
    }
    // value, Laplacian and d/dr_i rows: spin means over partners
    for (int rr = warp; rr < n_i * 5; rr += n_warps) {
      if (lane >= dg) continue;
      const int e_i = rr / 5, qq = rr - 5 * e_i, ie = i0 + e_i;
      const Cmp* src = gs + (e_i * sh.N * 5 + qq) * 33;
      Cmp up0 = 0, up1 = 0, dn0 = 0, dn1 = 0;
      for (int jj = 0; jj < sh.n_up; ++jj) { up0 += src[jj * 165 + c0]; up1 += src[jj * 165 + c1]; }
      for (int jj = sh.n_up; jj < sh.N; ++jj) { dn0 += src[jj * 165 + c0]; dn1 += src[jj * 165 + c1]; }
      const Cmp iu = sh.n_up ? (Cmp)1 / (Cmp)sh.n_up : (Cmp)0, id = sh.n_dn ? (Cmp)1 / (Cmp)sh.n_dn : (Cmp)0;
      const int t = qq == 0 ? 0 : (qq == 1 ? sh.T - 1 : 1 + 3 * ie + (qq - 2));
      const Cmp m0 = half0 ? dn0 * id : up0 * iu, m1 = half1 ? dn1 * id : up1 * iu;
      const int64_t o = tile_row(w, ie, sh.N, sh.wpt) * ldx + col;
      st2(Xc + t * slab + o, m0, m1);
      if (SplitValue<Act>::value) st2_lo(Xc + (sh.T + t) * slab + o, m0, m1);
    }
    if (l == a.L - 1) break;
    __syncthreads();
    Cmp z[kMaxH2];
    pair_matvec(sW + l * kMaxH2 * kMaxH2, sc + l * kMaxH2, q == 0, dg, g, z);
#pragma unroll
    for (int c = 0; c < kMaxH2; ++c) {
      // h and 1 - h^2 from the value lane; the 6 tangent rows give 2 (z_x^2 + z_y^2 + z_z^2)
      const Cmp zv = __shfl_sync(0xffffffffu, z[c], base);
      const Cmp zx = __shfl_sync(0xffffffffu, z[c], base + 1);
      const Cmp zy = __shfl_sync(0xffffffffu, z[c], base + 2);
      const Cmp zz = __shfl_sync(0xffffffffu, z[c], base + 3);
      const Cmp h = act_tanh<Act>(zv);
      const Cmp dh = (Cmp)1 - h * h;
      Cmp out = q == 0 ? h : dh * z[c];
      if (q == 4) out -= (Cmp)4 * h * dh * (zx * zx + zy * zy + zz * zz);
      if (c >= a.h2) out = 0;
      g[c] = (l > 0 ? g[c] : (Cmp)0) + out;
    }
  }
}

// Value pass: CTA per walker, threads loop over pairs.  The pair values live in shared
// memory between layers; per layer the spin means over j are summed per
// (i, spin, channel), then every pair is advanced through the next pair layer.
template <typename Act, typename Cmp, typename Wlk>
__global__ void __launch_bounds__(512) k_pair_value(const Wlk* __restrict__ r, Shape sh, PairArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cmp* sW = (Cmp*)smem_raw;
  Cmp* sc = sW + (a.L - 1) * kMaxH2 * kMaxH2;
  Cmp* gs = sc + (a.L - 1) * kMaxH2;                        // [N*N][33]
  const int w = blockIdx.x;
  const int N = sh.N, NP = N * N;
  stage_pair_weights(a, sW, sc);
  const Wlk* rw = r + (int64_t)w * N * 3;
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {
    const int i = p / N, j = p % N;
    Cmp* gp = gs + p * 33;
    for (int c = 0; c < 4; ++c) gp[c] = 0;
    if (j != i) {
      double d[3];
      for (int c = 0; c < 3; ++c) d[c] = (double)rw[3 * i + c] - (double)rw[3 * j + c];
      gp[0] = (Cmp)d[0]; gp[1] = (Cmp)d[1]; gp[2] = (Cmp)d[2];
      gp[3] = (Cmp)sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
  }
  for (int l = 0; l < a.L; ++l) {
    const int dg = a.d_g[l];
    __syncthreads();
    Act* X = (Act*)a.X[l];
    for (int e = threadIdx.x; e < N * 2 * dg; e += blockDim.x) {
      const int ii = e / (2 * dg), s2 = (e / dg) % 2, c = e % dg;
      const int lo = s2 ? sh.n_up : 0, hi = s2 ? N : sh.n_up;
      Cmp sum = 0;
      for (int jj = lo; jj < hi; ++jj) sum += gs[(ii * N + jj) * 33 + c];
      const int64_t rowi = tile_row(w, ii, N, sh.wpt);
      const Cmp mean = hi > lo ? sum / (Cmp)(hi - lo) : (Cmp)0;
      Act* o = X + rowi * a.ldx[l] + a.col0[l] + s2 * dg + c;
      st(o, mean);
      if (SplitValue<Act>::value) st_lo(o + sh.T * sh.R * a.ldx[l], mean);
    }
    if (l == a.L - 1) break;
    __syncthreads();
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
      Cmp* gp = gs + p * 33;
      Cmp g[kMaxH2], z[kMaxH2];
#pragma unroll
      for (int c = 0; c < kMaxH2; ++c) g[c] = c < dg ? gp[c] : (Cmp)0;
      pair_matvec(sW + l * kMaxH2 * kMaxH2, sc + l * kMaxH2, true, dg, g, z);
#pragma unroll
      for (int c = 0; c < kMaxH2; ++c) g[c] = (l > 0 ? g[c] : (Cmp)0) + (c < a.h2 ? act_tanh<Act>(z[c]) : (Cmp)0);
#pragma unroll
      for (int c = 0; c < kMaxH2; ++c)
        if (c < a.h2) gp[c] = g[c];
      if (a.gstore[l + 1]) {
        const int i = p / N, j = p % N;
        Cmp* gsto = (Cmp*)a.gstore[l + 1] + (((int64_t)w * N + i) * N + j) * a.h2;
#pragma unroll
        for (int c = 0; c < kMaxH2; ++c)
          if (c < a.h2) gsto[c] = g[c];
      }
    }
  }
}

// Spin means of a BF16 stream-layer output, the next layer's mean-field input:
// Hbar[t][w][s h1 + c] = mean over the electrons i of spin s of Y[t][row(w, i)][c].
// The value slab adds its low part (slab T of Y); every mean is stored as a hi/lo pair
// (the low part of slab t in slab T + t of Hbar).  One thread per (slab, walker, spin, 8
// columns); a warp reads 512 contiguous bytes of a row.
__global__ void k_spin_means_bf16(Shape sh, const __nv_bfloat16* __restrict__ Y, int ldy, int h1,
                                  __nv_bfloat16* __restrict__ Hbar) {
  const int g8 = h1 >> 3;
  const int64_t n = (int64_t)sh.T * sh.B * 2 * g8;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int c8 = (int)(e % g8);
    const int64_t rest = e / g8;
    const int s2 = (int)(rest & 1);
    const int64_t tw = rest >> 1;
    const int w = (int)(tw % sh.B), t = (int)(tw / sh.B);
    const int lo = s2 ? sh.n_up : 0, hi = s2 ? sh.N : sh.n_up;
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;
    const int parts = t == 0 ? 2 : 1;
    const int64_t row0 = tile_row(w, 0, sh.N, sh.wpt);            // a walker's rows are consecutive
    for (int part = 0; part < parts; ++part) {
      const __nv_bfloat16* base = Y + ((int64_t)(part ? sh.T : t) * sh.R + row0) * ldy + 8 * c8;
      // the rows of up to 8 electrons are loaded together (one memory round trip), then
      // summed in electron order
      for (int i0 = lo; i0 < hi; i0 += 8) {
        uint4 u[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          u[k] = i0 + k < hi ? __ldg((const uint4*)(base + (int64_t)(i0 + k) * ldy)) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (i0 + k >= hi) break;
          const __nv_bfloat162* p2 = (const __nv_bfloat162*)&u[k];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const float2 f = __bfloat1622float2(p2[m]);
            acc[2 * m] += f.x;
            acc[2 * m + 1] += f.y;
          }
        }
      }
    }
    const float sc = hi > lo ? 1.0f / (float)(hi - lo) : 0.f;
    uint4 o, ol;
    __nv_bfloat162* q = (__nv_bfloat162*)&o;
    __nv_bfloat162* ql = (__nv_bfloat162*)&ol;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float a0 = acc[2 * k] * sc, a1 = acc[2 * k + 1] * sc;
      q[k] = __floats2bfloat162_rn(a0, a1);
      ql[k] = __floats2bfloat162_rn(bf16_rem(a0), bf16_rem(a1));
    }
    const int64_t off = ((int64_t)t * sh.B + w) * 2 * h1 + s2 * h1 + 8 * c8;
    *(uint4*)(Hbar + off) = o;
    *(uint4*)(Hbar + (int64_t)sh.T * sh.B * 2 * h1 + off) = ol;
  }
}

// Value pass of the two-electron stream in BF16 mode.  Per walker the products
// [N^2 pairs x d_g] x [d_g x h2] of every pair layer run on warp-level BF16 tensor-core
// MMAs (m16n8k16, FP32 accumulation).  Activations and weights are split into hi/lo BF16
// parts and the three leading products are accumulated (about 16 significant bits, the
// precision the BF16 storage keeps for the pair means).  One CTA per walker, 4 warps over
// 16-pair row tiles; the pair activations stay in shared memory (FP32) between layers.

template <typename Wlk>
__global__ void __launch_bounds__(128) k_pair_value_mma(const Wlk* __restrict__ r, Shape sh, PairArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L1 = a.L - 1;
  __nv_bfloat16* wh = (__nv_bfloat16*)smem_raw;                  // [L-1][32 n][kPairWLd]: bf16(W[n][k])
  __nv_bfloat16* wl = wh + L1 * 32 * kPairWLd;                    // bf16(W - bf16(W))
  float* sc = (float*)(wl + L1 * 32 * kPairWLd);                  // [L-1][32] biases
  float* gs = sc + L1 * 32;                                       // [16-padded N^2][33] activations
  const int N = sh.N, NP = N * N, NPp = (NP + 15) & ~15;
  for (int l = 0; l < L1; ++l) {
    const float* W = (const float*)a.W[l];                        // [h2][d_g]
    const int dg = a.d_g[l];
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      const int n = e >> 5, k = e & 31;
      const float v = (n < a.h2 && k < dg) ? W[n * dg + k] : 0.f;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      wh[(l * 32 + n) * kPairWLd + k] = h;
      wl[(l * 32 + n) * kPairWLd + k] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
    for (int c = threadIdx.x; c < 32; c += blockDim.x) sc[l * 32 + c] = c < a.h2 ? ((const float*)a.c[l])[c] : 0.f;
  }
  // CTAs loop over walkers, so the weights are staged once per CTA
  for (int w = blockIdx.x; w < sh.B; w += gridDim.x) {
  __syncthreads();
  // the layer-0 input occupies columns 0..15 of each row (features, zero padding, and the
  // zero features of the i = j pairs); every later column is written by the layer-0 product
  // before it is read
  for (int e = threadIdx.x; e < NPp * 16; e += blockDim.x) gs[(e >> 4) * 33 + (e & 15)] = 0.f;
  __syncthreads();
  const Wlk* rw = r + (int64_t)w * N * 3;
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {
    const int i = p / N, j = p - (p / N) * N;
    if (j == i) continue;
    const float d0 = (float)rw[3 * i] - (float)rw[3 * j], d1 = (float)rw[3 * i + 1] - (float)rw[3 * j + 1],
                d2 = (float)rw[3 * i + 2] - (float)rw[3 * j + 2];
    float* gp = gs + p * 33;
    gp[0] = d0; gp[1] = d1; gp[2] = d2;
    gp[3] = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane >> 2, tig = lane & 3;
  for (int l = 0; l < a.L; ++l) {
    const int dg = a.d_g[l];
    __syncthreads();
    __nv_bfloat16* X = (__nv_bfloat16*)a.X[l];
    // spin means over the partners j of each electron i: warp per (i, spin) row, lane per channel
    const int64_t xrow0 = tile_row(w, 0, N, sh.wpt);       // a walker's rows are consecutive
    for (int e2 = warp; e2 < N * 2; e2 += (int)(blockDim.x >> 5)) {
      const int ii = e2 >> 1, s2 = e2 & 1, c = lane;
      if (c >= dg) continue;
      const int lo = s2 ? sh.n_up : 0, hi = s2 ? N : sh.n_up;
      float sum = 0.f;
      for (int jj = lo; jj < hi; ++jj) sum += gs[(ii * N + jj) * 33 + c];
      const float mean = hi > lo ? sum / (float)(hi - lo) : 0.f;
      __nv_bfloat16* o = X + (xrow0 + ii) * a.ldx[l] + a.col0[l] + s2 * dg + c;
      st(o, mean);
      st_lo(o + sh.T * sh.R * a.ldx[l], mean);
    }
    if (l == a.L - 1) break;
    __syncthreads();
    const int nks = (dg + 15) / 16;
    const __nv_bfloat16* whl = wh + l * 32 * kPairWLd;
    const __nv_bfloat16* wll = wl + l * 32 * kPairWLd;
    for (int mt = warp; mt < NPp / 16; mt += (int)(blockDim.x >> 5)) {
      const int p0 = mt * 16;
      float c[4][4];
#pragma unroll
      for (int nb = 0; nb < 4; ++nb) {
        const float b0 = sc[l * 32 + 8 * nb + 2 * tig], b1 = sc[l * 32 + 8 * nb + 2 * tig + 1];
        c[nb][0] = b0; c[nb][1] = b1; c[nb][2] = b0; c[nb][3] = b1;
      }
      for (int ks = 0; ks < nks; ++ks) {
        const int k0 = ks * 16;
        const float* r0 = gs + (p0 + grp) * 33 + k0 + 2 * tig;
        const float* r1 = gs + (p0 + grp + 8) * 33 + k0 + 2 * tig;
        uint32_t ah[4], al[4];
        split_pack(r0[0], r0[1], ah[0], al[0]);
        split_pack(r1[0], r1[1], ah[1], al[1]);
        split_pack(r0[8], r0[9], ah[2], al[2]);
        split_pack(r1[8], r1[9], ah[3], al[3]);
#pragma unroll
        for (int nb = 0; nb < 4; ++nb) {
          const int off = (8 * nb + grp) * kPairWLd + k0 + 2 * tig;
          const uint32_t bh0 = *(const uint32_t*)(whl + off), bh1 = *(const uint32_t*)(whl + off + 8);
          const uint32_t bl0 = *(const uint32_t*)(wll + off), bl1 = *(const uint32_t*)(wll + off + 8);
          mma_16816(c[nb], ah, bh0, bh1);
          mma_16816(c[nb], ah, bl0, bl1);
          mma_16816(c[nb], al, bh0, bh1);
        }
      }
      __syncwarp();                                              // every lane's A reads precede the writes
#pragma unroll
      for (int nb = 0; nb < 4; ++nb)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = p0 + grp + (q >= 2 ? 8 : 0), col = 8 * nb + 2 * tig + (q & 1);
          float* gp = gs + row * 33 + col;
          const float h = col < a.h2 ? tanh_fast(c[nb][q]) : 0.f;
          *gp = (l > 0 ? *gp : 0.f) + h;
        }
    }
    if (a.gstore[l + 1]) {
      __syncthreads();
      float* gsto = (float*)a.gstore[l + 1] + (int64_t)w * NP * a.h2;
      for (int e = threadIdx.x; e < NP * a.h2; e += blockDim.x) gsto[e] = gs[(e / a.h2) * 33 + e % a.h2];
    }
  }
  }
}

// Full (E_L) pass of the two-electron stream in BF16 mode.  The 5-row pair jets of one CTA
// (walker w, electrons i0 .. i0 + ib - 1, all partners j) are the rows of one matrix; every
// pair layer is (1) its product with the layer weights on warp-level BF16 MMAs (hi/lo
// splits of activations and weights, three products) into a shared-memory buffer, (2) the
// tanh forward-Laplacian rule, one thread per (pair, channel), and (3) the coalesced write
// of the spin means and d/dr_j slabs to the next layer input, as in k_pair_full.
template <typename Wlk>
__global__ void __launch_bounds__(256) k_pair_full_mma(const Wlk* __restrict__ r, Shape sh, PairArgs a, int ib) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L1 = a.L - 1;
  __nv_bfloat16* wh = (__nv_bfloat16*)smem_raw;                  // [L-1][32 n][kPairWLd]: bf16(W[n][k])
  __nv_bfloat16* wl = wh + L1 * 32 * kPairWLd;                    // bf16(W - bf16(W))
  float* sc = (float*)(wl + L1 * 32 * kPairWLd);                  // [L-1][32] biases
  const int rows_p = (ib * sh.N * 5 + 15) & ~15;
  float* gs = sc + L1 * 32;                                       // [rows_p][33]: pair p, row srow at p * 5 + srow
  float* zs = gs + rows_p * 33;                                   // [rows_p][33]: products of the current layer
  const int blocks_per_walker = (sh.N + ib - 1) / ib;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  const int grp = lane >> 2, tig = lane & 3;
  for (int l = 0; l < L1; ++l) {
    const float* W = (const float*)a.W[l];
    const int dg = a.d_g[l];
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      const int n = e >> 5, k = e & 31;
      const float v = (n < a.h2 && k < dg) ? W[n * dg + k] : 0.f;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      wh[(l * 32 + n) * kPairWLd + k] = h;
      wl[(l * 32 + n) * kPairWLd + k] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
    for (int c = threadIdx.x; c < 32; c += blockDim.x) sc[l * 32 + c] = c < a.h2 ? ((const float*)a.c[l])[c] : 0.f;
  }
  // CTAs loop over (walker, run of electrons) items, so the weights are staged once per CTA
  for (int item = blockIdx.x; item < sh.B * blocks_per_walker; item += gridDim.x) {
  const int w = item / blocks_per_walker, i0 = (item % blocks_per_walker) * ib;
  const int n_i = min(ib, sh.N - i0);
  const int npair = n_i * sh.N;
  __syncthreads();
  for (int e = threadIdx.x; e < rows_p * 33; e += blockDim.x) gs[e] = 0.f;
  __syncthreads();
  // layer-0 jets of the pair features [r_i - r_j, |r_i - r_j|]: value, Laplacian over both
  // electrons, d/dr_i along x, y, z
  const Wlk* rw = r + (int64_t)w * sh.N * 3;
  for (int p = threadIdx.x; p < npair; p += blockDim.x) {
    const int i = i0 + p / sh.N, j = p % sh.N;
    if (j == i) continue;
    const float d[3] = {(float)rw[3 * i] - (float)rw[3 * j], (float)rw[3 * i + 1] - (float)rw[3 * j + 1],
                        (float)rw[3 * i + 2] - (float)rw[3 * j + 2]};
    const float dist = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    float* g0 = gs + p * 5 * 33;
    g0[0] = d[0]; g0[1] = d[1]; g0[2] = d[2]; g0[3] = dist;
    g0[33 + 3] = 4.f / dist;
    for (int c = 0; c < 3; ++c) {
      g0[(2 + c) * 33 + c] = 1.f;
      g0[(2 + c) * 33 + 3] = d[c] / dist;
    }
  }
  for (int l = 0; l < a.L; ++l) {
    const int dg = a.d_g[l];
    __nv_bfloat16* X = (__nv_bfloat16*)a.X[l];
    const int64_t slab = sh.R * a.ldx[l];
    __syncthreads();
    // (3) layer-l input: spin means and d/dr_j slabs, adjacent column pairs per lane
    const int64_t ldx = a.ldx[l];
    __nv_bfloat16* Xc = X + a.col0[l];
    const int col = 2 * lane, half0 = col < dg ? 0 : 1, half1 = col + 1 < dg ? 0 : 1;
    const int c0 = col - half0 * dg, c1 = col + 1 - half1 * dg;
    for (int pp = warp; pp < npair; pp += n_warps) {
      const int e_i = pp / sh.N, jj = pp - e_i * sh.N;
      if (jj == i0 + e_i || lane >= dg) continue;
      const int sjj = jj < sh.n_up ? 0 : 1;
      const float scale = -1.f / (float)(sjj ? sh.n_dn : sh.n_up);
      const int64_t row = tile_row(w, i0 + e_i, sh.N, sh.wpt) * ldx;
#pragma unroll
      for (int axis = 0; axis < 3; ++axis) {
        const float* src = gs + (pp * 5 + 2 + axis) * 33;
        const float v0 = half0 == sjj ? src[c0] * scale : 0.f, v1 = half1 == sjj ? src[c1] * scale : 0.f;
        st2(Xc + (1 + 3 * jj + axis) * slab + row + col, v0, v1);
        st2_lo(Xc + (sh.T + 1 + 3 * jj + axis) * slab + row + col, v0, v1);
      }
    }
    for (int rr = warp; rr < n_i * 5; rr += n_warps) {
      if (lane >= dg) continue;
      const int e_i = rr / 5, qq = rr - 5 * e_i, ie = i0 + e_i;
      const float* src = gs + (e_i * sh.N * 5 + qq) * 33;
      float up0 = 0.f, up1 = 0.f, dn0 = 0.f, dn1 = 0.f;
      for (int jj = 0; jj < sh.n_up; ++jj) { up0 += src[jj * 165 + c0]; up1 += src[jj * 165 + c1]; }
      for (int jj = sh.n_up; jj < sh.N; ++jj) { dn0 += src[jj * 165 + c0]; dn1 += src[jj * 165 + c1]; }
      const float iu = sh.n_up ? 1.f / (float)sh.n_up : 0.f, id = sh.n_dn ? 1.f / (float)sh.n_dn : 0.f;
      const int t = qq == 0 ? 0 : (qq == 1 ? sh.T - 1 : 1 + 3 * ie + (qq - 2));
      const float m0 = half0 ? dn0 * id : up0 * iu, m1 = half1 ? dn1 * id : up1 * iu;
      const int64_t o = tile_row(w, ie, sh.N, sh.wpt) * ldx + col;
      st2(Xc + t * slab + o, m0, m1);
      st2_lo(Xc + (sh.T + t) * slab + o, m0, m1);
    }
    if (l == a.L - 1) break;
    // (1) products of every jet row with the layer weights (no bias) into zs
    const int nks = (dg + 15) / 16;
    const __nv_bfloat16* whl = wh + l * 32 * kPairWLd;
    const __nv_bfloat16* wll = wl + l * 32 * kPairWLd;
    for (int mt = warp; mt < rows_p / 16; mt += n_warps) {
      const int p0 = mt * 16;
      float c[4][4];
#pragma unroll
      for (int nb = 0; nb < 4; ++nb) c[nb][0] = c[nb][1] = c[nb][2] = c[nb][3] = 0.f;
      for (int ks = 0; ks < nks; ++ks) {
        const int k0 = ks * 16;
        const float* r0 = gs + (p0 + grp) * 33 + k0 + 2 * tig;
        const float* r1 = gs + (p0 + grp + 8) * 33 + k0 + 2 * tig;
        uint32_t ah[4], al[4];
        split_pack(r0[0], r0[1], ah[0], al[0]);
        split_pack(r1[0], r1[1], ah[1], al[1]);
        split_pack(r0[8], r0[9], ah[2], al[2]);
        split_pack(r1[8], r1[9], ah[3], al[3]);
#pragma unroll
        for (int nb = 0; nb < 4; ++nb) {
          const int off = (8 * nb + grp) * kPairWLd + k0 + 2 * tig;
          const uint32_t bh0 = *(const uint32_t*)(whl + off), bh1 = *(const uint32_t*)(whl + off + 8);
          const uint32_t bl0 = *(const uint32_t*)(wll + off), bl1 = *(const uint32_t*)(wll + off + 8);
          mma_16816(c[nb], ah, bh0, bh1);
          mma_16816(c[nb], ah, bl0, bl1);
          mma_16816(c[nb], al, bh0, bh1);
        }
      }
#pragma unroll
      for (int nb = 0; nb < 4; ++nb)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          zs[(p0 + grp + (q >= 2 ? 8 : 0)) * 33 + 8 * nb + 2 * tig + (q & 1)] = c[nb][q];
    }
    __syncthreads();
    // (2) tanh forward-Laplacian rule per (pair, channel); the 6 tangent rows of a pair
    // (d/dr_j = -d/dr_i) give 2 (z_x^2 + z_y^2 + z_z^2)
    for (int e = threadIdx.x; e < npair * 32; e += blockDim.x) {
      const int pp = e >> 5, ch = e & 31;
      const float* zr = zs + pp * 5 * 33 + ch;
      float* gr = gs + pp * 5 * 33 + ch;
      float ov = 0.f, ol = 0.f, ox = 0.f, oy = 0.f, oz = 0.f;
      if (ch < a.h2) {
        const float zv = zr[0] + sc[l * 32 + ch], zl = zr[33], zx = zr[66], zy = zr[99], zz = zr[132];
        const float h = tanh_fast(zv), dh = 1.f - h * h;
        ov = h;
        ox = dh * zx; oy = dh * zy; oz = dh * zz;
        ol = dh * zl - 4.f * h * dh * (zx * zx + zy * zy + zz * zz);
      }
      const bool res = l > 0;
      gr[0] = (res ? gr[0] : 0.f) + ov;
      gr[33] = (res ? gr[33] : 0.f) + ol;
      gr[66] = (res ? gr[66] : 0.f) + ox;
      gr[99] = (res ? gr[99] : 0.f) + oy;
      gr[132] = (res ? gr[132] : 0.f) + oz;
    }
  }
  }
}

// ---------------------------------------------------------------------------------------
// one-electron layer: for every 128-row walker tile and 64 output columns, loop over
// the tangent slabs: value first (h = tanh z), then every gradient slab
// ((1 - h^2) z_t, accumulating sum_t z_t^2), then the Laplacian slab
// ((1 - h^2) z_lap - 2 h (1 - h^2) sum_t z_t^2); plus the residual and the spin means
// of the output for the next layer.
// ---------------------------------------------------------------------------------------
struct LayerArgs {
  const void* X; int ldx; int k_self;
  const void* VsT;      // [k_self][h1]
  const void* Mterm;    // [T][B][h1]
  void* Y; int ldy;     // output [T][R][ldy]
  int residual;
  void* Hbar_out;       // [T][B][2 h1] or null
  void* act_out;        // [R][h1] tanh values (value pass) or null
  int h1;
};

template <typename Act, typename Cmp, bool FULL>
__global__ void __launch_bounds__(256) k_layer(Shape sh, LayerArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cmp* xs = (Cmp*)smem_raw;                // [32][132]
  Cmp* ws = xs + 32 * 132;                 // [32][64]
  Cmp* ys = ws + 32 * 64;                  // [128][65]
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int tile = blockIdx.x, n0 = blockIdx.y * 64;
  const int64_t row0 = (int64_t)tile * 128;
  const Act* X = (const Act*)a.X;
  const Cmp* VsT = (const Cmp*)a.VsT;
  const Cmp* Mt = (const Cmp*)a.Mterm;
  Act* Y = (Act*)a.Y;
  const int64_t xslab = sh.R * a.ldx, yslab = sh.R * a.ldy;
  Cmp hv[8][4], sq[8][4];
  int wv[8];
  for (int q = 0; q < 8; ++q) {
    const int rl = ty * 8 + q, wl = rl / sh.N;
    const int w = tile * sh.wpt + wl;
    wv[q] = (wl < sh.wpt && w < sh.B) ? w : -1;
  }
  for (int t = 0; t < sh.T; ++t) {
    Cmp acc[8][4] = {};
    const Act* Xt = X + t * xslab + row0 * a.ldx;
    for (int k0 = 0; k0 < a.k_self; k0 += 32) {
      for (int e = tid; e < 128 * 32; e += 256) {
        const int rr = e / 32, kk = e % 32;
        const int k = k0 + kk;
        xs[kk * 132 + rr] = k < a.k_self ? (Cmp)ld(Xt + (int64_t)rr * a.ldx + k) : (Cmp)0;
      }
      for (int e = tid; e < 32 * 64; e += 256) {
        const int kk = e / 64, nn = e % 64;
        const int k = k0 + kk, n = n0 + nn;
        ws[kk * 64 + nn] = (k < a.k_self && n < a.h1) ? VsT[(int64_t)k * a.h1 + n] : (Cmp)0;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < 32; ++kk) {
        Cmp av[8], bv[4];
#pragma unroll
        for (int q = 0; q < 8; ++q) av[q] = xs[kk * 132 + ty * 8 + q];
#pragma unroll
        for (int p = 0; p < 4; ++p) bv[p] = ws[kk * 64 + tx * 4 + p];
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
          for (int p = 0; p < 4; ++p) acc[q][p] += av[q] * bv[p];
      }
      __syncthreads();
    }
    // epilogue
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int rl = ty * 8 + q;
      const int64_t row = row0 + rl;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int cl = tx * 4 + p, col = n0 + cl;
        Cmp out = 0;
        if (wv[q] >= 0 && col < a.h1) {
          const Cmp z = acc[q][p] + Mt[((int64_t)t * sh.B + wv[q]) * a.h1 + col];
          if (t == 0) {
            const Cmp h = f_tanh(z);
            hv[q][p] = h;
            sq[q][p] = 0;
            out = h;
            if (a.act_out) ((Cmp*)a.act_out)[row * a.h1 + col] = h;
          } else if (t < sh.T - 1) {
            const Cmp h = hv[q][p];
            out = ((Cmp)1 - h * h) * z;
            sq[q][p] += z * z;
          } else {
            const Cmp h = hv[q][p], d = (Cmp)1 - h * h;
            out = d * z - (Cmp)2 * h * d * sq[q][p];
          }
          if (a.residual) out += (Cmp)ld(X + t * xslab + row * a.ldx + col);
          st(Y + t * yslab + row * a.ldy + col, out);
        }
        ys[rl * 65 + cl] = out;
      }
    }
    if (a.Hbar_out) {
      __syncthreads();
      Act* Hb = (Act*)a.Hbar_out;
      for (int e = tid; e < sh.wpt * 2 * 64; e += 256) {
        const int wl = e / 128, s = (e / 64) % 2, cl = e % 64, col = n0 + cl;
        const int w = tile * sh.wpt + wl;
        if (w >= sh.B || col >= a.h1) continue;
        const int lo = s ? sh.n_up : 0, hi = s ? sh.N : sh.n_up;
        Cmp sum = 0;
        for (int i = lo; i < hi; ++i) sum += ys[(wl * sh.N + i) * 65 + cl];
        st(Hb + ((int64_t)t * sh.B + w) * 2 * a.h1 + s * a.h1 + col, hi > lo ? sum / (Cmp)(hi - lo) : (Cmp)0);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------------------
// orbitals: phi^{k}_i(r_j) = (w_ki . h_j + g_ki) * env_ki(r_j), with the product rule
// over the tangent slabs; envelope derivatives only along r_j.
// ---------------------------------------------------------------------------------------
struct OrbArgs {
  const void* HL;               // [T][R][h1]
  const void* wT[2]; const void* g[2]; const void* pi[2]; const void* sig[2];
  void* Phi;                    // [B][PW]
  int64_t PW;                   // elements per walker
  int h1, K, aniso;
};

// Envelope sum_m pi exp(-s_m) of orbital ko at electron position rj (Eq. 4), its gradient
// along rj and its Laplacian.  Isotropic: s = sigma |d|; anisotropic: s = |Sigma d|, with
// grad s = Sigma^T u / s and lap s = (|Sigma|_F^2 - |Sigma^T u|^2 / s^2) / s.
template <typename Cmp, typename Wlk>
__device__ __forceinline__ void env_jet(const OrbArgs& a, int spin, int ko, const Wlk* rj, const double* nuc, int M,
                                        Cmp* env_out, Cmp* ge, Cmp* le_out) {
  const Cmp* pi = (const Cmp*)a.pi[spin] + (int64_t)ko * M;
  Cmp env = 0, le = 0;
  ge[0] = ge[1] = ge[2] = 0;
  for (int m = 0; m < M; ++m) {
    const Cmp d[3] = {(Cmp)((double)rj[0] - nuc[3 * m]), (Cmp)((double)rj[1] - nuc[3 * m + 1]),
                      (Cmp)((double)rj[2] - nuc[3 * m + 2])};
    Cmp s, gs[3], ls;
    if (!a.aniso) {
      const Cmp sg = ((const Cmp*)a.sig[spin])[(int64_t)ko * M + m];
      const Cmp dist = f_sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      s = sg * dist;
      for (int c = 0; c < 3; ++c) gs[c] = sg * d[c] / dist;
      ls = (Cmp)2 * sg / dist;
    } else {
      const Cmp* S = (const Cmp*)a.sig[spin] + ((int64_t)ko * M + m) * 9;
      Cmp u[3];
      for (int x = 0; x < 3; ++x) u[x] = S[3 * x] * d[0] + S[3 * x + 1] * d[1] + S[3 * x + 2] * d[2];
      s = f_sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      Cmp stu[3], frob = 0, n2 = 0;
      for (int y = 0; y < 3; ++y) stu[y] = S[y] * u[0] + S[3 + y] * u[1] + S[6 + y] * u[2];
      for (int q = 0; q < 9; ++q) frob += S[q] * S[q];
      for (int y = 0; y < 3; ++y) { gs[y] = stu[y] / s; n2 += stu[y] * stu[y]; }
      ls = (frob - n2 / (s * s)) / s;
    }
    const Cmp e = pi[m] * f_exp(-s);
    env += e;
    Cmp g2 = 0;
    for (int c = 0; c < 3; ++c) { ge[c] -= e * gs[c]; g2 += gs[c] * gs[c]; }
    le += e * (g2 - ls);
  }
  *env_out = env;
  *le_out = le;
}

// Envelope-derivative terms of the tensor-core orbital pass: on the slabs of the row's own
// coordinates phi += P_0 d_c env, on the Laplacian slab phi += 2 sum_c P_c d_c env + P_0 lap env.
template <typename PhiT, typename Wlk>
__global__ void k_orbital_fixup(const Wlk* __restrict__ r, const double* __restrict__ nuc, Shape sh, OrbArgs a,
                                const float* __restrict__ orbP) {
  const int w = blockIdx.x / sh.N, j = blockIdx.x % sh.N;
  const int spin = j < sh.n_up ? 0 : 1;
  const int n_s = spin ? sh.n_dn : sh.n_up;
  const int ko = threadIdx.x;
  if (ko >= a.K * n_s) return;
  const int jj = j - (spin ? sh.n_up : 0);
  const int64_t row = tile_row(w, j, sh.N, sh.wpt);
  const int ldp = a.K * sh.N, poff = spin ? a.K * sh.n_up : 0;
  float env, ge[3], le;
  env_jet<float, Wlk>(a, spin, ko, r + ((int64_t)w * sh.N + j) * 3, nuc, sh.M, &env, ge, &le);
  const float* pr = orbP + row * 4 * ldp + poff + ko;
  const float P0 = pr[0];
  const int k = ko / n_s, i = ko % n_s;
  const int64_t nn = (int64_t)n_s * n_s;
  PhiT* base = (PhiT*)a.Phi + (int64_t)w * a.PW + (spin ? (int64_t)a.K * sh.T * sh.n_up * sh.n_up : 0) +
               (int64_t)k * sh.T * nn + i * n_s + jj;
  float lap = P0 * le;
  for (int c = 0; c < 3; ++c) {
    base[(1 + 3 * j + c) * nn] += (PhiT)(P0 * ge[c]);
    lap += 2.f * pr[(1 + c) * ldp] * ge[c];
  }
  base[(sh.T - 1) * nn] += (PhiT)lap;
}

// Envelope values of every (electron, own-spin orbital), one thread each (tensor-core pass).
template <typename Wlk>
__global__ void k_envelope_values(const Wlk* __restrict__ r, const double* __restrict__ nuc, Shape sh, OrbArgs a,
                                  float* __restrict__ envv) {
  // one thread per (walker, electron j, orbital of j's spin); K n_s orbitals per electron.
  // Nuclei as FP32 in shared memory: the envelope values are FP32 in this mode, and FP64
  // arithmetic (conversions included) runs at a small fraction of the FP32 rate on this part.
  __shared__ float nucf[3 * kMaxNuclei];
  for (int q = threadIdx.x; q < 3 * sh.M; q += blockDim.x) nucf[q] = (float)nuc[q];
  __syncthreads();
  const int per_walker = a.K * (sh.n_up * sh.n_up + sh.n_dn * sh.n_dn);
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;       // the host checks B * per_walker < 2^31
  if (gid >= sh.B * per_walker) return;
  const int w = gid / per_walker;
  int rem = gid - w * per_walker;
  const int up_block = a.K * sh.n_up * sh.n_up;
  const int spin = rem < up_block ? 0 : 1;
  if (spin) rem -= up_block;
  const int n_s = spin ? sh.n_dn : sh.n_up;
  const int jj = rem / (a.K * n_s);
  const int j = (spin ? sh.n_up : 0) + jj;
  const int ko = rem - jj * (a.K * n_s);
  const int64_t row = tile_row(w, j, sh.N, sh.wpt);
  const Wlk* rj = r + ((int64_t)w * sh.N + j) * 3;
  const float* pi = (const float*)(spin ? a.pi[1] : a.pi[0]) + ko * sh.M;
  const float* sg = (const float*)(spin ? a.sig[1] : a.sig[0]);
  const float x = (float)rj[0], y = (float)rj[1], z = (float)rj[2];
  float env = 0.f;
  for (int m = 0; m < sh.M; ++m) {
    const float d0 = x - nucf[3 * m], d1 = y - nucf[3 * m + 1], d2 = z - nucf[3 * m + 2];
    float s2;
    if (!a.aniso) {
      s2 = sg[ko * sh.M + m] * sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    } else {
      const float* S = sg + (ko * sh.M + m) * 9;
      const float u0 = S[0] * d0 + S[1] * d1 + S[2] * d2;
      const float u1 = S[3] * d0 + S[4] * d1 + S[5] * d2;
      const float u2 = S[6] * d0 + S[7] * d1 + S[8] * d2;
      s2 = sqrtf(u0 * u0 + u1 * u1 + u2 * u2);
    }
    env += pi[m] * __expf(-s2);
  }
  envv[row * a.K * sh.N + (spin ? a.K * sh.n_up : 0) + ko] = env;
}

// The same values with the envelope parameters staged in shared memory, transposed so that
// the consecutive orbitals of a warp read consecutive words (the global layout puts each
// orbital's 9 M values 36 M bytes apart: 18 scattered cache lines per load instruction).
// Grid: (ceil(K (n_up^2 + n_dn^2) / 256), rows striding over the walkers).  Shared memory
// per spin s: sigma [M][9 or 1][K n_s], then pi [M][K n_s].
template <typename Wlk>
__global__ void k_envelope_values_smem(const Wlk* __restrict__ r, const double* __restrict__ nuc, Shape sh,
                                       OrbArgs a, float* __restrict__ envv) {
  extern __shared__ __align__(16) float env_smem[];
  __shared__ float nucf[3 * kMaxNuclei];
  const int M = sh.M, nc = a.aniso ? 9 : 1;
  const int off1 = M * (nc + 1) * a.K * sh.n_up;             // spin 1's parameters
  for (int q = threadIdx.x; q < 3 * M; q += blockDim.x) nucf[q] = (float)nuc[q];
  for (int sp = 0; sp < 2; ++sp) {
    const int Kn = a.K * (sp ? sh.n_dn : sh.n_up);
    float* sig_sp = env_smem + (sp ? off1 : 0);
    float* pi_sp = sig_sp + M * nc * Kn;
    const float* sg = (const float*)a.sig[sp];
    const float* pg = (const float*)a.pi[sp];
    for (int q = threadIdx.x; q < Kn * M * nc; q += blockDim.x) {
      const int ko = q / (M * nc), mc = q - ko * (M * nc);           // source order (ko, m, c)
      sig_sp[mc * Kn + ko] = sg[q];
    }
    for (int q = threadIdx.x; q < Kn * M; q += blockDim.x) {
      const int ko = q / M, m = q - ko * M;
      pi_sp[m * Kn + ko] = pg[q];
    }
  }
  __syncthreads();
  const int up_block = a.K * sh.n_up * sh.n_up;
  const int per_walker = up_block + a.K * sh.n_dn * sh.n_dn;
  int rem = blockIdx.x * blockDim.x + threadIdx.x;
  if (rem >= per_walker) return;
  const int spin = rem < up_block ? 0 : 1;
  if (spin) rem -= up_block;
  const int n_s = spin ? sh.n_dn : sh.n_up, Kn = a.K * n_s;
  const int jj = rem / Kn;
  const int j = (spin ? sh.n_up : 0) + jj;
  const int ko = rem - jj * Kn;
  const float* S0 = env_smem + (spin ? off1 : 0) + ko;
  const float* P0 = S0 + M * nc * Kn;
  const int64_t col = (spin ? a.K * sh.n_up : 0) + ko;
  // the grid's rows stride over the walkers, so the parameters are staged once per CTA
  for (int w = blockIdx.y; w < sh.B; w += gridDim.y) {
    const int64_t row = tile_row(w, j, sh.N, sh.wpt);
    const Wlk* rj = r + ((int64_t)w * sh.N + j) * 3;
    const float x = (float)rj[0], y = (float)rj[1], z = (float)rj[2];
    float env = 0.f;
    for (int m = 0; m < M; ++m) {
      const float d0 = x - nucf[3 * m], d1 = y - nucf[3 * m + 1], d2 = z - nucf[3 * m + 2];
      float s2;
      if (!a.aniso) {
        s2 = S0[m * Kn] * sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
      } else {
        const float* S = S0 + m * 9 * Kn;
        const float u0 = S[0] * d0 + S[Kn] * d1 + S[2 * Kn] * d2;
        const float u1 = S[3 * Kn] * d0 + S[4 * Kn] * d1 + S[5 * Kn] * d2;
        const float u2 = S[6 * Kn] * d0 + S[7 * Kn] * d1 + S[8 * Kn] * d2;
        s2 = sqrtf(u0 * u0 + u1 * u1 + u2 * u2);
      }
      env += P0[m * Kn] * __expf(-s2);
    }
    envv[row * a.K * sh.N + col] = env;
  }
}

template <typename Act, typename Cmp, typename PhiT, typename Wlk, bool FULL>
__global__ void k_orbitals(const Wlk* __restrict__ r, const double* __restrict__ nuc, Shape sh, OrbArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cmp* hs = (Cmp*)smem_raw;     // [h1]
  const int w = blockIdx.x / sh.N, j = blockIdx.x % sh.N;
  const int spin = j < sh.n_up ? 0 : 1;
  const int n_s = spin ? sh.n_dn : sh.n_up;
  const int jj = j - (spin ? sh.n_up : 0);
  const int n_ko = a.K * n_s;
  const int ko = threadIdx.x;
  const bool active = ko < n_ko;
  const int64_t row = tile_row(w, j, sh.N, sh.wpt);
  const Cmp* wT = (const Cmp*)a.wT[spin];
  // envelope value, gradient along r_j and Laplacian
  Cmp env = 0, ge[3] = {0, 0, 0}, le = 0;
  const Wlk* rj = r + ((int64_t)w * sh.N + j) * 3;
  if (active) env_jet<Cmp, Wlk>(a, spin, ko, rj, nuc, sh.M, &env, ge, &le);
  const int k = active ? ko / n_s : 0, i = active ? ko % n_s : 0;
  PhiT* out = (PhiT*)a.Phi + (int64_t)w * a.PW +
             (spin ? (int64_t)a.K * sh.T * sh.n_up * sh.n_up : 0) + (int64_t)k * sh.T * n_s * n_s +
             (int64_t)i * n_s + jj;
  const int64_t tstride = (int64_t)n_s * n_s;
  const int64_t hslab = sh.R * a.h1;
  const Act* HL = (const Act*)a.HL;
  Cmp p0 = 0, pj[3] = {0, 0, 0};
  for (int t = 0; t < sh.T; ++t) {
    for (int c = threadIdx.x; c < a.h1; c += blockDim.x) hs[c] = (Cmp)ld(HL + t * hslab + row * a.h1 + c);
    __syncthreads();
    if (active) {
      Cmp p = t == 0 ? ((const Cmp*)a.g[spin])[ko] : (Cmp)0;
      for (int c = 0; c < a.h1; ++c) p += hs[c] * wT[(int64_t)c * n_ko + ko];
      Cmp phi;
      if (t == 0) {
        p0 = p;
        phi = p * env;
      } else if (t < sh.T - 1) {
        const int e = (t - 1) / 3, c = (t - 1) % 3;
        phi = p * env;
        if (e == j) { pj[c] = p; phi += p0 * ge[c]; }
      } else {
        phi = p * env + (Cmp)2 * (pj[0] * ge[0] + pj[1] * ge[1] + pj[2] * ge[2]) + p0 * le;
      }
      out[t * tstride] = (PhiT)phi;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// orchestration
// ---------------------------------------------------------------------------------------
template <class Mode>
void launch_forward(const fn_system* s, const void* walkers, const Shape& sh, bool keep, cudaStream_t st) {
  using Act = typename Mode::Act; using Cmp = typename Mode::Cmp; using Det = typename Mode::Det;
  using Wlk = typename Mode::Wlk;
  const Workspace& ws = s->ws;
  const int L = s->cfg.n_layers, h1 = s->cfg.h1, h2 = s->cfg.h2;
  const Cmp* prep = (const Cmp*)ws.prep;
  const bool full = sh.T > 1;
  const Wlk* r = (const Wlk*)walkers;
  // inputs
  {
    const int64_t n = (int64_t)sh.B * sh.N;
    ProfScope ps(s->prof, kProfFeatures, st);
    k_features_en<Act, Wlk><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(r, s->d_nuclei, sh, (Act*)ws.X[0],
                                                                           s->layer[0].ldx);
    const int64_t m = (int64_t)sh.B * 2 * sh.M;
    k_features_mean<Act, Wlk><<<(unsigned)((m + 127) / 128), 128, 0, st>>>(r, s->d_nuclei, sh, (Act*)ws.Hbar[0]);
  }
  {
    PairArgs pa{};
    pa.L = L;
    pa.h2 = h2;
    for (int l = 0; l < L; ++l) {
      pa.X[l] = ws.X[l];
      pa.ldx[l] = s->layer[l].ldx;
      pa.col0[l] = s->layer[l].d_h;
      pa.d_g[l] = s->layer[l].d_g;
      if (l < L - 1) { pa.W[l] = prep + s->prep.W[l]; pa.c[l] = prep + s->prep.c[l]; }
      pa.gstore[l] = (keep && l >= 1) ? ws.gpair[l] : nullptr;
    }
    ProfScope ps(s->prof, full ? kProfPairFull : kProfPair, st);
    if (full) {
      const int ib = pair_full_ib(sh.N);
      const int warps = (ib * sh.N + kPairGroups - 1) / kPairGroups;
      if (Mode::kMode == FN_BF16_MIXED) {
        const int ibm = pair_full_mma_ib(sh.N);
        const size_t smem_m = smem_pair_full_mma(sh.N, L, ibm);
        const int64_t blocks_m =
            std::min<int64_t>((int64_t)sh.B * ((sh.N + ibm - 1) / ibm), (int64_t)s->sm_count * 8);
        cudaFuncSetAttribute(k_pair_full_mma<Wlk>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_m);
        k_pair_full_mma<Wlk><<<(unsigned)blocks_m, 256, smem_m, st>>>(r, sh, pa, ibm);
      } else {
      const size_t smem = smem_pair_full(sizeof(Cmp), sh.N, L, ib);
      const int64_t blocks = (int64_t)sh.B * ((sh.N + ib - 1) / ib);
      cudaFuncSetAttribute(k_pair_full<Act, Cmp, Wlk>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_pair_full<Act, Cmp, Wlk><<<(unsigned)blocks, 32 * warps, smem, st>>>(r, sh, pa, ib);
      }
    } else {
      if (Mode::kMode == FN_BF16_MIXED) {
        const size_t smem = smem_pair_value_mma(sh.N, L);
        cudaFuncSetAttribute(k_pair_value_mma<Wlk>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int64_t blocks_v = std::min<int64_t>(sh.B, (int64_t)s->sm_count * 16);
        k_pair_value_mma<Wlk><<<(unsigned)blocks_v, 128, smem, st>>>(r, sh, pa);
      } else {
        const size_t smem = smem_pair_value(sizeof(Cmp), sh.N, L);
        const int threads = (int)std::min<int64_t>(512, round_up((int64_t)sh.N * sh.N, 32));
        cudaFuncSetAttribute(k_pair_value<Act, Cmp, Wlk>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_pair_value<Act, Cmp, Wlk><<<(unsigned)sh.B, threads, smem, st>>>(r, sh, pa);
      }
    }
  }
  for (int l = 0; l < L; ++l) {
    const LayerDims& d = s->layer[l];
    // mean-field term M = Hbar_l U_l^T + b_l (bias on the value slab only)
    const Act* Hb = (const Act*)ws.Hbar[l];
    {
      ProfScope ps(s->prof, kProfMeanGemm, st);
      if (Mode::kMode == FN_BF16_MIXED) {
        const __nv_bfloat16* U16 = (const __nv_bfloat16*)ws.prep16 + s->prep.U16[l];
        // the spin means are hi/lo pairs: rows T B .. 2 T B hold the low parts
        if (!launch_gemm_tc(sh.T * sh.B, 2 * d.d_h, Hb, 2 * d.d_h, U16, 4 * d.d_h, 2 * d.d_h, h1, (float*)ws.Mterm, h1,
                            (const float*)(prep + s->prep.b[l]), sh.B, 1, false, ws.status, st, sh.T * sh.B))
          const_cast<fn_system*>(s)->host_error = FN_ERR_CUDA;
      } else {
        gemm<Act, Cmp, Cmp, Cmp>(st, sh.T * sh.B, h1, 2 * d.d_h, Hb, 2 * d.d_h, 1, prep + s->prep.UT[l], h1, 1,
                                 (Cmp*)ws.Mterm, h1, 1, prep + s->prep.b[l], sh.B, 1, false);
      }
    }
    LayerArgs la{};
    la.X = ws.X[l]; la.ldx = d.ldx; la.k_self = d.k_self;
    la.VsT = prep + s->prep.VsT[l];
    la.Mterm = ws.Mterm;
    const bool last = l == L - 1;
    la.Y = last ? ws.HL : ws.X[l + 1];
    la.ldy = last ? h1 : s->layer[l + 1].ldx;
    la.residual = l > 0;
    la.Hbar_out = last ? nullptr : ws.Hbar[l + 1];
    la.act_out = keep ? ws.act[l] : nullptr;
    la.h1 = h1;
    ProfScope ps(s->prof, full ? kProfLayerFull : kProfLayerValue, st);
    if (Mode::kMode == FN_BF16_MIXED) {
      const __nv_bfloat16* Vs16 = (const __nv_bfloat16*)ws.prep16 + s->prep.Vs16[l];
      if (!launch_layer_tc(sh, la.X, la.ldx, la.k_self, d.d_h, Vs16, (const float*)la.Mterm, la.Y, la.ldy, la.residual,
                           (float*)la.act_out, h1, ws.status, st))
        const_cast<fn_system*>(s)->host_error = FN_ERR_CUDA;
      if (!last) {
        ProfScope pm(s->prof, kProfSpinMeans, st);
        const int64_t n = (int64_t)sh.T * sh.B * 2 * (h1 / 8);
        const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)s->sm_count * 64);
        k_spin_means_bf16<<<blocks, 256, 0, st>>>(sh, (const __nv_bfloat16*)la.Y, la.ldy, h1,
                                                  (__nv_bfloat16*)la.Hbar_out);
      }
      continue;
    }
    const size_t smem = sizeof(Cmp) * (32 * 132 + 32 * 64 + 128 * 65);
    dim3 grid(sh.tiles, (h1 + 63) / 64);
    if (full) {
      cudaFuncSetAttribute(k_layer<Act, Cmp, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_layer<Act, Cmp, true><<<grid, 256, smem, st>>>(sh, la);
    } else {
      cudaFuncSetAttribute(k_layer<Act, Cmp, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_layer<Act, Cmp, false><<<grid, 256, smem, st>>>(sh, la);
    }
  }
  {
    OrbArgs oa{};
    oa.HL = ws.HL;
    for (int a = 0; a < 2; ++a) {
      oa.wT[a] = prep + s->prep.wT[a]; oa.g[a] = prep + s->prep.g[a];
      oa.pi[a] = prep + s->prep.pi[a]; oa.sig[a] = prep + s->prep.sig[a];
    }
    oa.Phi = ws.Phi;
    oa.PW = phi_walker_stride(s, sh.T);
    oa.h1 = h1; oa.K = s->cfg.n_dets; oa.aniso = s->cfg.envelope == FN_ENV_ANISOTROPIC;
    const int ko_max = s->cfg.n_dets * std::max(s->n_up, s->n_dn);
    const int threads = (int)std::min<int64_t>(1024, round_up(ko_max, 32));
    if (Mode::kMode == FN_BF16_MIXED) {
      {
      ProfScope ps(s->prof, full ? kProfOrbFull : kProfOrbValue, st);
      const int64_t n_env = (int64_t)sh.B * s->cfg.n_dets * (s->n_up * s->n_up + s->n_dn * s->n_dn);
      if (n_env >= ((int64_t)1 << 31)) {
        const_cast<fn_system*>(s)->host_error = FN_ERR_UNSUPPORTED;
        return;
      }
      const int nc = oa.aniso ? 9 : 1;
      const size_t env_smem = sizeof(float) * (size_t)s->M * (nc + 1) * s->cfg.n_dets * (s->n_up + s->n_dn);
      const int per_walker = s->cfg.n_dets * (s->n_up * s->n_up + s->n_dn * s->n_dn);
      if (env_smem <= 160 * 1024) {
        const unsigned gx = (unsigned)((per_walker + 255) / 256);
        const unsigned gy = (unsigned)std::max(1, std::min(sh.B, (s->sm_count * 8 + (int)gx - 1) / (int)gx));
        cudaFuncSetAttribute(k_envelope_values_smem<Wlk>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)env_smem);
        k_envelope_values_smem<Wlk><<<dim3(gx, gy), 256, env_smem, st>>>(r, s->d_nuclei, sh, oa, ws.envv);
      } else {
        k_envelope_values<Wlk><<<(unsigned)((n_env + 255) / 256), 256, 0, st>>>(r, s->d_nuclei, sh, oa, ws.envv);
      }
      const float* wb[2] = {(const float*)oa.g[0], (const float*)oa.g[1]};
      const float* pis[2] = {(const float*)oa.pi[0], (const float*)oa.pi[1]};
      const float* sgs[2] = {(const float*)oa.sig[0], (const float*)oa.sig[1]};
      if (!launch_orbitals_tc(sh, ws.HL, h1, (const __nv_bfloat16*)ws.prep16 + s->prep.W16, wb, pis, sgs,
                              s->cfg.n_dets, oa.aniso, (const float*)walkers, s->d_nuclei, ws.Phi, oa.PW, ws.orbP,
                              ws.envv, ws.status, st))
        const_cast<fn_system*>(s)->host_error = FN_ERR_CUDA;
      }
      if (full) {
        const int ko_max = s->cfg.n_dets * std::max(s->n_up, s->n_dn);
        ProfScope ps2(s->prof, kProfOrbFix, st);
        k_orbital_fixup<typename Mode::PhiT, Wlk><<<(unsigned)((int64_t)sh.B * sh.N), (unsigned)round_up(ko_max, 32), 0,
                                                    st>>>(r, s->d_nuclei, sh, oa, ws.orbP);
      }
      return;
    }
    ProfScope ps(s->prof, full ? kProfOrbFull : kProfOrbValue, st);
    const size_t smem = sizeof(Cmp) * h1;
    const unsigned blocks = (unsigned)((int64_t)sh.B * sh.N);
    using PhiT = typename Mode::PhiT;
    if (full) k_orbitals<Act, Cmp, PhiT, Wlk, true><<<blocks, threads, smem, st>>>(r, s->d_nuclei, sh, oa);
    else k_orbitals<Act, Cmp, PhiT, Wlk, false><<<blocks, threads, smem, st>>>(r, s->d_nuclei, sh, oa);
  }
}

template void launch_prep_params<ModeF64>(const fn_system*, const void*, cudaStream_t);
template void launch_prep_params<ModeF32>(const fn_system*, const void*, cudaStream_t);
template void launch_prep_params<ModeBF16>(const fn_system*, const void*, cudaStream_t);
template void launch_forward<ModeF64>(const fn_system*, const void*, const Shape&, bool, cudaStream_t);
template void launch_forward<ModeF32>(const fn_system*, const void*, const Shape&, bool, cudaStream_t);
template void launch_forward<ModeBF16>(const fn_system*, const void*, const Shape&, bool, cudaStream_t);

}  // namespace fn
