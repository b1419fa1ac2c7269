// Host side of the C ABI: argument checks, parameter-blob layout, Algorithm 1
// (ionic charge initialisation) and the spin split, workspace management and the
// orchestration of the kernel chain for every entry point.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "fn_internal.cuh"

namespace fn {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

fn_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FN_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FN_ERR_OOM : FN_ERR_CUDA;
}

Shape make_shape(const fn_system* s, int B, int T) {
  Shape sh;
  sh.B = B;
  sh.N = s->N;
  sh.n_up = s->n_up;
  sh.n_dn = s->n_dn;
  sh.M = s->M;
  sh.T = T;
  sh.wpt = kTileRows / s->N;
  sh.tiles = (B + sh.wpt - 1) / sh.wpt;
  sh.R = (int64_t)sh.tiles * kTileRows;
  return sh;
}

int64_t phi_walker_stride(const fn_system* s, int T) {
  return (int64_t)s->cfg.n_dets * T * ((int64_t)s->n_up * s->n_up + (int64_t)s->n_dn * s->n_dn);
}

// ---------------------------------------------------------------------------------------
// Algorithm 1 and the spin split (host, integer arithmetic, charges in double)
// ---------------------------------------------------------------------------------------
static fn_status ionic_counts(const std::vector<double>& Z, const double* partial, int t,
                              std::vector<int>* out) {
  const int m_atoms = (int)Z.size();
  std::vector<double> charge(m_atoms);
  std::vector<int> electron(m_atoms);
  for (int a = 0; a < m_atoms; ++a) {
    charge[a] = partial ? partial[a] : (double)t / (double)m_atoms;
    electron[a] = (int)std::lround(Z[a]);
  }
  while (t != 0) {
    if (t < 0) {                      // anion: lowest partial charge receives an electron
      int idx = 0;
      for (int a = 1; a < m_atoms; ++a)
        if (charge[a] < charge[idx]) idx = a;
      electron[idx] += 1;
      t += 1;
      charge[idx] += 1.0;
    } else {                          // cation: highest partial charge loses one
      int idx = -1;
      for (int a = 0; a < m_atoms; ++a)
        if (electron[a] > 0 && (idx < 0 || charge[a] > charge[idx])) idx = a;
      if (idx < 0) {
        set_error("ionic charge exceeds the number of electrons");
        return FN_ERR_ARG;
      }
      electron[idx] -= 1;
      t -= 1;
      charge[idx] -= 1.0;
    }
  }
  *out = electron;
  return FN_OK;
}

static void spin_assign(const std::vector<int>& counts, int n_up, int n_dn, std::vector<int>* atoms) {
  const int m_atoms = (int)counts.size();
  std::vector<int> up(m_atoms), dn(m_atoms);
  int su = 0;
  for (int a = 0; a < m_atoms; ++a) {
    up[a] = (counts[a] + 1) / 2;
    dn[a] = counts[a] / 2;
    su += up[a];
  }
  while (su > n_up) {                 // flip up -> down where up - down is largest
    int best = -1;
    for (int a = 0; a < m_atoms; ++a)
      if (up[a] > 0 && (best < 0 || up[a] - dn[a] > up[best] - dn[best])) best = a;
    up[best] -= 1; dn[best] += 1; su -= 1;
  }
  while (su < n_up) {
    int best = -1;
    for (int a = 0; a < m_atoms; ++a)
      if (dn[a] > 0 && (best < 0 || dn[a] - up[a] > dn[best] - up[best])) best = a;
    dn[best] -= 1; up[best] += 1; su += 1;
  }
  atoms->clear();
  for (int a = 0; a < m_atoms; ++a)
    for (int k = 0; k < up[a]; ++k) atoms->push_back(a);
  for (int a = 0; a < m_atoms; ++a)
    for (int k = 0; k < dn[a]; ++k) atoms->push_back(a);
  (void)n_dn;
}

// ---------------------------------------------------------------------------------------
// layouts
// ---------------------------------------------------------------------------------------
static void build_layout(fn_system* s) {
  const int L = s->cfg.n_layers, h1 = s->cfg.h1, h2 = s->cfg.h2, K = s->cfg.n_dets, M = s->M;
  int64_t off = 0;
  for (int l = 0; l < L; ++l) {
    LayerDims& d = s->layer[l];
    d.d_h = l == 0 ? 4 * M : h1;
    d.d_g = l == 0 ? 4 : h2;
    d.k_self = d.d_h + 2 * d.d_g;
    d.ldx = (int)round_up(d.k_self, 8);
    const int f_in = 3 * d.d_h + 2 * d.d_g;
    d.off_V = off; off += (int64_t)h1 * f_in;
    d.off_b = off; off += h1;
    if (l < L - 1) {
      d.off_W = off; off += (int64_t)h2 * d.d_g;
      d.off_c = off; off += h2;
    } else {
      d.off_W = d.off_c = -1;
    }
  }
  const int nsp[2] = {s->n_up, s->n_dn};
  for (int a = 0; a < 2; ++a) {
    if (!nsp[a]) continue;
    s->off_w[a] = off; off += (int64_t)K * nsp[a] * h1;
    s->off_g[a] = off; off += (int64_t)K * nsp[a];
  }
  const int sig_sz = s->cfg.envelope == FN_ENV_ANISOTROPIC ? 9 : 1;
  for (int a = 0; a < 2; ++a) {
    if (!nsp[a]) continue;
    s->off_pi[a] = off; off += (int64_t)K * nsp[a] * M;
    s->off_sig[a] = off; off += (int64_t)K * nsp[a] * M * sig_sz;
  }
  s->P = off;

  PrepLayout& p = s->prep;
  int64_t q = 0, q16 = 0;
  const int ns[2] = {s->n_up, s->n_dn};
  for (int l = 0; l < L; ++l) {
    const LayerDims& d = s->layer[l];
    p.VsT[l] = q; q += (int64_t)d.k_self * h1;
    p.UT[l] = q; q += (int64_t)2 * d.d_h * h1;
    p.b[l] = q; q += h1;
    if (l < L - 1) {
      p.W[l] = q; q += (int64_t)h2 * d.d_g;
      p.c[l] = q; q += h2;
    }
    p.Vs16[l] = q16; q16 += (int64_t)h1 * 2 * d.ldx;
    q16 = round_up(q16, 64);
    p.U16[l] = q16; q16 += (int64_t)h1 * 4 * d.d_h;
    q = round_up(q, 4);
    q16 = round_up(q16, 64);
  }
  p.W16 = q16; q16 += (int64_t)K * (ns[0] + ns[1]) * 2 * h1;
  q16 = round_up(q16, 64);
  for (int l = 0; l < L; ++l) {
    p.VsT16[l] = q16; q16 += (int64_t)s->layer[l].k_self * 2 * h1;
    q16 = round_up(q16, 64);
  }
  p.ldWT = (int)round_up((int64_t)K * (ns[0] + ns[1]), 64);
  p.W16T = q16; q16 += (int64_t)h1 * 2 * p.ldWT;
  q16 = round_up(q16, 64);
  for (int a = 0; a < 2; ++a) {
    const int64_t ko = (int64_t)K * ns[a];
    p.wT[a] = q; q += ko * h1;
    p.g[a] = q; q += ko;
    p.pi[a] = q; q += ko * M;
    p.sig[a] = q; q += ko * M * sig_sz;
    q = round_up(q, 4);
  }
  p.total = q;
  p.total16 = q16;
}

template <class Mode>
static size_t workspace_layout(fn_system* s, int B, Workspace* ws) {
  using Act = typename Mode::Act; using Cmp = typename Mode::Cmp; using Det = typename Mode::Det;
  using Wlk = typename Mode::Wlk;
  const int T = 3 * s->N + 2;
  const Shape sh = make_shape(s, B, T);
  const int L = s->cfg.n_layers, h1 = s->cfg.h1, h2 = s->cfg.h2, N = s->N;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = (size_t)round_up((int64_t)(off + bytes), 256); return o; };
  std::vector<std::pair<void**, size_t>> items;
  size_t o_X[kMaxLayers], o_Hbar[kMaxLayers], o_act[kMaxLayers], o_gp[kMaxLayers];
  int max_ldx = 0, max_dh = 0;
  // BF16 storage pairs slabs with low parts: X_l and the spin means get slabs T..2T-1
  // (low part of slab t in slab T + t), h_L one (the value slab's)
  const bool pairs = Mode::kMode == FN_BF16_MIXED;
  const int Tx = pairs ? 2 * T : T, Th = T + (pairs ? 1 : 0);
  for (int l = 0; l < L; ++l) {
    o_X[l] = take((size_t)Tx * sh.R * s->layer[l].ldx * sizeof(Act));
    o_Hbar[l] = take((size_t)Tx * B * 2 * s->layer[l].d_h * sizeof(Act));
    o_act[l] = take((size_t)sh.R * h1 * sizeof(Cmp));
    o_gp[l] = take((size_t)B * N * N * h2 * sizeof(Cmp));
    max_ldx = std::max(max_ldx, s->layer[l].ldx);
    max_dh = std::max(max_dh, s->layer[l].d_h);
  }
  const size_t o_HL = take((size_t)Th * sh.R * h1 * sizeof(Act));
  const size_t o_M = take((size_t)T * B * h1 * sizeof(Cmp));
  const size_t o_Phi = take((size_t)B * phi_walker_stride(s, T) * sizeof(typename Mode::PhiT));
  const size_t o_prep = take((size_t)s->prep.total * sizeof(Cmp));
  const size_t o_prep16 = take((size_t)s->prep.total16 * sizeof(__nv_bfloat16));
  const size_t o_walk2 = take((size_t)B * N * 3 * sizeof(Wlk));
  const size_t o_lp2 = take((size_t)B * sizeof(double));
  const size_t o_scr = take((size_t)B * sizeof(double) * 2);
  const size_t o_dX = take((size_t)sh.R * max_ldx * sizeof(Cmp));
  const size_t o_dH = take((size_t)sh.R * h1 * sizeof(Cmp));
  const size_t o_dZ = take((size_t)sh.R * h1 * sizeof(Cmp));
  const size_t o_dZw = take((size_t)B * h1 * sizeof(Cmp));
  const size_t o_dHbar = take((size_t)B * 2 * max_dh * sizeof(Cmp));
  const size_t o_dG = take((size_t)B * N * N * h2 * sizeof(Cmp));
  const size_t o_dPhi = take((size_t)B * phi_walker_stride(s, 1) * sizeof(Det));
  const size_t o_gradc = take((size_t)s->prep.total * sizeof(Cmp));
  const size_t o_dP = take((size_t)sh.R * s->cfg.n_dets * N * sizeof(Cmp));
  const size_t o_orbP = take(Mode::kMode == FN_BF16_MIXED ? (size_t)sh.R * 4 * s->cfg.n_dets * N * sizeof(float) : 0);
  const size_t o_envv = take(Mode::kMode == FN_BF16_MIXED ? (size_t)sh.R * s->cfg.n_dets * N * sizeof(float) : 0);
  const bool bf16 = Mode::kMode == FN_BF16_MIXED;
  int max_k = 0;
  for (int l = 0; l < L; ++l) max_k = std::max(max_k, s->layer[l].k_self);
  const int64_t KN = (int64_t)s->cfg.n_dets * N;
  const size_t o_g16 = take(bf16 ? (size_t)sh.R * std::max<int64_t>(h1, s->prep.ldWT) * 2 : 0);
  const size_t o_t16a = take(bf16 ? (size_t)std::max(max_k, h1) * sh.R * 2 : 0);
  const size_t o_t16b = take(bf16 ? (size_t)std::max<int64_t>(h1, KN) * sh.R * 2 : 0);
  const size_t o_counter = take(sizeof(int64_t) * 4);
  if (ws && ws->base) {
    char* b = (char*)ws->base;
    for (int l = 0; l < L; ++l) {
      ws->X[l] = b + o_X[l]; ws->Hbar[l] = b + o_Hbar[l]; ws->act[l] = b + o_act[l];
      ws->gpair[l] = b + o_gp[l];
    }
    ws->HL = b + o_HL; ws->Mterm = b + o_M; ws->Phi = b + o_Phi; ws->prep = b + o_prep;
    ws->prep16 = b + o_prep16; ws->walk2 = b + o_walk2; ws->lp2 = (double*)(b + o_lp2);
    ws->scratch_d = (double*)(b + o_scr); ws->dX = b + o_dX; ws->dH = b + o_dH; ws->dZ = b + o_dZ;
    ws->dZw = b + o_dZw; ws->dHbar = b + o_dHbar; ws->dG = b + o_dG; ws->dPhi = b + o_dPhi;
    ws->gradc = b + o_gradc; ws->dP = b + o_dP; ws->orbP = (float*)(b + o_orbP); ws->envv = (float*)(b + o_envv); ws->status = s->d_status; ws->counter = (int64_t*)(b + o_counter);
    ws->g16 = b + o_g16; ws->t16a = b + o_t16a; ws->t16b = b + o_t16b;
  }
  return off;
}

template <class F>
static auto dispatch(const fn_system* s, F&& f) {
  switch (s->cfg.precision) {
    case FN_FP64: return f(ModeF64{});
    case FN_FP32: return f(ModeF32{});
    default: return f(ModeBF16{});
  }
}

static size_t workspace_bytes(fn_system* s, int B) {
  return dispatch(s, [&](auto m) { return workspace_layout<decltype(m)>(s, B, nullptr); });
}

// The workspace grows in stream order: the new block is allocated and cleared on the call's
// stream and the old one is freed there (cudaMallocAsync / cudaFreeAsync), so growing never
// waits for the device and never stalls work of other handles on other streams.
static fn_status ensure_workspace(fn_system* s, int B, cudaStream_t st) {
  s->last_stream = (void*)st;
  s->stream_seen = true;
  if (B <= s->ws.cap_B && s->ws.base) return FN_OK;
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) return cuda_status(e, "cudaSetDevice");
  const size_t bytes = workspace_bytes(s, B);
  void* p = nullptr;
  e = cudaMallocAsync(&p, bytes, st);
  if (e != cudaSuccess) return cuda_status(e, "workspace allocation");
  e = cudaMemsetAsync(p, 0, bytes, st);
  if (e != cudaSuccess) { cudaFreeAsync(p, st); return cuda_status(e, "workspace clear"); }
  if (s->ws.base) cudaFreeAsync(s->ws.base, st);
  s->ws.base = p;
  s->ws.bytes = bytes;
  s->ws.cap_B = B;
  dispatch(s, [&](auto m) { return workspace_layout<decltype(m)>(s, B, &s->ws); });
  return FN_OK;
}

static void note_stream(fn_system* s, void* st) {
  s->last_stream = st;
  s->stream_seen = true;
}

// The per-walker kernels keep one walker's pair activations or determinant matrices in
// shared memory; a configuration whose largest such block exceeds the device's per-CTA
// maximum cannot be launched.  Returns the first stage that does not fit (or nullptr) and
// its byte count.
static const char* shared_memory_overflow(const fn_system* s, size_t limit, size_t* need) {
  const int N = s->N, L = s->cfg.n_layers, K = s->cfg.n_dets, nmax = std::max(s->n_up, s->n_dn);
  const bool bf16 = s->cfg.precision == FN_BF16_MIXED;
  const int cmp = s->cfg.precision == FN_FP64 ? 8 : 4;
  const int det = s->cfg.precision == FN_FP32 ? 4 : 8;
  struct Stage { const char* name; size_t bytes; };
  const Stage stages[] = {
      {"two-electron stream, value pass", bf16 ? smem_pair_value_mma(N, L) : smem_pair_value(cmp, N, L)},
      {"two-electron stream, local-energy pass",
       bf16 ? smem_pair_full_mma(N, L, pair_full_mma_ib(N)) : smem_pair_full(cmp, N, L, pair_full_ib(N))},
      {"two-electron stream, gradient", (bf16 && L > 1) ? smem_pair_bwd_mma(N) : 0},
      {"determinant stage, local energy", smem_det_energy(det, nmax, N, K, bf16)},
      {"determinant stage, value pass", nmax > 8 ? smem_det_value(det, nmax, K, false) : 0},
      {"determinant stage, gradient", smem_det_value(det, nmax, K, true)},
  };
  for (const Stage& st : stages)
    if (st.bytes > limit) {
      *need = st.bytes;
      return st.name;
    }
  return nullptr;
}

static fn_status check_launch(fn_system* s, const char* what) {
  if (s->host_error != FN_OK) {
    const fn_status e = s->host_error;
    s->host_error = FN_OK;
    set_error(std::string(what) + (e == FN_ERR_UNSUPPORTED
                                       ? ": batch too large (walkers x determinants x orbitals must stay below 2^31)"
                                       : ": a TMA tensor map could not be encoded or a GEMM shape is not covered"));
    return e;
  }
  return cuda_status(cudaGetLastError(), what);
}

}  // namespace fn

using namespace fn;

// ---------------------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------------------
extern "C" {

const char* fn_last_error(void) { return g_last_error.c_str(); }

fn_status fn_create_system(const double* h_nuclei, const double* h_charges, int n_nuclei,
                           int n_up, int n_down, const fn_net_config* cfg, fn_system_t* out) {
  if (!out || !cfg || !h_nuclei || !h_charges) { set_error("null argument"); return FN_ERR_ARG; }
  *out = nullptr;
  if (n_nuclei < 1 || n_nuclei > kMaxNuclei) { set_error("1..16 nuclei supported"); return FN_ERR_ARG; }
  if (n_up < 0 || n_down < 0) { set_error("negative electron count"); return FN_ERR_ARG; }
  if (n_up + n_down == 0) { set_error("system has no electrons"); return FN_ERR_EMPTY; }
  if (n_up + n_down > kMaxElectrons || n_up > kMaxSpin || n_down > kMaxSpin) {
    set_error("at most 32 electrons and 16 per spin"); return FN_ERR_UNSUPPORTED;
  }
  if (cfg->n_layers < 1 || cfg->n_layers > kMaxLayers || cfg->h1 < 1 || cfg->h1 > 1024 ||
      cfg->h2 < 1 || cfg->h2 > 32 || cfg->n_dets < 1 || cfg->n_dets > 64 ||
      (cfg->envelope != FN_ENV_ISOTROPIC && cfg->envelope != FN_ENV_ANISOTROPIC) ||
      cfg->precision < FN_FP64 || cfg->precision > FN_BF16_MIXED) {
    set_error("network configuration out of range"); return FN_ERR_ARG;
  }
  if (cfg->precision == FN_BF16_MIXED && cfg->h1 % 32 != 0) {
    set_error("h1 must be a multiple of 32 in FN_BF16_MIXED"); return FN_ERR_ARG;
  }
  double zsum = 0.0;
  for (int m = 0; m < n_nuclei; ++m) {
    if (!(h_charges[m] >= 1.0) || std::fabs(h_charges[m] - std::round(h_charges[m])) > 1e-12) {
      set_error("nuclear charges must be positive integers"); return FN_ERR_ARG;
    }
    zsum += h_charges[m];
  }
  fn_system* s = new fn_system();
  s->M = n_nuclei; s->n_up = n_up; s->n_dn = n_down; s->N = n_up + n_down; s->cfg = *cfg;
  s->nuclei.assign(h_nuclei, h_nuclei + 3 * n_nuclei);
  s->charges.assign(h_charges, h_charges + n_nuclei);
  s->total_charge = (int)std::lround(zsum) - s->N;
  for (int m = 0; m < n_nuclei; ++m)
    for (int k = m + 1; k < n_nuclei; ++k) {
      const double dx = h_nuclei[3 * m] - h_nuclei[3 * k], dy = h_nuclei[3 * m + 1] - h_nuclei[3 * k + 1],
                   dz = h_nuclei[3 * m + 2] - h_nuclei[3 * k + 2];
      s->v_nn += h_charges[m] * h_charges[k] / std::sqrt(dx * dx + dy * dy + dz * dz);
    }
  build_layout(s);
  fn_status st = ionic_counts(s->charges, nullptr, s->total_charge, &s->counts);
  if (st != FN_OK) { delete s; return st; }
  spin_assign(s->counts, n_up, n_down, &s->elec_atom);
  int smem_optin = 0;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
  if (e == cudaSuccess) {
    size_t need = 0;
    if (const char* stage = shared_memory_overflow(s, (size_t)smem_optin, &need)) {
      set_error(std::string(stage) + ": " + std::to_string(s->n_up) + "+" + std::to_string(s->n_dn) +
                " electrons, " + std::to_string(cfg->n_dets) + " determinants and " + std::to_string(cfg->n_layers) +
                " layers need " + std::to_string(need) + " bytes of shared memory per CTA; the device allows " +
                std::to_string(smem_optin));
      delete s;
      return FN_ERR_UNSUPPORTED;
    }
  }
  // nuclei [M][3], charges [M] and the device status word (4 ints) in one allocation; the
  // handle's device buffers are stream-ordered allocations made on the per-thread stream (no
  // ordering with other streams), waited for here, and freed in stream order by
  // fn_destroy_system
  const cudaStream_t pst = cudaStreamPerThread;
  if (e == cudaSuccess) e = cudaMallocAsync(&s->d_nuclei, sizeof(double) * (3 * n_nuclei + n_nuclei) + 4 * sizeof(int), pst);
  if (e == cudaSuccess) e = cudaMallocAsync(&s->d_elec_atom, sizeof(int) * kMaxElectrons, pst);
  if (e != cudaSuccess) { fn_status r = cuda_status(e, "create_system"); fn_destroy_system(s); return r; }
  s->d_charges = s->d_nuclei + 3 * n_nuclei;
  s->d_status = (int*)(s->d_nuclei + 4 * n_nuclei);
  e = cudaMemsetAsync(s->d_status, 0, 4 * sizeof(int), pst);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_nuclei, h_nuclei, sizeof(double) * 3 * n_nuclei, cudaMemcpyHostToDevice, pst);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_charges, h_charges, sizeof(double) * n_nuclei, cudaMemcpyHostToDevice, pst);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_elec_atom, s->elec_atom.data(), sizeof(int) * s->N, cudaMemcpyHostToDevice, pst);
  if (e == cudaSuccess) e = cudaStreamSynchronize(pst);
  if (e != cudaSuccess) { fn_status r = cuda_status(e, "create_system copy"); fn_destroy_system(s); return r; }
  st = upload_prep_descs(s);
  if (st != FN_OK) { fn_destroy_system(s); return st; }
  if (cfg->precision == FN_BF16_MIXED && !tc_available()) {
    set_error("the driver does not provide cuTensorMapEncodeTiled"); fn_destroy_system(s); return FN_ERR_UNSUPPORTED;
  }
  *out = s;
  return FN_OK;
}

// The device buffers are freed in stream order on the stream of the handle's latest call
// (its work there finishes first); the host does not wait.  Work of this handle enqueued on
// other streams must be ordered before that stream by the caller, as for every call.
fn_status fn_destroy_system(fn_system_t s) {
  if (!s) return FN_OK;
  const cudaStream_t st = s->stream_seen ? (cudaStream_t)s->last_stream : cudaStreamPerThread;
  void* bufs[5] = {s->ws.base, s->d_nuclei, s->d_elec_atom, s->d_descs, s->d_hf};
  for (void* p : bufs) {
    if (!p) continue;
    if (cudaFreeAsync(p, st) != cudaSuccess) {
      cudaGetLastError();
      cudaDeviceSynchronize();
      cudaFree(p);
    }
  }
  delete s->prof;
  delete s;
  return FN_OK;
}

int64_t fn_param_count(fn_system_t s) { return s ? s->P : -1; }

int64_t fn_workspace_bytes(fn_system_t s, int n_walkers) {
  if (!s || n_walkers < 1) return -1;
  return (int64_t)workspace_bytes(s, n_walkers);
}

fn_status fn_set_walker_offset(fn_system_t s, uint64_t off) {
  if (!s) { set_error("null system"); return FN_ERR_ARG; }
  s->walker_offset = off;
  return FN_OK;
}

fn_status fn_assign_electrons(fn_system_t s, const double* partial, int* counts_out, int* atoms_out) {
  if (!s) { set_error("null system"); return FN_ERR_ARG; }
  std::vector<int> counts, atoms;
  fn_status st = ionic_counts(s->charges, partial, s->total_charge, &counts);
  if (st != FN_OK) return st;
  spin_assign(counts, s->n_up, s->n_dn, &atoms);
  s->counts = counts;
  s->elec_atom = atoms;
  cudaError_t e = cudaMemcpy(s->d_elec_atom, atoms.data(), sizeof(int) * s->N, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e, "assign_electrons copy");
  if (counts_out) std::memcpy(counts_out, counts.data(), sizeof(int) * s->M);
  if (atoms_out) std::memcpy(atoms_out, atoms.data(), sizeof(int) * s->N);
  return FN_OK;
}

fn_status fn_init_params(fn_system_t s, uint64_t seed, void* d_params, void* stream) {
  if (!s || !d_params) { set_error("null argument"); return FN_ERR_ARG; }
  note_stream(s, stream);
  dispatch(s, [&](auto m) { launch_init_params<decltype(m)>(s, seed, d_params, (cudaStream_t)stream); return 0; });
  return check_launch(s, "init_params");
}

fn_status fn_init_walkers(fn_system_t s, int B, uint64_t seed, double init_std, const double* partial,
                          void* d_walkers, int* counts_out, void* stream) {
  if (!s || !d_walkers || B < 1 || !(init_std >= 0.0)) { set_error("invalid argument"); return FN_ERR_ARG; }
  if (partial) {
    fn_status st = fn_assign_electrons(s, partial, nullptr, nullptr);
    if (st != FN_OK) return st;
  }
  if (counts_out) std::memcpy(counts_out, s->counts.data(), sizeof(int) * s->M);
  note_stream(s, stream);
  dispatch(s, [&](auto m) { launch_init_walkers<decltype(m)>(s, B, seed, init_std, d_walkers, (cudaStream_t)stream); return 0; });
  return check_launch(s, "init_walkers");
}

fn_status fn_log_psi(fn_system_t s, const void* d_params, const void* d_walkers, int B,
                     double* d_log_psi, int8_t* d_sign, void* stream) {
  if (!s || !d_params || !d_walkers || B < 1 || !d_log_psi) { set_error("invalid argument"); return FN_ERR_ARG; }
  fn_status st = ensure_workspace(s, B, (cudaStream_t)stream);
  if (st != FN_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  dispatch(s, [&](auto m) {
    using Mode = decltype(m);
    const Shape sh = make_shape(s, B, 1);
    launch_prep_params<Mode>(s, d_params, cs);
    launch_forward<Mode>(s, d_walkers, sh, false, cs);
    launch_det_energy<Mode>(s, d_walkers, sh, nullptr, d_log_psi, d_sign, false, cs);
    return 0;
  });
  return check_launch(s, "log_psi");
}

fn_status fn_local_energy(fn_system_t s, const void* d_params, const void* d_walkers, int B,
                          double* d_e_local, double* d_log_psi, int8_t* d_sign, void* stream) {
  if (!s || !d_params || !d_walkers || B < 1 || !d_e_local) { set_error("invalid argument"); return FN_ERR_ARG; }
  fn_status st = ensure_workspace(s, B, (cudaStream_t)stream);
  if (st != FN_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  dispatch(s, [&](auto m) {
    using Mode = decltype(m);
    const Shape sh = make_shape(s, B, 3 * s->N + 2);
    launch_prep_params<Mode>(s, d_params, cs);
    launch_forward<Mode>(s, d_walkers, sh, false, cs);
    launch_det_energy<Mode>(s, d_walkers, sh, d_e_local, d_log_psi, d_sign, false, cs);
    return 0;
  });
  return check_launch(s, "local_energy");
}

fn_status fn_mcmc_steps(fn_system_t s, const void* d_params, void* d_walkers, double* d_log_psi, int B,
                        int n_steps, double step_size, uint64_t seed, uint64_t step_offset,
                        int64_t* d_accept, void* stream) {
  if (!s || !d_params || !d_walkers || !d_log_psi || B < 1 || n_steps < 0 || !(step_size >= 0.0)) {
    set_error("invalid argument"); return FN_ERR_ARG;
  }
  if (n_steps == 0) return FN_OK;
  fn_status st = ensure_workspace(s, B, (cudaStream_t)stream);
  if (st != FN_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  dispatch(s, [&](auto m) {
    using Mode = decltype(m);
    const Shape sh = make_shape(s, B, 1);
    launch_prep_params<Mode>(s, d_params, cs);
    for (int k = 0; k < n_steps; ++k) {
      const uint32_t step = (uint32_t)(step_offset + (uint64_t)k);
      launch_propose<Mode>(s, B, d_walkers, s->ws.walk2, step_size, seed, step, cs);
      launch_forward<Mode>(s, s->ws.walk2, sh, false, cs);
      launch_det_energy<Mode>(s, s->ws.walk2, sh, nullptr, s->ws.lp2, nullptr, false, cs);
      launch_accept<Mode>(s, B, d_walkers, s->ws.walk2, d_log_psi, s->ws.lp2, seed, step, d_accept, cs);
    }
    return 0;
  });
  return check_launch(s, "mcmc_steps");
}

fn_status fn_energy_grad(fn_system_t s, const void* d_params, const void* d_walkers, const double* d_e_local,
                         int B, void* d_grad, double* d_e_mean, void* stream) {
  if (!s || !d_params || !d_walkers || !d_e_local || !d_grad || B < 1) {
    set_error("invalid argument"); return FN_ERR_ARG;
  }
  fn_status st = ensure_workspace(s, B, (cudaStream_t)stream);
  if (st != FN_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  dispatch(s, [&](auto m) {
    using Mode = decltype(m);
    const Shape sh = make_shape(s, B, 1);
    launch_prep_params<Mode>(s, d_params, cs);
    launch_forward<Mode>(s, d_walkers, sh, true, cs);
    launch_det_energy<Mode>(s, d_walkers, sh, nullptr, s->ws.lp2, nullptr, true, cs);
    launch_energy_weights<Mode>(s, B, d_e_local, s->ws.scratch_d, d_e_mean, cs);
    launch_backward<Mode>(s, d_walkers, sh, s->ws.scratch_d, d_grad, cs);
    return 0;
  });
  return check_launch(s, "energy_grad");
}

fn_status fn_log_psi_vjp(fn_system_t s, const void* d_params, const void* d_walkers, const double* d_weights,
                         int B, void* d_grad, void* stream) {
  if (!s || !d_params || !d_walkers || !d_weights || !d_grad || B < 1) {
    set_error("invalid argument"); return FN_ERR_ARG;
  }
  fn_status st = ensure_workspace(s, B, (cudaStream_t)stream);
  if (st != FN_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  dispatch(s, [&](auto m) {
    using Mode = decltype(m);
    const Shape sh = make_shape(s, B, 1);
    launch_prep_params<Mode>(s, d_params, cs);
    launch_forward<Mode>(s, d_walkers, sh, true, cs);
    launch_det_energy<Mode>(s, d_walkers, sh, nullptr, s->ws.lp2, nullptr, true, cs);
    launch_backward<Mode>(s, d_walkers, sh, d_weights, d_grad, cs);
    return 0;
  });
  return check_launch(s, "log_psi_vjp");
}

static bool adam_args_ok(double lr, double beta1, double beta2, double eps) {
  return std::isfinite(lr) && beta1 >= 0.0 && beta1 < 1.0 && beta2 >= 0.0 && beta2 < 1.0 && eps >= 0.0 &&
         std::isfinite(eps);
}

fn_status fn_adam_step(fn_system_t s, void* d_params, const void* d_grad, void* d_m, void* d_v, int64_t t,
                       double lr, double beta1, double beta2, double eps, void* stream) {
  if (!s || !d_params || !d_grad || !d_m || !d_v || t < 1 || !adam_args_ok(lr, beta1, beta2, eps)) {
    set_error("invalid argument"); return FN_ERR_ARG;
  }
  fn_status st = ensure_workspace(s, 1, (cudaStream_t)stream);   // holds the device status word
  if (st != FN_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  dispatch(s, [&](auto m) {
    launch_adam<decltype(m)>(s, d_params, d_grad, d_m, d_v, t, lr, beta1, beta2, eps, cs);
    return 0;
  });
  return check_launch(s, "adam_step");
}

fn_status fn_sgd_step(fn_system_t s, void* d_params, const void* d_grad, double lr, void* stream) {
  if (!s || !d_params || !d_grad || !std::isfinite(lr)) { set_error("invalid argument"); return FN_ERR_ARG; }
  fn_status st = ensure_workspace(s, 1, (cudaStream_t)stream);
  if (st != FN_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  dispatch(s, [&](auto m) {
    launch_sgd<decltype(m)>(s, d_params, d_grad, lr, cs);
    return 0;
  });
  return check_launch(s, "sgd_step");
}

fn_status fn_clip_local_energy(fn_system_t s, const double* d_e_local, int B, double width, double* d_e_clipped,
                               double* d_stats, void* stream) {
  if (!s || !d_e_local || !d_e_clipped || B < 1 || !std::isfinite(width)) {
    set_error("invalid argument"); return FN_ERR_ARG;
  }
  fn_status st = ensure_workspace(s, 1, (cudaStream_t)stream);
  if (st != FN_OK) return st;
  launch_clip_energy(s, B, d_e_local, width, d_e_clipped, d_stats, (cudaStream_t)stream);
  return check_launch(s, "clip_local_energy");
}

fn_status fn_vmc_iteration(fn_system_t s, const fn_train_config* c, void* d_params, void* d_walkers, int B,
                           int64_t iteration, void* d_opt_state, void* d_grad, double* d_log_psi, double* d_e_local,
                           double* d_e_mean, int64_t* d_accept, void* stream) {
  if (!s || !c || !d_params || !d_walkers || !d_grad || !d_log_psi || !d_e_local || B < 1 || iteration < 0 ||
      c->n_mcmc_steps < 0 || !(c->step_size >= 0.0) || !std::isfinite(c->clip_width) ||
      (c->optimizer != FN_OPT_ADAM && c->optimizer != FN_OPT_SGD) || !std::isfinite(c->lr) ||
      (c->optimizer == FN_OPT_ADAM && (!d_opt_state || !adam_args_ok(c->lr, c->beta1, c->beta2, c->eps)))) {
    set_error("invalid argument"); return FN_ERR_ARG;
  }
  fn_status st = ensure_workspace(s, B, (cudaStream_t)stream);
  if (st != FN_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  const size_t par_bytes = s->cfg.precision == FN_FP64 ? sizeof(double) : sizeof(float);
  dispatch(s, [&](auto m) {
    using Mode = decltype(m);
    const Shape value = make_shape(s, B, 1);
    const Shape full = make_shape(s, B, 3 * s->N + 2);
    launch_prep_params<Mode>(s, d_params, cs);
    // log|psi| of the persistent walkers under the current parameters
    launch_forward<Mode>(s, d_walkers, value, false, cs);
    launch_det_energy<Mode>(s, d_walkers, value, nullptr, d_log_psi, nullptr, false, cs);
    // Metropolis, step indices iteration * n + k
    for (int k = 0; k < c->n_mcmc_steps; ++k) {
      const uint32_t step = (uint32_t)((uint64_t)iteration * (uint64_t)c->n_mcmc_steps + (uint64_t)k);
      launch_propose<Mode>(s, B, d_walkers, s->ws.walk2, c->step_size, c->seed, step, cs);
      launch_forward<Mode>(s, s->ws.walk2, value, false, cs);
      launch_det_energy<Mode>(s, s->ws.walk2, value, nullptr, s->ws.lp2, nullptr, false, cs);
      launch_accept<Mode>(s, B, d_walkers, s->ws.walk2, d_log_psi, s->ws.lp2, c->seed, step, d_accept, cs);
    }
    // local energies (Eqs. 2-3)
    launch_forward<Mode>(s, d_walkers, full, false, cs);
    launch_det_energy<Mode>(s, d_walkers, full, d_e_local, nullptr, nullptr, false, cs);
    // clipping, then the Eq. 6 gradient with the clipped energies held fixed
    const double* e_used = d_e_local;
    if (c->clip_width > 0.0) {
      launch_clip_energy(s, B, d_e_local, c->clip_width, s->ws.scratch_d, nullptr, cs);
      e_used = s->ws.scratch_d;   // the weights below are formed in place
    }
    launch_forward<Mode>(s, d_walkers, value, true, cs);
    launch_det_energy<Mode>(s, d_walkers, value, nullptr, s->ws.lp2, nullptr, true, cs);
    launch_energy_weights<Mode>(s, B, e_used, s->ws.scratch_d, d_e_mean, cs);
    launch_backward<Mode>(s, d_walkers, value, s->ws.scratch_d, d_grad, cs);
    // parameter update
    if (c->optimizer == FN_OPT_ADAM) {
      void* v = (char*)d_opt_state + (size_t)s->P * par_bytes;
      launch_adam<Mode>(s, d_params, d_grad, d_opt_state, v, iteration + 1, c->lr, c->beta1, c->beta2, c->eps, cs);
    } else {
      launch_sgd<Mode>(s, d_params, d_grad, c->lr, cs);
    }
    return 0;
  });
  return check_launch(s, "vmc_iteration");
}

fn_status fn_pretrain_setup(fn_system_t s, double* h_energy) {
  if (!s) { set_error("null system"); return FN_ERR_ARG; }
  return upload_hf_state(s, h_energy);
}

fn_status fn_pretrain_grad(fn_system_t s, const void* d_params, const void* d_walkers, int B, void* d_grad,
                           double* d_loss, void* stream) {
  if (!s || !d_params || !d_walkers || !d_grad || B < 1) { set_error("invalid argument"); return FN_ERR_ARG; }
  if (!s->d_hf) { set_error("fn_pretrain_setup has not been called for this system"); return FN_ERR_ARG; }
  fn_status st = ensure_workspace(s, B, (cudaStream_t)stream);
  if (st != FN_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  dispatch(s, [&](auto m) {
    using Mode = decltype(m);
    const Shape sh = make_shape(s, B, 1);
    launch_prep_params<Mode>(s, d_params, cs);
    launch_forward<Mode>(s, d_walkers, sh, true, cs);
    launch_pretrain_seed<Mode>(s, d_walkers, sh, d_loss, cs);
    launch_backward<Mode>(s, d_walkers, sh, s->ws.scratch_d, d_grad, cs);
    return 0;
  });
  return check_launch(s, "pretrain_grad");
}

fn_status fn_energy_moments(fn_system_t s, const double* d_e_local, int B, double* d_moments, void* stream) {
  if (!s || !d_e_local || !d_moments || B < 1) { set_error("invalid argument"); return FN_ERR_ARG; }
  note_stream(s, stream);
  launch_energy_moments(s, B, d_e_local, d_moments, (cudaStream_t)stream);
  return check_launch(s, "energy_moments");
}

fn_status fn_energy_stats(fn_system_t s, const double* d_moments, double* d_stats, void* stream) {
  if (!s || !d_moments || !d_stats) { set_error("invalid argument"); return FN_ERR_ARG; }
  note_stream(s, stream);
  launch_energy_stats(s, d_moments, d_stats, (cudaStream_t)stream);
  return check_launch(s, "energy_stats");
}

fn_status fn_energy_weights(fn_system_t s, const double* d_e_local, int B, const double* d_moments, double* d_weights,
                            void* stream) {
  if (!s || !d_e_local || !d_moments || !d_weights || B < 1) { set_error("invalid argument"); return FN_ERR_ARG; }
  note_stream(s, stream);
  launch_energy_weights_from(s, B, d_e_local, d_moments, d_weights, (cudaStream_t)stream);
  return check_launch(s, "energy_weights");
}

fn_status fn_selftest_expired_wait(fn_system_t s, int wait_us, void* stream) {
  if (!s || wait_us < 1 || wait_us > 100000) { set_error("invalid argument"); return FN_ERR_ARG; }
  fn_status st = ensure_workspace(s, 1, (cudaStream_t)stream);   // holds the device status word
  if (st != FN_OK) return st;
  launch_expired_wait(s, wait_us, (cudaStream_t)stream);
  return check_launch(s, "selftest_expired_wait");
}

fn_status fn_profile_enable(fn_system_t s, int enable) {
  if (!s) { set_error("null system"); return FN_ERR_ARG; }
  if (!s->prof) s->prof = new Profiler();
  s->prof->reset();
  s->prof->on = enable != 0;
  return FN_OK;
}

int fn_profile_read(fn_system_t s, int index, const char** name, int64_t* launches, double* total_ms) {
  if (!s) return -1;
  if (s->prof) s->prof->collect();
  if (index >= 0 && index < kProfCount) {
    if (name) *name = prof_name(index);
    if (launches) *launches = s->prof ? s->prof->launches[index] : 0;
    if (total_ms) *total_ms = s->prof ? s->prof->ms[index] : 0.0;
  }
  return kProfCount;
}

fn_status fn_sync(fn_system_t s, void* stream, int timeout_ms) {
  if (!s) { set_error("null system"); return FN_ERR_ARG; }
  cudaStream_t cs = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaStreamQuery(cs);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return cuda_status(q, "stream");
    const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_ms >= 0 && el > timeout_ms) { set_error("fn_sync deadline passed"); return FN_ERR_TIMEOUT; }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  // the status word is read and cleared in the order of this stream (already drained)
  int word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_status(e, "status read");
  if (word) {
    cudaMemsetAsync(s->d_status, 0, sizeof(int), cs);
    cudaStreamSynchronize(cs);
    set_error(word & kStatusTimeout ? "a bounded kernel wait expired (timeout bit)"
              : (word & kStatusSingular ? "all determinants singular for some walker" : "non-finite result"));
    if (word & kStatusTimeout) return FN_ERR_TIMEOUT;
    return FN_ERR_NUMERIC;
  }
  return FN_OK;
}

}  // extern "C"
