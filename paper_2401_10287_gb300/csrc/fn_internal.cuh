// Internal declarations of the fnvmc CUDA library: precision traits, the system
// handle, the device workspace layout and the kernel launchers shared between
// translation units.
//
// Data layout in device memory (B walkers, N electrons, T tangent slabs):
//   * T = 1 for value-only passes (Metropolis, log|psi|, energy gradient) and
//     T = 3N + 2 for the local energy: slab 0 is the value, slab 1 + 3e + c the
//     derivative along coordinate c of electron e, slab 3N + 1 the Laplacian.
//   * Electron rows are grouped in walker-aligned tiles of 128 rows: tile q holds
//     walkers q*wpt .. q*wpt + wpt - 1 (wpt = floor(128 / N)), row
//     q*128 + (w - q*wpt)*N + i; the last 128 - wpt*N rows of a tile are padding.
//     A tile therefore contains every electron of its walkers, so spin means
//     over electrons never cross a tile.
//   * Stream-layer inputs X_l are [T][R][ldx_l] (R = tiles*128 rows), columns
//     [h_i (d_h) | mean-up g_i. (d_g) | mean-down g_i. (d_g)].
//   * Spin means of h, Hbar_l, are [T][B][2 d_h]; the mean-field term
//     M_l = Hbar_l U_l^T (+ b_l on slab 0) is [T][B][h1].
//   * Orbital matrices Phi are [B][spin block][K][T][n_s][n_s] with element
//     (i, j) = orbital i evaluated at electron j of that spin.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/fnvmc.h"
#include "fn_profile.cuh"

namespace fn {

constexpr int kTileRows = 128;
constexpr int kMaxLayers = 8;
constexpr int kMaxElectrons = 32;
constexpr int kMaxSpin = 16;
constexpr int kMaxNuclei = 16;

// Status bits written by kernels into the device status word.
constexpr int kStatusNonFinite = 1;
constexpr int kStatusSingular = 2;
constexpr int kStatusTimeout = 4;

// ---- precision traits ------------------------------------------------------------
// Act: storage of stream activations; Cmp: elementwise arithmetic; Det: determinant
// stage; Wlk: walker coordinates; Par: parameter blob.
struct ModeF64 {
  using Act = double; using Cmp = double; using Det = double; using Wlk = double; using Par = double;
  using PhiT = double;
  static constexpr fn_precision kMode = FN_FP64;
};
struct ModeF32 {
  using Act = float; using Cmp = float; using Det = float; using Wlk = float; using Par = float;
  using PhiT = float;
  static constexpr fn_precision kMode = FN_FP32;
};
struct ModeBF16 {
  using Act = __nv_bfloat16; using Cmp = float; using Det = double; using Wlk = float; using Par = float;
  using PhiT = float;          // orbital matrices stored in FP32, factorised in FP64
  static constexpr fn_precision kMode = FN_BF16_MIXED;
};

__host__ __device__ inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ---- dynamic shared memory of the per-walker kernels ------------------------------
// One function per launch; the launchers and fn_create_system both use them, so a
// configuration whose kernels would need more than the device's per-CTA maximum is
// rejected when the system is created instead of failing at its first launch.
constexpr int kMaxH2 = 32;       // widest two-electron stream
constexpr int kPairLanes = 5, kPairGroups = 6;   // k_pair_full: 5 lanes per pair, 6 pairs per warp
constexpr int kPairWLd = 40;     // bf16 row stride of staged pair weights: conflict-free fragment loads
constexpr int kBwdWLd = 40;      // the same for the pair backward

inline size_t pair_weight_bytes(int cmp_bytes, int L) {
  return (size_t)cmp_bytes * ((L - 1) * kMaxH2 * kMaxH2 + (L - 1) * kMaxH2);
}
// k_pair_value (FP32/FP64): staged weights and every pair activation of one walker
inline size_t smem_pair_value(int cmp_bytes, int N, int L) {
  return pair_weight_bytes(cmp_bytes, L) + (size_t)cmp_bytes * N * N * 33;
}
// k_pair_value_mma (BF16)
inline size_t smem_pair_value_mma(int N, int L) {
  return (size_t)(L - 1) * (2 * 32 * kPairWLd * 2 + 32 * 4) + (size_t)((N * N + 15) & ~15) * 33 * 4;
}
// k_pair_full (FP32/FP64): electrons per CTA, the fewest warps per walker with at most 8 warps per CTA
inline int pair_full_ib(int N) {
  int ib = 1, best = 0x7fffffff;
  for (int c = 1; c <= N && c * N <= 8 * kPairGroups; ++c) {
    const int full = N / c, rem = N % c;
    const int warps = full * ((c * N + kPairGroups - 1) / kPairGroups) + (rem ? (rem * N + kPairGroups - 1) / kPairGroups : 0);
    if (warps <= best) { best = warps; ib = c; }
  }
  return ib;
}
inline size_t smem_pair_full(int cmp_bytes, int N, int L, int ib) {
  return pair_weight_bytes(cmp_bytes, L) + (size_t)cmp_bytes * ib * N * 5 * 33;
}
// k_pair_full_mma (BF16): electrons per CTA, at most 256 jet rows (5 per pair)
inline int pair_full_mma_ib(int N) { return std::max(1, std::min(N, 256 / (5 * N))); }
inline size_t smem_pair_full_mma(int N, int L, int ibm) {
  const int rows_p = (ibm * N * 5 + 15) & ~15;
  return (size_t)(L - 1) * (2 * 32 * kPairWLd * 2 + 32 * 4) + (size_t)2 * rows_p * 33 * 4;
}
// k_pair_bwd_mma (BF16)
inline size_t smem_pair_bwd_mma(int N) { return 2 * 32 * kBwdWLd * 2 + (size_t)2 * ((N * N + 15) & ~15) * 33 * 4; }
// k_det_energy: every (determinant, spin) matrix of one walker with its 3N tangent traces;
// with split = true (BF16-mixed mode) also the double-FP32 copy of every inverse of at most
// 8 x 8 (larger blocks keep the FP64 products)
inline size_t smem_det_energy(int det_bytes, int nmax, int N, int K, bool split = false) {
  split = split && nmax <= 8;
  const int ST = (int)round_up(2 * K, 32), NC = 3 * N;
  return (size_t)det_bytes * ((size_t)2 * nmax * nmax * ST + (size_t)nmax * ST + 4 * K + 4 * K * NC + 2 * K + K * NC +
                              2 * K + 128) + sizeof(int) * (size_t)nmax * ST +
         (split ? sizeof(float) * 2 * (size_t)nmax * nmax * ST : 0);
}
// k_det_value (value passes with more than 8 electrons of a spin, and the gradient's pass with inverses)
inline size_t smem_det_value(int det_bytes, int nmax, int K, bool inv) {
  const int threads = (int)round_up(2 * K, 32);
  return (size_t)det_bytes * ((size_t)(inv ? 2 : 1) * nmax * nmax * threads + (size_t)nmax * threads + 5 * K) +
         sizeof(int) * (size_t)nmax * threads;
}

// ---- geometry of one call ----------------------------------------------------------
struct Shape {
  int B = 0;        // walkers in the call
  int N = 0, n_up = 0, n_dn = 0, M = 0;
  int T = 1;        // tangent slabs of this pass
  int wpt = 0;      // walkers per 128-row tile
  int tiles = 0;
  int64_t R = 0;    // padded electron rows
};

// ---- per-layer sizes -----------------------------------------------------------------
struct LayerDims {
  int d_h, d_g;     // input widths of the one- and two-electron features
  int k_self;       // d_h + 2 d_g
  int ldx;          // row stride of X_l (k_self rounded up to 8)
  int64_t off_V, off_b, off_W, off_c;   // offsets in the parameter blob
};

// ---- prepared (internal layout) parameters ------------------------------------------
// All offsets are element offsets into a Cmp-typed array, except the bf16 copies.
struct PrepLayout {
  int64_t VsT[kMaxLayers];   // [k_self][h1]   self part of V, transposed
  int64_t UT[kMaxLayers];    // [2 d_h][h1]    mean-field part of V, transposed
  int64_t b[kMaxLayers];     // [h1]
  int64_t W[kMaxLayers];     // [h2][d_g]      pair weights (as in the blob)
  int64_t c[kMaxLayers];     // [h2]
  int64_t wT[2];             // [h1][K n_s]    orbital projection, transposed
  int64_t g[2];              // [K n_s]
  int64_t pi[2];             // [K n_s][M]
  int64_t sig[2];            // [K n_s][M] or [K n_s][M][9]
  int64_t total;
  // BF16 mode, each a [rows][2 ld] matrix: bf16(W) in columns [0, k), bf16(W - bf16(W)) from column ld
  int64_t Vs16[kMaxLayers];  // self part of V, rows h1, ld = ldx_l
  int64_t U16[kMaxLayers];   // mean-field part of V, rows h1, ld = 2 d_h
  int64_t W16;               // orbital projections, rows K (n_up + n_dn) (up block first), ld = h1
  // backward operands (same split layout): rows are the GEMM's output columns
  int64_t VsT16[kMaxLayers]; // V_self^T: rows k_self, ld = h1  (dX = dZ V_self)
  int64_t W16T;              // orbital projections transposed: rows h1, ld = ldWT (dh_L = dP W)
  int ldWT;                  // K (n_up + n_dn) rounded up to 64 (the hi part of a k-block never reaches the lo part)
  int64_t total16;
};

// One strided copy of the parameter preparation: blob -> internal layout.
struct CopyDesc {
  int64_t src, s_rs, s_cs;   // source offset and strides (row, col) in the blob
  int64_t dst, d_rs, d_cs;   // destination offset and strides
  int rows, cols;
  int to16;                  // 0: Cmp array; 1: bf16 array, bf16(v); 2: bf16 array, bf16(v - bf16(v));
                             // 3: bf16 array, zero (padding columns; the source is not read)
};

struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
  int cap_B = 0;
  // carved pointers (valid for cap_B walkers, full T)
  void* X[kMaxLayers] = {};
  void* HL = nullptr;            // last layer output [T][R][h1] (Act)
  void* Hbar[kMaxLayers] = {};   // [T][B][2 d_h] (Act)
  void* Mterm = nullptr;         // [T][B][h1] (Cmp)
  void* Phi = nullptr;           // [B][per-walker orbital block] (PhiT)
  void* prep = nullptr;          // prepared params (Cmp)
  void* prep16 = nullptr;        // bf16 weights
  void* walk2 = nullptr;         // proposal walkers [B][N][3] (Wlk)
  double* lp2 = nullptr;         // proposal log|psi| [B]
  double* scratch_d = nullptr;   // [B] doubles (per-walker weights etc.)
  // backward (value-only) storage
  void* act[kMaxLayers] = {};    // tanh outputs a_l [R][h1] (Cmp)
  void* gpair[kMaxLayers] = {};  // pair stream g^l [B][N][N][h2] (Cmp), l = 1..L-1
  void* dX = nullptr;            // [R][max ldx] (Cmp)
  void* dH = nullptr;            // [R][h1] (Cmp) running gradient wrt h
  void* dZ = nullptr;            // [R][h1] (Cmp)
  void* dZw = nullptr;           // [B][h1] (Cmp) walker sums of dZ
  void* dHbar = nullptr;         // [B][2 max d_h] (Cmp)
  void* dG = nullptr;            // [B][N][N][h2] (Cmp) gradient wrt the pair stream
  void* dPhi = nullptr;          // [B][orbital block, value slab] (Det)
  void* gradc = nullptr;         // prepared-layout gradient accumulator (Cmp)
  void* dP = nullptr;            // [R][K (n_up + n_dn)] gradient wrt orbital projections (Cmp)
  float* orbP = nullptr;         // [R][4][K N] projections for the orbital envelope fix-up (BF16 mode)
  float* envv = nullptr;         // [R][K N] envelope values (BF16 mode)
  // BF16-mode backward operands for the tensor-core GEMMs
  void* g16 = nullptr;           // [R][max(h1, ldWT)] bf16 copy of dZ or dP
  void* t16a = nullptr;          // [max(k_self, h1)][R] bf16 transposed activations (X_l^T, h_L^T)
  void* t16b = nullptr;          // [max(h1, K N)][R] bf16 transposed gradients (dZ^T, dP^T)
  int* status = nullptr;         // device status word (the handle's d_status)
  int64_t* counter = nullptr;    // scratch counter
};

}  // namespace fn

struct fn_system {
  int M = 0, n_up = 0, n_dn = 0, N = 0;
  fn_net_config cfg{};
  std::vector<double> nuclei, charges;
  int total_charge = 0;
  std::vector<int> counts, elec_atom;
  fn::LayerDims layer[fn::kMaxLayers];
  int64_t off_w[2] = {0, 0}, off_g[2] = {0, 0}, off_pi[2] = {0, 0}, off_sig[2] = {0, 0};
  int64_t P = 0;
  fn::PrepLayout prep{};
  uint64_t walker_offset = 0;
  double v_nn = 0.0;
  int device = 0;
  int sm_count = 0;
  fn::Workspace ws;
  // small device constants
  double* d_nuclei = nullptr;    // [M][3]
  double* d_charges = nullptr;   // [M]
  int* d_status = nullptr;       // device status word (kStatus* bits), read and cleared by fn_sync
  int* d_elec_atom = nullptr;    // [N]
  void* d_descs = nullptr;       // parameter-preparation copy descriptors
  int n_descs = 0;
  double* d_hf = nullptr;        // UHF state for the Eq. 5 pretraining loss (fn_pretrain_setup)
  int hf_nbf = 0;                // its basis functions (0: not set up)
  void* last_stream = nullptr;   // stream of the latest call that enqueued work (frees are ordered on it)
  bool stream_seen = false;
  fn::Profiler* prof = nullptr;  // kernel-class timing (fn_profile_enable)
  fn_status host_error = FN_OK;  // set by a launcher that could not enqueue its kernel
};

namespace fn {

void set_error(const std::string& msg);
fn_status cuda_status(cudaError_t e, const char* what);

fn_status upload_prep_descs(fn_system* s);

// Tensor-core one-electron layer (BF16 mode); false if a TMA tensor map could not be built.
bool launch_layer_tc(const Shape& sh, const void* X, int ldx, int k_self, int lo_col0, const void* Vs16,
                     const float* Mterm, void* Y, int ldy, int residual, float* act_out, int h1, int* status,
                     cudaStream_t st);
bool launch_gemm_tc(int rows, int k, const void* A, int lda, const void* Bw, int ldb, int bsplit, int ncols, float* C,
                    int ldc, const float* bias, int bias_rows, int ksplit, bool atomic, int* status, cudaStream_t st,
                    int a_lo_row = 0);
bool launch_orbitals_tc(const Shape& sh, const void* HL, int h1, const void* W16, const float* const* wbias,
                        const float* const* pi, const float* const* sig, int K, int aniso, const float* walkers,
                        const double* nuclei, void* Phi, int64_t PW, float* orbP, const float* envv, int* status,
                        cudaStream_t st);
bool tc_available();

// Shapes and sizes
Shape make_shape(const fn_system* s, int B, int T);
int64_t phi_walker_stride(const fn_system* s, int T);   // elements per walker of Phi

// ---- launchers (one instantiation per precision mode) --------------------------------
template <class Mode> void launch_prep_params(const fn_system* s, const void* params, cudaStream_t st);
template <class Mode> void launch_forward(const fn_system* s, const void* walkers, const Shape& sh,
                                          bool keep_for_backward, cudaStream_t st);
template <class Mode> void launch_det_energy(const fn_system* s, const void* walkers, const Shape& sh,
                                             double* e_local, double* log_psi, int8_t* sign,
                                             bool keep_inverse, cudaStream_t st);
template <class Mode> void launch_init_walkers(const fn_system* s, int B, uint64_t seed, double std_,
                                               void* walkers, cudaStream_t st);
template <class Mode> void launch_init_params(const fn_system* s, uint64_t seed, void* params,
                                              cudaStream_t st);
template <class Mode> void launch_propose(const fn_system* s, int B, const void* walkers, void* out,
                                          double step, uint64_t seed, uint32_t step_idx, cudaStream_t st);
template <class Mode> void launch_accept(const fn_system* s, int B, void* walkers, const void* prop,
                                         double* lp, const double* lp_new, uint64_t seed,
                                         uint32_t step_idx, int64_t* accept_count, cudaStream_t st);
template <class Mode> void launch_energy_weights(const fn_system* s, int B, const double* e_local, double* weights,
                                                 double* e_mean, cudaStream_t st);
template <class Mode> void launch_backward(const fn_system* s, const void* walkers, const Shape& sh,
                                           const double* weights, void* grad, cudaStream_t st);

// Training loop (fn_optim.cu): parameter updates on the flat blob and local-energy clipping.
template <class Mode> void launch_adam(const fn_system* s, void* params, const void* grad, void* m, void* v,
                                       int64_t t, double lr, double beta1, double beta2, double eps,
                                       cudaStream_t st);
template <class Mode> void launch_sgd(const fn_system* s, void* params, const void* grad, double lr,
                                      cudaStream_t st);
void launch_clip_energy(const fn_system* s, int B, const double* e, double width, double* out, double* stats,
                        cudaStream_t st);
// Eq. 5 pretraining (fn_pretrain.cu, fn_scf.cu): UHF state upload, the loss and its seeds.
fn_status upload_hf_state(fn_system* s, double* e_out);
template <class Mode> void launch_pretrain_seed(const fn_system* s, const void* walkers, const Shape& sh,
                                                double* loss, cudaStream_t st);
// Eq. 1 statistics and Eq. 6 weights from summable moments [count, sum E_L, sum E_L^2] (fn_optim.cu).
void launch_energy_moments(const fn_system* s, int B, const double* e, double* mom, cudaStream_t st);
void launch_energy_stats(const fn_system* s, const double* mom, double* stats, cudaStream_t st);
void launch_energy_weights_from(const fn_system* s, int B, const double* e, const double* mom, double* w,
                                cudaStream_t st);
// Failure-path self-test (fn_selftest.cu): a barrier wait that expires after wait_us.
void launch_expired_wait(const fn_system* s, int wait_us, cudaStream_t st);

}  // namespace fn
