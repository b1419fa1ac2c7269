/*
 * fnvmc.h - C ABI of the GB300 (sm_103a) variational Monte Carlo hot path.
 *
 * The library evaluates a permutation-equivariant fermionic neural-network
 * wavefunction (method section "FermiNet Model", Eq. 4 envelope) for batches of
 * walkers, its exact local energy (Eqs. 1-3, exact forward-mode Laplacian), runs
 * Metropolis-Hastings on |psi|^2 (section "Electron Sampler"), assigns electrons
 * to atoms with the ionic charge initialisation (Algorithm 1) and computes the
 * VMC energy gradient (Eq. 6).  Every step runs in the library's CUDA kernels;
 * there is no CPU fallback.
 *
 * Conventions shared by all entry points
 *   - Lengths in bohr, energies in hartree.
 *   - d_* pointers are device memory owned by the caller; h_* pointers are host
 *     memory owned by the caller.  The library owns the system handle and an
 *     internal device workspace that grows on demand (a stream-ordered
 *     allocation on the call's stream happens only when a call needs more
 *     walkers than any previous call on that handle).
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream).  Argument errors return
 *     immediately and leave device memory untouched.  Numerical problems found
 *     on the device (non-finite log|psi| or local energy, singular
 *     determinants of every term) are recorded in a device status word and
 *     reported by fn_sync() as FN_ERR_NUMERIC.
 *   - Precision modes fix the dtypes:
 *       FN_FP64        params double, walkers double, all arithmetic FP64;
 *       FN_FP32        params float,  walkers float,  all arithmetic FP32
 *                      (energies accumulated and returned in FP64);
 *       FN_BF16_MIXED  params float,  walkers float; stream-layer and
 *                      Laplacian-tangent contractions on tcgen05 tensor cores
 *                      with BF16 operands and FP32 accumulation; elementwise
 *                      work FP32; determinants, their inverse-based gradient and
 *                      Laplacian terms and the local-energy assembly in FP64.
 *   - Walkers are stored [B][N][3]; electrons 0..n_up-1 are spin up, the rest
 *     spin down.  Walker index w in a call is global index walker_offset + w
 *     for the random streams (see fn_set_walker_offset).
 *   - The handle is not thread-safe: calls on one handle must not overlap in
 *     time from different host threads, and calls on one handle enqueued on
 *     different streams must be ordered by the caller (they share a workspace).
 *   - fn_last_error() returns a thread-local message for the last failing call.
 *   - Environment: FN_LAYER_KERNEL=pair selects, for BF16 stream layers whose
 *     output width is a multiple of 128, the CTA-pair tensor-core kernel
 *     (cta_group::2) instead of the default one-CTA kernel; the outputs are
 *     the same bits.  FN_DET_KERNEL=thread selects, for the BF16 local-energy
 *     determinant stage with blocks of 5 to 8 electrons, one thread per block
 *     instead of 8-lane groups; the results agree to rounding.  Both are read
 *     at every launch.
 */
#ifndef FNVMC_H
#define FNVMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FN_OK = 0,
  FN_ERR_ARG = 1,         /* invalid argument or size                           */
  FN_ERR_OOM = 2,         /* device allocation failed                           */
  FN_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed        */
  FN_ERR_TIMEOUT = 4,     /* fn_sync deadline passed before the stream drained  */
  FN_ERR_NUMERIC = 5,     /* non-finite or singular result recorded on device   */
  FN_ERR_EMPTY = 6,       /* system with no electrons                           */
  FN_ERR_UNSUPPORTED = 7  /* configuration outside the compiled kernel limits   */
} fn_status;

typedef enum { FN_FP64 = 0, FN_FP32 = 1, FN_BF16_MIXED = 2 } fn_precision;
typedef enum { FN_ENV_ISOTROPIC = 0, FN_ENV_ANISOTROPIC = 1 } fn_envelope;

/* Network sizes ("FermiNet Model" section):
 *   n_layers  one-electron stream layers L >= 1 (the two-electron stream has L-1);
 *   h1        one-electron width, 1..1024, multiple of 32 in FN_BF16_MIXED;
 *   h2        two-electron width, 1..32;
 *   n_dets    determinants K, 1..64;
 *   envelope  fn_envelope: scalar sigma per (k, i, m, spin) or 3x3 sigma (Eq. 4);
 *   precision fn_precision.                                                      */
typedef struct {
  int n_layers, h1, h2, n_dets;
  int envelope;
  int precision;
} fn_net_config;

typedef struct fn_system* fn_system_t;

/* Creates a system: M nuclei at h_nuclei[M][3] with charges h_charges[M]
 * (integer-valued), n_up + n_down electrons (1..32 in total, each spin <= 16),
 * and a network configuration.  The ionic charge t = sum Z - n_up - n_down is
 * derived.  The default electron assignment is Algorithm 1 with partial
 * charges t/M for every atom.  Returns FN_ERR_EMPTY for zero electrons.
 * The per-walker kernels keep one walker's pair activations (N^2 rows) and its
 * 2 n_dets determinant matrices in shared memory, so the sizes above combine
 * into smaller limits on a device with 227 KB per CTA: FN_FP32 reaches 32
 * electrons, and n_dets 32 at 16 electrons of one spin; FN_FP64 reaches 29
 * electrons with 2 layers (25 with 8); FN_BF16_MIXED reaches 29 electrons;
 * FN_FP64 and FN_BF16_MIXED reach n_dets 16 at 16 electrons of one spin.  A
 * configuration that does not fit returns FN_ERR_UNSUPPORTED, and
 * fn_last_error() names the stage and the bytes it needs.                   */
fn_status fn_create_system(const double* h_nuclei, const double* h_charges, int n_nuclei,
                           int n_up, int n_down, const fn_net_config* cfg, fn_system_t* out);
fn_status fn_destroy_system(fn_system_t sys);

/* Number of entries of the flat parameter blob (dtype per precision mode).
 * Blob order: for each layer l: V_l [h1][3 d_h + 2 d_g] (columns: h_i, mean
 * up h, mean down h, mean up g_i., mean down g_i.), b_l [h1], and for
 * l < L-1: W_l [h2][d_g], c_l [h2]  (d_h = 4M, d_g = 4 at l = 0, else h1, h2);
 * then w_up [K n_up][h1], g_up [K n_up], w_down, g_down; then pi_up [K n_up][M],
 * sigma_up [K n_up][M] or [K n_up][M][3][3], pi_down, sigma_down.  Orbital rows
 * are ordered k * n_spin + i.  Spin blocks with no electron are absent.      */
int64_t fn_param_count(fn_system_t sys);

/* Device workspace bytes a call with n_walkers walkers needs (for admission). */
int64_t fn_workspace_bytes(fn_system_t sys, int n_walkers);

/* Global index of walker 0 in the random streams (default 0), so that a batch
 * split across devices draws the same numbers as one device.               */
fn_status fn_set_walker_offset(fn_system_t sys, uint64_t walker_offset);

/* Algorithm 1 (ionic charge initialisation) followed by the spin split, on
 * the host.  h_partial_charges[M] are Mulliken-style partial charges, or NULL
 * for t/M each.  Ties go to the lowest atom index; an atom with no electron
 * left is skipped when removing.  Writes per-atom counts h_counts_out[M] and
 * the atom of every electron h_electron_atoms_out[N] (either may be NULL) and
 * makes this the system's assignment for fn_init_walkers.                   */
fn_status fn_assign_electrons(fn_system_t sys, const double* h_partial_charges,
                              int* h_counts_out, int* h_electron_atoms_out);

/* Parameter initialisation: dense weights and biases N(0,1)/sqrt(fan_in) from
 * the Philox4x32-10 stream (counter (j>>1, 0, 0, 3), key = seed), envelope
 * pi = 1 and sigma = 1 (identity).  Bit-identical to the FP64 definition,
 * then rounded to the blob dtype.                                           */
fn_status fn_init_params(fn_system_t sys, uint64_t seed, void* d_params, void* stream);

/* Walker initialisation ("Electron Sampler"): runs fn_assign_electrons with
 * h_partial_charges (NULL: keep the current assignment), then
 * r[w][e] = R[atom(e)] + init_std * z, z from the Philox stream
 * (counter (j>>1, w, 0, 0), j = 3e + axis), computed in FP64 without fused
 * multiply-add and rounded to the walker dtype: bit-exact.
 * d_walkers [n_walkers][N][3]; h_atom_counts_out [M] or NULL.              */
fn_status fn_init_walkers(fn_system_t sys, int n_walkers, uint64_t seed, double init_std,
                          const double* h_partial_charges, void* d_walkers,
                          int* h_atom_counts_out, void* stream);

/* log|psi| and sign of psi for every walker (value-only forward pass).
 * d_log_psi [n_walkers] double, d_sign [n_walkers] int8 (+1/-1, 0 if psi = 0). */
fn_status fn_log_psi(fn_system_t sys, const void* d_params, const void* d_walkers,
                     int n_walkers, double* d_log_psi, int8_t* d_sign, void* stream);

/* n_steps Metropolis-Hastings steps on |psi|^2: r' = r + step_size * z for all
 * 3N coordinates (proposal stream counter (j>>1, w, step, 1)), accept iff
 * log U <= 2 (log|psi(r')| - log|psi(r)|), U = (m+1) 2^-53 from counter
 * (0, w, step, 2); step = step_offset + s (low 32 bits).  d_log_psi holds
 * log|psi| of the incoming walkers on entry (e.g. from fn_log_psi) and of the
 * outgoing walkers on exit.  d_accept_count [1] int64 is incremented by the
 * number of accepted moves (NULL to skip).                                  */
fn_status fn_mcmc_steps(fn_system_t sys, const void* d_params, void* d_walkers, double* d_log_psi,
                        int n_walkers, int n_steps, double step_size, uint64_t seed,
                        uint64_t step_offset, int64_t* d_accept_count, void* stream);

/* Local energy with the exact Laplacian (Eqs. 2-3):
 * E_L = -1/2 sum_c [(d_c log|psi|)^2 + d_c^2 log|psi|] + V_ee + V_ne + V_nn.
 * d_e_local, d_log_psi [n_walkers] double; d_sign [n_walkers] int8 (either of
 * the last two may be NULL).                                                */
fn_status fn_local_energy(fn_system_t sys, const void* d_params, const void* d_walkers,
                          int n_walkers, double* d_e_local, double* d_log_psi, int8_t* d_sign,
                          void* stream);

/* VMC energy gradient (Eq. 6): grad = (2/B) sum_w (E_L,w - mean E_L) d log|psi_w| / d theta,
 * with E_L held fixed.  The value-only forward pass is recomputed; gradients
 * are written to d_grad [fn_param_count] in blob order and blob dtype.
 * d_e_mean_out [1] double receives mean E_L (NULL to skip).                 */
fn_status fn_energy_grad(fn_system_t sys, const void* d_params, const void* d_walkers,
                         const double* d_e_local, int n_walkers, void* d_grad,
                         double* d_e_mean_out, void* stream);

/* Weighted parameter gradient of log|psi|: d_grad = sum_w d_weights[w] d log|psi_w| / d theta
 * (the vector-Jacobian product of the value-only forward pass).  fn_energy_grad is this
 * with weights 2 (E_L,w - mean E_L) / B; a batch split across devices uses it with
 * weights built from the global mean and count, then sums the gradients (Eq. 6).
 * d_weights [n_walkers] double; d_grad [fn_param_count] blob dtype.           */
fn_status fn_log_psi_vjp(fn_system_t sys, const void* d_params, const void* d_walkers,
                         const double* d_weights, int n_walkers, void* d_grad, void* stream);

/* log|psi| and sign, like fn_log_psi, for callers that cannot let the library allocate
 * device memory: programs whose device memory belongs to a pool or framework allocator
 * that must account for every byte, and processes with a memory budget fixed before the
 * library was loaded.  No cudaMalloc or cudaFree happens in this call.  Its scratch is one
 * static 64 MiB device array that every device loading the library holds until the
 * process exits; the array's address is looked up on the first call made on each
 * device (cudaGetSymbolAddress), so make that first call before any stream capture.
 * Calls share the array: two calls whose work overlaps on the GPU race, so order them
 * on one stream.  Each call writes every part of the array it reads, so what an earlier
 * call (of any system) left there never reaches the result.  A batch whose scratch
 * exceeds 64 MiB returns FN_ERR_ARG, with the walker count that fits in fn_last_error().
 * The handle's own workspace is untouched; errors found on the device (non-finite or
 * singular results, an expired bounded wait) are recorded in the handle's status word
 * and reported by the next fn_sync, as for fn_log_psi.
 * The method has no counterpart of this entry point; it is a deployment variant.  */
fn_status fn_log_psi_noalloc(fn_system_t sys, const void* d_params, const void* d_walkers,
                             int n_walkers, double* d_log_psi, int8_t* d_sign, void* stream);

/* ---- Eq. 5 pretraining -------------------------------------------------------------------
 * Before the energy is optimised, the method fits the network's orbitals to Hartree-Fock
 * orbitals at the sampled positions (Eq. 5): L = (1/B) sum_w sum_spin sum_{k,i,j}
 * (Phi_kij - Phi^HF_ij)^2, k the determinant, i the orbital, j the electron of that spin,
 * B the walkers; the same occupied UHF orbital i (STO-6G, in order of orbital energy, signed
 * so that its largest-magnitude coefficient is positive) is the target of every determinant. */

/* Runs unrestricted Hartree-Fock in STO-6G for the system (nuclei H..Ne, at most 20 basis
 * functions, the system's n_up and n_down) on the host and keeps its occupied orbitals on the
 * device for fn_pretrain_grad.  h_energy [1] receives the UHF energy (NULL to skip).
 * FN_ERR_ARG for other elements, FN_ERR_UNSUPPORTED above 20 functions or when occupied
 * levels are degenerate (the target is then not unique), FN_ERR_NUMERIC if it does not
 * converge.  Synchronous; call it once per system.                                          */
fn_status fn_pretrain_setup(fn_system_t sys, double* h_energy);

/* Eq. 5 loss of the walkers and its parameter gradient: the value-only forward pass, the
 * HF orbitals at every electron, dL/dPhi, and the hand-written reverse pass of fn_energy_grad
 * from that seed.  d_grad [fn_param_count] blob dtype; d_loss [1] double (NULL to skip).
 * FN_ERR_ARG if fn_pretrain_setup was not called.                                           */
fn_status fn_pretrain_grad(fn_system_t sys, const void* d_params, const void* d_walkers, int n_walkers,
                           void* d_grad, double* d_loss, void* stream);

/* ---- Eq. 1 estimator and Eq. 6 weights from summable moments ------------------------
 * The VMC energy is the mean local energy over the sampled walkers (Eq. 1); its error bar
 * follows from their variance.  The moments [count, sum E_L, sum E_L^2] (FP64) add up over
 * batches and devices, so a batch split across GPUs all-reduces these three numbers (a sum)
 * and then forms the statistics or the Eq. 6 weights from the global moments.            */

/* d_moments [3] double <- [n_walkers, sum E_L, sum E_L^2] of d_e_local [n_walkers] double
 * (one CTA, fixed summation order).                                                      */
fn_status fn_energy_moments(fn_system_t sys, const double* d_e_local, int n_walkers, double* d_moments,
                            void* stream);

/* d_stats [3] double <- [count, mean = sum / count, variance = sum2 / count - mean^2 (>= 0)]
 * from d_moments [3] (Eq. 1; the standard error is sqrt(variance / count)).  A non-finite
 * mean or variance sets the numeric bit reported by fn_sync.                               */
fn_status fn_energy_stats(fn_system_t sys, const double* d_moments, double* d_stats, void* stream);

/* Eq. 6 weights with the mean and count of d_moments [3] (e.g. all-reduced over devices):
 * d_weights[w] = 2 (d_e_local[w] - sum / count) / count, [n_walkers] double; the input of
 * fn_log_psi_vjp.                                                                           */
fn_status fn_energy_weights(fn_system_t sys, const double* d_e_local, int n_walkers, const double* d_moments,
                            double* d_weights, void* stream);

/* ---- VMC training loop ------------------------------------------------------------
 * The training phase of the method updates the parameters with the Eq. 6 gradient
 * between rounds of the electron sampler.  The method names no optimiser: the library
 * offers Adam (Kingma & Ba 2015, Algorithm 1) and plain gradient descent, and an optional
 * clamp of the local energies to a window around their median before Eq. 6.           */

/* Adam update of the flat parameter blob, in place, with step count t >= 1:
 *   m <- beta1 m + (1 - beta1) g,   v <- beta2 v + (1 - beta2) g^2,
 *   theta <- theta - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
 * d_params, d_grad, d_m, d_v [fn_param_count] blob dtype, caller-owned; d_m and d_v are
 * zero before the first step and must not alias each other, d_params or d_grad.
 * Requires 0 <= beta1, beta2 < 1, eps >= 0 and a finite lr; arithmetic in the blob dtype.
 * A non-finite updated parameter sets the numeric bit reported by fn_sync.          */
fn_status fn_adam_step(fn_system_t sys, void* d_params, const void* d_grad, void* d_m, void* d_v,
                       int64_t t, double lr, double beta1, double beta2, double eps, void* stream);

/* Gradient descent, in place: theta <- theta - lr g (blob dtype, [fn_param_count]).  */
fn_status fn_sgd_step(fn_system_t sys, void* d_params, const void* d_grad, double lr, void* stream);

/* Local-energy clipping: centre = the lower median (the element of rank
 * floor((B - 1) / 2) of the sorted batch, an exact member of it), spread = mean |E_L - centre|
 * (summed in FP64), and every energy clamped to centre +- width * spread; width <= 0
 * copies the energies unchanged.  d_e_local, d_e_clipped [n_walkers] double; they may be
 * the same buffer.  d_stats [2] double receives (centre, spread), NULL to skip.  One CTA
 * does the work (a selection pass reads the batch 8 times).  A non-finite energy makes
 * the spread non-finite: nothing is clamped and fn_sync reports FN_ERR_NUMERIC.     */
fn_status fn_clip_local_energy(fn_system_t sys, const double* d_e_local, int n_walkers, double width,
                               double* d_e_clipped, double* d_stats, void* stream);

typedef enum { FN_OPT_ADAM = 0, FN_OPT_SGD = 1 } fn_optimizer;

/* Settings of one training iteration.
 *   n_mcmc_steps  Metropolis steps per iteration (>= 0);
 *   step_size     proposal standard deviation in bohr (>= 0);
 *   seed          key of the sampler's random streams;
 *   clip_width    local-energy clipping width (fn_clip_local_energy), <= 0 for none;
 *   optimizer     fn_optimizer;
 *   lr, beta1, beta2, eps   rate and Adam settings (beta and eps unused by FN_OPT_SGD). */
typedef struct {
  int n_mcmc_steps;
  double step_size;
  uint64_t seed;
  double clip_width;
  int optimizer;
  double lr, beta1, beta2, eps;
} fn_train_config;

/* One VMC training iteration with index `iteration` >= 0 on walkers that persist between
 * iterations, in this order:
 *   1. log|psi| of d_walkers under the current parameters (value-only pass);
 *   2. n_mcmc_steps Metropolis steps (fn_mcmc_steps) with step indices
 *      iteration * n_mcmc_steps + k, k = 0 .. n_mcmc_steps - 1 (taken modulo 2^32);
 *   3. local energies of the moved walkers (fn_local_energy);
 *   4. clipping with cfg->clip_width (the clipped copy is internal);
 *   5. the Eq. 6 gradient with the clipped energies held fixed (fn_energy_grad);
 *   6. the update: Adam with step count iteration + 1, or gradient descent.
 * d_params updated in place; d_walkers [B][N][3] updated in place; d_opt_state
 * [2 fn_param_count] blob dtype = (m, v) of Adam, zero before iteration 0 (NULL for SGD);
 * d_grad [fn_param_count] blob dtype receives the gradient of step 5; d_log_psi [B] double
 * receives log|psi| of the moved walkers under the parameters before the update;
 * d_e_local [B] double receives the unclipped energies; d_e_mean [1] double receives the
 * mean of the clipped energies (NULL to skip); d_accept [1] int64 is incremented by the
 * accepted moves (NULL to skip).  Errors as the calls it is made of.                   */
fn_status fn_vmc_iteration(fn_system_t sys, const fn_train_config* cfg, void* d_params, void* d_walkers,
                           int n_walkers, int64_t iteration, void* d_opt_state, void* d_grad,
                           double* d_log_psi, double* d_e_local, double* d_e_mean, int64_t* d_accept,
                           void* stream);

/* Mulliken partial charges for Algorithm 1 (fn_assign_electrons, fn_init_walkers): the
 * ionic charge initialisation takes them from a Hartree-Fock calculation in the STO-6G
 * basis.  Unrestricted Hartree-Fock in STO-6G (Hehre, Stewart & Pople 1969; standard
 * molecular exponents) for nuclei of H..Ne (integer Z 1..10, at most 20 basis functions:
 * four first-row atoms), n_up + n_down electrons; q_A = Z_A - sum over the functions mu on A
 * of (P S)_mu,mu.  Host computation (no device memory, no stream): h_partial_charges [M]
 * receives the charges (they sum to the ionic charge), h_energy [1] the UHF energy in
 * hartree (NULL to skip).  FN_ERR_ARG for other elements, FN_ERR_UNSUPPORTED above 20
 * functions, FN_ERR_NUMERIC if the iterations do not converge.                         */
fn_status fn_mulliken_charges(const double* h_nuclei, const double* h_charges, int n_nuclei, int n_up,
                              int n_down, double* h_partial_charges, double* h_energy);

/* Failure-path self-test: launches one CTA whose threads wait on a shared-memory
 * mbarrier that nothing arrives at, each wait bounded by wait_us microseconds
 * (1..100000) of %globaltimer and by an iteration cap.  On expiry the kernel sets the
 * timeout bit of the device status word and returns, as the tensor-core kernels do when
 * one of their waits expires; fn_sync then returns FN_ERR_TIMEOUT and clears the bit, and
 * the context stays usable.  It tests error reporting without a fault or a hang.        */
fn_status fn_selftest_expired_wait(fn_system_t sys, int wait_us, void* stream);

/* Kernel timing: while enabled, every kernel the handle launches is bracketed by a
 * CUDA event pair on its stream (adds a few microseconds per launch).  Enabling or
 * disabling clears the counters.  fn_profile_read waits for the recorded events and
 * returns the number of kernel classes; for 0 <= index < that number it writes the
 * class name (static storage), the launch count and the summed device time in ms. */
fn_status fn_profile_enable(fn_system_t sys, int enable);
int fn_profile_read(fn_system_t sys, int index, const char** name, int64_t* launches, double* total_ms);

/* Waits for the stream with a deadline (polling, no blocking sync), then reads
 * and clears the device status word.  FN_ERR_TIMEOUT if the deadline passes
 * (work keeps running) or if a kernel gave up on a bounded wait,
 * FN_ERR_NUMERIC if a kernel flagged a numerical error.                     */
fn_status fn_sync(fn_system_t sys, void* stream, int timeout_ms);

const char* fn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FNVMC_H */
