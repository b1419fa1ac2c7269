// log|psi| without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: applications whose device memory
// is owned by a pool or a framework allocator that must see every byte, and processes
// under a hard memory budget that was fixed before the library was loaded.  For them this entry point runs
// the value-only forward pass (the same kernels as fn_log_psi) with all of its scratch
// in one file-scope device array, so the call itself never allocates.  The caller still
// provides parameters, walkers and outputs.
//
// The array is kNoAllocScratchBytes (64 MiB) and exists on every device that loads the
// library, for the life of the process.  Its device address is looked up once per device
// (cudaGetSymbolAddress with that device current) on the first call made on that device,
// so that first call should come before any stream capture.
// All calls share the array, so two calls whose work overlaps on the GPU race.  A call
// sees whatever the previous one left there; every buffer of the array is written before
// it is read (the parameter preparation writes the zero padding of the BF16 weight
// matrices itself), so no leftover value reaches a result.  Errors found on the device
// (a non-finite or singular result, a bounded wait that expired) go to the handle's own
// status word, which lives outside the array, and fn_sync reports them as it does for
// fn_log_psi.
#include <mutex>

#include "fn_internal.cuh"

namespace fn {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
static void* g_scratch_addr[kNoAllocMaxDevices] = {};
static std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (looked up once per device).
static fn_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("device index beyond the no-allocation table");
    return FN_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress of the no-allocation scratch");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return FN_OK;
}

// Carves the value-pass buffers (T = 1) out of `base`; returns the bytes needed.
template <class Mode>
static size_t value_pass_layout(const fn_system* s, int B, unsigned char* base, Workspace* ws) {
  using Act = typename Mode::Act; using Cmp = typename Mode::Cmp;
  const Shape sh = make_shape(s, B, 1);
  const int L = s->cfg.n_layers, h1 = s->cfg.h1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (size_t)round_up((int64_t)(off + bytes), 256);
    return o;
  };
  size_t o_X[kMaxLayers], o_Hbar[kMaxLayers];
  const int Tx = Mode::kMode == FN_BF16_MIXED ? 2 : 1;       // value slab and, in BF16 storage, its low part
  for (int l = 0; l < L; ++l) {
    o_X[l] = take((size_t)Tx * sh.R * s->layer[l].ldx * sizeof(Act));
    o_Hbar[l] = take((size_t)Tx * B * 2 * s->layer[l].d_h * sizeof(Act));
  }
  const size_t o_HL = take((size_t)Tx * sh.R * h1 * sizeof(Act));
  const size_t o_M = take((size_t)B * h1 * sizeof(Cmp));
  const size_t o_Phi = take((size_t)B * phi_walker_stride(s, 1) * sizeof(typename Mode::PhiT));
  const size_t o_prep = take((size_t)s->prep.total * sizeof(Cmp));
  const size_t o_prep16 = take((size_t)s->prep.total16 * sizeof(__nv_bfloat16));
  const size_t o_envv = take(Mode::kMode == FN_BF16_MIXED ? (size_t)sh.R * s->cfg.n_dets * s->N * sizeof(float) : 0);
  if (base && ws) {
    *ws = Workspace();
    for (int l = 0; l < L; ++l) {
      ws->X[l] = base + o_X[l];
      ws->Hbar[l] = base + o_Hbar[l];
    }
    ws->HL = base + o_HL;
    ws->Mterm = base + o_M;
    ws->Phi = base + o_Phi;
    ws->prep = base + o_prep;
    ws->prep16 = base + o_prep16;
    ws->status = s->d_status;            // kernels report into the handle's word, read by fn_sync
    ws->envv = (float*)(base + o_envv);
    ws->base = base;
    ws->bytes = off;
    ws->cap_B = B;
  }
  return off;
}

template <class Mode>
static fn_status log_psi_noalloc(fn_system* s, const void* params, const void* walkers, int B, double* log_psi,
                                 int8_t* sign, cudaStream_t st) {
  const size_t need = value_pass_layout<Mode>(s, B, nullptr, nullptr);
  if (need > kNoAllocScratchBytes) {
    int fit = B;
    while (fit > 1 && value_pass_layout<Mode>(s, fit, nullptr, nullptr) > kNoAllocScratchBytes) fit = fit * 3 / 4;
    set_error("fn_log_psi_noalloc: " + std::to_string(B) + " walkers need " + std::to_string(need >> 20) +
              " MiB of scratch; the static scratch holds 64 MiB (about " + std::to_string(fit) +
              " walkers of this system)");
    return FN_ERR_ARG;
  }
  s->last_stream = (void*)st;          // the handle's small buffers are in use on this stream
  s->stream_seen = true;
  void* base = nullptr;
  fn_status r = scratch_address(&base);
  if (r != FN_OK) return r;
  Workspace arena;
  value_pass_layout<Mode>(s, B, (unsigned char*)base, &arena);
  // run the value pass of fn_log_psi against the arena, leaving the handle's own workspace untouched
  const Workspace saved = s->ws;
  Profiler* saved_prof = s->prof;
  s->ws = arena;
  s->prof = nullptr;
  const Shape sh = make_shape(s, B, 1);
  launch_prep_params<Mode>(s, params, st);
  launch_forward<Mode>(s, walkers, sh, false, st);
  launch_det_energy<Mode>(s, walkers, sh, nullptr, log_psi, sign, false, st);
  s->ws = saved;
  s->prof = saved_prof;
  if (s->host_error != FN_OK) {
    const fn_status he = s->host_error;
    s->host_error = FN_OK;
    set_error("fn_log_psi_noalloc: a TMA tensor map could not be encoded");
    return he;
  }
  return cuda_status(cudaGetLastError(), "fn_log_psi_noalloc");
}

}  // namespace fn

using namespace fn;

extern "C" fn_status fn_log_psi_noalloc(fn_system_t s, const void* d_params, const void* d_walkers, int n_walkers,
                                        double* d_log_psi, int8_t* d_sign, void* stream) {
  if (!s || !d_params || !d_walkers || n_walkers < 1 || !d_log_psi) {
    set_error("invalid argument");
    return FN_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  switch (s->cfg.precision) {
    case FN_FP64: return log_psi_noalloc<ModeF64>(s, d_params, d_walkers, n_walkers, d_log_psi, d_sign, st);
    case FN_FP32: return log_psi_noalloc<ModeF32>(s, d_params, d_walkers, n_walkers, d_log_psi, d_sign, st);
    default: return log_psi_noalloc<ModeBF16>(s, d_params, d_walkers, n_walkers, d_log_psi, d_sign, st);
  }
}
