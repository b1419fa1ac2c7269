// One-electron stream layer on the 5th-generation tensor cores (BF16 operands, FP32
// accumulation in tensor memory), with the forward-Laplacian epilogue fused.
//
// Per CTA: 128 electron rows (one walker-aligned tile) x N_t output columns, looping
// over every tangent slab t (value, 3N gradient slabs, Laplacian):
//   warp 0      TMA producer: X_l[t] tile (128 x 64 bf16) and V_self tile (N_t x 64) per
//               k-block into a 4-stage shared-memory ring (128B swizzle);
//   warp 1      allocates tensor memory; one lane issues tcgen05.mma (M=128, N=N_t, K=16)
//               into a double-buffered accumulator and commits to mbarriers;
//   warps 2..5  epilogue, one TMEM lane (= row) per thread: z = acc + M[t][walker];
//               slab 0: h = tanh z (kept in TMEM), slabs 1..3N: (1 - h^2) z and the running
//               sum of z^2 (kept in TMEM), Laplacian slab: (1 - h^2) z - 2 h (1 - h^2) sum;
//               plus the residual, the BF16 store and the spin means of the output.
// Tensor memory columns: [0, 2 N_t) accumulators, [2 N_t, 3 N_t) h, [3 N_t, 4 N_t) sum z^2.
//
// Every wait is bounded (1 s of %globaltimer); on expiry the CTA records a timeout bit in
// the device status word, the producer waits (bounded) for its copies in flight, tensor
// memory is freed and the CTA returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "fn_device.cuh"
#include "fn_internal.cuh"

namespace fn {
namespace tc {

constexpr int kStages = 4;
constexpr int kBlockK = 64;                     // bf16 elements per 128-byte swizzled row
constexpr int kThreads = 192;
constexpr uint64_t kWaitNs = 1000000000ull;     // 1 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Waits until the phase of the given parity has completed; false after the deadline.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t deadline) {
  const uint32_t addr = smem_u32(bar);
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer() > deadline) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// OR of a predicate over the 128 epilogue threads (named barrier 1).
__device__ __forceinline__ bool epilogue_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, 128, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"(v ? 1u : 0u)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

#define FN_R32(v)                                                                                                 \
  "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),    \
      "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),      \
      "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),     \
      "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
#define FN_W32(v)                                                                                                  \
  "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),   \
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), \
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),  \
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])

// 32 consecutive 32-bit columns of this warp's 32 TMEM lanes (one lane per thread).  The
// load and its completion wait are one asm statement, so the registers are defined only
// once the data has arrived.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : FN_R32(v)
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      FN_W32(v)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

struct TcArgs {
  Shape sh;
  int nkb;               // k-blocks of 64
  int nt;                // output columns per CTA (32, 64 or 128)
  int h1;
  const float* Mterm;    // [T][B][h1]
  const __nv_bfloat16* X; int ldx;    // input (residual source)
  __nv_bfloat16* Y; int ldy;          // output
  int residual;
  float* Hbar_out;       // [T][B][2 h1] or null
  float* act_out;        // [R][h1] or null
  int* status;
  uint32_t tmem_cols;
};

template <bool FULL>
__global__ void __launch_bounds__(kThreads, 1)
    k_layer_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned carve-up
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int nt = a.nt;
  const uint32_t bytesA = 128 * 128, bytesB = (uint32_t)nt * 128;
  unsigned char* sA = base;                                   // kStages x 16 KB
  unsigned char* sB = sA + kStages * bytesA;                  // kStages x nt*128
  float* ys = (float*)(sB + kStages * bytesB);                // [128][33]
  uint64_t* bars = (uint64_t*)(ys + 128 * 33);                // full[S], empty[S], accf[2], acce[2]
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* accf = bars + 2 * kStages;
  uint64_t* acce = accf + 2;
  uint64_t* mma_done = acce + 2;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Shape& sh = a.sh;
  const int tile = blockIdx.x, n0 = blockIdx.y * nt;
  const int T = sh.T, nkb = a.nkb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(accf + b, 1); mbar_init(acce + b, 4); }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint64_t deadline = globaltimer() + kWaitNs * 8;   // whole-CTA budget; each wait checks it

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      for (int t = 0; t < T && ok; ++t) {
        for (int kb = 0; kb < nkb; ++kb, ++issued) {
          const int stage = issued % kStages;
          const uint32_t round = (uint32_t)(issued / kStages);
          if (*abort_flag || !mbar_wait(empty + stage, (round & 1u) ^ 1u, deadline)) { ok = false; break; }
          mbar_expect_tx(full + stage, bytesA + bytesB);
          tma_load_2d(sA + stage * bytesA, &tmA, full + stage, kb * kBlockK, (int)(t * sh.R + (int64_t)tile * 128));
          tma_load_2d(sB + stage * bytesB, &tmB, full + stage, kb * kBlockK, n0);
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.status, kStatusTimeout);
      }
      // drain: every armed stage must have received its bytes before shared memory is released
      const uint64_t dl2 = globaltimer() + kWaitNs;
      for (int q = std::max(0, issued - kStages); q < issued; ++q)
        mbar_wait(full + (q % kStages), (uint32_t)((q / kStages) & 1), dl2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, nt);
      int consumed = 0;
      bool ok = true;
      for (int t = 0; t < T && ok; ++t) {
        const int buf = t & 1;
        const uint32_t use = (uint32_t)(t >> 1);
        if (*abort_flag || !mbar_wait(acce + buf, (use & 1u) ^ 1u, deadline)) { ok = false; break; }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * nt);
        for (int kb = 0; kb < nkb; ++kb, ++consumed) {
          const int stage = consumed % kStages;
          const uint32_t round = (uint32_t)(consumed / kStages);
          if (*abort_flag || !mbar_wait(full + stage, round & 1u, deadline)) { ok = false; break; }
          fence_after();
          const uint64_t da = sdesc(smem_u32(sA + stage * bytesA));
          const uint64_t db = sdesc(smem_u32(sB + stage * bytesB));
#pragma unroll
          for (int k4 = 0; k4 < kBlockK / 16; ++k4)
            mma_bf16(d, da + (uint64_t)(2 * k4), db + (uint64_t)(2 * k4), idesc, (kb | k4) != 0 ? 1u : 0u);
          mma_commit(empty + stage);
        }
        if (ok) mma_commit(accf + buf);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.status, kStatusTimeout);
      }
      // every MMA issued by this thread has completed before tensor memory is released
      mma_commit(mma_done);
      mbar_wait(mma_done, 0u, globaltimer() + kWaitNs);
    }
  } else {
    // epilogue: thread = TMEM lane = row of the tile
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const int64_t row = (int64_t)tile * 128 + r;
    const int wl = r / sh.N;
    const int w = tile * sh.wpt + wl;
    const bool valid = wl < sh.wpt && w < sh.B;
    const int ethread = threadIdx.x - 64;        // 0..127 across the four epilogue warps
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const int64_t xslab = sh.R * a.ldx, yslab = sh.R * a.ldy;
    for (int t = 0; t < T; ++t) {
      const int buf = t & 1;
      const uint32_t use = (uint32_t)(t >> 1);
      const bool ok = !*abort_flag && mbar_wait(accf + buf, use & 1u, deadline);
      if (epilogue_any(!ok)) {
        if (ethread == 0) {
          *abort_flag = 1;
          atomicOr(a.status, kStatusTimeout);
        }
        break;
      }
      fence_after();
      for (int cc = 0; cc < nt / 32; ++cc) {
        const int col0 = n0 + cc * 32;
        uint32_t acc[32], hv[32], sq[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(buf * nt + cc * 32), acc);
        if (FULL && t > 0) {
          tmem_ld32(tmem + lane_base + (uint32_t)(2 * nt + cc * 32), hv);
          tmem_ld32(tmem + lane_base + (uint32_t)(3 * nt + cc * 32), sq);
        }
        const bool live = valid && col0 < a.h1;
        float out[32];
        if (live) {
          const float4* mt = (const float4*)(a.Mterm + ((int64_t)t * sh.B + w) * a.h1 + col0);
          float mv[32];
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const float4 m4 = mt[v];
            mv[4 * v] = m4.x; mv[4 * v + 1] = m4.y; mv[4 * v + 2] = m4.z; mv[4 * v + 3] = m4.w;
          }
          float res[32];
          if (a.residual) {
            const uint4* xr = (const uint4*)(a.X + t * xslab + row * a.ldx + col0);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const uint4 u = xr[v];
              const __nv_bfloat162* p2 = (const __nv_bfloat162*)&u;
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(p2[e]);
                res[8 * v + 2 * e] = f.x;
                res[8 * v + 2 * e + 1] = f.y;
              }
            }
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float z = __uint_as_float(acc[j]) + mv[j];
            float o;
            if (t == 0) {
              const float h = tanhf(z);
              hv[j] = __float_as_uint(h);
              sq[j] = 0u;
              o = h;
            } else {
              const float h = __uint_as_float(hv[j]);
              const float d = 1.0f - h * h;
              if (t < T - 1) {
                o = d * z;
                sq[j] = __float_as_uint(__uint_as_float(sq[j]) + z * z);
              } else {
                o = d * z - 2.0f * h * d * __uint_as_float(sq[j]);
              }
            }
            out[j] = a.residual ? o + res[j] : o;
          }
          uint4* yo = (uint4*)(a.Y + t * yslab + row * a.ldy + col0);
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            uint4 u;
            __nv_bfloat162* p2 = (__nv_bfloat162*)&u;
#pragma unroll
            for (int e = 0; e < 4; ++e) p2[e] = __floats2bfloat162_rn(out[8 * v + 2 * e], out[8 * v + 2 * e + 1]);
            yo[v] = u;
          }
          if (t == 0 && a.act_out) {
            float4* ao = (float4*)(a.act_out + row * a.h1 + col0);
#pragma unroll
            for (int v = 0; v < 8; ++v)
              ao[v] = make_float4(__uint_as_float(hv[4 * v]), __uint_as_float(hv[4 * v + 1]),
                                  __uint_as_float(hv[4 * v + 2]), __uint_as_float(hv[4 * v + 3]));
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) { out[j] = 0.f; hv[j] = 0u; sq[j] = 0u; }
        }
        if (FULL) {
          if (t == 0) {
            tmem_st32(tmem + lane_base + (uint32_t)(2 * nt + cc * 32), hv);
            tmem_st32(tmem + lane_base + (uint32_t)(3 * nt + cc * 32), sq);
          } else if (t < T - 1) {
            tmem_st32(tmem + lane_base + (uint32_t)(3 * nt + cc * 32), sq);
          }
          tmem_wait_st();
        }
        if (a.Hbar_out && col0 < a.h1) {
#pragma unroll
          for (int j = 0; j < 32; ++j) ys[r * 33 + j] = out[j];
          asm volatile("bar.sync 1, 128;" ::: "memory");
          for (int e = ethread; e < sh.wpt * 2 * 32; e += 128) {
            const int wl2 = e / 64, s = (e / 32) & 1, j = e & 31;
            const int w2 = tile * sh.wpt + wl2;
            if (w2 >= sh.B) continue;
            const int lo = s ? sh.n_up : 0, hi = s ? sh.N : sh.n_up;
            float sum = 0.f;
            for (int i = lo; i < hi; ++i) sum += ys[(wl2 * sh.N + i) * 33 + j];
            a.Hbar_out[((int64_t)t * sh.B + w2) * 2 * a.h1 + s * a.h1 + col0 + j] = hi > lo ? sum / (float)(hi - lo) : 0.f;
          }
          asm volatile("bar.sync 1, 128;" ::: "memory");
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce + buf);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

}  // namespace tc

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D bf16 tensor map: inner dimension `cols` (elements), `rows` rows of stride ld elements,
// box 64 x box_rows, 128-byte swizzle, out-of-bounds elements read as zero.
static bool make_map(CUtensorMap* m, const void* base, int64_t cols, int64_t rows, int64_t ld, int box_rows) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)tc::kBlockK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_available() { return encode_fn() != nullptr; }

int tc_columns(int h1) {
  if (h1 % 128 == 0) return 128;
  if (h1 % 64 == 0) return 64;
  return 32;
}

size_t tc_smem_bytes(int nt) {
  return 1024 + tc::kStages * (128 * 128 + (size_t)nt * 128) + 128 * 33 * sizeof(float) + 8 * (2 * tc::kStages + 5) + 16;
}

// Launches the tensor-core layer; returns false (nothing launched) if a tensor map could not be built.
bool launch_layer_tc(const Shape& sh, const void* X, int ldx, int k_self, const void* Vs16, const float* Mterm, void* Y,
                     int ldy, int residual, float* Hbar_out, float* act_out, int h1, int* status, cudaStream_t st) {
  const int nt = tc_columns(h1);
  CUtensorMap ta, tb;
  if (!make_map(&ta, X, k_self, (int64_t)sh.T * sh.R, ldx, 128)) return false;
  if (!make_map(&tb, Vs16, k_self, h1, ldx, nt)) return false;
  tc::TcArgs a{};
  a.sh = sh;
  a.nkb = (k_self + tc::kBlockK - 1) / tc::kBlockK;
  a.nt = nt;
  a.h1 = h1;
  a.Mterm = Mterm;
  a.X = (const __nv_bfloat16*)X;
  a.ldx = ldx;
  a.Y = (__nv_bfloat16*)Y;
  a.ldy = ldy;
  a.residual = residual;
  a.Hbar_out = Hbar_out;
  a.act_out = act_out;
  a.status = status;
  const bool full = sh.T > 1;
  a.tmem_cols = (uint32_t)(full ? 4 * nt : std::max(32, 2 * nt));
  const size_t smem = tc_smem_bytes(nt);
  dim3 grid(sh.tiles, h1 / nt);
  if (full) {
    cudaFuncSetAttribute(tc::k_layer_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc::k_layer_tc<true><<<grid, tc::kThreads, smem, st>>>(ta, tb, a);
  } else {
    cudaFuncSetAttribute(tc::k_layer_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc::k_layer_tc<false><<<grid, tc::kThreads, smem, st>>>(ta, tb, a);
  }
  return true;
}

}  // namespace fn
