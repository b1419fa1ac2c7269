// One-electron stream layer on the 5th-generation tensor cores (BF16 operands, FP32
// accumulation in tensor memory), with the forward-Laplacian epilogue fused.
//
// Per CTA: 128 electron rows (one walker-aligned tile) x N_t output columns, looping
// over every tangent slab t (value, 3N gradient slabs, Laplacian):
//   warp 0      TMA producer: X_l[t] tile (128 x 64 bf16) and the V_self tiles (N_t x 64,
//               high and low BF16 parts) per k-block into a 3-stage shared-memory
//               ring (128B swizzle);
//   warp 1      allocates tensor memory; one lane issues tcgen05.mma (M=128, N=N_t, K=16)
//               into a double-buffered accumulator and commits to mbarriers;
//   warps 2..9  epilogue, one TMEM lane (= row) per thread, two warps per lane quarter
//               (column halves): z = acc + M[t][walker] (M[t] staged in shared memory by
//               cp.async one slab ahead); slab 0: h = tanh z (kept in TMEM), slabs 1..3N:
//               (1 - h^2) z and the running sum of z^2 (kept in TMEM), Laplacian slab:
//               (1 - h^2) z - 2 h (1 - h^2) sum; plus the residual (loaded before the
//               accumulator wait) and the BF16 store.
// Tensor memory columns: [0, 2 N_t) accumulators, [2 N_t, 3 N_t) h, [3 N_t, 4 N_t) sum z^2.
//
// Every wait is bounded (1 s of %globaltimer); on expiry the CTA records a timeout bit in
// the device status word, the producer waits (bounded) for its copies in flight, tensor
// memory is freed and the CTA returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "fn_device.cuh"
#include "fn_internal.cuh"

namespace fn {
namespace tc {

constexpr int kStages = 4;                      // TMA ring depth (the layer kernel uses 3, see stages_for)
constexpr int kBlockK = 64;                     // bf16 elements per 128-byte swizzled row
constexpr int kEpiWarps = 8;                   // two warps per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;
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

// OR of a predicate over the epilogue threads (named barrier 1).
__device__ __forceinline__ bool epilogue_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, 256, q;\n\t"
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

// Three 16-column loads (accumulator, h, sum of squares) under one completion wait.
__device__ __forceinline__ void tmem_ld16x3(uint32_t ta, uint32_t tb, uint32_t tc_, uint32_t (&a)[16],
                                            uint32_t (&b)[16], uint32_t (&c)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%48];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
      "%29, %30, %31}, [%49];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, "
      "%45, %46, %47}, [%50];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]),
        "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]), "=r"(b[0]),
        "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]), "=r"(b[8]), "=r"(b[9]),
        "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15]), "=r"(c[0]), "=r"(c[1]),
        "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7]), "=r"(c[8]), "=r"(c[9]), "=r"(c[10]),
        "=r"(c[11]), "=r"(c[12]), "=r"(c[13]), "=r"(c[14]), "=r"(c[15])
      : "r"(ta), "r"(tb), "r"(tc_)
      : "memory");
}

// 16-byte asynchronous global -> shared copy (no register staging), grouped per thread.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
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

enum { kEpiLayer = 0, kEpiPlain = 1, kEpiOrbital = 2 };

// Ring depth per kernel: the layer kernel gives one stage's worth of shared memory to the
// double-buffered residual tiles.
__host__ __device__ constexpr int stages_for(int epi) { return epi == kEpiLayer ? 3 : kStages; }
constexpr uint32_t kResBox = 128 * 128;          // one residual box: 128 rows x 64 bf16 (128B swizzle)

struct TcArgs {
  Shape sh;
  int tiles;             // row tiles of 128; CTA y index strides over them (persistent)
  int nkb;               // k-blocks of 64
  int nt;                // output columns per CTA (32, 64 or 128)
  int h1;
  int* status;
  uint32_t tmem_cols;
  // layer epilogue
  const float* Mterm;    // [T][B][h1]
  const __nv_bfloat16* X; int ldx;    // input (residual source)
  __nv_bfloat16* Y; int ldy;          // output
  int residual;
  float* act_out;        // [R][h1] or null
  int mt_stage;          // 1: the epilogue stages M[t] rows of the tile in shared memory
  // plain epilogue: C[row][col] = acc + bias[col] (rows < bias_rows), or C += acc (atomic);
  // the K range may be split over `ksplit` CTAs per output tile (requires atomic)
  int rows; float* C; int ldc; const float* bias; int bias_rows;
  int ksplit, atomic;
  // hi/lo pairs of A (BF16 storage): the low part of slab t sits at A row alo_row + t R +
  // tile row (0: no low parts).  Slab 0 is paired in every column; a tangent slab only
  // from k-block kb_lo_t on (the pair-mean columns of a layer input).  The low part is
  // multiplied by the high part of B in extra k-blocks of the item.
  int64_t alo_row;
  int kb_lo_t;
  // orbital epilogue
  const float* wbias[2];              // orbital bias g, [K n_s]
  const float* pi[2]; const float* sig[2];
  const float* walkers;               // [B][N][3]
  const double* nuclei;
  int K, aniso, ctiles_up;            // column tiles of the up block
  float* Phi; int64_t PW;             // [B][PW] (float)
  float* orbP;                        // [R][4][K N]: value projection and the row's own-coordinate ones
  const float* envv;                  // [R][K N]: envelope values (k_envelope_values)
  // split weights: columns [0, k) hold bf16(W), columns [bsplit, bsplit + k) hold
  // bf16(W - bf16(W)); every k-block is multiplied by both (0 = no split)
  int bsplit;
  int stages;            // A ring depth of the resident-weight layer kernel
};


// Packed two-lane FP32 arithmetic (one instruction for two values) for the epilogue.
__device__ __forceinline__ uint64_t pack_f2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack_f2(uint64_t v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t add_f2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub_f2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t mul_f2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t fma_f2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// ---- epilogue: stream layer ------------------------------------------------------------
// One 32-column chunk, in two 16-column halves (register budget).  `res` holds the
// chunk's residual (8 bf16 per uint4), loaded before the accumulator wait; `mrow` is the
// walker's mean-field row for this tile's columns (shared memory or global).  The spin
// means of the output, the next layer's mean-field input, are taken by a separate pass.
template <bool FULL>
__device__ __forceinline__ void epi_layer(const TcArgs& a, int t, int cc, bool has_chunk, int r, uint32_t tmem,
                                          uint32_t lane_base, int buf, int n0, int tile, const unsigned char* rs,
                                          const float* mrow) {
  const Shape& sh = a.sh;
  const int nt = a.nt, T = sh.T;
  const int64_t row = (int64_t)tile * 128 + r;
  const int wl = r / sh.N;
  const int w = tile * sh.wpt + wl;
  const bool valid = wl < sh.wpt && w < sh.B;
  const int64_t yslab = sh.R * a.ldy;
  const int col0 = n0 + cc * 32;
  const bool live = has_chunk && valid && col0 < a.h1;
  const int kind = t == 0 ? 0 : (t < T - 1 ? 1 : 2);           // value, gradient, Laplacian slab
  if (has_chunk) {
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int cb = cc * 32 + hh * 16;
      uint32_t acc[16], hv[16], sq[16];
      if (FULL && t > 0) {
        tmem_ld16x3(tmem + lane_base + (uint32_t)(buf * nt + cb), tmem + lane_base + (uint32_t)(2 * nt + cb),
                    tmem + lane_base + (uint32_t)(3 * nt + cb), acc, hv, sq);
      } else {
        tmem_ld16(tmem + lane_base + (uint32_t)(buf * nt + cb), acc);
      }
      float out[16];
      if (live) {
        const float4* mt = (const float4*)(mrow + cc * 32 + hh * 16);
        // residual of this piece from the shared-memory tile (TMA, 128B swizzle: 16-byte chunk j
        // of row r sits at chunk j ^ (r % 8) of the row's 128 bytes); zero without a residual
        float rv[16];
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const int cl = cc * 32 + hh * 16 + 8 * v;
          uint4 u = make_uint4(0u, 0u, 0u, 0u);
          if (a.residual) u = *(const uint4*)(rs + (cl >> 6) * kResBox + r * 128 + ((((cl & 63) >> 3) ^ (r & 7)) << 4));
          const __nv_bfloat162* p2 = (const __nv_bfloat162*)&u;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(p2[e]);
            rv[8 * v + 2 * e] = f.x;
            rv[8 * v + 2 * e + 1] = f.y;
          }
        }
        if (kind == 0) {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const float4 m4 = mt[v];
            const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int j = 4 * v + e;
              const float h = tanh_fast(__uint_as_float(acc[j]) + mv[e]);
              hv[j] = __float_as_uint(h);
              sq[j] = 0u;
              out[j] = h + rv[j];
            }
          }
          if (a.residual && a.alo_row > 0) {
            // the value slab's residual is a pair: add its low part (slab T of X)
            const uint4* xl = (const uint4*)(a.X + (int64_t)T * sh.R * a.ldx + row * a.ldx + col0 + hh * 16);
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              const uint4 u = xl[v];
              const __nv_bfloat162* p2 = (const __nv_bfloat162*)&u;
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(p2[e]);
                out[8 * v + 2 * e] += f.x;
                out[8 * v + 2 * e + 1] += f.y;
              }
            }
          }
        } else {
          // tangent and Laplacian slabs on packed two-lane FP32 operations:
          //   z = acc + M,  -(1 - h^2) = h h - 1,  out = residual - (-(1 - h^2)) w,
          //   w = z (tangent; and sum z^2 += z z) or z - 2 h sum z^2 (Laplacian)
          const uint64_t m1 = pack_f2(-1.f, -1.f), m2 = pack_f2(-2.f, -2.f);
#pragma unroll
          for (int jp = 0; jp < 8; ++jp) {
            const float4 m4 = mt[jp >> 1];
            const uint64_t z2 = add_f2(pack_f2(__uint_as_float(acc[2 * jp]), __uint_as_float(acc[2 * jp + 1])),
                                       (jp & 1) ? pack_f2(m4.z, m4.w) : pack_f2(m4.x, m4.y));
            const uint64_t h2 = pack_f2(__uint_as_float(hv[2 * jp]), __uint_as_float(hv[2 * jp + 1]));
            const uint64_t s2 = pack_f2(__uint_as_float(sq[2 * jp]), __uint_as_float(sq[2 * jp + 1]));
            const uint64_t nd2 = fma_f2(h2, h2, m1);
            uint64_t w2;
            if (kind == 1) {
              w2 = z2;
              float s0, s1;
              unpack_f2(fma_f2(z2, z2, s2), s0, s1);
              sq[2 * jp] = __float_as_uint(s0);
              sq[2 * jp + 1] = __float_as_uint(s1);
            } else {
              w2 = fma_f2(mul_f2(h2, s2), m2, z2);
            }
            unpack_f2(sub_f2(pack_f2(rv[2 * jp], rv[2 * jp + 1]), mul_f2(nd2, w2)), out[2 * jp], out[2 * jp + 1]);
          }
        }
        uint4* yo = (uint4*)(a.Y + t * yslab + row * a.ldy + col0 + hh * 16);
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          uint4 u;
          __nv_bfloat162* p2 = (__nv_bfloat162*)&u;
#pragma unroll
          for (int e = 0; e < 4; ++e) p2[e] = __floats2bfloat162_rn(out[8 * v + 2 * e], out[8 * v + 2 * e + 1]);
          yo[v] = u;
        }
        if (kind == 0 && a.alo_row > 0) {
          // and the output's value slab is stored as a pair (slab T of Y)
          uint4* yl = (uint4*)(a.Y + (int64_t)T * yslab + row * a.ldy + col0 + hh * 16);
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            uint4 u;
            __nv_bfloat162* p2 = (__nv_bfloat162*)&u;
#pragma unroll
            for (int e = 0; e < 4; ++e)
              p2[e] = __floats2bfloat162_rn(bf16_rem(out[8 * v + 2 * e]), bf16_rem(out[8 * v + 2 * e + 1]));
            yl[v] = u;
          }
        }
        if (kind == 0 && a.act_out) {
          float4* ao = (float4*)(a.act_out + row * a.h1 + col0 + hh * 16);
#pragma unroll
          for (int v = 0; v < 4; ++v)
            ao[v] = make_float4(__uint_as_float(hv[4 * v]), __uint_as_float(hv[4 * v + 1]),
                                __uint_as_float(hv[4 * v + 2]), __uint_as_float(hv[4 * v + 3]));
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) { out[j] = 0.f; hv[j] = 0u; sq[j] = 0u; }
      }
      if (FULL) {
        if (kind == 0) {
          tmem_st16(tmem + lane_base + (uint32_t)(2 * nt + cb), hv);
          tmem_st16(tmem + lane_base + (uint32_t)(3 * nt + cb), sq);
        } else if (kind == 1) {
          tmem_st16(tmem + lane_base + (uint32_t)(3 * nt + cb), sq);
        }
      }
    }
    if (FULL) tmem_wait_st();
  }
}

// Issues the copies of M[t] (the tile's walkers, this CTA's nt columns) into a staging
// buffer of rows nt + 4 floats; one commit group per call and thread.
__device__ __forceinline__ void stage_mterm(const TcArgs& a, int t, int tile, int n0, float* dst, int ethread) {
  const Shape& sh = a.sh;
  const int q4 = a.nt >> 2;                                   // 16-byte pieces per walker row
  const int w0 = tile * sh.wpt;
  const int nw = min(sh.wpt, sh.B - w0);
  for (int e = ethread; e < nw * q4; e += 32 * kEpiWarps) {
    const int wl = e / q4, c4 = e - wl * q4;
    cp_async16(dst + wl * (a.nt + 4) + 4 * c4, a.Mterm + ((int64_t)t * sh.B + w0 + wl) * a.h1 + n0 + 4 * c4);
  }
  cp_async_commit();
}

// First k-block whose low part an item multiplies (kb1: none).
template <int EPI>
__device__ __forceinline__ int lo_first(const TcArgs& a, int t, int kb0, int kb1) {
  if (a.alo_row <= 0) return kb1;
  if (EPI == kEpiPlain) return kb0;
  return t == 0 ? kb0 : max(kb0, min(kb1, a.kb_lo_t));
}

// Work item -> (row tile, k-block range): split-K GEMMs give every (tile, split) pair its
// own item; the other kernels cover all k-blocks of a tile.
template <int EPI>
__device__ __forceinline__ void item_range(const TcArgs& a, int pidx, int nkb, int& tile, int& kb0, int& kb1) {
  tile = pidx; kb0 = 0; kb1 = nkb;
  if (EPI == kEpiPlain && a.ksplit > 1) {
    tile = pidx / a.ksplit;
    const int sp = pidx - tile * a.ksplit;
    kb0 = (int)((int64_t)sp * nkb / a.ksplit);
    kb1 = (int)((int64_t)(sp + 1) * nkb / a.ksplit);
  }
}

// ---- epilogue: plain GEMM with bias ----------------------------------------------------
__device__ __forceinline__ void epi_plain(const TcArgs& a, int cc, int r, uint32_t tmem, uint32_t lane_base, int buf,
                                          int n0, int tile) {
  const int64_t row = (int64_t)tile * 128 + r;
  const int col0 = n0 + cc * 32;
  uint32_t acc[32];
  tmem_ld32(tmem + lane_base + (uint32_t)(buf * a.nt + cc * 32), acc);
  if (row >= a.rows || col0 >= a.h1) return;
  float* co = a.C + row * a.ldc + col0;
  if (a.atomic) {
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (col0 + q < a.h1) atomicAdd(co + q, __uint_as_float(acc[q]));
    return;
  }
  const bool with_bias = a.bias && row < a.bias_rows;
  if (col0 + 32 <= a.h1 && (a.ldc & 3) == 0) {
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      float o[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) o[e] = __uint_as_float(acc[4 * v + e]) + (with_bias ? a.bias[col0 + 4 * v + e] : 0.f);
      ((float4*)co)[v] = make_float4(o[0], o[1], o[2], o[3]);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (col0 + q < a.h1) co[q] = __uint_as_float(acc[q]) + (with_bias ? a.bias[col0 + q] : 0.f);
  }
}

// ---- epilogue: orbitals x envelope, common product term ------------------------------------
// phi_t = P_t env for every slab (P_0 includes the orbital bias).  The envelope-derivative
// terms (own-coordinate slabs and the Laplacian) are added by k_orbital_fixup from the value
// projection P_0 and the own-coordinate projections, stored here with predicated stores.
// TMEM columns: [0, 2 nt) accumulators, [2 nt, 3 nt) envelope value.
template <bool FULL>
__device__ __forceinline__ void epi_orbital(const TcArgs& a, int t, int cc, int r, uint32_t tmem, uint32_t lane_base,
                                            int buf, int spin, int ko0, int tile) {
  const Shape& sh = a.sh;
  const int nt = a.nt, T = sh.T;
  const int wl = r / sh.N, j = r % sh.N;
  const int w = tile * sh.wpt + wl;
  const int n_s = spin ? sh.n_dn : sh.n_up;
  const int n_ko = a.K * n_s;
  const bool valid = wl < sh.wpt && w < sh.B && (j < sh.n_up ? 0 : 1) == spin;
  const int jj = j - (spin ? sh.n_up : 0);
  const int colb = cc * 32;
  uint32_t acc[32], ev[32];
  tmem_ld32(tmem + lane_base + (uint32_t)(buf * nt + colb), acc);
  if (t > 0) tmem_ld32(tmem + lane_base + (uint32_t)(2 * nt + colb), ev);
  const int own_c = (t >= 1 && t <= 3 * sh.N && (t - 1) / 3 == j) ? (t - 1) % 3 : -1;
  const int64_t row = (int64_t)tile * 128 + r;
  const int ldp = a.K * sh.N;
  float* orbp = a.orbP + row * 4 * ldp + (spin ? a.K * sh.n_up : 0);
  const int64_t nn = (int64_t)n_s * n_s;
  float* Phi = a.Phi + (int64_t)w * a.PW + (spin ? (int64_t)a.K * T * sh.n_up * sh.n_up : 0) + t * nn + jj;
  const float* envrow = a.envv + row * ldp + (spin ? a.K * sh.n_up : 0);
  int k = (ko0 + colb) / (n_s ? n_s : 1), i = (ko0 + colb) - k * n_s;
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    const int ko = ko0 + colb + q;
    if (valid && ko < n_ko) {
      float P = __uint_as_float(acc[q]);
      float e;
      if (t == 0) {
        P += a.wbias[spin][ko];
        e = envrow[ko];
        ev[q] = __float_as_uint(e);
        if (FULL) orbp[ko] = P;
      } else {
        e = __uint_as_float(ev[q]);
        if (own_c >= 0) orbp[(1 + own_c) * ldp + ko] = P;
      }
      Phi[(int64_t)k * T * nn + i * n_s] = P * e;
    } else if (t == 0) {
      ev[q] = 0u;
    }
    if (++i == n_s) { i = 0; ++k; }
  }
  if (t == 0 && FULL) {
    tmem_st32(tmem + lane_base + (uint32_t)(2 * nt + colb), ev);
    tmem_wait_st();
  }
}

template <int EPI, bool FULL>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int nt = a.nt;
  const int nbparts = a.bsplit ? 2 : 1;                       // B_hi (and B_lo) per stage
  const uint32_t bytesA = 128 * 128, bytesB = (uint32_t)nt * 128;
  constexpr int NS = stages_for(EPI);
  const bool rstage = EPI == kEpiLayer && a.residual;         // residual tiles staged by TMA
  const int nbox = (nt + 63) / 64;
  unsigned char* sA = base;                                   // NS x 16 KB
  unsigned char* sB = sA + NS * bytesA;                       // NS x nbparts x nt*128
  unsigned char* sR = sB + NS * nbparts * bytesB;             // [2][nbox] residual boxes (layer)
  float* mts = (float*)(sR + (rstage ? 2 * nbox * kResBox : 0));   // [2][wpt][nt + 4] M[t] staging (layer)
  const size_t mt_floats = (EPI == kEpiLayer && a.mt_stage) ? (size_t)2 * a.sh.wpt * (nt + 4) : 0;
  uint64_t* bars = (uint64_t*)(mts + mt_floats);
  uint64_t* full = bars;
  uint64_t* empty = bars + NS;
  uint64_t* accf = bars + 2 * NS;
  uint64_t* acce = accf + 2;
  uint64_t* mma_done = acce + 2;
  uint64_t* resf = mma_done + 1;
  uint64_t* rese = resf + 2;
  uint32_t* tmem_slot = (uint32_t*)(rese + 2);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Shape& sh = a.sh;
  // blockIdx.x runs over the column tiles (fastest), so the CTAs that share an A tile run together;
  // blockIdx.y strides over the row tiles (persistent CTAs, one per SM)
  const int ctile = blockIdx.x;
  const int my_tiles = a.tiles > (int)blockIdx.y ? (a.tiles - 1 - (int)blockIdx.y) / (int)gridDim.y + 1 : 0;
  // column tile: for orbitals it selects (spin, tile within the spin block)
  int spin = 0, ko0 = 0, brow0 = ctile * nt;
  if (EPI == kEpiOrbital) {
    spin = ctile >= a.ctiles_up ? 1 : 0;
    ko0 = (spin ? ctile - a.ctiles_up : ctile) * nt;
    brow0 = (spin ? a.K * sh.n_up : 0) + ko0;
  }
  const int T = EPI == kEpiPlain ? 1 : sh.T;
  const int nkb = a.nkb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf + b, 1); mbar_init(acce + b, kEpiWarps);
      mbar_init(resf + b, 1); mbar_init(rese + b, kEpiWarps);
    }
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
  const uint64_t deadline = globaltimer() + kWaitNs * 8 * (uint64_t)(my_tiles > 0 ? my_tiles : 1);

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0, res_issued = 0;
      bool ok = true;
      for (int item = 0; item < my_tiles * T && ok; ++item) {
        const int pidx = (int)blockIdx.y + (item / T) * (int)gridDim.y, t = item % T;
        int tile, kb0, kb1;
        item_range<EPI>(a, pidx, nkb, tile, kb0, kb1);
        const int arow = EPI == kEpiPlain ? tile * 128 : (int)(t * sh.R + (int64_t)tile * 128);
        const int nk = kb1 - kb0, lf = lo_first<EPI>(a, t, kb0, kb1);
        const int n_k = nk + (kb1 - lf);
        const int lo_row = (int)(a.alo_row + (int64_t)t * sh.R + (int64_t)tile * 128);
        if (rstage) {
          // this item's residual tile (the layer input's first h1 columns of these rows)
          const int rb = item & 1;
          if (*abort_flag || !mbar_wait(rese + rb, ((uint32_t)(item >> 1) & 1u) ^ 1u, deadline)) { ok = false; break; }
          mbar_expect_tx(resf + rb, (uint32_t)nbox * kResBox);
          for (int bx = 0; bx < nbox; ++bx)
            tma_load_2d(sR + (rb * nbox + bx) * kResBox, &tmA, resf + rb, ctile * nt + bx * 64, arow);
          ++res_issued;
        }
        for (int kk = 0; kk < n_k; ++kk, ++issued) {
          const bool lo = kk >= nk;
          const int kb = lo ? lf + (kk - nk) : kb0 + kk;
          const int parts = lo ? 1 : nbparts;
          const int stage = issued % NS;
          const uint32_t round = (uint32_t)(issued / NS);
          if (*abort_flag || !mbar_wait(empty + stage, (round & 1u) ^ 1u, deadline)) { ok = false; break; }
          mbar_expect_tx(full + stage, bytesA + parts * bytesB);
          tma_load_2d(sA + stage * bytesA, &tmA, full + stage, kb * kBlockK, lo ? lo_row : arow);
          for (int part = 0; part < parts; ++part)
            tma_load_2d(sB + (stage * nbparts + part) * bytesB, &tmB, full + stage, part * a.bsplit + kb * kBlockK,
                        brow0);
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.status, kStatusTimeout);
      }
      const uint64_t dl2 = globaltimer() + kWaitNs;
      for (int q = issued > NS ? issued - NS : 0; q < issued; ++q)
        mbar_wait(full + (q % NS), (uint32_t)((q / NS) & 1), dl2);
      for (int q = res_issued > 2 ? res_issued - 2 : 0; q < res_issued; ++q)
        mbar_wait(resf + (q & 1), (uint32_t)((q >> 1) & 1), dl2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, nt);
      int consumed = 0;
      bool ok = true;
      for (int item = 0; item < my_tiles * T && ok; ++item) {
        const int buf = item & 1;
        const uint32_t use = (uint32_t)(item >> 1);
        if (*abort_flag || !mbar_wait(acce + buf, (use & 1u) ^ 1u, deadline)) { ok = false; break; }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * nt);
        int tile, kb0, kb1;
        item_range<EPI>(a, (int)blockIdx.y + (item / T) * (int)gridDim.y, nkb, tile, kb0, kb1);
        (void)tile;
        const int t = item % T;
        const int nk = kb1 - kb0;
        const int n_k = nk + (kb1 - lo_first<EPI>(a, t, kb0, kb1));
        for (int kk = 0; kk < n_k; ++kk, ++consumed) {
          const int parts = kk >= nk ? 1 : nbparts;
          const int stage = consumed % NS;
          const uint32_t round = (uint32_t)(consumed / NS);
          if (*abort_flag || !mbar_wait(full + stage, round & 1u, deadline)) { ok = false; break; }
          fence_after();
          const uint64_t da = sdesc(smem_u32(sA + stage * bytesA));
          for (int part = 0; part < parts; ++part) {
            const uint64_t db = sdesc(smem_u32(sB + (stage * nbparts + part) * bytesB));
#pragma unroll
            for (int k4 = 0; k4 < kBlockK / 16; ++k4)
              mma_bf16(d, da + (uint64_t)(2 * k4), db + (uint64_t)(2 * k4), idesc,
                       (kk != 0 || k4 != 0 || part != 0) ? 1u : 0u);
          }
          mma_commit(empty + stage);
        }
        if (ok) mma_commit(accf + buf);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.status, kStatusTimeout);
      }
      mma_commit(mma_done);
      mbar_wait(mma_done, 0u, globaltimer() + kWaitNs);
    }
  } else {
    const int q = warp & 3;                       // TMEM lane quarter this warp may access
    const int r = q * 32 + lane;
    const int ethread = threadIdx.x - 64;         // 0..255
    const int ehalf = (warp - 2) >> 2;            // column half: chunks cc with cc % 2 == ehalf
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const int nchunks = nt / 32;
    const int n_items = my_tiles * T;
    if (EPI == kEpiLayer && a.mt_stage && n_items > 0) stage_mterm(a, 0, (int)blockIdx.y, ctile * nt, mts, ethread);
    for (int item = 0; item < n_items; ++item) {
      const int t = item % T;
      int tile, kb0_, kb1_;
      item_range<EPI>(a, (int)blockIdx.y + (item / T) * (int)gridDim.y, a.nkb, tile, kb0_, kb1_);
      const int buf = item & 1;
      const uint32_t use = (uint32_t)(item >> 1);
      if (EPI == kEpiLayer && a.mt_stage) cp_async_wait_all();
      bool ok = !*abort_flag && mbar_wait(accf + buf, use & 1u, deadline);
      if (rstage) ok = ok && mbar_wait(resf + buf, use & 1u, deadline);
      // (the barrier also publishes every thread's staged M[t] copies)
      if (epilogue_any(!ok)) {
        if (ethread == 0) {
          *abort_flag = 1;
          atomicOr(a.status, kStatusTimeout);
        }
        break;
      }
      fence_after();
      const float* mrow = nullptr;
      if (EPI == kEpiLayer) {
        if (a.mt_stage) {
          // prefetch the next slab's M[t] into the other buffer (its readers passed the barrier)
          if (item + 1 < n_items) {
            const int tile1 = (int)blockIdx.y + ((item + 1) / T) * (int)gridDim.y, t1 = (item + 1) % T;
            stage_mterm(a, t1, tile1, ctile * nt, mts + ((item + 1) & 1) * sh.wpt * (nt + 4), ethread);
          }
          const int wl = min(r / sh.N, sh.wpt - 1);
          mrow = mts + ((item & 1) * sh.wpt + wl) * (nt + 4);
        } else {
          const int w = min(tile * sh.wpt + r / sh.N, sh.B - 1);
          mrow = a.Mterm + ((int64_t)t * sh.B + w) * a.h1 + ctile * nt;
        }
      }
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        if (it >= (nchunks + 1) / 2) break;
        const int cc = 2 * it + ehalf;
        const bool has = cc < nchunks;
        if (EPI == kEpiLayer) {
          epi_layer<FULL>(a, t, has ? cc : 0, has, r, tmem, lane_base, buf, ctile * nt, tile,
                          sR + buf * nbox * kResBox, mrow);
        } else if (has) {
          if (EPI == kEpiPlain) epi_plain(a, cc, r, tmem, lane_base, buf, ctile * nt, tile);
          else epi_orbital<FULL>(a, t, cc, r, tmem, lane_base, buf, spin, ko0, tile);
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(acce + buf);
        if (rstage) mbar_arrive(rese + buf);
      }
    }
  }
  if (EPI == kEpiLayer) cp_async_wait_all();
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}


// ---- stream layer with the weights resident in shared memory ----------------------------
// The layer's split weights for this CTA's nt output columns (hi and lo parts of every
// k-block, nkb x 2 x nt x 128 B: 160 KB at k_self = 320, nt = 128) are loaded by TMA once
// per CTA; the ring then carries only the A tiles (16 KB per k-block), as many stages as
// the remaining shared memory holds.  The epilogue reads the residual (the layer input's
// first h1 columns of the same rows, just loaded through L2 for the A operand) and the
// walker's mean-field row with plain vector loads issued before the accumulator wait, and
// processes 32 columns per tensor-memory round trip (accumulator, h and sum z^2 loaded
// together under one wait).
struct ResLayout {
  uint32_t b_bytes;      // resident weights
  int stages;            // A ring depth
  uint32_t mt_bytes;     // M[t] staging: [2][wpt][nt + 4] floats
  uint32_t y_bytes;      // output staging of the TMA stores: 1 KB per epilogue warp
  size_t total;          // dynamic shared memory of the launch
};

__host__ __device__ inline ResLayout res_layout(int nkb, int nt, int stages, int wpt) {
  ResLayout l;
  l.b_bytes = (uint32_t)nkb * 2u * (uint32_t)nt * 128u;
  l.stages = stages;
  // rounded up to 128 B: the output staging after it is the source of TMA stores, which
  // must start on a 128-byte boundary
  l.mt_bytes = (2u * (uint32_t)wpt * (uint32_t)(nt + 4) * 4u + 127u) & ~127u;
  l.y_bytes = (uint32_t)kEpiWarps * 1024u;
  l.total = 1024 + (size_t)l.b_bytes + (size_t)stages * 128 * 128 + l.mt_bytes + l.y_bytes +
            8 * (2 * (size_t)stages + 6) + 16;
  return l;
}

// Tile store shared -> global through the tensor map (bulk group of the issuing thread).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"((uint64_t)map),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Wait for the tensor-memory loads in flight; the registers are operands so that no use of
// them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld48(uint32_t (&a)[16], uint32_t (&b)[16], uint32_t (&c)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                 "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]),
                 "+r"(a[15]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]),
                 "+r"(b[7]), "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]),
                 "+r"(b[14]), "+r"(b[15]), "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3]), "+r"(c[4]), "+r"(c[5]),
                 "+r"(c[6]), "+r"(c[7]), "+r"(c[8]), "+r"(c[9]), "+r"(c[10]), "+r"(c[11]), "+r"(c[12]),
                 "+r"(c[13]), "+r"(c[14]), "+r"(c[15])
               :
               : "memory");
}

__device__ __forceinline__ void tmem_wait_ld32(uint32_t (&a)[16], uint32_t (&b)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                 "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]),
                 "+r"(a[15]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]),
                 "+r"(b[7]), "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]),
                 "+r"(b[14]), "+r"(b[15])
               :
               : "memory");
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ float2 bf2_to_f2(uint32_t u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
__device__ __forceinline__ uint32_t f2_to_bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *(const uint32_t*)&h;
}

// Threads of the resident-weight layer kernel: warpgroup 0 (producer warp, MMA warp, two idle
// warps) gives registers back (setmaxnreg) to the two epilogue warpgroups, whose threads keep
// h and sum z^2 of their 64 columns in registers across the slabs of a tile.
constexpr int kResThreads = 384;
constexpr int kResRegsLow = 40;        // warpgroup 0 after setmaxnreg.dec
constexpr int kResRegsHigh = 232;      // epilogue warpgroups after setmaxnreg.inc
// The launch holds 384 x 168 registers (ptxas gives 168 per thread at 384 threads, one CTA per
// SM); the split must not exceed it: 128 x 40 + 256 x 232 = 64512 = 384 x 168.
static_assert(128 * kResRegsLow + 256 * kResRegsHigh <= kResThreads * 168, "register split above the launch");

template <bool FULL>
__global__ void __launch_bounds__(kResThreads, 1)
    k_layer_res(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const __grid_constant__ CUtensorMap tmY, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int nt = a.nt, nkb = a.nkb;
  const uint32_t bytesA = 128 * 128, bytesB = (uint32_t)nt * 128;
  const ResLayout lay = res_layout(nkb, nt, a.stages, a.sh.wpt);
  const int NS = lay.stages;
  unsigned char* sB = base;                                   // [nkb][hi rows, lo rows] weight tiles
  unsigned char* sA = sB + lay.b_bytes;                       // NS A tiles
  float* mts = (float*)(sA + (size_t)NS * bytesA);            // [2][wpt][nt + 4] M[t] rows
  uint4* ystage = (uint4*)((unsigned char*)mts + lay.mt_bytes);   // [8 warps][32 rows][2] x 16 B
  uint64_t* bars = (uint64_t*)((unsigned char*)ystage + lay.y_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + NS;
  uint64_t* accf = bars + 2 * NS;
  uint64_t* acce = accf + 2;
  uint64_t* bfull = acce + 2;
  uint64_t* mma_done = bfull + 1;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Shape& sh = a.sh;
  const int ctile = blockIdx.x;
  const int my_tiles = a.tiles > (int)blockIdx.y ? (a.tiles - 1 - (int)blockIdx.y) / (int)gridDim.y + 1 : 0;
  const int T = sh.T;
  const int n_items = my_tiles * T;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(accf + b, 1); mbar_init(acce + b, kEpiWarps); }
    mbar_init(bfull, 1);
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
  const uint64_t deadline = globaltimer() + kWaitNs * 8 * (uint64_t)(my_tiles > 0 ? my_tiles : 1);

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kResRegsLow));
    if (warp == 0 && lane == 0 && n_items > 0) {
      // the CTA's weights, once: k-block kb holds W_hi rows then W_lo rows (2 nt rows)
      mbar_expect_tx(bfull, lay.b_bytes);
      for (int kb = 0; kb < nkb; ++kb)
        for (int part = 0; part < 2; ++part)
          tma_load_2d(sB + (size_t)(kb * 2 + part) * bytesB, &tmB, bfull, part * a.bsplit + kb * kBlockK, ctile * nt);
      // ring position (stage, phase) and item (tile, t) advance by increments: no division
      int issued = 0, stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int tile = (int)blockIdx.y, t = 0;
      for (int item = 0; item < n_items && ok; ++item) {
        const int arow = (int)(t * sh.R + (int64_t)tile * 128);
        const int lo_row = (int)(a.alo_row + (int64_t)t * sh.R + (int64_t)tile * 128);
        const int lf = lo_first<kEpiLayer>(a, t, 0, nkb);
        const int n_k = nkb + (nkb - lf);
        for (int kk = 0; kk < n_k; ++kk) {
          const bool lo = kk >= nkb;
          const int kb = lo ? lf + (kk - nkb) : kk;
          if (*abort_flag || !mbar_wait(empty + stage, phase ^ 1u, deadline)) { ok = false; break; }
          mbar_expect_tx(full + stage, bytesA);
          tma_load_2d(sA + (size_t)stage * bytesA, &tmA, full + stage, kb * kBlockK, lo ? lo_row : arow);
          ++issued;
          if (++stage == NS) { stage = 0; phase ^= 1u; }
        }
        if (++t == T) { t = 0; tile += (int)gridDim.y; }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.status, kStatusTimeout);
      }
      // wait (bounded) for the copies still in flight before the CTA can exit
      const uint64_t dl2 = globaltimer() + kWaitNs;
      mbar_wait(bfull, 0u, dl2);
      for (int q = issued > NS ? issued - NS : 0; q < issued; ++q)
        mbar_wait(full + (q % NS), (uint32_t)((q / NS) & 1), dl2);
    } else if (warp == 1 && lane == 0) {
      // one MMA of N = 2 nt multiplies the A tile by the stacked [hi; lo] weight rows of a
      // k-block: accumulator columns [0, nt) get A W_hi, [nt, 2 nt) get A W_lo; two
      // accumulators of 2 nt columns alternate between items
      const uint32_t idesc = idesc_bf16(128, 2 * nt);
      int stage = 0;
      uint32_t phase = 0;
      int t = 0;
      bool ok = n_items == 0 || (!*abort_flag && mbar_wait(bfull, 0u, deadline));
      const uint32_t sA_u = smem_u32(sA), sB_u = smem_u32(sB);
      for (int item = 0; item < n_items && ok; ++item) {
        const int buf = item & 1;
        const uint32_t use = (uint32_t)(item >> 1);
        if (*abort_flag || !mbar_wait(acce + buf, (use & 1u) ^ 1u, deadline)) { ok = false; break; }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * 2 * nt);
        const int lf = lo_first<kEpiLayer>(a, t, 0, nkb);
        const int n_k = nkb + (nkb - lf);
        for (int kk = 0; kk < n_k; ++kk) {
          const bool lo = kk >= nkb;
          const int kb = lo ? lf + (kk - nkb) : kk;
          if (*abort_flag || !mbar_wait(full + stage, phase, deadline)) { ok = false; break; }
          fence_after();
          const uint64_t da = sdesc(sA_u + (uint32_t)stage * bytesA);
          const uint64_t db = sdesc(sB_u + (uint32_t)(kb * 2) * bytesB);
#pragma unroll
          for (int k4 = 0; k4 < kBlockK / 16; ++k4)
            mma_bf16(d, da + (uint64_t)(2 * k4), db + (uint64_t)(2 * k4), idesc, (kk != 0 || k4 != 0) ? 1u : 0u);
          mma_commit(empty + stage);
          if (++stage == NS) { stage = 0; phase ^= 1u; }
        }
        if (ok) mma_commit(accf + buf);
        if (++t == T) t = 0;
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.status, kStatusTimeout);
      }
      mma_commit(mma_done);
      mbar_wait(mma_done, 0u, globaltimer() + kWaitNs);
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kResRegsHigh));
    const int q = warp & 3;                       // TMEM lane quarter this warp may access
    const int r = q * 32 + lane;
    const int ehalf = (warp - 4) >> 2;            // column half: chunks cc with cc % 2 == ehalf
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const int nchunks = nt / 32;
    const int n0 = ctile * nt;
    const int wl = r / sh.N;
    const int ethread = threadIdx.x - 128;
    uint4* ystg = ystage + (warp - 4) * 64;
    // the 16-column pieces of this thread: chunk cc = 2 (pc / 2) + ehalf (where it exists), half pc % 2
    const int npieces = (ehalf < nchunks ? 2 : 0) + (2 + ehalf < nchunks ? 2 : 0);
    // h = tanh z of the value slab and the running sum of z^2 over the tangent slabs, for this
    // thread's row and columns, kept across the slabs of a tile
    float hreg[4][16], sreg[4][16];
    if (n_items > 0) stage_mterm(a, 0, (int)blockIdx.y, n0, mts, ethread);
    int tile = (int)blockIdx.y, t = 0;
    for (int item = 0; item < n_items; ++item) {
      const int buf = item & 1;
      const uint32_t use = (uint32_t)(item >> 1);
      const int64_t row = (int64_t)tile * 128 + r;
      const int w = tile * sh.wpt + wl;
      const bool valid = wl < sh.wpt && w < sh.B;
      const int kind = t == 0 ? 0 : (t < T - 1 ? 1 : 2);
      // residual pieces (the layer input's columns of this thread), loaded before the wait
      uint4 res[4][2];
      const bool has_res = a.residual && valid;
      const uint4* xres = (const uint4*)(a.X + t * sh.R * (int64_t)a.ldx + row * a.ldx + n0);
#pragma unroll
      for (int pc = 0; pc < 4; ++pc) {
        res[pc][0] = make_uint4(0u, 0u, 0u, 0u);
        res[pc][1] = make_uint4(0u, 0u, 0u, 0u);
        if (pc < npieces && has_res) {
          const int cb = (2 * (pc >> 1) + ehalf) * 32 + (pc & 1) * 16;
          res[pc][0] = __ldg(xres + cb / 8);
          res[pc][1] = __ldg(xres + cb / 8 + 1);
        }
      }
      cp_async_wait_all();
      bool ok = !*abort_flag && mbar_wait(accf + buf, use & 1u, deadline);
      // (the barrier also publishes every thread's staged M[t] copies)
      if (epilogue_any(!ok)) {
        if (ethread == 0) {
          *abort_flag = 1;
          atomicOr(a.status, kStatusTimeout);
        }
        break;
      }
      fence_after();
      // the next item's M[t] rows into the other buffer (its readers passed the barrier)
      int tile1 = tile, t1 = t + 1;
      if (t1 == T) { t1 = 0; tile1 += (int)gridDim.y; }
      if (item + 1 < n_items) stage_mterm(a, t1, tile1, n0, mts + ((item + 1) & 1) * sh.wpt * (nt + 4), ethread);
      const float* mrow = mts + ((item & 1) * sh.wpt + min(wl, sh.wpt - 1)) * (nt + 4);
      const uint32_t accb = tmem + lane_base + (uint32_t)(buf * 2 * nt);
#pragma unroll
      for (int pc = 0; pc < 4; ++pc) {
        if (pc >= npieces) break;                 // warp-uniform
        const int cb = (2 * (pc >> 1) + ehalf) * 32 + (pc & 1) * 16;
        const int col0 = n0 + cb;
        uint32_t ah[16], al[16], unused[16];
        tmem_ld16_nowait(accb + (uint32_t)cb, ah);
        tmem_ld16_nowait(accb + (uint32_t)(nt + cb), al);
        float4 m[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) m[v] = *((const float4*)(mrow + cb) + v);
        tmem_wait_ld48(ah, al, unused);
        const uint32_t* rr = (const uint32_t*)res[pc];
        uint32_t o[8];
        if (kind == 0) {
          float outf[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float mv = (j & 3) == 0 ? m[j >> 2].x : ((j & 3) == 1 ? m[j >> 2].y : ((j & 3) == 2 ? m[j >> 2].z : m[j >> 2].w));
            const float h = tanh_fast(__uint_as_float(ah[j]) + __uint_as_float(al[j]) + mv);
            if (FULL) { hreg[pc][j] = h; sreg[pc][j] = 0.f; }
            const float2 r2 = bf2_to_f2(rr[j >> 1]);
            outf[j] = h + ((j & 1) ? r2.y : r2.x);
            al[j] = __float_as_uint(h);           // h of this piece, for act_out
          }
          if (valid && a.residual && a.alo_row > 0) {
            // the value slab's residual is a pair: add its low part (slab T of X)
            const uint4* xl = (const uint4*)(a.X + (int64_t)T * sh.R * a.ldx + row * a.ldx + col0);
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              const uint4 u = xl[v];
              const uint32_t* uu = (const uint32_t*)&u;
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 f = bf2_to_f2(uu[e]);
                outf[8 * v + 2 * e] += f.x;
                outf[8 * v + 2 * e + 1] += f.y;
              }
            }
          }
          // the value slab and its low part (slab T) as TMA tile stores, like the tangent slabs
          const int yrow = (int)((int64_t)tile * 128 + q * 32);
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            if (part == 1 && a.alo_row <= 0) break;
#pragma unroll
            for (int p = 0; p < 8; ++p)
              o[p] = !valid ? 0u
                            : (part == 0 ? f2_to_bf2(outf[2 * p], outf[2 * p + 1])
                                         : f2_to_bf2(bf16_rem(outf[2 * p]), bf16_rem(outf[2 * p + 1])));
            if (lane == 0) bulk_wait_read0();
            __syncwarp();
            ystg[2 * lane] = make_uint4(o[0], o[1], o[2], o[3]);
            ystg[2 * lane + 1] = make_uint4(o[4], o[5], o[6], o[7]);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
              tma_store_2d(&tmY, ystg, col0, (int)(part ? (int64_t)T * sh.R + yrow : yrow));
              bulk_commit();
            }
          }
          if (valid) {
            if (a.act_out) {
              float4* ao = (float4*)(a.act_out + row * a.h1 + col0);
#pragma unroll
              for (int v = 0; v < 4; ++v)
                ao[v] = make_float4(__uint_as_float(al[4 * v]), __uint_as_float(al[4 * v + 1]),
                                    __uint_as_float(al[4 * v + 2]), __uint_as_float(al[4 * v + 3]));
            }
          }
        } else if (FULL) {
          // tangent slab: out = res + (1 - h^2) z, sum z^2 += z^2; Laplacian slab:
          // out = res + (1 - h^2) (z - 2 h sum z^2); packed two-lane FP32 arithmetic
          const uint64_t m1 = pack_f2(-1.f, -1.f), m2 = pack_f2(-2.f, -2.f);
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const float4 m4 = m[p >> 1];
            const uint64_t z2 = add_f2(add_f2(pack_f2(__uint_as_float(ah[2 * p]), __uint_as_float(ah[2 * p + 1])),
                                              pack_f2(__uint_as_float(al[2 * p]), __uint_as_float(al[2 * p + 1]))),
                                       (p & 1) ? pack_f2(m4.z, m4.w) : pack_f2(m4.x, m4.y));
            const uint64_t h2 = pack_f2(hreg[pc][2 * p], hreg[pc][2 * p + 1]);
            const uint64_t s2 = pack_f2(sreg[pc][2 * p], sreg[pc][2 * p + 1]);
            const uint64_t nd2 = fma_f2(h2, h2, m1);              // -(1 - h^2)
            uint64_t w2;
            if (kind == 1) {
              w2 = z2;
              unpack_f2(fma_f2(z2, z2, s2), sreg[pc][2 * p], sreg[pc][2 * p + 1]);
            } else {
              w2 = fma_f2(mul_f2(h2, s2), m2, z2);                // z - 2 h sum z^2
            }
            const float2 r2 = bf2_to_f2(rr[p]);
            float a0, a1;
            unpack_f2(sub_f2(pack_f2(r2.x, r2.y), mul_f2(nd2, w2)), a0, a1);
            o[p] = valid ? f2_to_bf2(a0, a1) : 0u;  // rows without an electron are written as zero
          }
          // the warp's 32 rows x 16 columns go out as one TMA tile store (coalesced) from a
          // 1 KB staging buffer; its previous store must have finished reading the buffer
          if (lane == 0) bulk_wait_read0();
          __syncwarp();
          ystg[2 * lane] = make_uint4(o[0], o[1], o[2], o[3]);
          ystg[2 * lane + 1] = make_uint4(o[4], o[5], o[6], o[7]);
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&tmY, ystg, col0, (int)(t * sh.R + (int64_t)tile * 128 + q * 32));
            bulk_commit();
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce + buf);
      if (++t == T) { t = 0; tile += (int)gridDim.y; }
    }
    cp_async_wait_all();
    if (lane == 0) bulk_wait0();          // the output stores have completed
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}


// ---- stream layer on CTA pairs (cta_group::2) ---------------------------------------
// The two CTAs of a cluster (the two SMs of one TPC) share every MMA: M = 256 rows, CTA
// rank 0 supplying its row tile as rows 0..127 and rank 1 the next row tile as rows
// 128..255.  Each CTA holds half of the weight tile, the high and low BF16 parts of 64 of
// the pair's 128 output columns stacked as one 128-row operand (80 KB at k_self = 320),
// and every MMA is N = 256: accumulator columns [0, 64) hold A W_hi and [64, 128) A W_lo
// for rank 0's 64 columns, [128, 256) the same for rank 1's.  Per CTA:
//   warp 0       TMA producer: the CTA's weight half once, then its A tiles (16 KB per
//                k-block) into a ring; every copy of both CTAs completes on the rank-0
//                CTA's barrier
//   warp 1       allocates the pair's tensor memory; on rank 0 one lane issues the MMAs
//                and commits to the barriers of both CTAs (multicast)
//   warps 4..19  epilogue on the CTA's own 128 rows: a TMEM lane quarter and 32 output
//                columns per warp.  Each warp first moves its accumulator columns (high +
//                low) to registers and hands the accumulator back, then computes, with h
//                and sum z^2 kept in tensor memory, and writes its 32 x 32 output tile by
//                one TMA store.  Warps proceed independently: the mean-field rows M[t] of
//                a warp's walkers are staged per warp (cp.async, one item ahead).
// Tensor memory (512 columns): the accumulator [0, 256) and, in the tangent pass, h
// [256, 384) and sum z^2 [384, 512); the value-only pass double-buffers the accumulator.
struct PairLayout {
  uint32_t b_bytes;      // resident weight half
  int stages;            // A ring depth
  uint32_t mt_bytes;     // M[t] staging: [16 warps][2][wpw][32] floats (rounded up to 1 KB)
  uint32_t y_bytes;      // output staging: 2 KB per epilogue warp
  size_t total;
};

constexpr int kPairEpiWarps = 16;
constexpr int kPairThreads = 128 + 32 * kPairEpiWarps;     // 640
constexpr int kPairRegsLow = 40;                           // warpgroup 0 after setmaxnreg.dec
constexpr int kPairRegsHigh = 104;                         // epilogue warpgroups after setmaxnreg.inc
// 640 threads launch with 96 registers each (65536 / 640 rounded down to 8); the split must
// fit in them: 128 x 40 + 512 x 104 = 58368 <= 640 x 96 = 61440.  The host checks the launch count.
constexpr int kPairLaunchRegs = 96;
static_assert(128 * kPairRegsLow + 32 * kPairEpiWarps * kPairRegsHigh <= kPairThreads * kPairLaunchRegs,
              "register split above the launch");

// Walkers whose rows meet 32 consecutive rows of a tile: at most 32 / N + 2.
__host__ __device__ inline int pair_wpw(int N) { return 32 / N + 2; }

__host__ __device__ inline PairLayout pair_layout(int nkb, int stages, int N) {
  PairLayout l;
  l.b_bytes = (uint32_t)nkb * 2u * 64u * 128u;
  l.stages = stages;
  l.mt_bytes = ((uint32_t)kPairEpiWarps * 2u * (uint32_t)pair_wpw(N) * 128u + 1023u) & ~1023u;
  l.y_bytes = (uint32_t)kPairEpiWarps * 2048u;
  l.total = 1024 + (size_t)l.b_bytes + (size_t)stages * 128 * 128 + l.mt_bytes + l.y_bytes +
            8 * (2 * (size_t)stages + 6) + 16;
  return l;
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Address of the same shared variable in CTA `rank` of the cluster (shared::cluster window).
__device__ __forceinline__ uint32_t mapa_rank(const void* p, uint32_t rank) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(smem_u32(p)), "r"(rank));
  return d;
}
// Arrival on a barrier of the peer CTA.  The ordering it carries is that of the tensor-memory
// loads before it (tcgen05.wait::ld and fence::before_thread_sync), not of generic memory.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// TMA load into this CTA's shared memory whose completion is counted on a barrier of either
// CTA of the pair (here always rank 0's).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cluster, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(bar_cluster), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// Arrive (once the pair's MMAs issued so far complete) on the barrier at this offset in both CTAs.
__device__ __forceinline__ void mma_commit_pair_mc(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// The M[t] rows of the walkers that meet this warp's rows (walkers wa .. wa + nwm - 1 of the
// tile), this CTA's columns n0 + cg0 .. + 31, into the warp's staging rows of 32 floats;
// one commit group per call and lane.
__device__ __forceinline__ void stage_mterm_warp(const TcArgs& a, int t, int tile, int wa, int nwm, int col,
                                                 float* dst, int lane) {
  const Shape& sh = a.sh;
  const int w0 = tile * sh.wpt + wa;
  for (int e = lane; e < nwm * 8; e += 32) {
    const int j = e >> 3, c = e & 7;
    if (w0 + j < sh.B) cp_async16(dst + j * 32 + 4 * c, a.Mterm + ((int64_t)t * sh.B + w0 + j) * a.h1 + col + 4 * c);
  }
  cp_async_commit();
}

template <bool FULL>
__global__ void __launch_bounds__(kPairThreads, 1)
    k_layer_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ CUtensorMap tmY, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int nt = 128;
  constexpr int NACC = FULL ? 1 : 2;                          // accumulators of 256 columns
  constexpr uint32_t bytesA = 128 * 128, bytesB = 128 * 128;  // B: 64 W_hi rows then 64 W_lo rows
  const int nkb = a.nkb;
  const Shape& sh = a.sh;
  const PairLayout lay = pair_layout(nkb, a.stages, sh.N);
  const int NS = lay.stages;
  const int wpw = pair_wpw(sh.N);
  unsigned char* sB = base;                                   // [nkb][128 rows] weight tiles
  unsigned char* sA = sB + lay.b_bytes;                       // NS A tiles
  float* mts = (float*)(sA + (size_t)NS * bytesA);            // [16 warps][2][wpw][32] M[t] rows
  unsigned char* ystage = (unsigned char*)mts + lay.mt_bytes; // [16 warps][32 rows][64 B]
  uint64_t* bars = (uint64_t*)(ystage + lay.y_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + NS;
  uint64_t* accf = bars + 2 * NS;
  uint64_t* acce = accf + 2;
  uint64_t* bfull = acce + 2;
  uint64_t* mma_done = bfull + 1;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int ctile = (int)(blockIdx.x >> 1);
  const int pairs = (a.tiles + 1) >> 1;
  const int my_pairs = pairs > (int)blockIdx.y ? (pairs - 1 - (int)blockIdx.y) / (int)gridDim.y + 1 : 0;
  const int T = sh.T;
  const int n_items = my_pairs * T;                           // the same in both CTAs of the pair

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(accf + b, 1); mbar_init(acce + b, 2 * kPairEpiWarps); }
    mbar_init(bfull, 1);
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    // one warp of each CTA of the pair allocates, together, the same columns in both
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  // both CTAs' barriers are initialised before any copy or arrival of the peer reaches them
  fence_before();
  cluster_sync_all();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint64_t deadline = globaltimer() + kWaitNs * 8 * (uint64_t)(my_pairs > 0 ? my_pairs : 1);

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kPairRegsLow));
    if (warp == 0 && lane == 0 && n_items > 0) {
      // this CTA's weight half, once: k-block kb holds 64 W_hi rows then 64 W_lo rows
      if (rank == 0) mbar_expect_tx(bfull, 2 * lay.b_bytes);
      const uint32_t bfull0 = mapa_rank(bfull, 0);
      for (int kb = 0; kb < nkb; ++kb)
        for (int part = 0; part < 2; ++part)
          tma_load_2d_pair(sB + (size_t)kb * bytesB + part * (bytesB / 2), &tmB, bfull0,
                           part * a.bsplit + kb * kBlockK, ctile * nt + (int)rank * 64);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int pr = (int)blockIdx.y, t = 0;
      for (int item = 0; item < n_items && ok; ++item) {
        const int tile = 2 * pr + (int)rank;
        // (rank 1's tile of the last pair may lie past the rows: its copies read rows of
        // the next slab or the zero fill, and its epilogue stores nothing)
        const int arow = (int)(t * sh.R + (int64_t)tile * 128);
        const int lo_row = (int)(a.alo_row + (int64_t)t * sh.R + (int64_t)tile * 128);
        const int lf = lo_first<kEpiLayer>(a, t, 0, nkb);
        const int n_k = nkb + (nkb - lf);
        for (int kk = 0; kk < n_k; ++kk) {
          const bool lo = kk >= nkb;
          const int kb = lo ? lf + (kk - nkb) : kk;
          if (*abort_flag || !mbar_wait(empty + stage, phase ^ 1u, deadline)) { ok = false; break; }
          if (rank == 0) mbar_expect_tx(full + stage, 2 * bytesA);
          tma_load_2d_pair(sA + (size_t)stage * bytesA, &tmA, mapa_rank(full + stage, 0), kb * kBlockK,
                           lo ? lo_row : arow);
          if (++stage == NS) { stage = 0; phase ^= 1u; }
        }
        if (++t == T) { t = 0; pr += (int)gridDim.y; }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.status, kStatusTimeout);
        // the copies in flight complete on rank 0's barriers, which this thread cannot
        // wait on: give them a bounded 200 us before the CTA leaves
        const uint64_t until = globaltimer() + 200000ull;
        while (globaltimer() < until) {}
      }
    } else if (warp == 1 && lane == 0 && rank == 0) {
      // per k-block of the A tile, 4 MMAs (K = 16, N = 256) against the stacked weight rows
      const uint32_t idesc = idesc_bf16(256, 256);
      int stage = 0;
      uint32_t phase = 0;
      int t = 0;
      bool ok = n_items == 0 || (!*abort_flag && mbar_wait(bfull, 0u, deadline));
      fence_after();
      const uint32_t sA_u = smem_u32(sA), sB_u = smem_u32(sB);
      for (int item = 0; item < n_items && ok; ++item) {
        const int buf = NACC == 1 ? 0 : (item & 1);
        const uint32_t use = (uint32_t)(NACC == 1 ? item : item >> 1);
        if (*abort_flag || !mbar_wait(acce + buf, (use & 1u) ^ 1u, deadline)) { ok = false; break; }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * 256);
        const int lf = lo_first<kEpiLayer>(a, t, 0, nkb);
        const int n_k = nkb + (nkb - lf);
        for (int kk = 0; kk < n_k; ++kk) {
          const int kb = kk >= nkb ? lf + (kk - nkb) : kk;
          if (*abort_flag || !mbar_wait(full + stage, phase, deadline)) { ok = false; break; }
          fence_after();
          const uint64_t da = sdesc(sA_u + (uint32_t)stage * bytesA);
          const uint64_t db = sdesc(sB_u + (uint32_t)kb * bytesB);
#pragma unroll
          for (int k4 = 0; k4 < kBlockK / 16; ++k4)
            mma_bf16_pair(d, da + (uint64_t)(2 * k4), db + (uint64_t)(2 * k4), idesc, (kk != 0 || k4 != 0) ? 1u : 0u);
          mma_commit_pair_mc(empty + stage);
          if (++stage == NS) { stage = 0; phase ^= 1u; }
        }
        if (ok) mma_commit_pair_mc(accf + buf);
        if (++t == T) t = 0;
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.status, kStatusTimeout);
      }
      mma_commit_pair(mma_done);
      mbar_wait(mma_done, 0u, globaltimer() + kWaitNs);
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kPairRegsHigh));
    const int q = warp & 3;                       // TMEM lane quarter this warp may access
    const int r = q * 32 + lane;                  // row in the CTA's tile
    const int cg0 = ((warp - 4) >> 2) * 32;       // the warp's 32 output columns within the 128
    // accumulator columns of those outputs' W_hi products (the W_lo ones follow 64 later)
    const uint32_t dhi = (uint32_t)(cg0 < 64 ? cg0 : cg0 + 64);
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const int n0 = ctile * nt;
    const int wl = r / sh.N;
    const int wa = (q * 32) / sh.N;               // first walker meeting the warp's rows
    const int nwm = min(sh.wpt, (q * 32 + 31) / sh.N + 1) - wa;   // walkers of the warp's rows
    const int wrow = min(wl, sh.wpt - 1) - wa;    // this row's walker in the warp's staging
    float* mw = mts + (size_t)(warp - 4) * 2 * wpw * 32;
    unsigned char* ystg = ystage + (warp - 4) * 2048;
    uint4* yrow = (uint4*)(ystg + lane * 64);     // this thread's row of the 32 x 32 output tile
    const uint32_t hcol = 256, scol = 384;        // tensor-memory columns of h and sum z^2
    const uint32_t acce0 = mapa_rank(acce, 0);
    int pr = (int)blockIdx.y, t = 0;
    if (n_items > 0 && nwm > 0) stage_mterm_warp(a, 0, 2 * pr + (int)rank, wa, nwm, n0 + cg0, mw, lane);
    else cp_async_commit();
    for (int item = 0; item < n_items; ++item) {
      const int buf = NACC == 1 ? 0 : (item & 1);
      const uint32_t use = (uint32_t)(NACC == 1 ? item : item >> 1);
      const int tile = 2 * pr + (int)rank;
      const bool tile_ok = tile < a.tiles;
      const int64_t row = (int64_t)tile * 128 + r;
      const int w = tile * sh.wpt + wl;
      const bool valid = tile_ok && wl < sh.wpt && w < sh.B;
      const uint32_t tl = tmem + lane_base;
      const int yr = (int)((int64_t)tile * 128 + q * 32);
      const uint4* xr = (const uint4*)(a.X + t * sh.R * (int64_t)a.ldx + row * a.ldx + n0 + cg0);
      // Waits for the item's M[t] rows and accumulator (false: timed out), moves z without the
      // mean-field term (the W_hi and W_lo products of the warp's 32 columns) to registers,
      // hands the accumulator back to the MMA, stages the next item's M[t] rows and waits
      // until the previous item's stores have read the staging tile.
      auto begin_item = [&](float (&zr)[2][16]) -> bool {
        cp_async_wait_all();
        __syncwarp();
        if (*abort_flag || !mbar_wait(accf + buf, use & 1u, deadline)) {
          *abort_flag = 1;
          if (lane == 0) atomicOr(a.status, kStatusTimeout);
          return false;
        }
        fence_after();
#pragma unroll
        for (int pc = 0; pc < 2; ++pc) {
          uint32_t ah[16], al[16];
          tmem_ld16_nowait(tl + (uint32_t)(buf * 256) + dhi + (uint32_t)(pc * 16), ah);
          tmem_ld16_nowait(tl + (uint32_t)(buf * 256) + dhi + 64u + (uint32_t)(pc * 16), al);
          tmem_wait_ld32(ah, al);
#pragma unroll
          for (int j = 0; j < 16; ++j) zr[pc][j] = __uint_as_float(ah[j]) + __uint_as_float(al[j]);
        }
        fence_before();
        __syncwarp();
        if (lane == 0) {
          if (rank == 0) mbar_arrive(acce + buf);
          else mbar_arrive_remote(acce0 + 8u * (uint32_t)buf);
        }
        // the next item's M[t] rows into the warp's other buffer (its last reader was this
        // warp at the previous item)
        int pr1 = pr, t1 = t + 1;
        if (t1 == T) { t1 = 0; pr1 += (int)gridDim.y; }
        if (item + 1 < n_items && nwm > 0)
          stage_mterm_warp(a, t1, 2 * pr1 + (int)rank, wa, nwm, n0 + cg0, mw + ((item + 1) & 1) * wpw * 32, lane);
        else cp_async_commit();
        if (lane == 0) bulk_wait_read0();
        __syncwarp();
        return true;
      };
      const float* mrow = mw + ((item & 1) * wpw + max(wrow, 0)) * 32;
      // The warp's 32 rows x 32 columns leave as one TMA tile store (none for a tile past the rows).
      auto store_tile = [&](int64_t slab_row) {
        fence_proxy_async();
        __syncwarp();
        if (lane == 0 && tile_ok) {
          tma_store_2d(&tmY, ystg, n0 + cg0, (int)(slab_row + yr));
          bulk_commit();
        }
      };
      if (t == 0) {
        // value slab: h = tanh(z), out = h + residual (a hi/lo pair in and out); the residual
        // and its low part (slab T) are loaded before the accumulator wait
        uint4 res[2][2], rlo[2][2];
#pragma unroll
        for (int pc = 0; pc < 2; ++pc)
#pragma unroll
          for (int v = 0; v < 2; ++v) { res[pc][v] = make_uint4(0u, 0u, 0u, 0u); rlo[pc][v] = res[pc][v]; }
        const uint4* xl = (const uint4*)(a.X + (int64_t)T * sh.R * a.ldx + row * a.ldx + n0 + cg0);
        const bool has_lo = valid && a.residual && a.alo_row > 0;
        if (valid && a.residual) {
#pragma unroll
          for (int pc = 0; pc < 2; ++pc) { res[pc][0] = __ldg(xr + 2 * pc); res[pc][1] = __ldg(xr + 2 * pc + 1); }
          if (!FULL && has_lo) {
#pragma unroll
            for (int pc = 0; pc < 2; ++pc) { rlo[pc][0] = __ldg(xl + 2 * pc); rlo[pc][1] = __ldg(xl + 2 * pc + 1); }
          }
        }
        float zr[2][16];
        if (!begin_item(zr)) break;
        if (FULL && has_lo) {
          // (in the tangent pass the value slab is one item in 3N + 2: its low-part loads wait
          // here rather than hold registers through the accumulator hand-back)
#pragma unroll
          for (int pc = 0; pc < 2; ++pc) { rlo[pc][0] = __ldg(xl + 2 * pc); rlo[pc][1] = __ldg(xl + 2 * pc + 1); }
        }
        uint32_t olo[2][8];
#pragma unroll
        for (int pc = 0; pc < 2; ++pc) {
          const float4* mt = (const float4*)(mrow + pc * 16);
          const uint32_t* rr = (const uint32_t*)res[pc];
          const uint32_t* rl = (const uint32_t*)rlo[pc];
          uint32_t hv[16], o[8];
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const float4 m4 = mt[p >> 1];
            const float h0 = tanh_fast(zr[pc][2 * p] + ((p & 1) ? m4.z : m4.x));
            const float h1 = tanh_fast(zr[pc][2 * p + 1] + ((p & 1) ? m4.w : m4.y));
            hv[2 * p] = __float_as_uint(h0);
            hv[2 * p + 1] = __float_as_uint(h1);
            const float2 r2 = bf2_to_f2(rr[p]);
            const float2 l2 = bf2_to_f2(rl[p]);
            const float y0 = h0 + r2.x + l2.x, y1 = h1 + r2.y + l2.y;
            o[p] = valid ? f2_to_bf2(y0, y1) : 0u;
            olo[pc][p] = valid ? f2_to_bf2(bf16_rem(y0), bf16_rem(y1)) : 0u;
          }
          if (FULL) tmem_st16(tl + hcol + (uint32_t)(cg0 + pc * 16), hv);   // h, for the tangent slabs
          if (valid && a.act_out) {
            float4* ao = (float4*)(a.act_out + row * a.h1 + n0 + cg0 + pc * 16);
#pragma unroll
            for (int v = 0; v < 4; ++v)
              ao[v] = make_float4(__uint_as_float(hv[4 * v]), __uint_as_float(hv[4 * v + 1]),
                                  __uint_as_float(hv[4 * v + 2]), __uint_as_float(hv[4 * v + 3]));
          }
          yrow[2 * pc] = make_uint4(o[0], o[1], o[2], o[3]);
          yrow[2 * pc + 1] = make_uint4(o[4], o[5], o[6], o[7]);
        }
        store_tile(0);
        if (a.alo_row > 0) {
          // the value slab's low part (slab T of Y) from the same staging tile
          if (lane == 0) bulk_wait_read0();
          __syncwarp();
#pragma unroll
          for (int pc = 0; pc < 2; ++pc) {
            yrow[2 * pc] = make_uint4(olo[pc][0], olo[pc][1], olo[pc][2], olo[pc][3]);
            yrow[2 * pc + 1] = make_uint4(olo[pc][4], olo[pc][5], olo[pc][6], olo[pc][7]);
          }
          store_tile((int64_t)T * sh.R);
        }
        if (FULL) tmem_wait_st();
      } else if (FULL) {
        // tangent slab: out = res + (1 - h^2) z, sum z^2 += z^2; Laplacian slab:
        // out = res + (1 - h^2) (z - 2 h sum z^2); packed two-lane FP32 arithmetic
        const bool lap = t == T - 1;
        uint4 res[2][2];
#pragma unroll
        for (int pc = 0; pc < 2; ++pc) {
          res[pc][0] = make_uint4(0u, 0u, 0u, 0u);
          res[pc][1] = res[pc][0];
          if (valid && a.residual) { res[pc][0] = __ldg(xr + 2 * pc); res[pc][1] = __ldg(xr + 2 * pc + 1); }
        }
        float zr[2][16];
        if (!begin_item(zr)) break;
        const uint64_t m1 = pack_f2(-1.f, -1.f), m2 = pack_f2(-2.f, -2.f);
#pragma unroll
        for (int pc = 0; pc < 2; ++pc) {
          const int c = cg0 + pc * 16;
          uint32_t hv[16], sq[16];
          tmem_ld16_nowait(tl + hcol + (uint32_t)c, hv);
          if (t > 1) tmem_ld16_nowait(tl + scol + (uint32_t)c, sq);   // the first tangent slab starts the sum
          tmem_wait_ld32(hv, sq);
          const float4* mt = (const float4*)(mrow + pc * 16);
          const uint32_t* rr = (const uint32_t*)res[pc];
          uint32_t o[8];
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const float4 m4 = mt[p >> 1];
            const uint64_t z2 = add_f2(pack_f2(zr[pc][2 * p], zr[pc][2 * p + 1]),
                                       (p & 1) ? pack_f2(m4.z, m4.w) : pack_f2(m4.x, m4.y));
            const uint64_t h2 = pack_f2(__uint_as_float(hv[2 * p]), __uint_as_float(hv[2 * p + 1]));
            const uint64_t s2 = pack_f2(__uint_as_float(sq[2 * p]), __uint_as_float(sq[2 * p + 1]));
            const uint64_t nd2 = fma_f2(h2, h2, m1);              // -(1 - h^2)
            uint64_t w2;
            if (!lap) {
              w2 = z2;
              float s0, s1;
              unpack_f2(t == 1 ? mul_f2(z2, z2) : fma_f2(z2, z2, s2), s0, s1);
              sq[2 * p] = __float_as_uint(s0);
              sq[2 * p + 1] = __float_as_uint(s1);
            } else {
              w2 = fma_f2(mul_f2(h2, s2), m2, z2);                // z - 2 h sum z^2
            }
            const float2 r2 = bf2_to_f2(rr[p]);
            float a0, a1;
            unpack_f2(sub_f2(pack_f2(r2.x, r2.y), mul_f2(nd2, w2)), a0, a1);
            o[p] = valid ? f2_to_bf2(a0, a1) : 0u;  // rows without an electron are written as zero
          }
          if (!lap) tmem_st16(tl + scol + (uint32_t)c, sq);
          yrow[2 * pc] = make_uint4(o[0], o[1], o[2], o[3]);
          yrow[2 * pc + 1] = make_uint4(o[4], o[5], o[6], o[7]);
        }
        store_tile(t * sh.R);
        tmem_wait_st();
      }
      if (++t == T) { t = 0; pr += (int)gridDim.y; }
    }
    cp_async_wait_all();
    if (lane == 0) bulk_wait0();          // the output stores have completed
  }
  // neither CTA leaves (or frees tensor memory) while the pair's MMAs or the peer's
  // arrivals may still reach it
  fence_before();
  cluster_sync_all();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
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

// 2-D bf16 tensor map for tile stores: box 16 columns x 32 rows, no swizzle.
static bool make_store_map(CUtensorMap* m, const void* base, int64_t cols, int64_t rows, int64_t ld,
                           int box_cols = 16) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, 32};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_available() { return encode_fn() != nullptr; }

int tc_columns(int h1) {
  if (h1 % 128 == 0) return 128;
  if (h1 % 64 == 0) return 64;
  return 32;
}

static uint32_t pow2_cols(int c) {
  uint32_t v = 32;
  while ((int)v < c) v <<= 1;
  return v;
}

// Dynamic shared memory of a launch: alignment slack, the A/B ring, the layer epilogue's
// M[t] staging (mt_rows walkers, double-buffered), barriers.
static size_t tc_smem_bytes(int nt, int epi, bool split, int mt_rows = 0, bool res = false) {
  const int ns = tc::stages_for(epi);
  const size_t mt = (size_t)2 * mt_rows * (nt + 4) * 4;
  const size_t rs = res ? (size_t)2 * ((nt + 63) / 64) * tc::kResBox : 0;
  return 1024 + ns * (128 * 128 + (size_t)nt * 128 * (split ? 2 : 1)) + rs + mt + 8 * (2 * ns + 9) + 16;
}
constexpr size_t kMaxDynamicSmem = 227 * 1024;

static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Grid of column tiles x enough row-tile strides to give every SM one CTA.
static dim3 persistent_grid(int ctiles, int tiles) {
  const int per_col = std::max(1, sm_count() / std::max(1, ctiles));
  return dim3(ctiles, std::min(tiles, per_col));
}

template <int EPI>
static void launch_tc(const CUtensorMap& ta, const CUtensorMap& tb, const tc::TcArgs& a, dim3 grid, bool full,
                      cudaStream_t st) {
  const size_t smem = tc_smem_bytes(a.nt, EPI, a.bsplit != 0, (EPI == tc::kEpiLayer && a.mt_stage) ? a.sh.wpt : 0,
                                   EPI == tc::kEpiLayer && a.residual);
  if (full) {
    cudaFuncSetAttribute(tc::k_tc<EPI, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc::k_tc<EPI, true><<<grid, tc::kThreads, smem, st>>>(ta, tb, a);
  } else {
    cudaFuncSetAttribute(tc::k_tc<EPI, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc::k_tc<EPI, false><<<grid, tc::kThreads, smem, st>>>(ta, tb, a);
  }
}

// The stream layer runs on the one-CTA resident-weight kernel; FN_LAYER_KERNEL=pair selects
// the CTA-pair kernel where it applies (output columns in tiles of 128).  Both produce the
// same bits: the same products, accumulated in the same order.  On the N2 network at 4096
// walkers the pair kernel issues its MMAs at the full N = 256 rate but is not faster (1.17 ms
// per launch against 1.11 ms): both are bound by their epilogues' memory operations, not by
// the A-tile stream, which alone takes 0.41 ms through a 3-stage ring and 0.28 ms through a
// 6-stage one.
static bool layer_pair_enabled() {
  const char* v = getenv("FN_LAYER_KERNEL");
  return v && strcmp(v, "pair") == 0;
}

// Largest number of 2-CTA clusters of the pair kernel resident at once (0: none).
template <bool FULL>
static int pair_max_clusters(size_t smem) {
  static int cached = -1;
  static size_t cached_smem = 0;
  if (cached >= 0 && cached_smem == smem) return cached;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2, 1, 1);
  cfg.blockDim = dim3(tc::kPairThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, tc::k_layer_pair<FULL>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cached = n;
  cached_smem = smem;
  return n;
}

// The stream layer on CTA pairs (output columns in tiles of 128); false when this device
// or shape cannot run it (nothing launched).
template <bool FULL>
static bool launch_layer_pair(const CUtensorMap& ta, const CUtensorMap& tbp, const CUtensorMap& ty,
                              const tc::TcArgs& a, size_t smem, cudaStream_t st) {
  static int regs_ok = -1;
  if (regs_ok < 0) {
    cudaFuncAttributes fa;
    regs_ok = cudaFuncGetAttributes(&fa, tc::k_layer_pair<FULL>) == cudaSuccess &&
              fa.numRegs >= tc::kPairLaunchRegs;
    cudaGetLastError();
  }
  if (!regs_ok) return false;
  if (cudaFuncSetAttribute(tc::k_layer_pair<FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int ctiles = a.h1 / 128;
  const int clusters = pair_max_clusters<FULL>(smem);
  if (clusters < ctiles) return false;
  const int pairs = (a.tiles + 1) / 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * ctiles, std::min(pairs, clusters / ctiles), 1);
  cfg.blockDim = dim3(tc::kPairThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, tc::k_layer_pair<FULL>, ta, tbp, ty, a) != cudaSuccess) {
    cudaGetLastError();          // a refused launch is not an error of the call: the caller falls back
    return false;
  }
  return true;
}

// Stream layer on the tensor cores; returns false (nothing launched) if a tensor map could not be built.
bool launch_layer_tc(const Shape& sh, const void* X, int ldx, int k_self, int lo_col0, const void* Vs16,
                     const float* Mterm, void* Y, int ldy, int residual, float* act_out, int h1, int* status,
                     cudaStream_t st) {
  const int nt = tc_columns(h1);
  CUtensorMap ta, tb;
  // slabs 0..T-1 and their low parts (slabs T..2T-1)
  if (!make_map(&ta, X, k_self, (int64_t)2 * sh.T * sh.R, ldx, 128)) return false;
  if (!make_map(&tb, Vs16, ldx + k_self, h1, 2 * ldx, nt)) return false;
  tc::TcArgs a{};
  a.sh = sh;
  a.nkb = (k_self + tc::kBlockK - 1) / tc::kBlockK;
  a.nt = nt;
  a.h1 = h1;
  a.status = status;
  a.Mterm = Mterm;
  a.X = (const __nv_bfloat16*)X;
  a.ldx = ldx;
  a.Y = (__nv_bfloat16*)Y;
  a.ldy = ldy;
  a.residual = residual;
  a.act_out = act_out;
  a.bsplit = ldx;
  a.alo_row = (int64_t)sh.T * sh.R;
  a.kb_lo_t = lo_col0 / tc::kBlockK;
  // stage M[t] in shared memory when the tile's walkers fit beside the ring
  a.mt_stage = tc_smem_bytes(nt, tc::kEpiLayer, true, sh.wpt, residual != 0) <= kMaxDynamicSmem ? 1 : 0;
  const bool full = sh.T > 1;
  a.tmem_cols = pow2_cols(full ? 4 * nt : 2 * nt);
  a.tiles = sh.tiles;
  // weights resident in shared memory when they fit beside an A ring of two or more stages
  if (nt == 128 && layer_pair_enabled()) {
    // CTA pairs: each CTA holds half of the weight tile; A ring as deep as shared memory allows
    int pstages = 0;
    while (pstages < 8 && tc::pair_layout(a.nkb, pstages + 1, sh.N).total <= kMaxDynamicSmem) ++pstages;
    CUtensorMap tbp, ty;
    if (pstages >= 3 && make_map(&tbp, Vs16, ldx + k_self, h1, 2 * ldx, 64) &&
        make_store_map(&ty, Y, ldy, (int64_t)(sh.T + 1) * sh.R, ldy, 32)) {
      tc::TcArgs ap = a;
      ap.stages = pstages;
      ap.tmem_cols = 512;
      const size_t smem = tc::pair_layout(a.nkb, pstages, sh.N).total;
      if (full ? launch_layer_pair<true>(ta, tbp, ty, ap, smem, st) : launch_layer_pair<false>(ta, tbp, ty, ap, smem, st))
        return true;
    }
  }
  const uint32_t b_bytes = tc::res_layout(a.nkb, nt, 0, sh.wpt).b_bytes;
  int stages = 0;
  while (stages < 8 && tc::res_layout(a.nkb, nt, stages + 1, sh.wpt).total <= kMaxDynamicSmem) ++stages;
  if (b_bytes > 0 && stages >= 2) {
    a.stages = stages;
    // two accumulators of 2 nt columns (A W_hi | A W_lo); h and sum z^2 live in registers
    a.tmem_cols = pow2_cols(4 * nt);
    // output tiles of 16 columns x 32 rows (tangent slabs), no swizzle
    CUtensorMap ty;
    const int64_t y_rows = (int64_t)(sh.T + 1) * sh.R;        // slabs 0..T-1 and the value's low part
    if (!make_store_map(&ty, Y, ldy, y_rows, ldy)) return false;
    const size_t smem = tc::res_layout(a.nkb, nt, stages, sh.wpt).total;
    const dim3 grid = persistent_grid(h1 / nt, sh.tiles);
    if (full) {
      cudaFuncSetAttribute(tc::k_layer_res<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      tc::k_layer_res<true><<<grid, tc::kResThreads, smem, st>>>(ta, tb, ty, a);
    } else {
      cudaFuncSetAttribute(tc::k_layer_res<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      tc::k_layer_res<false><<<grid, tc::kResThreads, smem, st>>>(ta, tb, ty, a);
    }
    return true;
  }
  launch_tc<tc::kEpiLayer>(ta, tb, a, persistent_grid(h1 / nt, sh.tiles), full, st);
  return true;
}

// C[rows][ncols] (row stride ldc, fp32) = A[rows][k] B[ncols][k]^T (+ bias[col] on rows <
// bias_rows), or C += A B^T by atomic adds with the k range split over `ksplit` CTAs per
// output tile.  A: bf16 K-major, row stride lda elements.  B: bf16 K-major, row stride ldb;
// with bsplit > 0 it holds bf16(W) in columns [0, k) and bf16(W - bf16(W)) in
// [bsplit, bsplit + k), and both are multiplied.  With a_lo_row > 0, A row a_lo_row + r
// holds the low part of row r (a hi/lo BF16 pair), multiplied by the high part of B in
// extra k-blocks.  Returns false (nothing launched) if a tensor map could not be built or
// the shapes are outside what the kernel covers.
bool launch_gemm_tc(int rows, int k, const void* A, int lda, const void* Bw, int ldb, int bsplit, int ncols, float* C,
                    int ldc, const float* bias, int bias_rows, int ksplit, bool atomic, int* status, cudaStream_t st,
                    int a_lo_row) {
  if (rows <= 0 || k <= 0 || ncols <= 0) return true;
  const int nt = ncols >= 128 ? 128 : (ncols > 64 ? 128 : (ncols > 32 ? 64 : 32));
  const int ctiles = (ncols + nt - 1) / nt;
  const int nkb = (k + tc::kBlockK - 1) / tc::kBlockK;
  ksplit = std::max(1, std::min(ksplit, nkb));
  if (ksplit > 1 && !atomic) return false;
  if (a_lo_row > 0 && (ksplit > 1 || a_lo_row < rows)) return false;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, k, a_lo_row > 0 ? (int64_t)a_lo_row + rows : rows, lda, 128)) return false;
  if (!make_map(&tb, Bw, bsplit ? bsplit + k : k, ncols, ldb, nt)) return false;
  tc::TcArgs a{};
  a.sh.T = 1;
  a.nkb = nkb;
  a.nt = nt;
  a.h1 = ncols;
  a.status = status;
  a.rows = rows;
  a.C = C;
  a.ldc = ldc;
  a.bias = bias;
  a.bias_rows = bias_rows;
  a.bsplit = bsplit;
  a.ksplit = ksplit;
  a.atomic = atomic ? 1 : 0;
  a.alo_row = a_lo_row;
  a.tmem_cols = pow2_cols(2 * nt);
  a.tiles = (rows + 127) / 128 * ksplit;
  launch_tc<tc::kEpiPlain>(ta, tb, a, persistent_grid(ctiles, a.tiles), false, st);
  return true;
}

// Orbitals: Phi (double) from h_L (bf16) and the bf16 orbital weights [K (n_up + n_dn)][h1].
bool launch_orbitals_tc(const Shape& sh, const void* HL, int h1, const void* W16, const float* const* wbias,
                        const float* const* pi, const float* const* sig, int K, int aniso, const float* walkers,
                        const double* nuclei, void* Phi, int64_t PW, float* orbP, const float* envv, int* status,
                        cudaStream_t st) {
  const int nmax = std::max(sh.n_up, sh.n_dn);
  const int nt = (int)std::min<int64_t>(128, round_up((int64_t)K * nmax, 32));
  CUtensorMap ta, tb;
  if (!make_map(&ta, HL, h1, (int64_t)(sh.T + 1) * sh.R, h1, 128)) return false;
  if (!make_map(&tb, W16, 2 * h1, (int64_t)K * sh.N, 2 * h1, nt)) return false;
  tc::TcArgs a{};
  a.sh = sh;
  a.nkb = (h1 + tc::kBlockK - 1) / tc::kBlockK;
  a.nt = nt;
  a.h1 = h1;
  a.status = status;
  for (int q = 0; q < 2; ++q) { a.wbias[q] = wbias[q]; a.pi[q] = pi[q]; a.sig[q] = sig[q]; }
  a.walkers = walkers;
  a.nuclei = nuclei;
  a.K = K;
  a.aniso = aniso;
  a.ctiles_up = (K * sh.n_up + nt - 1) / nt;
  const int ctiles_dn = (K * sh.n_dn + nt - 1) / nt;
  a.Phi = (float*)Phi;
  a.PW = PW;
  a.orbP = orbP;
  a.bsplit = h1;
  a.envv = envv;
  a.alo_row = (int64_t)sh.T * sh.R;          // h_L: only the value slab has a low part
  a.kb_lo_t = a.nkb;
  const bool full = sh.T > 1;
  a.tmem_cols = pow2_cols(3 * nt);
  a.tiles = sh.tiles;
  launch_tc<tc::kEpiOrbital>(ta, tb, a, persistent_grid(a.ctiles_up + ctiles_dn, sh.tiles), full, st);
  return true;
}

}  // namespace fn
