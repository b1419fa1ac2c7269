// Tiled SIMT GEMM with arbitrary strides (transposes by stride), optional bias on the
// first rows and split-K accumulation by atomics.  Used for the mean-field term of the
// forward pass and for the parameter-gradient contractions of the backward pass.
#pragma once
#include <algorithm>

#include "fn_device.cuh"

namespace fn {

// ---------------------------------------------------------------------------------------
// tiled SIMT GEMM: C(m,n) (+)= sum_k A(m,k) B(k,n) + bias[n] (rows m < bias_rows)
// ---------------------------------------------------------------------------------------
template <typename TA, typename TB, typename TC, typename Cmp>
__global__ void __launch_bounds__(256) k_gemm(int Mr, int Nc, int Kd, const TA* __restrict__ A, int64_t sam,
                                              int64_t sak, const TB* __restrict__ Bm, int64_t sbk, int64_t sbn,
                                              TC* __restrict__ C, int64_t scm, int64_t scn,
                                              const Cmp* __restrict__ bias, int64_t bias_rows, int atomic_acc) {
  __shared__ Cmp As[16][64 + 1];
  __shared__ Cmp Bs[16][64 + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
  const int kchunk = (Kd + gridDim.z - 1) / gridDim.z;
  const int kbeg = blockIdx.z * kchunk, kend = min(Kd, kbeg + kchunk);
  Cmp acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int e = tid; e < 16 * 64; e += 256) {
      const int kk = e / 64, mm = e % 64;
      const int64_t m = m0 + mm;
      const int k = k0 + kk;
      As[kk][mm] = (m < Mr && k < kend) ? (Cmp)ld(A + m * sam + k * sak) : (Cmp)0;
      const int64_t n = n0 + mm;
      Bs[kk][mm] = (n < Nc && k < kend) ? (Cmp)ld(Bm + k * sbk + n * sbn) : (Cmp)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      Cmp av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { av[q] = As[kk][ty * 4 + q]; bv[q] = Bs[kk][tx * 4 + q]; }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[q][p] += av[q] * bv[p];
    }
    __syncthreads();
  }
  for (int q = 0; q < 4; ++q) {
    const int64_t m = m0 + ty * 4 + q;
    if (m >= Mr) continue;
    for (int p = 0; p < 4; ++p) {
      const int64_t n = n0 + tx * 4 + p;
      if (n >= Nc) continue;
      Cmp v = acc[q][p];
      if (bias && m < bias_rows && blockIdx.z == 0) v += bias[n];
      TC* o = C + m * scm + n * scn;
      if (atomic_acc) atomicAdd(o, (TC)v);
      else st(o, v);
    }
  }
}

template <typename TA, typename TB, typename TC, typename Cmp>
inline void gemm(cudaStream_t st, int Mr, int Nc, int Kd, const TA* A, int64_t sam, int64_t sak, const TB* Bm,
          int64_t sbk, int64_t sbn, TC* C, int64_t scm, int64_t scn, const Cmp* bias, int64_t bias_rows,
          int split_k, bool atomic_acc) {
  if (Mr <= 0 || Nc <= 0 || Kd <= 0) return;
  dim3 grid((Nc + 63) / 64, (Mr + 63) / 64, std::max(1, split_k));
  k_gemm<TA, TB, TC, Cmp><<<grid, 256, 0, st>>>(Mr, Nc, Kd, A, sam, sak, Bm, sbk, sbn, C, scm, scn, bias,
                                                 bias_rows, (atomic_acc || split_k > 1) ? 1 : 0);
}

}  // namespace fn
