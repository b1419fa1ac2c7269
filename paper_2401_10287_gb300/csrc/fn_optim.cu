// Parameter updates and local-energy clipping of the VMC training loop.
//
// The training phase updates the network parameters with the Eq. 6 gradient between
// rounds of the electron sampler.  The method names no optimiser; the library offers
// Adam (Kingma & Ba 2015, Algorithm 1) and plain gradient descent on the flat parameter
// blob, and an optional clamp of the local energies to a window around their median
// before they enter Eq. 6 (lower median +- width * mean absolute deviation).
//
//   k_adam          elementwise over the P parameters, grid-stride; memory bound
//                   (4 reads + 3 writes of the blob dtype per parameter).
//   k_sgd           theta -= lr * g.
//   k_clip_energy   one CTA of 1024 threads: the lower median (rank floor((B - 1) / 2))
//                   by radix selection over the order-preserving 64-bit keys of the
//                   energies (8 passes of 8 bits, warp-aggregated shared-memory
//                   histograms), the mean absolute deviation by a block reduction in
//                   FP64, then the clamp.  The median is an exact member of the batch.
#include <math.h>

#include <algorithm>

#include "fn_internal.cuh"

namespace fn {

// ---- Adam / gradient descent -------------------------------------------------------------
template <typename P>
struct AdamCoef {
  P lr, b1, one_b1, b2, one_b2, eps;
  P d1, d2;   // bias-correction denominators 1 - beta1^t and 1 - beta2^t
};

template <typename P>
__global__ void k_adam(int64_t n, P* __restrict__ p, const P* __restrict__ g, P* __restrict__ m,
                       P* __restrict__ v, AdamCoef<P> c, int* __restrict__ status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const P gi = g[i];
    const P mi = c.b1 * m[i] + c.one_b1 * gi;
    const P vi = c.b2 * v[i] + c.one_b2 * (gi * gi);
    m[i] = mi;
    v[i] = vi;
    const P pi = p[i] - c.lr * (mi / c.d1) / (sqrt(vi / c.d2) + c.eps);
    p[i] = pi;
    bad |= !isfinite(pi);
  }
  if (bad) atomicOr(status, kStatusNonFinite);
}

template <typename P>
__global__ void k_sgd(int64_t n, P* __restrict__ p, const P* __restrict__ g, P lr, int* __restrict__ status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const P pi = p[i] - lr * g[i];
    p[i] = pi;
    bad |= !isfinite(pi);
  }
  if (bad) atomicOr(status, kStatusNonFinite);
}

static unsigned elementwise_grid(const fn_system* s, int64_t n) {
  const int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)std::max(1, s->sm_count) * 8;
  return (unsigned)std::max<int64_t>(1, std::min(blocks, cap));
}

template <class Mode>
void launch_adam(const fn_system* s, void* params, const void* grad, void* m, void* v, int64_t t, double lr,
                 double beta1, double beta2, double eps, cudaStream_t st) {
  using P = typename Mode::Par;
  AdamCoef<P> c;
  c.lr = (P)lr;
  c.b1 = (P)beta1;
  c.one_b1 = (P)(1.0 - beta1);
  c.b2 = (P)beta2;
  c.one_b2 = (P)(1.0 - beta2);
  c.eps = (P)eps;
  c.d1 = (P)(1.0 - pow(beta1, (double)t));
  c.d2 = (P)(1.0 - pow(beta2, (double)t));
  ProfScope ps(s->prof, kProfOptim, st);
  k_adam<P><<<elementwise_grid(s, s->P), 256, 0, st>>>(s->P, (P*)params, (const P*)grad, (P*)m, (P*)v, c,
                                                        s->ws.status);
}

template <class Mode>
void launch_sgd(const fn_system* s, void* params, const void* grad, double lr, cudaStream_t st) {
  using P = typename Mode::Par;
  ProfScope ps(s->prof, kProfOptim, st);
  k_sgd<P><<<elementwise_grid(s, s->P), 256, 0, st>>>(s->P, (P*)params, (const P*)grad, (P)lr, s->ws.status);
}

// ---- local-energy clipping ------------------------------------------------------------------
// Order-preserving map of an IEEE double to an unsigned 64-bit key: positive values get
// the sign bit set, negative values are bit-inverted, so unsigned order = numeric order.
__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_value(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

constexpr int kClipThreads = 1024;

__global__ void __launch_bounds__(kClipThreads) k_clip_energy(int B, const double* e, double width, double* out,
                                                               double* __restrict__ stats,
                                                               int* __restrict__ status) {
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long s_prefix;
  __shared__ unsigned int s_rank;
  __shared__ double red[kClipThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  // Radix selection of the element of rank (B - 1) / 2, most significant byte first.
  // Invariant: `rank` < number of keys whose bits above `shift` + 8 equal `prefix`.
  unsigned long long prefix = 0, mask = 0;
  unsigned int rank = (unsigned int)(B - 1) / 2u;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int b = tid; b < 256; b += kClipThreads) hist[b] = 0;
    __syncthreads();
    for (int64_t base = 0; base < B; base += kClipThreads) {   // uniform trip count: full warps below
      const int64_t i = base + tid;
      const bool in = i < B;
      const unsigned long long k = in ? order_key(e[i]) : 0ull;
      const bool hit = in && (k & mask) == prefix;
      const unsigned int bin = hit ? (unsigned int)((k >> shift) & 255ull) : 256u;
      const unsigned int peers = __match_any_sync(0xffffffffu, bin);
      if (hit && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned int)__popc(peers));
    }
    __syncthreads();
    if (wid == 0) {   // warp 0: lane l owns bins 8l .. 8l + 7
      unsigned int cnt[8], own = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        cnt[j] = hist[lane * 8 + j];
        own += cnt[j];
      }
      unsigned int incl = own;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned int excl = incl - own;
      if (rank >= excl && rank < incl) {
        unsigned int c = excl;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (rank < c + cnt[j]) {
            s_prefix = prefix | ((unsigned long long)(lane * 8 + j) << shift);
            s_rank = rank - c;
            break;
          }
          c += cnt[j];
        }
      }
    }
    __syncthreads();
    prefix = s_prefix;
    rank = s_rank;
    mask |= 0xffull << shift;
  }
  const double centre = key_value(prefix);

  // Mean absolute deviation from the centre.
  double acc = 0.0;
  for (int64_t i = tid; i < B; i += kClipThreads) acc += fabs(e[i] - centre);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    double x = red[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[0] = x;
  }
  __syncthreads();
  const double spread = red[0] / (double)B;

  // Clamp (every read of e is behind the barrier above, so out may alias e); the
  // comparisons keep a NaN energy as it is.
  const bool on = width > 0.0;
  const double lo = centre - width * spread, hi = centre + width * spread;
  for (int64_t i = tid; i < B; i += kClipThreads) {
    const double x = e[i];
    out[i] = on ? (x < lo ? lo : (x > hi ? hi : x)) : x;
  }
  if (tid == 0) {
    if (stats) {
      stats[0] = centre;
      stats[1] = spread;
    }
    if (!isfinite(spread)) atomicOr(status, kStatusNonFinite);
  }
}

void launch_clip_energy(const fn_system* s, int B, const double* e, double width, double* out, double* stats,
                        cudaStream_t st) {
  ProfScope ps(s->prof, kProfOptim, st);
  k_clip_energy<<<1, kClipThreads, 0, st>>>(B, e, width, out, stats, s->ws.status);
}

// ---- Eq. 1 estimator and the Eq. 6 weights ------------------------------------------------
// The VMC energy is the mean local energy over the walkers (Eq. 1) and its statistical
// error follows from their variance; Eq. 6 weights every walker by 2 (E_L - mean) / count.
// The moments [count, sum E_L, sum E_L^2] add up across batches (and across devices), so a
// batch split over several GPUs sums them (one all-reduce of three numbers) before the
// statistics or the weights are formed.  One CTA, FP64, fixed summation order.
constexpr int kStatThreads = 1024;

__global__ void __launch_bounds__(kStatThreads) k_energy_moments(int B, const double* __restrict__ e,
                                                                  double* __restrict__ mom) {
  __shared__ double s1[kStatThreads], s2[kStatThreads];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < B; i += kStatThreads) {
    const double x = e[i];
    a += x;
    b += x * x;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int off = kStatThreads / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      s1[threadIdx.x] += s1[threadIdx.x + off];
      s2[threadIdx.x] += s2[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    mom[0] = (double)B;
    mom[1] = s1[0];
    mom[2] = s2[0];
  }
}

__global__ void k_energy_stats(const double* __restrict__ mom, double* __restrict__ stats, int* __restrict__ status) {
  const double n = mom[0], mean = mom[1] / n;
  const double var = fmax(0.0, mom[2] / n - mean * mean);
  stats[0] = n;
  stats[1] = mean;
  stats[2] = var;
  if (!isfinite(mean) || !isfinite(var)) atomicOr(status, kStatusNonFinite);
}

__global__ void k_energy_weights_from(int B, const double* __restrict__ e, const double* __restrict__ mom,
                                      double* __restrict__ w) {
  const double n = mom[0], mean = mom[1] / n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x)
    w[i] = 2.0 * (e[i] - mean) / n;
}

void launch_energy_moments(const fn_system* s, int B, const double* e, double* mom, cudaStream_t st) {
  ProfScope ps(s->prof, kProfOptim, st);
  k_energy_moments<<<1, kStatThreads, 0, st>>>(B, e, mom);
}

void launch_energy_stats(const fn_system* s, const double* mom, double* stats, cudaStream_t st) {
  ProfScope ps(s->prof, kProfOptim, st);
  k_energy_stats<<<1, 1, 0, st>>>(mom, stats, s->d_status);
}

void launch_energy_weights_from(const fn_system* s, int B, const double* e, const double* mom, double* w,
                                cudaStream_t st) {
  ProfScope ps(s->prof, kProfOptim, st);
  k_energy_weights_from<<<elementwise_grid(s, B), 256, 0, st>>>(B, e, mom, w);
}

#define FN_INST_OPTIM(M)                                                                                        \
  template void launch_adam<M>(const fn_system*, void*, const void*, void*, void*, int64_t, double, double,      \
                               double, double, cudaStream_t);                                                    \
  template void launch_sgd<M>(const fn_system*, void*, const void*, double, cudaStream_t);
FN_INST_OPTIM(ModeF64)
FN_INST_OPTIM(ModeF32)
FN_INST_OPTIM(ModeBF16)

}  // namespace fn
