// Device random numbers: Philox4x32-10 (Salmon et al., SC'11) and Box-Muller
// normals built on project-written log and sin/cos.
//
// Every floating-point step uses an explicitly rounded intrinsic (__dadd_rn,
// __dmul_rn, __ddiv_rn, __dsqrt_rn) so that the compiler can neither contract
// nor reorder it; the sequence of operations is fixed, which makes the draws
// reproducible bit for bit by any IEEE-754 implementation of the same
// definition:
//   uniforms  U1 = (m + 1) 2^-53 in (0, 1] and U2 = m 2^-53 in [0, 1), m the top
//             53 bits of a 64-bit word formed from two Philox output words;
//   log x     x = m 2^e with m in [sqrt(1/2), sqrt(2)), s = (m - 1)/(m + 1),
//             log x = e ln2 + 2 s sum_{k=0}^{11} s^{2k}/(2k+1) (Horner);
//   sincos    q = nearest quarter of u, f = u - q/4, t = 2 pi f, Taylor series of
//             sin t to t^17 and cos t to t^18 (Horner), rotated by q;
//   normals   z0 = sqrt(-2 log U1) cos(2 pi U2), z1 = sqrt(-2 log U1) sin(2 pi U2).
// Counter convention: normal j of stream (c1, c2, c3) uses counter
// (j >> 1, c1, c2, c3) and key (seed lo, seed hi); even j takes z0, odd j z1.
#pragma once
#include <stdint.h>

namespace fn {

enum : uint32_t { kStreamInit = 0, kStreamProposal = 1, kStreamAccept = 2, kStreamParams = 3 };

struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox10(U4 ctr, uint64_t seed) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t a = ctr.x, c = ctr.z;
    const uint32_t hi_a = __umulhi(0xD2511F53u, a), lo_a = 0xD2511F53u * a;
    const uint32_t hi_c = __umulhi(0xCD9E8D57u, c), lo_c = 0xCD9E8D57u * c;
    ctr.x = hi_c ^ ctr.y ^ k0;
    ctr.y = lo_c;
    ctr.z = hi_a ^ ctr.w ^ k1;
    ctr.w = lo_a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return ctr;
}

__device__ __forceinline__ double top53(uint32_t hi, uint32_t lo) {
  const uint64_t word = ((uint64_t)hi << 32) | (uint64_t)lo;
  return (double)(word >> 11);   // exact: < 2^53
}

// 2^-53 as an exactly representable constant
__device__ __forceinline__ double two_m53() { return 1.1102230246251565e-16; }

__device__ __forceinline__ double log_rn(double x) {
  int e;
  double m = frexp(x, &e);                       // exact, m in [0.5, 1)
  if (m < 0.7071067811865476) { m = __dmul_rn(m, 2.0); e -= 1; }
  const double s = __ddiv_rn(__dadd_rn(m, -1.0), __dadd_rn(m, 1.0));
  const double s2 = __dmul_rn(s, s);
  double p = __ddiv_rn(1.0, 23.0);
#pragma unroll
  for (int k = 10; k >= 0; --k) p = __dadd_rn(__dmul_rn(p, s2), __ddiv_rn(1.0, (double)(2 * k + 1)));
  const double log_m = __dmul_rn(__dmul_rn(s, 2.0), p);
  return __dadd_rn(__dmul_rn((double)e, 0.6931471805599453), log_m);
}

__device__ __forceinline__ void sincos2pi_rn(double u, double* s_out, double* c_out) {
  const double q = rint(__dmul_rn(u, 4.0));
  const double f = __dadd_rn(u, -__dmul_rn(q, 0.25));
  const double t = __dmul_rn(f, 6.283185307179586);
  const double t2 = __dmul_rn(t, t);
  // Taylor coefficients (-1)^k / (2k+1)! and (-1)^k / (2k)!, each an exact integer
  // reciprocal correctly rounded at compile time.
  const double sc[9] = {1.0, -1.0 / 6.0, 1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0,
                        -1.0 / 39916800.0, 1.0 / 6227020800.0, -1.0 / 1307674368000.0,
                        1.0 / 355687428096000.0};
  const double cc[10] = {1.0, -1.0 / 2.0, 1.0 / 24.0, -1.0 / 720.0, 1.0 / 40320.0,
                         -1.0 / 3628800.0, 1.0 / 479001600.0, -1.0 / 87178291200.0,
                         1.0 / 20922789888000.0, -1.0 / 6402373705728000.0};
  double ps = sc[8];
#pragma unroll
  for (int k = 7; k >= 0; --k) ps = __dadd_rn(__dmul_rn(ps, t2), sc[k]);
  const double sin_t = __dmul_rn(t, ps);
  double pc = cc[9];
#pragma unroll
  for (int k = 8; k >= 0; --k) pc = __dadd_rn(__dmul_rn(pc, t2), cc[k]);
  const double cos_t = pc;
  const int quad = ((int)q) & 3;
  double s, c;
  switch (quad) {
    case 0: s = sin_t; c = cos_t; break;
    case 1: s = cos_t; c = -sin_t; break;
    case 2: s = -sin_t; c = -cos_t; break;
    default: s = -cos_t; c = sin_t; break;
  }
  *s_out = s;
  *c_out = c;
}

// Box-Muller pair from one Philox block
__device__ __forceinline__ void normal_pair(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint64_t seed, double* z0, double* z1) {
  const U4 r = philox10(U4{c0, c1, c2, c3}, seed);
  const double u1 = __dmul_rn(__dadd_rn(top53(r.x, r.y), 1.0), two_m53());
  const double u2 = __dmul_rn(top53(r.z, r.w), two_m53());
  const double rad = __dsqrt_rn(__dmul_rn(log_rn(u1), -2.0));
  double s, c;
  sincos2pi_rn(u2, &s, &c);
  *z0 = __dmul_rn(rad, c);
  *z1 = __dmul_rn(rad, s);
}

__device__ __forceinline__ double normal_at(uint64_t j, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint64_t seed) {
  double z0, z1;
  normal_pair((uint32_t)(j >> 1), c1, c2, c3, seed, &z0, &z1);
  return (j & 1) ? z1 : z0;
}

__device__ __forceinline__ double log_uniform_accept(uint32_t walker, uint32_t step, uint64_t seed) {
  const U4 r = philox10(U4{0u, walker, step, (uint32_t)kStreamAccept}, seed);
  const double u = __dmul_rn(__dadd_rn(top53(r.x, r.y), 1.0), two_m53());
  return log_rn(u);
}

}  // namespace fn
