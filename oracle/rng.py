"""Counter-based random numbers of the oracle (test infrastructure only).

The electron sampler draws Gaussian initial positions and Gaussian proposals
and a log-uniform acceptance variate (electron-sampler section).  To make the
CPU and GPU draws identical, both sides implement the same published
counter-based generator independently:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies with the
  multipliers 0xD2511F53 / 0xCD9E8D57 and the Weyl key increments
  0x9E3779B9 / 0xBB67AE85.
* 53-bit uniforms from two output words, Box-Muller normals.
* ``fn_log`` and ``fn_sincos2pi`` are written here from their series
  (log via 2*atanh((m-1)/(m+1)), sin/cos via Taylor series on a quarter-period
  reduced argument), using only IEEE add, multiply, divide and sqrt, each
  correctly rounded, in a fixed order with no fused multiply-add, so that the
  result is bit-identical on any IEEE-754 machine that follows the same
  sequence.

Counter convention (key = (seed low 32 bits, seed high 32 bits)):
  normal number j of stream (c1, c2, c3) comes from counter (j >> 1, c1, c2, c3),
  first Box-Muller output for even j, second for odd j.
  walker init:   c1 = walker, c2 = 0,    c3 = 0, j = 3*electron + axis
  proposal:      c1 = walker, c2 = step, c3 = 1, j = 3*electron + axis
  acceptance:    counter (0, walker, step, 2), words 0..1 -> U in (0, 1]
  parameters:    c1 = 0,      c2 = 0,    c3 = 3, j = parameter index
"""
from __future__ import annotations

import math

import numpy as np

_MASK32 = np.uint64(0xFFFFFFFF)
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85

PURPOSE_INIT = 0
PURPOSE_PROPOSAL = 1
PURPOSE_ACCEPT = 2
PURPOSE_PARAMS = 3


def philox4x32_10(c0, c1, c2, c3, seed: int):
    """Philox4x32-10 block function; counters are arrays of 32-bit values.

    Returns four uint64 arrays each holding a 32-bit output word.
    """
    x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) & _MASK32 for c in (c0, c1, c2, c3))
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    k0 = int(seed) & 0xFFFFFFFF
    k1 = (int(seed) >> 32) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _PHILOX_W0) & 0xFFFFFFFF
            k1 = (k1 + _PHILOX_W1) & 0xFFFFFFFF
        p0 = x0 * _PHILOX_M0           # < 2**64: exact in uint64
        p1 = x2 * _PHILOX_M1
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(k0), lo1, hi0 ^ x3 ^ np.uint64(k1), lo0)
    return x0, x1, x2, x3


def bits53(hi, lo):
    """Top 53 bits of the 64-bit word (hi:lo) as an integer-valued float64."""
    word = (np.asarray(hi, dtype=np.uint64) << np.uint64(32)) | np.asarray(lo, dtype=np.uint64)
    return (word >> np.uint64(11)).astype(np.float64)


_TWO_M53 = 2.0 ** -53


def uniform_open0(hi, lo):
    """U = (m + 1) * 2**-53 in (0, 1]; log U is always finite."""
    return (bits53(hi, lo) + 1.0) * _TWO_M53


def uniform_closed0(hi, lo):
    """U = m * 2**-53 in [0, 1)."""
    return bits53(hi, lo) * _TWO_M53


# Series coefficients, each the correctly rounded double of an exact rational.
_ATANH_COEF = [1.0 / (2 * k + 1) for k in range(12)]                      # 1, 1/3, ..., 1/23
_SIN_COEF = [(-1.0) ** k / float(math.factorial(2 * k + 1)) for k in range(9)]   # to t^17
_COS_COEF = [(-1.0) ** k / float(math.factorial(2 * k)) for k in range(10)]     # to t^18
_LN2 = 0.6931471805599453          # ln 2 rounded to double
_TWO_PI = 6.283185307179586        # 2*pi rounded to double
_SQRT_HALF = 0.7071067811865476    # sqrt(1/2) rounded to double


def fn_log(x):
    """Natural log for positive normal float64, from log m = 2 atanh((m-1)/(m+1)).

    x = m * 2**e with m in [sqrt(1/2), sqrt(2)); s = (m-1)/(m+1), |s| <= 0.172;
    the odd series 2 s (1 + s^2/3 + ... + s^22/23) is summed by Horner's rule.
    """
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # m in [0.5, 1)
    low = m < _SQRT_HALF
    m = np.where(low, m * 2.0, m)
    e = np.where(low, e - 1, e).astype(np.float64)
    s = (m - 1.0) / (m + 1.0)
    s2 = s * s
    p = np.full_like(s, _ATANH_COEF[11])
    for k in range(10, -1, -1):
        p = p * s2 + _ATANH_COEF[k]
    log_m = (s * 2.0) * p
    return e * _LN2 + log_m


def fn_sincos2pi(u):
    """(sin 2 pi u, cos 2 pi u) for u in [0, 1).

    q = rint(4u) picks the nearest quarter period, f = u - q/4 in [-1/8, 1/8]
    (exact), t = 2 pi f, and sin t, cos t come from their Taylor series to
    t^17 / t^18 (error below 2**-56 on |t| <= pi/4).  The quarter q rotates
    the pair.
    """
    u = np.asarray(u, dtype=np.float64)
    q = np.rint(u * 4.0)
    f = u - q * 0.25
    t = f * _TWO_PI
    t2 = t * t
    ps = np.full_like(t, _SIN_COEF[8])
    for k in range(7, -1, -1):
        ps = ps * t2 + _SIN_COEF[k]
    sin_t = t * ps
    pc = np.full_like(t, _COS_COEF[9])
    for k in range(8, -1, -1):
        pc = pc * t2 + _COS_COEF[k]
    cos_t = pc
    quad = q.astype(np.int64) & 3
    s = np.select([quad == 0, quad == 1, quad == 2, quad == 3], [sin_t, cos_t, -sin_t, -cos_t])
    c = np.select([quad == 0, quad == 1, quad == 2, quad == 3], [cos_t, -sin_t, -cos_t, sin_t])
    return s, c


def box_muller(u1, u2):
    """Two standard normals from U1 in (0,1] and U2 in [0,1)."""
    rad = np.sqrt(fn_log(u1) * -2.0)
    s, c = fn_sincos2pi(u2)
    return rad * c, rad * s


def normals(seed: int, c1, c2, c3, j):
    """Normal number j of the stream (c1, c2, c3) (arrays broadcast)."""
    j = np.asarray(j, dtype=np.uint64)
    x0, x1, x2, x3 = philox4x32_10(j >> np.uint64(1), c1, c2, c3, seed)
    z0, z1 = box_muller(uniform_open0(x0, x1), uniform_closed0(x2, x3))
    return np.where((j & np.uint64(1)) == 0, z0, z1)


def walker_normals(seed: int, n_walkers: int, n_coords: int, step: int, purpose: int,
                   walker_offset: int = 0):
    """[n_walkers, n_coords] normals for the init (purpose 0) or proposal (purpose 1) stream."""
    w = np.arange(n_walkers, dtype=np.uint64)[:, None] + np.uint64(walker_offset)
    j = np.arange(n_coords, dtype=np.uint64)[None, :]
    return normals(seed, w, np.uint64(step & 0xFFFFFFFF), np.uint64(purpose), j)


def accept_log_uniform(seed: int, n_walkers: int, step: int, walker_offset: int = 0):
    """log U per walker, U in (0, 1] from words 0..1 of counter (0, walker, step, 2)."""
    w = np.arange(n_walkers, dtype=np.uint64) + np.uint64(walker_offset)
    x0, x1, _, _ = philox4x32_10(np.uint64(0), w, np.uint64(step & 0xFFFFFFFF),
                                 np.uint64(PURPOSE_ACCEPT), seed)
    return fn_log(uniform_open0(x0, x1))
