"""Pins of the oracle's random streams: library Philox, libm/mpmath, normal statistics."""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import rng

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_philox_matches_library_philox():
    """Philox4x32-10 against the Philox of Triton's CPU interpreter (a library, run as one)."""
    pytest.importorskip("triton")
    code = textwrap.dedent("""
        import numpy as np, torch, triton, triton.language as tl
        @triton.jit
        def k(out_ptr, seed, BLOCK: tl.constexpr):
            offs = tl.arange(0, BLOCK)
            a, b, c, d = tl.randint4x(seed, offs)
            tl.store(out_ptr + offs * 4 + 0, a)
            tl.store(out_ptr + offs * 4 + 1, b)
            tl.store(out_ptr + offs * 4 + 2, c)
            tl.store(out_ptr + offs * 4 + 3, d)
        for seed in (0, 1, 12345678901, 2**64 - 1):
            out = torch.zeros(64 * 4, dtype=torch.int32)
            k[(1,)](out, seed, BLOCK=64)
            np.savetxt(__import__('sys').stdout, out.numpy().view(np.uint32).reshape(1, -1), fmt='%d')
    """)
    env = dict(os.environ, TRITON_INTERPRET="1")
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=300)
    if res.returncode != 0:
        pytest.skip("Triton interpreter unavailable: " + res.stderr[-200:])
    rows = [np.array(line.split(), dtype=np.uint64) for line in res.stdout.strip().splitlines()]
    for seed, row in zip((0, 1, 12345678901, 2**64 - 1), rows):
        x = rng.philox4x32_10(np.arange(64), 0, 0, 0, seed)
        ours = np.stack(x, 1).reshape(-1)
        np.testing.assert_array_equal(ours, row)


def test_philox_counter_sensitivity():
    """Every counter word and key word changes about half of the output bits."""
    base = np.stack(rng.philox4x32_10(5, 6, 7, 8, 99), -1).astype(np.uint32)
    variants = [(5 ^ 1, 6, 7, 8, 99), (5, 6 ^ 1, 7, 8, 99), (5, 6, 7 ^ 1, 8, 99),
                (5, 6, 7, 8 ^ 1, 99), (5, 6, 7, 8, 99 ^ (1 << 40))]
    for v in variants:
        out = np.stack(rng.philox4x32_10(*v), -1).astype(np.uint32)
        flipped = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(out, base))
        assert 32 <= flipped <= 96


def test_uniform_bits_are_uniform():
    x = rng.philox4x32_10(np.arange(200000), 3, 0, 1, 7)
    u = rng.uniform_closed0(x[0], x[1])
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2 = np.sum((hist - 200000 / 64) ** 2 / (200000 / 64))
    assert chi2 < 120          # 63 d.o.f.; p ~ 1e-5
    assert rng.uniform_open0(np.uint64(0), np.uint64(0)) == 2.0 ** -53
    assert rng.uniform_open0(np.uint64(0xFFFFFFFF), np.uint64(0xFFFFFFFF)) == 1.0


def _ulp_err(ours, exact):
    return abs(float(ours) - float(exact)) / math.ulp(abs(float(exact)) or 1.0)


def test_fn_log_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    rs = np.random.default_rng(0)
    xs = np.concatenate([rs.uniform(0, 1, 3000), 2.0 ** -rs.uniform(0, 53, 3000),
                         [2.0 ** -53, 1.0, 0.5, 0.7071067811865476, 0.7071067811865475, 1 - 2**-53]])
    ours = rng.fn_log(xs)
    worst = max(_ulp_err(o, mpmath.log(mpmath.mpf(float(x)))) if x != 1.0 else abs(o)
                for o, x in zip(ours, xs))
    assert worst <= 2.0
    assert rng.fn_log(np.array([1.0]))[0] == 0.0


def test_fn_sincos2pi_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    rs = np.random.default_rng(1)
    us = np.concatenate([rs.uniform(0, 1, 4000), [0.0, 0.125, 0.25, 0.375, 0.5, 0.75, 1 - 2**-53]])
    s, c = rng.fn_sincos2pi(us)
    for u, so, co in zip(us, s, c):
        ang = 2 * mpmath.pi * mpmath.mpf(float(u))
        assert abs(so - float(mpmath.sin(ang))) <= 4 * 2.0 ** -53
        assert abs(co - float(mpmath.cos(ang))) <= 4 * 2.0 ** -53
    s0, c0 = rng.fn_sincos2pi(np.array([0.0]))
    assert s0[0] == 0.0 and c0[0] == 1.0


def test_normals_statistics():
    scipy_stats = pytest.importorskip("scipy.stats")
    z = rng.normals(11, np.uint64(0), np.uint64(0), np.uint64(0), np.arange(400000, dtype=np.uint64))
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-4
    # the two outputs of one Box-Muller pair are uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 0.01
