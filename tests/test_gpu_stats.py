"""Eq. 1 estimator and Eq. 6 weights in the library (fn_energy_moments, fn_energy_stats,
fn_energy_weights) against the plain formulas in FP64 on the host, including moments summed
over two batches as a data-parallel run sums them."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_helpers import make_pair, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    torch.cuda.synchronize()


@pytest.mark.parametrize("B", [1, 7, 1024, 40000])
def test_energy_moments_stats_weights(B):
    _, gpu = make_pair(W.h2(), W.Ansatz(2, 32, 8, 1, "iso"), 0)
    e = np.random.default_rng(B).normal(-109.0, 3.0, B)
    ed = torch.as_tensor(e).cuda()
    mom = gpu.energy_moments(ed)
    st = gpu.energy_stats(mom)
    w = gpu.energy_weights(ed, mom)
    gpu.sync()
    mom, st, w = mom.cpu().numpy(), st.cpu().numpy(), w.cpu().numpy()
    assert mom[0] == B
    assert abs(mom[1] - e.sum()) <= 1e-12 * np.abs(e).sum()
    assert abs(mom[2] - (e * e).sum()) <= 1e-12 * (e * e).sum()
    assert abs(st[1] - e.mean()) <= 1e-12 * abs(e.mean())
    # the variance formed from the moments loses digits to the mean^2 / var ratio (1e3 here)
    assert abs(st[2] - e.var()) <= 1e-9 * max(e.var(), 1e-300) + 1e-12 * e.mean() ** 2
    np.testing.assert_allclose(w, 2.0 * (e - e.mean()) / B, rtol=0, atol=1e-12 * np.abs(e).max() / B * 4)


def test_moments_of_two_batches_add_up():
    _, gpu = make_pair(W.h2(), W.Ansatz(2, 32, 8, 1, "iso"), 0)
    e = np.random.default_rng(3).normal(-1.1, 0.2, 37)
    a, b = torch.as_tensor(e[:20]).cuda(), torch.as_tensor(e[20:]).cuda()
    mom = gpu.energy_moments(a) + gpu.energy_moments(b)
    st = gpu.energy_stats(mom)
    w = gpu.energy_weights(a, mom)
    gpu.sync()
    assert st[0].item() == 37
    assert abs(st[1].item() - e.mean()) < 1e-14
    np.testing.assert_allclose(w.cpu().numpy(), 2.0 * (e[:20] - e.mean()) / 37, rtol=0, atol=1e-15)
