"""fn_log_psi_noalloc: log|psi| computed from the library's static scratch array.

Callers that cannot let a library allocate device memory (an external allocator owns
it, or the memory budget is fixed) use this entry point; it must give the same result as
fn_log_psi.  This file is collected last so that a run stopping at the first failure has
run every other test first; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from gpu_helpers import make_pair, need_gpu, oracle_params, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec,ans,atol", [
    (0, W.Ansatz(3, 24, 8, 3, "aniso"), 1e-10),
    (1, W.Ansatz(3, 24, 8, 3, "aniso"), 1e-4),
    (2, W.Ansatz(3, 64, 16, 4, "aniso"), 1e-4),
])
def test_noalloc_matches_log_psi_two_calls(prec, ans, atol):
    from oracle import mcmc
    sysm = W.lih(-1)
    net, gpu = make_pair(sysm, ans, prec)
    dt = torch.float64 if prec == 0 else torch.float32
    npdt = np.float64 if prec == 0 else np.float32
    for call, (B, seed) in enumerate(((300, 1), (77, 2))):
        p = to_dev(oracle_params(net, seed, 0.05).astype(npdt), dt)
        r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, 3, 2, None, B, seed, 0.5, dtype=npdt)
        rd = to_dev(r, dt)
        lp_ref, sg_ref = gpu.log_psi(p, rd)
        lp, sg = gpu.log_psi_noalloc(p, rd)
        gpu.sync()
        tol = atol * np.maximum(1.0, np.abs(lp_ref.cpu().numpy()))
        assert np.all(np.abs(lp.cpu().numpy() - lp_ref.cpu().numpy()) <= tol), call
        assert torch.equal(sg, sg_ref), call


def test_noalloc_rejects_batches_beyond_the_scratch():
    import paper_2401_10287_gb300 as P
    sysm = W.n2()
    net, gpu = make_pair(sysm, W.Ansatz(4, 256, 32, 16, "aniso"), 1)
    p = gpu.init_params(0)
    walkers = torch.zeros((20000, 14, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(P.FnError) as err:
        gpu.log_psi_noalloc(p, walkers)
    assert err.value.code == 1 and "64 MiB" in str(err.value)
