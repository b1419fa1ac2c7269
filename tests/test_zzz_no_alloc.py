"""fn_log_psi_noalloc: log|psi| computed from the library's static scratch array.

Callers that cannot let a library allocate device memory (an external allocator owns
it, or the memory budget is fixed) use this entry point; it must give the same result as
fn_log_psi and as the FP64 oracle, whatever an earlier call left in the shared array, and
it must report device-side errors through fn_sync like every other call.  This file is
collected last so that a run stopping at the first failure has run every other test
first; it passes alone in a fresh process as well.
"""
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


@pytest.mark.parametrize("prec,name,make,ans,B", [
    (0, "LiH-", lambda: W.lih(-1), W.Ansatz(3, 24, 8, 3, "aniso"), 61),
    (1, "N2", W.n2, W.Ansatz(3, 32, 8, 2, "aniso"), 40),
    (2, "C", lambda: W.atom(6), W.Ansatz(3, 64, 16, 4, "aniso"), 48),
])
def test_noalloc_against_oracle(prec, name, make, ans, B):
    """log|psi| and sign of the no-allocation path against the FP64 oracle at the parameters
    and positions the GPU saw: 1e-10 absolute in FP64; in FP32, 1e-4 relative to
    max(1, |log psi|) times the condition number of the determinant sum,
    sum_k |D_k| / |sum_k D_k| (single-precision storage of every activation; near a node of
    psi the terms cancel and their rounding is amplified by that factor); in BF16-mixed mode
    the per-walker bound of the BF16 tests (1e-2 of max(1, |log psi|): activations stored
    with 8 to 16 significant bits)."""
    from oracle import ansatz, mcmc
    sysm = make()
    net, gpu = make_pair(sysm, ans, prec)
    npdt = np.float64 if prec == 0 else np.float32
    dt = torch.float64 if prec == 0 else torch.float32
    p = oracle_params(net, 3, 0.05).astype(npdt)
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, sysm.partial_charges, B, 3, 1.0,
                             dtype=npdt)
    lp, sg = gpu.log_psi_noalloc(to_dev(p, dt), to_dev(r, dt))
    gpu.sync()
    lp_ref, sg_ref = ansatz.log_psi(net, p.astype(np.float64), sysm.nuclei, r.astype(np.float64))
    lp = lp.cpu().numpy()
    scale = np.maximum(1.0, np.abs(lp_ref))
    if prec == 0:
        assert np.all(np.abs(lp - lp_ref) <= 1e-10)
    elif prec == 1:
        a_up, a_dn = ansatz.orbital_matrices(net, p.astype(np.float64), sysm.nuclei, r.astype(np.float64))
        l_k = ansatz.slogdet(a_up)[1] + ansatz.slogdet(a_dn)[1]
        cond = np.exp(l_k - lp_ref[:, None]).sum(1)
        assert np.all(np.abs(lp - lp_ref) <= 1e-4 * scale * cond)
    else:
        assert np.all(np.abs(lp - lp_ref) <= 1e-2 * scale)
    np.testing.assert_array_equal(sg.cpu().numpy(), sg_ref)


def test_noalloc_leftovers_and_status_word():
    """(1) A batch of non-finite walkers fills the shared array with NaN activations; the
    call records the non-finite result in the handle's status word and fn_sync reports
    FN_ERR_NUMERIC once, then FN_OK.  (2) A smaller batch of the same single-atom system
    then places its BF16 weight copies inside the region the first call filled with NaN;
    its layer-0 weight rows have zero padding (12 input columns stored with stride 16), so
    the result is finite and equal to fn_log_psi only if the call itself writes that
    padding.  Both calls use one stream, as the entry point requires."""
    import paper_2401_10287_gb300 as P
    sysm = W.atom(6)
    net, gpu = make_pair(sysm, W.Ansatz(3, 64, 16, 4, "aniso"), 2)
    p = to_dev(oracle_params(net, 5, 0.05).astype(np.float32), torch.float32)
    bad = torch.full((4096, sysm.n_electrons, 3), float("nan"), dtype=torch.float32, device="cuda")
    lp_bad, _ = gpu.log_psi_noalloc(p, bad)
    with pytest.raises(P.FnError) as err:
        gpu.sync()
    assert err.value.code == 5, str(err.value)
    assert not torch.isfinite(lp_bad).any()
    gpu.sync()                                   # the bit was cleared by the report
    from oracle import mcmc
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, None, 64, 6, 1.0,
                             dtype=np.float32)
    rd = to_dev(r, torch.float32)
    for _ in range(2):
        lp, sg = gpu.log_psi_noalloc(p, rd)
        lp_ref, sg_ref = gpu.log_psi(p, rd)
        gpu.sync()
        assert torch.isfinite(lp).all()
        tol = 1e-4 * np.maximum(1.0, np.abs(lp_ref.cpu().numpy()))
        assert np.all(np.abs(lp.cpu().numpy() - lp_ref.cpu().numpy()) <= tol)
        assert torch.equal(sg, sg_ref)


def test_noalloc_rejects_batches_beyond_the_scratch():
    import paper_2401_10287_gb300 as P
    sysm = W.n2()
    net, gpu = make_pair(sysm, W.Ansatz(4, 256, 32, 16, "aniso"), 1)
    p = gpu.init_params(0)
    walkers = torch.zeros((20000, 14, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(P.FnError) as err:
        gpu.log_psi_noalloc(p, walkers)
    assert err.value.code == 1 and "64 MiB" in str(err.value)
