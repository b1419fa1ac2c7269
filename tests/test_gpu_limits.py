"""The library at its size limits, against the oracle, with ragged walker counts.

The per-walker kernels hold one walker's pair activations (N^2 rows of up to 32 channels)
or its determinant matrices (2K matrices of n x n with their 3N tangent traces) in shared
memory, so the largest electron count, determinant count and depth depend on the mode:
FP32 reaches N = 32 (16 + 16) and, at 16 electrons of one spin, K = 32; FP64 reaches
N = 29 with 2 layers and N = 25 with 8; BF16 reaches N = 29 (the pair-stream gradient);
FP64 and BF16 reach K = 16 at 16 electrons of a spin.  Each dimension is taken to its
maximum on its own (h1 = 1024, K = 64 with 2 electrons per spin, 8 layers, 16 + 16
electrons), and one step beyond must be refused when the system is created."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import ansatz, mcmc
from gpu_helpers import make_pair, need_gpu, oracle_params, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    torch.cuda.synchronize()


def _system(name, z_a, z_b, n_up, n_dn, bond):
    s = W.diatomic(name, z_a, z_b, bond)
    return W.System(name, s.nuclei, s.charges, n_up, n_dn, None)


CASES = {
    # name: (system factory, ansatz, walkers)
    "S2 16+16": (lambda: _system("S2", 16, 16, 16, 16, 3.57), W.Ansatz(2, 32, 8, 2, "aniso"), 5),
    "PSi 15+14": (lambda: _system("PSi", 15, 14, 15, 14, 4.0), W.Ansatz(2, 32, 8, 2, "aniso"), 5),
    "AlMg 13+12, 8 layers": (lambda: _system("AlMg", 13, 12, 13, 12, 5.0), W.Ansatz(8, 32, 8, 2, "aniso"), 3),
    "O2 16+0, K=16": (lambda: _system("O2", 8, 8, 16, 0, 2.28), W.Ansatz(2, 32, 8, 16, "aniso"), 3),
    "LiH K=64": (lambda: W.lih(0), W.Ansatz(2, 32, 8, 64, "aniso"), 7),
    "H2 h1=1024": (W.h2, W.Ansatz(2, 1024, 32, 1, "iso"), 3),
    "LiH+ 8 layers": (lambda: W.lih(1), W.Ansatz(8, 64, 16, 2, "aniso"), 9),
}


def _fp_case(name, prec):
    make, ans, B = CASES[name]
    sysm = make()
    net, gpu = make_pair(sysm, ans, prec)
    npdt = np.float64 if prec == 0 else np.float32
    dt = torch.float64 if prec == 0 else torch.float32
    p = oracle_params(net, 0, 0.05).astype(npdt).astype(np.float64)
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, None, B, 1, 1.0, dtype=npdt)
    e, lp, sg = gpu.local_energy(to_dev(p, dt), to_dev(r, dt))
    lp2, sg2 = gpu.log_psi(to_dev(p, dt), to_dev(r, dt))
    gpu.sync()
    r64 = r.astype(np.float64)
    e_ref, lp_ref, sg_ref = ansatz.local_energy(net, p, sysm.nuclei, sysm.charges, r64)
    return (e.cpu().numpy(), lp.cpu().numpy(), sg.cpu().numpy(), lp2.cpu().numpy(), sg2.cpu().numpy()), \
        (e_ref, lp_ref, sg_ref), (net, sysm, p, r64)


@pytest.mark.parametrize("name", ["PSi 15+14", "AlMg 13+12, 8 layers", "O2 16+0, K=16", "LiH K=64", "H2 h1=1024",
                                  "LiH+ 8 layers"])
def test_limits_fp64_match_oracle(name):
    (e, lp, sg, lp2, sg2), (e_ref, lp_ref, sg_ref), _ = _fp_case(name, 0)
    np.testing.assert_array_equal(sg, sg_ref)
    np.testing.assert_array_equal(sg2, sg_ref)
    np.testing.assert_allclose(lp, lp_ref, rtol=0, atol=1e-10 * np.maximum(1.0, np.abs(lp_ref)).max())
    np.testing.assert_allclose(lp2, lp_ref, rtol=0, atol=1e-10 * np.maximum(1.0, np.abs(lp_ref)).max())
    assert np.all(np.abs(e - e_ref) <= 1e-8 * np.maximum(1.0, np.abs(e_ref)))


@pytest.mark.parametrize("name", ["S2 16+16", "LiH K=64", "LiH+ 8 layers"])
def test_limits_fp32_match_oracle(name):
    """FP32 bound of the parity tests: 1e-4 relative to the kinetic-term scale."""
    (e, lp, sg, _, _), (e_ref, lp_ref, sg_ref), (net, sysm, p, r) = _fp_case(name, 1)
    _, _, grad, lap = ansatz.log_psi_derivatives(net, p, sysm.nuclei, r)
    scale = np.maximum(np.maximum(1.0, np.abs(e_ref)), 0.5 * (np.sum(grad * grad, -1) + np.abs(lap)))
    assert np.all(np.abs(lp - lp_ref) <= 1e-4 * np.maximum(1.0, np.abs(lp_ref)))
    assert np.all(np.abs(e - e_ref) / scale <= 1e-4)


@pytest.mark.parametrize("name", ["PSi 15+14", "O2 16+0, K=16", "LiH K=64", "H2 h1=1024", "LiH+ 8 layers"])
def test_limits_bf16_against_oracle(name):
    """BF16-mixed at the limits: walkers equilibrated by the oracle's chain, median error
    relative to the kinetic-term scale below 1e-2 as in the BF16 parity tests, and a finite
    Eq. 6 gradient (which runs the pair-stream backward at its largest N)."""
    make, ans, B = CASES[name]
    sysm = make()
    net, gpu = make_pair(sysm, ans, 2)
    B = max(B, 8)
    p = oracle_params(net, 0, 0.05).astype(np.float32).astype(np.float64)
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, None, B, 1, 1.0)
    lp0, _ = ansatz.log_psi(net, p, sysm.nuclei, r)
    r, _, _ = mcmc.metropolis(net, p, sysm.nuclei, r, lp0, 2, 60, 0.3)
    r32 = r.astype(np.float32)
    pd, rd = to_dev(p, torch.float32), to_dev(r32, torch.float32)
    e, lp, _ = gpu.local_energy(pd, rd)
    g, _ = gpu.energy_grad(pd, rd, e)
    gpu.sync()
    r64 = r32.astype(np.float64)
    e_ref, lp_ref, _ = ansatz.local_energy(net, p, sysm.nuclei, sysm.charges, r64)
    _, _, grad, lap = ansatz.log_psi_derivatives(net, p, sysm.nuclei, r64)
    scale = np.maximum(np.maximum(1.0, np.abs(e_ref)), 0.5 * (np.sum(grad * grad, -1) + np.abs(lap)))
    rel = np.abs(e.cpu().numpy() - e_ref) / scale
    assert np.median(rel) < 1e-2, (np.median(rel), rel.max())
    assert np.all(np.isfinite(g.cpu().numpy()))


@pytest.mark.parametrize("prec,n_up,n_dn,L,K,stage", [
    (0, 16, 16, 2, 2, "two-electron stream, value pass"),     # FP64 pair activations of 32 electrons
    (2, 16, 16, 2, 2, "two-electron stream, gradient"),       # BF16 pair backward of 32 electrons
    (0, 13, 13, 8, 2, "two-electron stream, value pass"),     # FP64, 26 electrons with 8 layers
    (0, 16, 0, 2, 17, "determinant stage"),                   # FP64, 16 electrons of a spin, K = 17
    (1, 16, 0, 2, 33, "determinant stage"),                   # FP32, K = 33
])
def test_beyond_the_limits_is_refused_at_creation(prec, n_up, n_dn, L, K, stage):
    import paper_2401_10287_gb300 as P
    s = W.diatomic("X", 16, 16, 3.0)
    with pytest.raises(P.FnError) as err:
        P.System(s.nuclei, s.charges, n_up, n_dn, P.NetConfig(L, 32, 8, K, P.ANISO, prec))
    assert err.value.code == 7
    assert stage in str(err.value) and "shared memory" in str(err.value)
