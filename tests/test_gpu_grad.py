"""Energy gradient (Eq. 6) of the CUDA backward against central finite differences of the
FP64 oracle (h = 1e-5, Richardson-extrapolated with h/2 to remove the O(h^2) term), on 32
random parameter indices and along a random direction."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import ansatz, grad, mcmc
from gpu_helpers import make_pair, need_gpu, oracle_params, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    torch.cuda.synchronize()


def _case(sysm, ans, prec, B, seed=0, std=0.5, perturb=0.05):
    net, gpu = make_pair(sysm, ans, prec)
    p = oracle_params(net, seed, perturb)
    dt_np = np.float64 if prec == 0 else np.float32
    dt = torch.float64 if prec == 0 else torch.float32
    p = p.astype(dt_np).astype(np.float64)
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, sysm.partial_charges, B, seed + 3,
                             std, dtype=dt_np)
    e = np.random.default_rng(seed).normal(-8.0, 1.0, B)    # any fixed local energies
    g, mean = gpu.energy_grad(to_dev(p, dt), to_dev(r, dt), torch.as_tensor(e).cuda())
    gpu.sync()
    return net, gpu, p, r.astype(np.float64), e, g.cpu().numpy().astype(np.float64), float(mean.item())


@pytest.mark.parametrize("make", [lambda: W.lih(1), lambda: W.lih(-1), W.h2, W.n2])
def test_energy_grad_fp64_against_fd(make):
    sysm = make()
    ans = W.Ansatz(3, 16, 8, 3, "aniso")
    net, gpu, p, r, e, g, mean = _case(sysm, ans, 0, 24)
    assert abs(mean - e.mean()) < 1e-12
    idx = np.random.default_rng(1).choice(p.shape[0], 32, replace=False)
    g_fd = grad.energy_gradient_richardson(net, p, sysm.nuclei, r, e, idx, h=1e-5)
    np.testing.assert_allclose(g[idx], g_fd, rtol=1e-5, atol=1e-6 * max(1.0, np.abs(g_fd).max()))
    v = np.random.default_rng(2).standard_normal(p.shape[0])
    v /= np.linalg.norm(v)
    d = grad.directional_richardson(net, p, sysm.nuclei, r, e, v, h=1e-5)
    assert abs(g @ v - d) <= 1e-5 * max(1.0, abs(d))


def test_energy_grad_iso_envelope_fp64():
    sysm = W.h2()
    ans = W.Ansatz(2, 32, 8, 1, "iso")
    net, gpu, p, r, e, g, mean = _case(sysm, ans, 0, 50, std=1.0)
    v = np.random.default_rng(3).standard_normal(p.shape[0])
    v /= np.linalg.norm(v)
    d = grad.directional_richardson(net, p, sysm.nuclei, r, e, v, h=1e-5)
    assert abs(g @ v - d) <= 1e-5 * max(1.0, abs(d))


@pytest.mark.parametrize("charge", [1, -1])
def test_energy_grad_lih_ions_fp64_full_size(charge):
    """The same workload in FP64: the backward itself agrees with the Richardson differences
    to 1e-7 relative to the summed term magnitudes."""
    sysm = W.lih(charge)
    ans = W.Ansatz(4, 128, 16, 8, "aniso")
    net, gpu, p, r, e, g, mean = _case(sysm, ans, 0, 4096, seed=4, perturb=0.0)
    idx = np.random.default_rng(4).choice(p.shape[0], 32, replace=False)
    g_fd = grad.energy_gradient_richardson(net, p, sysm.nuclei, r, e, idx, h=1e-5)
    terms = grad.term_magnitude_fd(net, p, sysm.nuclei, r, e, idx, h=1e-5)
    ratio = np.abs(g[idx] - g_fd) / terms
    assert np.all(ratio <= 1e-7), (ratio.max(), np.median(ratio))


@pytest.mark.parametrize("charge", [1, -1])
def test_energy_grad_lih_ions_fp32_full_size(charge):
    """LiH+/LiH- workload: 4 layers 128/16, 8 determinants, anisotropic envelopes, 4096 walkers
    initialised N(0, 0.5) around the atoms chosen by Algorithm 1, FP32; 32 random indices.
    FP32 bound: relative to the summed term magnitudes sum_w |c_w d log|psi_w||, the scale an
    FP32 sum of those terms is accurate to, 1e-3 for every index and 3e-4 for the median: each
    walker's term carries the FP32 error of its determinant inverse, about kappa(A) * 6e-8
    with orbital-matrix condition numbers in the hundreds at random initialisation."""
    sysm = W.lih(charge)
    ans = W.Ansatz(4, 128, 16, 8, "aniso")
    net, gpu, p, r, e, g, mean = _case(sysm, ans, 1, 4096, seed=4, perturb=0.0)
    idx = np.random.default_rng(4).choice(p.shape[0], 32, replace=False)
    g_fd = grad.energy_gradient_richardson(net, p, sysm.nuclei, r, e, idx, h=1e-5)
    terms = grad.term_magnitude_fd(net, p, sysm.nuclei, r, e, idx, h=1e-5)
    ratio = np.abs(g[idx] - g_fd) / terms
    assert np.all(ratio <= 1e-3) and np.median(ratio) <= 3e-4, (ratio.max(), np.median(ratio))


def test_autograd_function_matches_library():
    import paper_2401_10287_gb300 as P
    sysm = W.lih(1)
    net, gpu = make_pair(sysm, W.Ansatz(2, 16, 8, 2, "aniso"), 0)
    params = gpu.init_params(3).requires_grad_(True)
    walkers, _ = gpu.init_walkers(64, 5, 0.5, sysm.partial_charges)
    e, _, _ = gpu.local_energy(params.detach(), walkers)
    loss = P.EnergyGrad.apply(params, walkers, e, gpu)
    loss.backward()
    g, mean = gpu.energy_grad(params.detach(), walkers, e)
    # split-K atomics reorder the FP64 sums between calls: equal to rounding
    torch.testing.assert_close(params.grad, g, rtol=1e-10, atol=1e-12)
    assert abs(float(loss.detach()) - float(e.mean())) < 1e-12


def test_log_psi_vjp_weights():
    """sum_w c_w d log|psi_w|: unit weight on one walker equals that walker's FD gradient."""
    sysm = W.lih(-1)
    net, gpu = make_pair(sysm, W.Ansatz(2, 16, 8, 2, "aniso"), 0)
    p = oracle_params(net, 7, 0.05)
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, 3, 2, None, 9, 1, 0.5)
    wts = np.zeros(9)
    wts[4] = 1.0
    g = gpu.log_psi_vjp(to_dev(p, torch.float64), to_dev(r, torch.float64), torch.as_tensor(wts).cuda())
    idx = np.random.default_rng(0).choice(p.shape[0], 16, replace=False)
    h = 1e-5
    for q in idx:
        pp, pm = p.copy(), p.copy()
        pp[q] += h
        pm[q] -= h
        fd = (ansatz.log_psi(net, pp, sysm.nuclei, r[4:5])[0] - ansatz.log_psi(net, pm, sysm.nuclei, r[4:5])[0]) / (2 * h)
        assert abs(g[q].item() - fd[0]) <= 1e-6 * max(1.0, abs(fd[0]))
