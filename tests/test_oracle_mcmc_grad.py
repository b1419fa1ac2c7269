"""Pins of the oracle sampler (detailed balance on a known density) and of the Eq. 6 gradient."""
import numpy as np
import pytest

import workloads as W
from oracle import ansatz, grad, mcmc, rng


def _hydrogen(env="iso"):
    s = W.hydrogen_atom()
    net = ansatz.Net(1, 1, 0, 1, 8, 4, 1, env)
    blob = ansatz.init_params(net, 0)
    p = ansatz.unpack(net, blob)
    p["w_up"][...] = 0.0
    p["g_up"][...] = 1.0
    return s, net, blob


def test_init_walkers_around_assigned_nuclei():
    s = W.lih(-1)
    r, counts = mcmc.init_walkers(s.nuclei, s.charges, s.n_up, s.n_down, None, 4000, 9, 0.5)
    assert counts == [4, 1]
    centres = s.nuclei[[0, 0, 1, 0, 0]]
    np.testing.assert_allclose(r.mean(0), centres, atol=0.05)
    np.testing.assert_allclose(r.std(0), 0.5, atol=0.03)


def test_proposal_zero_step_always_accepts():
    """step 0: r' = r, A = 0 and log U <= 0 for U in (0, 1]: ties accept."""
    s, net, blob = _hydrogen()
    r, _ = mcmc.init_walkers(s.nuclei, s.charges, 1, 0, None, 200, 0, 1.0)
    lp, _ = ansatz.log_psi(net, blob, s.nuclei, r)
    r2, lp2, acc = mcmc.metropolis(net, blob, s.nuclei, r, lp, 1, 3, 0.0)
    assert np.all(acc == 3)
    np.testing.assert_array_equal(r2, r)


@pytest.mark.slow
def test_detailed_balance_hydrogen_mean_radius():
    """|psi|^2 = exp(-2r): the exact mean radius is 3/2 bohr."""
    s, net, blob = _hydrogen()
    B = 4000
    r, _ = mcmc.init_walkers(s.nuclei, s.charges, 1, 0, None, B, 0, 1.0)
    lp, _ = ansatz.log_psi(net, blob, s.nuclei, r)
    r, lp, _ = mcmc.metropolis(net, blob, s.nuclei, r, lp, 5, 150, 0.7)
    radii = []
    for blk in range(30):
        r, lp, _ = mcmc.metropolis(net, blob, s.nuclei, r, lp, 5, 5, 0.7, step_offset=150 + 5 * blk)
        radii.append(np.linalg.norm(r[:, 0], axis=-1).mean())
    assert abs(np.mean(radii) - 1.5) < 0.02


def test_acceptance_decreases_with_step():
    s, net, blob = _hydrogen()
    r, _ = mcmc.init_walkers(s.nuclei, s.charges, 1, 0, None, 2000, 0, 1.0)
    lp, _ = ansatz.log_psi(net, blob, s.nuclei, r)
    rates = []
    for step in (0.1, 0.5, 2.0):
        _, _, acc = mcmc.metropolis(net, blob, s.nuclei, r, lp, 2, 5, step)
        rates.append(acc.mean() / 5)
    assert rates[0] > rates[1] > rates[2]


def test_gradient_closed_form_hydrogen():
    """log psi = log pi - sigma r: d/dsigma = -r, d/dpi = 1/pi; Eq. 6 with any fixed E_L."""
    s, net, blob = _hydrogen()
    p = ansatz.unpack(net, blob)
    p["sigma_up"][...] = 1.2
    p["pi_up"][...] = 0.8
    r, _ = mcmc.init_walkers(s.nuclei, s.charges, 1, 0, None, 50, 4, 1.0)
    e = np.random.default_rng(0).standard_normal(50)
    c = 2 * (e - e.mean()) / 50
    rad = np.linalg.norm(r[:, 0], axis=-1)
    names = [n for n, *_ in ansatz.param_layout(net)]
    offs = np.cumsum([0] + [int(np.prod(sh)) for _, sh, _, _ in ansatz.param_layout(net)])
    i_pi, i_sig = offs[names.index("pi_up")], offs[names.index("sigma_up")]
    g = grad.energy_gradient_fd(net, blob, s.nuclei, r, e, [i_pi, i_sig])
    np.testing.assert_allclose(g[0], np.sum(c) / 0.8, atol=1e-9)
    np.testing.assert_allclose(g[1], np.sum(c * -rad), rtol=1e-8, atol=1e-10)


def test_gradient_directional_linearity():
    s = W.lih(1)
    net = ansatz.Net(2, 2, 1, 2, 8, 4, 2, "aniso")
    blob = ansatz.init_params(net, 2)
    r, _ = mcmc.init_walkers(s.nuclei, s.charges, 2, 1, s.partial_charges, 12, 1, 0.5)
    e, _, _ = ansatz.local_energy(net, blob, s.nuclei, s.charges, r)
    idx = [3, 40, 100, 200, blob.shape[0] - 5]
    g = grad.energy_gradient_fd(net, blob, s.nuclei, r, e, idx)
    v = np.zeros_like(blob)
    w = np.array([0.3, -1.0, 0.5, 2.0, -0.7])
    v[idx] = w
    d = grad.directional_fd(net, blob, s.nuclei, r, e, v)
    assert abs(d - g @ w) < 1e-5 * max(1.0, abs(g @ w))


def test_richardson_removes_h2_term():
    """On a gradient with large curvature the extrapolated value is h-independent to ~1e-9."""
    s = W.lih(1)
    net = ansatz.Net(2, 2, 1, 2, 8, 4, 2, "aniso")
    blob = ansatz.init_params(net, 2)
    r, _ = mcmc.init_walkers(s.nuclei, s.charges, 2, 1, s.partial_charges, 12, 1, 0.5)
    e, _, _ = ansatz.local_energy(net, blob, s.nuclei, s.charges, r)
    a = grad.energy_gradient_richardson(net, blob, s.nuclei, r, e, [3], h=1e-4)
    b = grad.energy_gradient_richardson(net, blob, s.nuclei, r, e, [3], h=5e-5)
    plain = grad.energy_gradient_fd(net, blob, s.nuclei, r, e, [3], h=1e-4)
    assert abs(a[0] - b[0]) < 1e-7 * abs(a[0])
    assert abs(plain[0] - b[0]) > 10 * abs(a[0] - b[0])
