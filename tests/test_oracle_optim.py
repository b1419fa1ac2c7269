"""Pins of the oracle's optimisation loop: Adam (Kingma & Ba 2015, Algorithm 1), gradient
descent, local-energy clipping and the training iteration that chains the sampler, the local
energy (Eqs. 2-3) and the Eq. 6 gradient.  Each expected value is a closed form worked out by
hand or an invariant; none is computed by the function under test."""
import numpy as np
import pytest

import workloads as W
from oracle import ansatz, grad, mcmc, optim


# ---- Adam -----------------------------------------------------------------------------

def test_adam_first_step_is_normalised_gradient():
    """t = 1: m_hat = g and v_hat = g^2 exactly, so the step is -lr g / (|g| + eps).
    Without the bias correction the step would be -lr 0.1 g / (0.0316 |g| + eps)."""
    g = np.array([3.0, -0.5, 1e-3, 0.0, -7.0])
    p0 = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    p, m, v = optim.adam_step(p0, g, np.zeros(5), np.zeros(5), 1, lr=0.1, eps=1e-8)
    np.testing.assert_allclose(p - p0, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-13)


def test_adam_constant_gradient_steps_are_equal():
    """With a constant g, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so every corrected
    step equals the first one; an off-by-one exponent in the correction breaks this."""
    g = np.array([0.25, -2.0, 5.0])
    p = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for t in range(1, 8):
        prev = p
        p, m, v = optim.adam_step(p, g, m, v, t, lr=0.01, beta1=0.9, beta2=0.99, eps=0.0)
        np.testing.assert_allclose(p - prev, -0.01 * np.sign(g), rtol=1e-12)
        np.testing.assert_allclose(m, (1 - 0.9 ** t) * g, rtol=1e-12)
        np.testing.assert_allclose(v, (1 - 0.99 ** t) * g * g, rtol=1e-12)


def test_adam_two_steps_worked_example():
    """beta1 = 1/2, beta2 = 3/4, eps = 0, lr = 1, gradients 2 then 3.
    Step 1: m = 1, v = 1, m_hat = 2, v_hat = 4: step -1.
    Step 2: m = 1/2 + 3/2 = 2, v = 3/4 + 9/4 = 3, m_hat = 2 / (3/4) = 8/3,
            v_hat = 3 / (7/16) = 48/7: step -(8/3) sqrt(7/48)."""
    p, m, v = optim.adam_step(np.array([0.0]), np.array([2.0]), np.zeros(1), np.zeros(1), 1, 1.0, 0.5, 0.75, 0.0)
    assert p[0] == pytest.approx(-1.0, abs=1e-15)
    p2, m, v = optim.adam_step(p, np.array([3.0]), m, v, 2, 1.0, 0.5, 0.75, 0.0)
    assert m[0] == pytest.approx(2.0, abs=1e-15) and v[0] == pytest.approx(3.0, abs=1e-15)
    assert p2[0] - p[0] == pytest.approx(-(8.0 / 3.0) * np.sqrt(7.0 / 48.0), rel=1e-14)


def test_adam_is_invariant_to_gradient_scale():
    """With eps = 0 the update depends on g only through g / sqrt(E[g^2])."""
    rs = np.random.default_rng(3)
    gs = rs.standard_normal((6, 40))
    pa = pb = np.zeros(40)
    ma = va = mb = vb = np.zeros(40)
    for t, g in enumerate(gs, start=1):
        pa, ma, va = optim.adam_step(pa, g, ma, va, t, 0.05, eps=0.0)
        pb, mb, vb = optim.adam_step(pb, 1e4 * g, mb, vb, t, 0.05, eps=0.0)
    np.testing.assert_allclose(pa, pb, rtol=1e-10, atol=1e-14)


def test_adam_minimises_a_convex_quadratic():
    """f = 1/2 sum a_i x_i^2 (a_i from 0.1 to 10): Adam with a decaying rate drives every
    coordinate to the minimum at 0; a sign error would drive them away."""
    a = np.geomspace(0.1, 10.0, 12)
    x = np.linspace(-3.0, 3.0, 12)
    m = v = np.zeros(12)
    for t in range(1, 3001):
        x, m, v = optim.adam_step(x, a * x, m, v, t, lr=0.1 / np.sqrt(t))
    assert np.max(np.abs(x)) < 5e-3


def test_adam_rejects_step_zero():
    with pytest.raises(ValueError):
        optim.adam_step(np.zeros(1), np.ones(1), np.zeros(1), np.zeros(1), 0, 0.1)


def test_sgd_step():
    np.testing.assert_array_equal(optim.sgd_step([1.0, -2.0], [0.5, 4.0], 0.25), [0.875, -3.0])


# ---- clipping -------------------------------------------------------------------------

def test_lower_median():
    assert optim.lower_median([5.0]) == 5.0
    assert optim.lower_median([3.0, 1.0, 2.0]) == 2.0
    assert optim.lower_median([4.0, 1.0, 3.0, 2.0]) == 2.0       # rank floor(3/2) = 1
    e = np.random.default_rng(0).standard_normal(1001)
    assert optim.lower_median(e) == np.median(e)


def test_clip_single_outlier_closed_form():
    """Nine zeros and 100: centre 0, spread 100/10 = 10, window +-5*10: 100 -> 50."""
    e = np.zeros(10)
    e[7] = 100.0
    c, centre, spread = optim.clip_local_energy(e, 5.0)
    assert centre == 0.0 and spread == 10.0
    np.testing.assert_array_equal(c, np.where(np.arange(10) == 7, 50.0, 0.0))


def test_clip_symmetric_window():
    """[-2, -1, 0, 1, 2]: centre 0, spread 6/5, width 1 clamps the ends to +-1.2."""
    c, centre, spread = optim.clip_local_energy([-2.0, -1.0, 0.0, 1.0, 2.0], 1.0)
    assert centre == 0.0 and spread == pytest.approx(1.2, abs=1e-15)
    np.testing.assert_allclose(c, [-1.2, -1.0, 0.0, 1.0, 1.2], atol=1e-15)


def test_clip_off_and_inside_values_untouched():
    e = np.random.default_rng(1).standard_normal(257) - 40.0
    c0, _, _ = optim.clip_local_energy(e, 0.0)
    np.testing.assert_array_equal(c0, e)
    c, centre, spread = optim.clip_local_energy(e, 2.0)
    inside = np.abs(e - centre) <= 2.0 * spread
    np.testing.assert_array_equal(c[inside], e[inside])
    np.testing.assert_allclose(np.abs(c[~inside] - centre), 2.0 * spread, rtol=1e-14)
    assert (~inside).any()


def test_clip_is_permutation_equivariant():
    rs = np.random.default_rng(2)
    e = rs.standard_cauchy(300)
    perm = rs.permutation(300)
    a, _, _ = optim.clip_local_energy(e, 3.0)
    b, _, _ = optim.clip_local_energy(e[perm], 3.0)
    np.testing.assert_array_equal(a[perm], b)


# ---- training iteration ------------------------------------------------------------------

def _hydrogen_exact():
    """psi = (0 . h + 1) exp(-|r|): the hydrogen ground state, E = -1/2 at every point."""
    s = W.hydrogen_atom()
    net = ansatz.Net(1, 1, 0, 1, 4, 2, 1, "iso")
    blob = ansatz.init_params(net, 0)
    p = ansatz.unpack(net, blob)
    p["w_up"][...] = 0.0
    p["g_up"][...] = 1.0
    return s, net, blob


def test_train_iteration_zero_variance_at_the_ground_state():
    """At an eigenstate E_L is constant, so Eq. 6 gives a zero gradient and the update
    leaves the parameters where they are (zero-variance property)."""
    s, net, blob = _hydrogen_exact()
    r, _ = mcmc.init_walkers(s.nuclei, s.charges, 1, 0, None, 16, 5, 1.0)
    st = optim.TrainState(blob, r)
    out = optim.train_iteration(net, st, s.nuclei, s.charges, seed=5, n_mcmc=3, step_size=0.3,
                                clip_width=5.0, optimizer="adam", lr=0.01)
    np.testing.assert_allclose(out["e_local"], -0.5, atol=1e-10)
    assert np.max(np.abs(out["grad"])) < 1e-9
    assert np.max(np.abs(st.params - blob)) < 1e-5 * 0.01
    assert st.t == 1


def test_train_iteration_wiring_with_zero_rate():
    """lr = 0: the parameters stay, the walkers are those of Metropolis run directly with
    step indices t*n .. t*n + n - 1, and the second iteration continues the streams."""
    s = W.h2()
    net = ansatz.Net(2, 1, 1, 1, 4, 2, 1, "iso")
    blob = ansatz.init_params(net, 1)
    r0, _ = mcmc.init_walkers(s.nuclei, s.charges, 1, 1, None, 8, 2, 1.0)
    st = optim.TrainState(blob, r0)
    for t in range(2):
        r_prev = st.walkers.copy()
        out = optim.train_iteration(net, st, s.nuclei, s.charges, seed=9, n_mcmc=4, step_size=0.2,
                                    optimizer="sgd", lr=0.0)
        lp, _ = ansatz.log_psi(net, blob, s.nuclei, r_prev)
        r_ref, lp_ref, acc = mcmc.metropolis(net, blob, s.nuclei, r_prev, lp, 9, 4, 0.2, step_offset=4 * t)
        np.testing.assert_array_equal(st.walkers, r_ref)
        np.testing.assert_array_equal(out["accepted"], acc)
        np.testing.assert_array_equal(st.params, blob)
    assert st.t == 2


def test_train_iteration_uses_clipped_energies_in_eq6():
    """Eq. 6 takes the clipped energies: a narrow window changes the gradient, and the
    SGD update equals -lr times the gradient of the clipped surrogate."""
    s = W.h2()
    net = ansatz.Net(2, 1, 1, 1, 4, 2, 1, "iso")
    blob = ansatz.init_params(net, 1)
    r0, _ = mcmc.init_walkers(s.nuclei, s.charges, 1, 1, None, 12, 3, 1.0)
    a = optim.TrainState(blob, r0)
    b = optim.TrainState(blob, r0)
    oa = optim.train_iteration(net, a, s.nuclei, s.charges, seed=4, n_mcmc=2, step_size=0.2,
                               clip_width=0.0, optimizer="sgd", lr=0.1)
    ob = optim.train_iteration(net, b, s.nuclei, s.charges, seed=4, n_mcmc=2, step_size=0.2,
                               clip_width=0.25, optimizer="sgd", lr=0.1)
    np.testing.assert_array_equal(a.walkers, b.walkers)
    assert not np.array_equal(ob["e_clipped"], ob["e_local"])
    assert np.max(np.abs(oa["grad"] - ob["grad"])) > 1e-6
    idx = [0, 5, len(blob) - 1]
    g_ref = grad.energy_gradient_richardson(net, blob, s.nuclei, b.walkers, ob["e_clipped"], idx)
    np.testing.assert_allclose(b.params[idx], blob[idx] - 0.1 * g_ref, rtol=1e-12, atol=1e-14)
