"""CUDA path against the FP64 oracle, through the C ABI (needs a GB300).

Tolerances (method-fixed where the method fixes them, else derived):
  FP64 mode   |d log|psi|| <= 1e-10, |d E_L| <= 1e-8 relative (to max(1, |E_L|));
  FP32 mode   |d E_L| <= 1e-4 relative to the magnitude of the terms E_L is formed
              from, max(1, |E_L|, (|grad log psi|^2 + |lap log psi|)/2): near a node
              of psi the kinetic energy is a small difference of large terms, and an
              FP32 evaluation can only be accurate relative to those terms;
              log|psi| to 1e-4 relative;
  init        bit-exact walkers and parameters, integer electron counts exact.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import ansatz, ionic, mcmc
from gpu_helpers import make_pair, need_gpu, oracle_params, to_dev

pytestmark = pytest.mark.gpu

SMALL = W.Ansatz(2, 32, 8, 1, "iso")
MID = W.Ansatz(3, 24, 8, 3, "aniso")


def _systems():
    return {"H2": W.h2(), "LiH+": W.lih(1), "LiH-": W.lih(-1), "H": W.hydrogen_atom(), "N2": W.n2(),
            "C": W.atom(6), "Si-": W.atom(14, -1)}


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", ["H2", "LiH+", "LiH-", "N2"])
@pytest.mark.parametrize("prec", [0, 1])
def test_init_walkers_bit_exact(name, prec):
    sysm = _systems()[name]
    net, gpu = make_pair(sysm, SMALL, prec)
    dt = np.float64 if prec == 0 else np.float32
    for B, seed, std in ((7, 0, 1.0), (300, 5, 0.5)):
        r_gpu, counts = gpu.init_walkers(B, seed, std, sysm.partial_charges)
        r_ref, counts_ref = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down,
                                              sysm.partial_charges, B, seed, std, dtype=dt)
        assert counts == counts_ref
        np.testing.assert_array_equal(r_gpu.cpu().numpy(), r_ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_init_params_bit_exact(prec):
    sysm = W.lih(-1)
    net, gpu = make_pair(sysm, W.Ansatz(4, 128, 16, 8, "aniso"), prec)
    ref = ansatz.init_params(net, 4)
    got = gpu.init_params(4).cpu().numpy()
    np.testing.assert_array_equal(got, ref.astype(np.float64 if prec == 0 else np.float32))


@pytest.mark.parametrize("charges,z,t", [((0.88694, 0.11306), (3, 1), 1), (None, (3, 1), -1),
                                          ((0.6, 0.4), (3, 1), 2), ((-0.3, -0.2), (1, 1), -2)])
def test_assign_electrons_matches_algorithm1(charges, z, t):
    import paper_2401_10287_gb300 as P
    n = sum(z) - t
    sysm = W.System("x", np.array([[0, 0, 0], [0, 0, 2.0]]), np.array(z, dtype=float), (n + 1) // 2, n // 2)
    gpu = P.System(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, P.NetConfig(1, 8, 4, 1))
    counts, atoms = gpu.assign_electrons(charges)
    ref = ionic.ionic_electron_counts(list(z), charges, t)
    assert counts == ref
    assert atoms == list(ionic.electron_atoms(ref, sysm.n_up, sysm.n_down))


def _energy_case(name, ans, prec, B, seed=0, perturb=0.05, std=1.0):
    sysm = _systems()[name]
    net, gpu = make_pair(sysm, ans, prec)
    p = oracle_params(net, seed, perturb)
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, sysm.partial_charges, B, seed + 1,
                             std, dtype=np.float64 if prec == 0 else np.float32)
    dt = torch.float64 if prec == 0 else torch.float32
    e, lp, sg = gpu.local_energy(to_dev(p, dt), to_dev(r, dt))
    gpu.sync()
    # the oracle sees exactly the parameters and positions the GPU saw
    p_seen = p.astype(np.float64 if prec == 0 else np.float32).astype(np.float64)
    e_ref, lp_ref, sg_ref = ansatz.local_energy(net, p_seen, sysm.nuclei, sysm.charges, r.astype(np.float64))
    return (e.cpu().numpy(), lp.cpu().numpy(), sg.cpu().numpy()), (e_ref, lp_ref, sg_ref), (net, gpu, p_seen, r)


@pytest.mark.parametrize("name,B", [("H2", 150), ("LiH+", 100), ("LiH-", 61), ("H", 200), ("N2", 20), ("C", 33)])
def test_local_energy_fp64(name, B):
    (e, lp, sg), (e_ref, lp_ref, sg_ref), _ = _energy_case(name, MID, 0, B)
    np.testing.assert_array_equal(sg, sg_ref)
    np.testing.assert_allclose(lp, lp_ref, rtol=0, atol=1e-10)
    np.testing.assert_allclose(e, e_ref, rtol=0, atol=1e-8 * np.maximum(1.0, np.abs(e_ref)).max())
    assert np.all(np.abs(e - e_ref) <= 1e-8 * np.maximum(1.0, np.abs(e_ref)))


def test_local_energy_fp64_h2_workload():
    """Plain-method workload: H2, 2 layers 32/8, 1 determinant, isotropic envelope, 256 walkers."""
    (e, lp, sg), (e_ref, lp_ref, _), _ = _energy_case("H2", SMALL, 0, 256, seed=0, perturb=0.0)
    np.testing.assert_allclose(lp, lp_ref, rtol=0, atol=1e-10)
    assert np.all(np.abs(e - e_ref) <= 1e-8 * np.maximum(1.0, np.abs(e_ref)))


def test_hydrogen_zero_variance_gpu():
    import paper_2401_10287_gb300 as P
    sysm = W.hydrogen_atom()
    net, gpu = make_pair(sysm, W.Ansatz(2, 16, 8, 1, "iso"), 0)
    p = ansatz.init_params(net, 0)
    d = ansatz.unpack(net, p)
    d["w_up"][...] = 0.0
    d["g_up"][...] = 1.0
    r, _ = gpu.init_walkers(500, 3, 1.0)
    e, _, _ = gpu.local_energy(to_dev(p, torch.float64), r)
    np.testing.assert_allclose(e.cpu().numpy(), -0.5, atol=1e-12)


@pytest.mark.parametrize("name,B", [("H2", 150), ("LiH-", 61), ("N2", 12)])
def test_log_psi_value_pass_matches(name, B):
    (e, lp, sg), (e_ref, lp_ref, sg_ref), (net, gpu, p, r) = _energy_case(name, MID, 0, B)
    lp2, sg2 = gpu.log_psi(to_dev(p, torch.float64), to_dev(r, torch.float64))
    np.testing.assert_allclose(lp2.cpu().numpy(), lp_ref, rtol=0, atol=1e-10)
    np.testing.assert_array_equal(sg2.cpu().numpy(), sg_ref)


@pytest.mark.parametrize("name,B", [("H2", 150), ("LiH+", 100), ("N2", 20)])
def test_local_energy_fp32(name, B):
    """FP32 mode: 1e-4 relative to the kinetic-term scale (module docstring)."""
    (e, lp, sg), (e_ref, lp_ref, sg_ref), (net, gpu, p, r) = _energy_case(name, MID, 1, B)
    sysm = _systems()[name]
    _, _, grad, lap = ansatz.log_psi_derivatives(net, p, sysm.nuclei, r.astype(np.float64))
    scale = np.maximum(np.maximum(1.0, np.abs(e_ref)), 0.5 * (np.sum(grad * grad, -1) + np.abs(lap)))
    rel = np.abs(e - e_ref) / scale
    assert np.all(np.abs(lp - lp_ref) <= 1e-4 * np.maximum(1.0, np.abs(lp_ref)))
    assert np.median(rel) < 1e-5
    assert np.all(rel <= 1e-4), (rel.max(), np.argmax(rel))


def test_mcmc_step_fp64_matches_oracle():
    """One Metropolis step: proposals are bit-exact; every accept decision matches the oracle
    except where |log U - A| is below 1e-9 (a floating-point tie)."""
    from oracle import rng
    sysm = W.lih(1)
    net, gpu = make_pair(sysm, MID, 0)
    p = oracle_params(net, 1, 0.05)
    B = 300
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, 2, 1, sysm.partial_charges, B, 2, 0.5)
    pd, rd = to_dev(p, torch.float64), to_dev(r, torch.float64)
    lp, _ = gpu.log_psi(pd, rd)
    lp0 = lp.cpu().numpy()
    acc = torch.zeros(1, dtype=torch.int64, device="cuda")
    gpu.mcmc_steps(pd, rd, lp, 1, 0.3, seed=9, step_offset=17, accept_count=acc)
    gpu.sync()
    prop = mcmc.propose(r, 9, 17, 0.3)
    lp_prop, _ = ansatz.log_psi(net, p, sysm.nuclei, prop)
    log_u = rng.accept_log_uniform(9, B, 17)
    a = 2.0 * (lp_prop - lp0)
    ref_acc = log_u <= a
    moved = np.any(rd.cpu().numpy() != r, axis=(1, 2))
    clear = np.abs(log_u - a) > 1e-9
    np.testing.assert_array_equal(moved[clear], ref_acc[clear])
    np.testing.assert_array_equal(rd.cpu().numpy()[moved], prop[moved])
    assert int(acc.item()) == int(moved.sum())
    np.testing.assert_allclose(lp.cpu().numpy()[moved], lp_prop[moved], atol=1e-10)


def test_mcmc_chain_fp64_matches_oracle():
    """Ten steps of the H2 workload chain, oracle replaying the same draws."""
    sysm = W.h2()
    net, gpu = make_pair(sysm, SMALL, 0)
    p = oracle_params(net, 0)
    B = 70
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, 1, 1, None, B, 0, 1.0)
    pd, rd = to_dev(p, torch.float64), to_dev(r, torch.float64)
    lp, _ = gpu.log_psi(pd, rd)
    gpu.mcmc_steps(pd, rd, lp, 10, 0.02, seed=0)
    r_ref, lp_ref, _ = mcmc.metropolis(net, p, sysm.nuclei, r, lp.cpu().numpy() * 0 + ansatz.log_psi(net, p, sysm.nuclei, r)[0], 0, 10, 0.02)
    same = np.all(rd.cpu().numpy() == r_ref, axis=(1, 2))
    assert same.mean() > 0.97     # a rare accept-boundary flip may fork a chain
    np.testing.assert_allclose(lp.cpu().numpy()[same], lp_ref[same], atol=1e-10)
