"""BF16-mixed mode (tcgen05 tensor-core stream layers, FP64 determinants) against the FP64 oracle.

The BF16 mode stores stream activations in BF16 (8 significant bits), so its error is
not a rounding-order difference: the tests bound it loosely per walker and report the
mean-energy error, the quantity the precision mode is judged by."""
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


def _run(sysm, ans, B, seed=0, std=1.0, perturb=0.0, burn_in=150, step=0.3):
    """Walkers equilibrated on |psi|^2 by the oracle's own Metropolis chain (FP64), so that
    they are distributed like the walkers a VMC run evaluates."""
    net, gpu = make_pair(sysm, ans, 2)
    p = oracle_params(net, seed, perturb).astype(np.float32).astype(np.float64)
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, sysm.partial_charges, B, seed + 1,
                             std)
    lp0, _ = ansatz.log_psi(net, p, sysm.nuclei, r)
    r, _, _ = mcmc.metropolis(net, p, sysm.nuclei, r, lp0, seed + 2, burn_in, step)
    r = r.astype(np.float32)
    e, lp, sg = gpu.local_energy(to_dev(p, torch.float32), to_dev(r, torch.float32))
    gpu.sync()
    r64 = r.astype(np.float64)
    e_ref, lp_ref, _ = ansatz.local_energy(net, p, sysm.nuclei, sysm.charges, r64)
    _, _, grad, lap = ansatz.log_psi_derivatives(net, p, sysm.nuclei, r64)
    scale = np.maximum(np.maximum(1.0, np.abs(e_ref)), 0.5 * (np.sum(grad * grad, -1) + np.abs(lap)))
    return e.cpu().numpy(), lp.cpu().numpy(), e_ref, lp_ref, scale


@pytest.mark.parametrize("name,make,ans,B", [
    ("H2", W.h2, W.Ansatz(2, 32, 8, 1, "iso"), 256),
    ("LiH+", lambda: W.lih(1), W.Ansatz(4, 128, 16, 8, "aniso"), 130),
    ("N2", W.n2, W.Ansatz(4, 256, 32, 16, "aniso"), 40),
])
def test_bf16_local_energy_against_oracle(name, make, ans, B):
    e, lp, e_ref, lp_ref, scale = _run(make(), ans, B)
    rel = np.abs(e - e_ref) / scale
    mean_err = abs(e.mean() - e_ref.mean())
    worst = int(np.argmax(rel))
    print(f"{name}: median rel {np.median(rel):.2e} max rel {rel.max():.2e} (E_ref {e_ref[worst]:.3f}, scale "
          f"{scale[worst]:.1f}) mean-energy error {mean_err * 1e3:.3f} mHa of {e_ref.mean():.4f} Ha;"
          f" |d log psi| median {np.median(np.abs(lp - lp_ref)):.2e} max {np.abs(lp - lp_ref).max():.2e}")
    assert np.all(np.isfinite(e))
    assert np.median(rel) < 1e-2


def test_bf16_mcmc_and_grad_run():
    sysm = W.lih(-1)
    net, gpu = make_pair(sysm, W.Ansatz(4, 128, 16, 8, "aniso"), 2)
    params = gpu.init_params(4)
    walkers, counts = gpu.init_walkers(512, 4, 0.5)
    assert counts == [4, 1]
    lp, _ = gpu.log_psi(params, walkers)
    acc = torch.zeros(1, dtype=torch.int64, device="cuda")
    gpu.mcmc_steps(params, walkers, lp, 5, 0.05, seed=1, accept_count=acc)
    e, lp2, _ = gpu.local_energy(params, walkers)
    g, mean = gpu.energy_grad(params, walkers, e)
    gpu.sync()
    assert 0 < acc.item() <= 5 * 512
    assert torch.isfinite(e).all() and torch.isfinite(g).all()
    assert (lp - lp2).abs().max().item() < 5e-2 * max(1.0, lp.abs().max().item())


@pytest.mark.parametrize("name,make,ans,B", [
    ("LiH+", lambda: W.lih(1), W.Ansatz(4, 128, 16, 8, "aniso"), 96),
    ("N2", W.n2, W.Ansatz(4, 256, 32, 16, "aniso"), 32),
])
def test_bf16_energy_grad_against_fp64_and_oracle(name, make, ans, B):
    """Eq. 6 gradient of the BF16 mode (BF16 activations with the value slab kept as a
    hi/lo pair, BF16 gradient signals, split BF16 weights, tensor-core GEMMs) against the
    FP64 library gradient (itself pinned to oracle finite differences) and, along random
    directions, against the oracle's Richardson finite difference.  Error budget: the
    tangent-free backward stores every layer's backpropagated signal with 8 significant
    bits (relative 2^-9) and multiplies it by 8-bit activations, so a 4-layer gradient
    carries about 1e-2 relative error; the bound is 3e-2 of the gradient norm."""
    from oracle import grad as ograd
    sysm = make()
    net, g16 = make_pair(sysm, ans, 2)
    _, g64 = make_pair(sysm, ans, 0)
    p = oracle_params(net, 0, 0.02).astype(np.float32).astype(np.float64)
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, sysm.partial_charges, B, 1, 1.0)
    lp0, _ = ansatz.log_psi(net, p, sysm.nuclei, r)
    r, _, _ = mcmc.metropolis(net, p, sysm.nuclei, r, lp0, 2, 100, 0.3)
    r = r.astype(np.float32).astype(np.float64)
    e = np.random.default_rng(5).normal(-8.0, 1.0, B)
    ge = torch.as_tensor(e).cuda()
    gb, _ = g16.energy_grad(to_dev(p, torch.float32), to_dev(r, torch.float32), ge)
    gd, _ = g64.energy_grad(to_dev(p, torch.float64), to_dev(r, torch.float64), ge)
    g16.sync()
    gb = gb.cpu().numpy().astype(np.float64)
    gd = gd.cpu().numpy()
    assert np.all(np.isfinite(gb))
    rel = np.linalg.norm(gb - gd) / np.linalg.norm(gd)
    dirs = []
    for k in range(2):
        v = np.random.default_rng(10 + k).standard_normal(p.shape[0])
        v /= np.linalg.norm(v)
        d = ograd.directional_richardson(net, p, sysm.nuclei, r, e, v, h=1e-5)
        dirs.append((float(gb @ v), float(gd @ v), float(d)))
    print(f"{name}: |g_bf16 - g_fp64| / |g_fp64| = {rel:.3e}; directional (bf16, fp64, oracle FD): {dirs}")
    assert rel < 3e-2
    for b, f, d in dirs:
        assert abs(f - d) <= 1e-5 * max(1.0, abs(d))
        assert abs(b - d) <= 3e-2 * np.linalg.norm(gd)


def test_bf16_h2_precision_config_mean_energy():
    """Precision configuration: H2 at 1.4 bohr, 2 layers 32/8, 1 determinant, isotropic
    envelopes, 4096 walkers equilibrated by the oracle's Metropolis chain.  The BF16-mixed
    mean local energy must be within 1 mHa of the oracle's on the same walkers (the target
    of the precision mode); per-walker errors are reported."""
    sysm = W.h2()
    ans = W.Ansatz(2, 32, 8, 1, "iso")
    e, lp, e_ref, lp_ref, scale = _run(sysm, ans, 4096, seed=0, perturb=0.0, burn_in=200, step=0.3)
    d = e - e_ref
    err = abs(d.mean())
    se = d.std() / np.sqrt(d.size)
    print(f"H2 cfg3, 4096 walkers: mean-energy error {d.mean() * 1e3:.3f} +- {se * 1e3:.3f} mHa of "
          f"{e_ref.mean():.5f} Ha; per-walker median |dE| {np.median(np.abs(d)):.2e} Ha, max {np.abs(d).max():.2e}")
    assert np.all(np.isfinite(e))
    assert err <= 1e-3


@pytest.mark.parametrize("name,make", [
    ("H", W.hydrogen_atom),                 # one electron: no pairs, an empty spin group
    ("Li", lambda: W.atom(3)),              # 2 up / 1 down
    ("O-", lambda: W.atom(8, -1)),          # 5 up / 4 down
])
def test_bf16_atoms_unequal_spins_against_oracle(name, make):
    """BF16 mode on atoms with unequal (or empty) spin groups, against the FP64 oracle on
    oracle-equilibrated walkers: same per-walker bound as the molecules above."""
    e, lp, e_ref, lp_ref, scale = _run(make(), W.Ansatz(3, 64, 16, 4, "aniso"), 96, seed=1, burn_in=100)
    rel = np.abs(e - e_ref) / scale
    print(f"{name}: median rel {np.median(rel):.2e} max rel {rel.max():.2e}; mean-energy error "
          f"{abs(e.mean() - e_ref.mean()) * 1e3:.3f} mHa of {e_ref.mean():.4f} Ha")
    assert np.all(np.isfinite(e))
    assert np.median(rel) < 1e-2
    assert np.median(np.abs(lp - lp_ref)) < 1e-2


def test_bf16_layer_pair_kernel_matches_single(monkeypatch):
    """The CTA-pair stream-layer kernel (FN_LAYER_KERNEL=pair: cta_group::2 MMAs of M = 256,
    each CTA holding half of the weight tile) forms the same products, accumulated in the
    same order, as the default one-CTA kernel, so log psi and E_L are bit-identical.  N2 network
    (4 layers 256/32, 16 determinants), 256 walkers: 29 row tiles, so the last CTA pair has
    a rank-1 tile past the rows."""
    sysm = W.n2()
    cfg = W.N2_LARGE
    _, gpu = make_pair(sysm, cfg["ansatz"], 2)
    params = gpu.init_params(cfg["seed"])
    walkers, _ = gpu.init_walkers(256, cfg["seed"], cfg["init_std"])
    lp0, _ = gpu.log_psi(params, walkers)
    gpu.mcmc_steps(params, walkers, lp0, 3, 0.05, 7)
    out = {}
    for mode in ["single", "pair"]:
        monkeypatch.setenv("FN_LAYER_KERNEL", mode)
        lp, sg = gpu.log_psi(params, walkers)
        e, lp2, _ = gpu.local_energy(params, walkers)
        g, _ = gpu.energy_grad(params, walkers, e)
        gpu.sync()
        out[mode] = [x.clone() for x in (lp, sg, e, lp2, g)]
    for a, b in zip(out["single"][:4], out["pair"][:4]):
        assert torch.equal(a, b)
    # the gradient's sums over walkers end in FP32 atomic additions, whose order varies from
    # run to run: equal to that rounding
    g1, g2 = out["single"][4], out["pair"][4]
    assert torch.all((g1 - g2).abs() <= 1e-5 * g1.abs().max())


@pytest.mark.parametrize("name,make,ans", [
    ("N2", W.n2, W.Ansatz(2, 64, 16, 4, "aniso")),            # 7 + 7 electrons
    ("O-", lambda: W.atom(8, -1), W.Ansatz(2, 64, 16, 4, "iso")),   # 5 + 4 electrons, 27 coordinates
])
def test_bf16_group_det_kernel_matches_thread_kernel(monkeypatch, name, make, ans):
    """The local-energy determinant stage on 8-lane groups (default for blocks of 5 to 8
    electrons) against the one-thread-per-block kernel (FN_DET_KERNEL=thread) on the same
    orbitals.  Both choose the same pivots; the elimination order of their operations differs
    (Gauss-Jordan in registers against LU in shared memory, C = A^-1 by elimination against
    substitution, the traces summed in another order), so log psi agrees to 1e-12 of
    max(1, |log psi|) with the same signs, and E_L to 1e-9 of max(1, |E_L|).  Measured: 1e-14
    and 3e-12."""
    sysm = make()
    _, gpu = make_pair(sysm, ans, 2)
    params = gpu.init_params(3)
    walkers, _ = gpu.init_walkers(512, 3, 1.0)
    lp0, _ = gpu.log_psi(params, walkers)
    gpu.mcmc_steps(params, walkers, lp0, 20, 0.1, 5)
    out = {}
    for mode in ["thread", "group"]:
        monkeypatch.setenv("FN_DET_KERNEL", mode)
        e, lp, sg = gpu.local_energy(params, walkers)
        gpu.sync()
        out[mode] = (e.cpu().numpy(), lp.clone(), sg.clone())
    e1, lp1, s1 = out["thread"]
    e2, lp2, s2 = out["group"]
    dlp = (lp1 - lp2).abs().max().item()
    rel = np.abs(e1 - e2) / np.maximum(1.0, np.abs(e1))
    print(f"{name}: group vs thread determinant kernel, max |d log psi| {dlp:.2e}, sign mismatches "
          f"{int((s1 != s2).sum())}, max |dE_L| rel {rel.max():.2e}, median {np.median(rel):.2e}")
    assert torch.equal(s1, s2)
    assert torch.all((lp1 - lp2).abs() <= 1e-12 * torch.clamp(lp1.abs(), min=1.0))
    assert np.all(np.isfinite(e2))
    assert rel.max() <= 1e-9
