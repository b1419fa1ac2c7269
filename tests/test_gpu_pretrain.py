"""Eq. 5 pretraining on the GPU (fn_pretrain_setup, fn_pretrain_grad) against the oracle:
the loss against oracle.pretrain.pretrain_loss at the same parameters and positions, and the
parameter gradient along random directions against Richardson-extrapolated central
differences of that oracle loss.  The library's STO-6G expansion is the published table and
the oracle's is fitted from scratch; the two agree to about 1e-5, which sets the tolerance."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mcmc, pretrain
from gpu_helpers import make_pair, need_gpu, oracle_params, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    torch.cuda.synchronize()


def _oracle_loss(net, p, sysm, r, state):
    return pretrain.pretrain_loss(net, p, sysm.nuclei, r, state)


def _directional(net, p, sysm, r, state, v, h):
    def f(eps):
        return _oracle_loss(net, p + eps * v, sysm, r, state)
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("name,make,ans,B", [
    ("H2", W.h2, W.Ansatz(2, 32, 8, 1, "iso"), 64),
    ("LiH", lambda: W.lih(0), W.Ansatz(3, 32, 8, 2, "aniso"), 48),
    ("LiH+", lambda: W.lih(1), W.Ansatz(3, 32, 8, 2, "aniso"), 48),
])
def test_pretrain_loss_and_gradient_fp64(name, make, ans, B):
    sysm = make()
    net, gpu = make_pair(sysm, ans, 0)
    e_hf = gpu.pretrain_setup()
    state = pretrain.hf_state(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down)
    assert abs(e_hf - state["energy"]) < 1e-5
    p = oracle_params(net, 2, 0.05)
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, sysm.partial_charges, B, 5, 0.8)
    g, loss = gpu.pretrain_grad(to_dev(p, torch.float64), to_dev(r, torch.float64))
    gpu.sync()
    g = g.cpu().numpy()
    loss_ref = _oracle_loss(net, p, sysm, r, state)
    print(f"{name}: loss {loss.item():.8f} oracle {loss_ref:.8f}; |g| {np.linalg.norm(g):.4e}")
    assert abs(loss.item() - loss_ref) <= 1e-4 * loss_ref
    for k in range(2):
        v = np.random.default_rng(20 + k).standard_normal(p.shape[0])
        v /= np.linalg.norm(v)
        d = _directional(net, p, sysm, r, state, v, 1e-4)
        assert abs(float(g @ v) - d) <= 1e-4 * np.linalg.norm(g) + 1e-9, (float(g @ v), d)


def test_pretrain_bf16_against_fp64():
    """BF16-mixed mode (tensor-core forward and backward) against the FP64 path: the same
    loss to 1e-2 relative and the gradient to 3e-2 of its norm (the error budget of the BF16
    energy gradient: 8-bit storage of the backpropagated signals through every layer)."""
    sysm = W.lih(0)
    ans = W.Ansatz(3, 64, 16, 4, "aniso")
    net, g16 = make_pair(sysm, ans, 2)
    _, g64 = make_pair(sysm, ans, 0)
    g16.pretrain_setup()
    g64.pretrain_setup()
    p = oracle_params(net, 3, 0.05).astype(np.float32).astype(np.float64)
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, None, 256, 6, 0.8)
    r = r.astype(np.float32).astype(np.float64)
    gb, lb = g16.pretrain_grad(to_dev(p, torch.float32), to_dev(r, torch.float32))
    gd, ld = g64.pretrain_grad(to_dev(p, torch.float64), to_dev(r, torch.float64))
    g16.sync()
    gb = gb.cpu().numpy().astype(np.float64)
    gd = gd.cpu().numpy()
    rel = np.linalg.norm(gb - gd) / np.linalg.norm(gd)
    print(f"BF16 pretraining: loss {lb.item():.6f} vs {ld.item():.6f}; gradient rel {rel:.2e}")
    assert np.all(np.isfinite(gb))
    assert abs(lb.item() - ld.item()) <= 1e-2 * ld.item()
    assert rel < 3e-2


def test_pretrain_refusals():
    import paper_2401_10287_gb300 as P
    net, gpu = make_pair(W.n2(), W.Ansatz(2, 32, 8, 1, "aniso"), 0)
    with pytest.raises(P.FnError) as err:       # the degenerate pi levels of N2
        gpu.pretrain_setup()
    assert err.value.code == 7
    net, gpu = make_pair(W.h2(), W.Ansatz(2, 32, 8, 1, "iso"), 0)
    p = gpu.init_params(0)
    w, _ = gpu.init_walkers(8, 0, 1.0)
    with pytest.raises(P.FnError) as err:
        gpu.pretrain_grad(p, w)
    assert err.value.code == 1
