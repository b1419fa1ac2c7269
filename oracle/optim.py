"""Optimisation loop of the oracle (TEST INFRASTRUCTURE ONLY).

The training phase of the method updates the network parameters with the Eq. 6
gradient, sampling the walkers with the electron sampler between updates ("10 steps
between MCMC updates" in the Results section).  The paper names no optimiser and no
local-energy clipping; this module takes these readings:

* Adam, as defined by Kingma & Ba (ICLR 2015, Algorithm 1), and plain gradient
  descent as the degenerate alternative;
* optional clipping of the local energies before Eq. 6: centre = the lower median
  of the batch, spread = the mean absolute deviation from that centre, every energy
  clamped to centre +- width * spread (the scheme of the FermiNet line of work;
  width <= 0 turns it off);
* one training iteration on walkers that persist from the previous iteration:
  log|psi| of the walkers under the current parameters, n Metropolis steps with
  step indices t*n .. t*n + n - 1 of the random streams, local energies (Eqs. 2-3),
  clipping, the Eq. 6 gradient with the (clipped) energies held fixed, then the
  update (Adam step count t + 1).

The gradient here is the finite-difference one of ``oracle.grad`` (Richardson), so the
training iteration is only affordable for networks of a few hundred parameters.

Parity status: pinned by ``tests/test_oracle_optim.py`` (closed forms of Adam's bias
correction, scale invariance, a convex quadratic, the clipping window on constructed
data, and the zero-variance property of the hydrogen-atom ground state).
"""
from __future__ import annotations

import numpy as np

from . import ansatz, grad, mcmc


def sgd_step(params, g, lr: float):
    """theta <- theta - lr * g."""
    return np.asarray(params, np.float64) - float(lr) * np.asarray(g, np.float64)


def adam_step(params, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) with step count t >= 1.

    Returns (params, m, v).  The moment estimates are exponential averages of g and
    g**2; both are divided by (1 - beta**t) to remove the bias of their zero start.
    """
    if t < 1:
        raise ValueError("Adam step count starts at 1")
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return np.asarray(params, np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def lower_median(e) -> float:
    """Element of rank floor((B - 1) / 2) of the sorted batch (an exact batch member)."""
    e = np.sort(np.asarray(e, np.float64))
    return float(e[(e.shape[0] - 1) // 2])


def clip_local_energy(e, width: float):
    """Clamp to centre +- width * spread; returns (clipped, centre, spread).

    width <= 0 returns the energies unchanged (centre and spread are still reported).
    """
    e = np.asarray(e, np.float64)
    centre = lower_median(e)
    spread = float(np.mean(np.abs(e - centre)))
    if width <= 0:
        return e.copy(), centre, spread
    lo, hi = centre - width * spread, centre + width * spread
    return np.minimum(np.maximum(e, lo), hi), centre, spread


class TrainState:
    """Parameters, walkers and optimiser moments carried from one iteration to the next."""

    def __init__(self, params, walkers):
        self.params = np.array(params, np.float64)
        self.walkers = np.array(walkers)
        self.m = np.zeros_like(self.params)
        self.v = np.zeros_like(self.params)
        self.t = 0


def train_iteration(net, state: TrainState, nuclei, charges, seed: int, n_mcmc: int, step_size: float,
                    clip_width: float = 0.0, optimizer: str = "adam", lr: float = 1e-3,
                    beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, fd_h: float = 1e-5):
    """One VMC training iteration (see the module docstring); updates ``state`` in place.

    Returns a dict with the local energies before clipping, the clipped ones, the
    Eq. 6 gradient, log|psi| of the sampled walkers and the accepted moves per walker.
    """
    p = state.params
    lp, _ = ansatz.log_psi(net, p, nuclei, state.walkers)
    r, lp, acc = mcmc.metropolis(net, p, nuclei, state.walkers, lp, seed, n_mcmc, step_size,
                                 step_offset=state.t * n_mcmc)
    e, _, _ = ansatz.local_energy(net, p, nuclei, charges, r)
    e_c, _, _ = clip_local_energy(e, clip_width)
    g = grad.energy_gradient_richardson(net, p, nuclei, r, e_c, range(p.shape[0]), h=fd_h)
    if optimizer == "adam":
        state.params, state.m, state.v = adam_step(p, g, state.m, state.v, state.t + 1, lr, beta1, beta2, eps)
    elif optimizer == "sgd":
        state.params = sgd_step(p, g, lr)
    else:
        raise ValueError(optimizer)
    state.walkers = r
    state.t += 1
    return {"e_local": e, "e_clipped": e_c, "grad": g, "log_psi": lp, "accepted": acc}
