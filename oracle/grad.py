"""VMC energy gradient of the oracle (test infrastructure only).

Eq. 6: grad_theta L = 2 E_p[(E_p - E_p(E_p)) grad_theta log|psi|], with the
expectation taken as the mean over the B walkers and the local energies held
fixed.  Equivalently it is the gradient of the surrogate
S(theta) = (2/B) sum_w (E_L,w - mean E_L) log|psi_theta(r_w)|, which is what is
differentiated here by central finite differences in float64.
"""
from __future__ import annotations

import numpy as np

from . import ansatz


def surrogate(net, params, nuclei, r, e_local) -> float:
    e = np.asarray(e_local, dtype=np.float64)
    c = 2.0 * (e - e.mean()) / e.shape[0]
    lp, _ = ansatz.log_psi(net, params, nuclei, r)
    return float(np.sum(c * lp))


def energy_gradient_fd(net, params, nuclei, r, e_local, indices, h: float = 1e-5) -> np.ndarray:
    """Gradient entries for the given parameter indices by central differences."""
    params = np.asarray(params, dtype=np.float64)
    out = np.zeros(len(indices))
    for n, idx in enumerate(indices):
        pp = params.copy()
        pp[idx] += h
        pm = params.copy()
        pm[idx] -= h
        out[n] = (surrogate(net, pp, nuclei, r, e_local) - surrogate(net, pm, nuclei, r, e_local)) / (2 * h)
    return out


def directional_fd(net, params, nuclei, r, e_local, direction, h: float = 1e-5) -> float:
    """Derivative of the surrogate along ``direction`` (checks every entry at once)."""
    params = np.asarray(params, dtype=np.float64)
    v = np.asarray(direction, dtype=np.float64)
    return (surrogate(net, params + h * v, nuclei, r, e_local)
            - surrogate(net, params - h * v, nuclei, r, e_local)) / (2 * h)


# Central differences carry an O(h^2) truncation error, which near a node of psi (where
# log|psi| has large third derivatives) exceeds 1e-4 relative at h = 1e-5.  Richardson
# extrapolation of the steps h and h/2, (4 D(h/2) - D(h)) / 3, cancels that term.

def energy_gradient_richardson(net, params, nuclei, r, e_local, indices, h: float = 1e-5) -> np.ndarray:
    d1 = energy_gradient_fd(net, params, nuclei, r, e_local, indices, h)
    d2 = energy_gradient_fd(net, params, nuclei, r, e_local, indices, h / 2)
    return (4.0 * d2 - d1) / 3.0


def directional_richardson(net, params, nuclei, r, e_local, direction, h: float = 1e-5) -> float:
    d1 = directional_fd(net, params, nuclei, r, e_local, direction, h)
    d2 = directional_fd(net, params, nuclei, r, e_local, direction, h / 2)
    return (4.0 * d2 - d1) / 3.0


def term_magnitude_fd(net, params, nuclei, r, e_local, indices, h: float = 1e-5) -> np.ndarray:
    """sum_w |c_w d log|psi_w| / d theta_p| for the given indices (per-walker central
    differences).  The size of the terms that Eq. 6 sums: a reduced-precision gradient can
    only be accurate relative to it when the terms cancel."""
    params = np.asarray(params, dtype=np.float64)
    e = np.asarray(e_local, dtype=np.float64)
    c = 2.0 * (e - e.mean()) / e.shape[0]
    out = np.zeros(len(indices))
    for n, idx in enumerate(indices):
        pp = params.copy()
        pp[idx] += h
        pm = params.copy()
        pm[idx] -= h
        d = (ansatz.log_psi(net, pp, nuclei, r)[0] - ansatz.log_psi(net, pm, nuclei, r)[0]) / (2 * h)
        out[n] = float(np.sum(np.abs(c * d)))
    return out