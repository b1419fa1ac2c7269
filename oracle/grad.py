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
