"""Data-parallel VMC over walkers: the one exchange step of Eq. 6.

Walkers are independent, so each rank evaluates its own shard (its random streams are
offset by rank * shard size with fn_set_walker_offset).  Eq. 6 needs the mean local
energy over ALL walkers before the per-walker weights can be formed, and the gradient
is a sum over all walkers:

    E_bar = sum_r sum_w E_L / sum_r B_r
    g     = sum_r sum_w 2 (E_L,w - E_bar) / B_total * d log|psi_w| / d theta

so each rank all-reduces [sum E_L, B_r], forms its weights with the global mean and
count, computes its shard's weighted gradient (fn_log_psi_vjp) and all-reduces it.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def global_mean_and_count(e_local: torch.Tensor, group=None):
    """(global mean E_L, global walker count) by one all-reduce of [sum, count]."""
    stats = torch.stack([e_local.to(torch.float64).sum(),
                         torch.tensor(float(e_local.numel()), dtype=torch.float64, device=e_local.device)])
    dist.all_reduce(stats, group=group)
    return stats[0] / stats[1], stats[1]


def energy_weights(e_local: torch.Tensor, group=None) -> torch.Tensor:
    """Per-walker weights 2 (E_L,w - E_bar) / B_total of Eq. 6 with the global mean and count."""
    mean, count = global_mean_and_count(e_local, group)
    return 2.0 * (e_local.to(torch.float64) - mean) / count


def allreduce_gradient(grad: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of the shards' weighted gradients (in place)."""
    dist.all_reduce(grad, group=group)
    return grad


def energy_gradient(system, params, walkers, e_local, group=None):
    """Eq. 6 gradient of the whole data-parallel batch, computed shard-wise."""
    w = energy_weights(e_local, group)
    g = system.log_psi_vjp(params, walkers, w)
    return allreduce_gradient(g, group)
