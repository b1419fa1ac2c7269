"""Data-parallel VMC over walkers: the one exchange step of Eq. 6.

Walkers are independent, so each rank evaluates its own shard (its random streams are
offset by rank * shard size with fn_set_walker_offset).  Eq. 6 needs the mean local
energy over ALL walkers before the per-walker weights can be formed, and the gradient
is a sum over all walkers:

    E_bar = sum_r sum_w E_L / sum_r B_r
    g     = sum_r sum_w 2 (E_L,w - E_bar) / B_total * d log|psi_w| / d theta

so each rank all-reduces the moments [B_r, sum E_L, sum E_L^2] (fn_energy_moments), forms its
weights from the global moments (fn_energy_weights), computes its shard's weighted gradient
(fn_log_psi_vjp) and all-reduces it.

A training iteration (``train_step``) adds two things:
* clipping uses the window of the whole batch: every rank gathers all ranks' local energies
  (B_r doubles each), clips the gathered batch with fn_clip_local_energy and keeps its slice;
* the update (fn_adam_step / fn_sgd_step) then sees the same all-reduced gradient on every rank,
  so the replicas' parameters stay identical without any broadcast.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def global_moments(system, e_local: torch.Tensor, group=None) -> torch.Tensor:
    """[total count, sum E_L, sum E_L^2] over every rank: the library's moments of this rank's
    energies (fn_energy_moments), summed by one all-reduce of three numbers."""
    mom = system.energy_moments(e_local.to(torch.float64).contiguous())
    dist.all_reduce(mom, group=group)
    return mom


def global_mean_and_count(system, e_local: torch.Tensor, group=None):
    """(global mean E_L, global walker count) from the all-reduced moments (fn_energy_stats)."""
    stats = system.energy_stats(global_moments(system, e_local, group))
    return stats[1], stats[0]


def energy_weights(system, e_local: torch.Tensor, group=None) -> torch.Tensor:
    """Per-walker weights 2 (E_L,w - E_bar) / B_total of Eq. 6 with the global mean and count
    (fn_energy_weights on the all-reduced moments)."""
    return system.energy_weights(e_local.to(torch.float64).contiguous(), global_moments(system, e_local, group))


def allreduce_gradient(grad: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of the shards' weighted gradients (in place)."""
    dist.all_reduce(grad, group=group)
    return grad


def energy_gradient(system, params, walkers, e_local, group=None):
    """Eq. 6 gradient of the whole data-parallel batch, computed shard-wise."""
    w = energy_weights(system, e_local, group)
    g = system.log_psi_vjp(params, walkers, w)
    return allreduce_gradient(g, group)


def gather_energies(e_local: torch.Tensor, group=None):
    """(every rank's energies concatenated in rank order, this rank's offset in them)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n = torch.tensor([e_local.numel()], dtype=torch.int64, device=e_local.device)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    sizes = [int(c.item()) for c in counts]
    width = max(sizes)
    padded = torch.zeros(width, dtype=torch.float64, device=e_local.device)
    padded[: e_local.numel()] = e_local.to(torch.float64)
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    full = torch.cat([p[:k] for p, k in zip(parts, sizes)])
    return full, sum(sizes[:rank])


def clip_global(system, e_local: torch.Tensor, width: float, group=None) -> torch.Tensor:
    """This rank's energies clipped with the window (median, spread) of the whole batch."""
    full, offset = gather_energies(e_local, group)
    clipped, _ = system.clip_local_energy(full.contiguous(), width)
    return clipped[offset: offset + e_local.numel()].contiguous()


def train_step(system, cfg, params, walkers, iteration: int, m=None, v=None, group=None):
    """One data-parallel training iteration; every argument tensor is updated in place.

    The steps are those of fn_vmc_iteration: log|psi| of the rank's walkers, cfg.n_mcmc_steps
    Metropolis steps (step indices iteration * n + k; the rank's random streams are offset by
    fn_set_walker_offset), local energies, clipping with the global window, the Eq. 6 gradient
    with the global mean and count (all-reduced), and the update with Adam step count
    iteration + 1 (m, v: the moments, [param_count] each) or gradient descent.
    Returns (this rank's unclipped local energies, the all-reduced gradient).
    """
    lp, _ = system.log_psi(params, walkers)
    system.mcmc_steps(params, walkers, lp, cfg.n_mcmc_steps, cfg.step_size, cfg.seed,
                      step_offset=iteration * cfg.n_mcmc_steps)
    e, _, _ = system.local_energy(params, walkers)
    e_used = clip_global(system, e, cfg.clip_width, group) if cfg.clip_width > 0 else e
    g = energy_gradient(system, params, walkers, e_used, group)
    if cfg.optimizer == "adam":
        system.adam_step(params, g, m, v, iteration + 1, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps)
    else:
        system.sgd_step(params, g, cfg.lr)
    return e, g
