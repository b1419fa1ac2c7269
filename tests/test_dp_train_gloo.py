"""Data-parallel training step (dp.train_step) with gloo ranks on the CPU.

A stand-in for the library supplies per-walker local energies and gradients of log|psi|
from a toy model (smooth functions of the walkers and parameters); clipping and the Adam
update come from the oracle.  Two ranks with uneven shards (20 + 17 walkers) must reach,
iteration after iteration, exactly what one rank reaches on the whole batch: the clipping
window, the Eq. 6 mean and the gradient are those of the whole batch, and the replicas'
parameters stay identical."""
import os

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import optim
from paper_2401_10287_gb300 import TrainConfig, dp

P, B, N = 6, 37, 2


class CpuStandIn:
    """The System calls train_step makes, on CPU tensors (float64)."""

    def log_psi(self, params, walkers):
        return torch.zeros(walkers.shape[0], dtype=torch.float64), None

    def mcmc_steps(self, params, walkers, log_psi, n_steps, step_size, seed, step_offset=0, accept_count=None):
        walkers.mul_(1.0 - 0.01 * n_steps).add_(0.001 * (step_offset + 1))

    def _features(self, walkers):
        r = walkers.reshape(walkers.shape[0], -1)
        # no constant column: its Eq. 6 gradient would be zero up to rounding, which Adam's
        # g / (|g| + eps) turns into a summation-order-dependent step
        return torch.stack([r.sum(1), (r * r).sum(1), r[:, 0], torch.sin(r).sum(1), r.abs().sum(1),
                            r[:, 1] ** 3], 1)

    def local_energy(self, params, walkers):
        f = self._features(walkers)
        e = f @ params + 40.0 * torch.tan(1.4 * torch.tanh(f[:, 0]))        # heavy tails for clipping
        return e, None, None

    def clip_local_energy(self, e, width):
        c, centre, spread = optim.clip_local_energy(e.numpy(), width)
        return torch.from_numpy(c), torch.tensor([centre, spread])

    def log_psi_vjp(self, params, walkers, weights):
        return weights @ (self._features(walkers) * torch.cos(params))

    def adam_step(self, params, g, m, v, t, lr, beta1, beta2, eps):
        p2, m2, v2 = optim.adam_step(params.numpy(), g.numpy(), m.numpy(), v.numpy(), t, lr, beta1, beta2, eps)
        params.copy_(torch.from_numpy(p2))
        m.copy_(torch.from_numpy(m2))
        v.copy_(torch.from_numpy(v2))

    def sgd_step(self, params, g, lr):
        params.sub_(lr * g)

    def energy_moments(self, e):
        return torch.stack([torch.tensor(float(e.numel()), dtype=torch.float64), e.sum(), (e * e).sum()])

    def energy_weights(self, e, m):
        return 2.0 * (e - m[1] / m[0]) / m[0]


def _walkers():
    return torch.from_numpy(np.random.default_rng(7).standard_normal((B, N, 3)))


def _run(rank, world, port, out_path, shards, clip_per_shard):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shards[rank]
    walkers = _walkers()[lo:hi].clone()
    params = torch.linspace(-0.5, 0.5, P, dtype=torch.float64)
    m, v = torch.zeros(P, dtype=torch.float64), torch.zeros(P, dtype=torch.float64)
    cfg = TrainConfig(n_mcmc_steps=2, step_size=0.1, seed=1, clip_width=1.0, lr=0.05)
    sys_ = CpuStandIn()
    if clip_per_shard:                    # the mistake the global window avoids
        dp.clip_global = lambda s, e, w, group=None: s.clip_local_energy(e, w)[0]
    rows = []
    for it in range(3):
        e, g = dp.train_step(sys_, cfg, params, walkers, it, m, v)
        rows.append(np.concatenate([params.numpy(), g.numpy()]))
    gathered = [torch.zeros(3 * 2 * P, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, torch.from_numpy(np.concatenate(rows)))
    if rank == 0:
        np.save(out_path, torch.stack(gathered).numpy())
    dist.barrier()
    dist.destroy_process_group()


def _spawn(tmp_path, name, world, shards, clip_per_shard=False):
    out = str(tmp_path / f"{name}.npy")
    port = 29600 + (os.getpid() + 37 * world + (5 if clip_per_shard else 0)) % 1000
    mp.spawn(_run, args=(world, port, out, shards, clip_per_shard), nprocs=world, join=True)
    return np.load(out)


def test_two_rank_training_equals_one_rank(tmp_path):
    one = _spawn(tmp_path, "one", 1, [(0, B)])
    two = _spawn(tmp_path, "two", 2, [(0, 20), (20, B)])
    np.testing.assert_array_equal(two[0], two[1])                   # replicas stay identical
    np.testing.assert_allclose(two[0], one[0], rtol=1e-12, atol=1e-13)
    bad = _spawn(tmp_path, "bad", 2, [(0, 20), (20, B)], clip_per_shard=True)
    assert np.max(np.abs(bad[0] - one[0])) > 1e-6                  # per-shard clipping differs
