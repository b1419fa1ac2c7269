"""The data-parallel exchange of Eq. 6 with two gloo ranks on the CPU.

Each rank holds a shard of local energies and per-walker gradients of log|psi|
(synthetic, seeded); the weights and the all-reduced gradient must equal the formula
evaluated on the whole batch by one process."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2401_10287_gb300 import dp


def _data():
    rs = np.random.default_rng(0)
    e = rs.normal(-10.0, 2.0, 37)                # uneven shards: 20 + 17 walkers
    dlogpsi = rs.standard_normal((37, 11))
    return e, dlogpsi


class _Moments:
    """CPU stand-in for the library's Eq. 1 / Eq. 6 calls (fn_energy_moments, fn_energy_stats,
    fn_energy_weights, whose GPU versions are tested against numpy in tests/test_gpu_stats.py):
    the test here is the exchange, not the arithmetic."""

    def energy_moments(self, e):
        return torch.stack([torch.tensor(float(e.numel()), dtype=torch.float64), e.sum(), (e * e).sum()])

    def energy_stats(self, m):
        mean = m[1] / m[0]
        return torch.stack([m[0], mean, m[2] / m[0] - mean * mean])

    def energy_weights(self, e, m):
        return 2.0 * (e - m[1] / m[0]) / m[0]


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    e, d = _data()
    lo, hi = (0, 20) if rank == 0 else (20, 37)
    e_l = torch.tensor(e[lo:hi])
    sysm = _Moments()
    w = dp.energy_weights(sysm, e_l)
    g = torch.tensor(w.numpy() @ d[lo:hi])       # the shard's weighted gradient (what fn_log_psi_vjp returns)
    dp.allreduce_gradient(g)
    mean, count = dp.global_mean_and_count(sysm, e_l)
    if rank == 0:
        np.save(out_path, np.concatenate([g.numpy(), [mean.item(), count.item()]]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gradient_equals_single_process(tmp_path):
    out = str(tmp_path / "g.npy")
    port = 29500 + (os.getpid() % 1000)
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    got = np.load(out)
    e, d = _data()
    ref = (2.0 * (e - e.mean()) / e.size) @ d
    np.testing.assert_allclose(got[:-2], ref, rtol=1e-12, atol=1e-12)
    assert abs(got[-2] - e.mean()) < 1e-12 and got[-1] == e.size
