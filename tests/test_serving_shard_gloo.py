"""Serving split by job across GPUs (one process per GPU): two gloo ranks on the CPU, each
running the continuous-batching server with the fake backend on its shard of the stream.
Every job is served exactly once, with no collective while serving; the results gathered
afterwards are the whole stream on every rank."""
import os

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2401_10287_gb300 import serve

import workloads as W


def _requests():
    return serve.requests_from_jobs(W.serving_jobs(n_jobs=40, rate_per_s=2000.0, seed=4, mcmc_steps=10))


def _run(rank, world, port, out_path):
    from test_serving_scheduler import FakeBackend
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = serve.shard_requests(_requests(), rank, world)
    srv = serve.Server(FakeBackend(), memory_budget=12_000_000, slots=4)
    res = srv.run(mine)
    assert srv.peak_footprint <= 12_000_000
    everything = serve.gather_results(res)
    np.save(out_path + f".{rank}.npy", np.array([[r.job_id, r.energy, len(mine)] for r in everything]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_serving_covers_every_job_once(tmp_path):
    out = str(tmp_path / "res")
    port = 29700 + os.getpid() % 1000
    mp.spawn(_run, args=(2, port, out), nprocs=2, join=True)
    a, b = np.load(out + ".0.npy"), np.load(out + ".1.npy")
    np.testing.assert_array_equal(a[:, :2], b[:, :2])               # same gathered stream on both ranks
    reqs = _requests()
    assert sorted(a[:, 0].astype(int).tolist()) == sorted(r.job_id for r in reqs)
    for row, r in zip(a, sorted(reqs, key=lambda r: r.job_id)):
        assert row[1] == (-(r.n_up + r.n_down) if r.n_up + r.n_down else row[1])


def test_shards_partition_the_stream_in_arrival_order():
    reqs = _requests()
    shards = [serve.shard_requests(reqs, k, 3) for k in range(3)]
    ids = [r.job_id for s in shards for r in s]
    assert sorted(ids) == sorted(r.job_id for r in reqs)
    assert max(len(s) for s in shards) - min(len(s) for s in shards) <= 1
    for s in shards:
        assert [r.arrival_s for r in s] == sorted(r.arrival_s for r in s)
