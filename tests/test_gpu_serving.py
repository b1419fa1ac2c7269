"""Serving through the library: every job's energy is the same alone and in the mix."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    yield
    torch.cuda.synchronize()


def _mix():
    from paper_2401_10287_gb300 import serve
    systems = [W.hydrogen_atom(), W.atom(3, 1), W.atom(6), W.atom(8, -1), W.lih(), W.h2(), W.n2(), W.atom(1, 1),
               W.co(), W.atom(14, -1)]
    jobs = [W.Job(i, 0.0, s, nw, 10, 0.05, 1.0, 100 + i)
            for i, (s, nw) in enumerate(zip(systems, [300, 256, 128, 200, 256, 64, 128, 100, 96, 80]))]
    return serve.requests_from_jobs(jobs)


@pytest.mark.parametrize("prec", [1, 2])
def test_alone_equals_mix(prec):
    import paper_2401_10287_gb300 as P
    from paper_2401_10287_gb300 import serve
    cfg = P.NetConfig(2, 32, 8, 2, P.ANISO, prec)
    reqs = _mix()
    be = serve.LibraryBackend(cfg)
    srv = serve.Server(be, memory_budget=40 << 30, slots=4, chunk_steps=3)
    mixed = {r.job_id: r for r in srv.run(reqs, realtime=False)}
    assert srv.max_concurrent > 1
    for req in reqs:
        alone = serve.Server(serve.LibraryBackend(cfg), memory_budget=40 << 30, slots=1).run([req], realtime=False)[0]
        m = mixed[req.job_id]
        assert np.isfinite(m.energy)
        assert abs(m.energy - alone.energy) <= 1e-10 * max(1.0, abs(alone.energy)), req.key
        assert m.acceptance == alone.acceptance
    assert mixed[7].energy == 0.0          # H+ has no electrons


def test_serving_stream_workload_prefix():
    """The serving workload (Poisson arrivals, atoms and diatomics, 4/256/32/16 BF16) on a prefix."""
    import paper_2401_10287_gb300 as P
    from paper_2401_10287_gb300 import serve
    jobs = W.serving_jobs(n_jobs=12, rate_per_s=50.0, seed=4, mcmc_steps=5)
    reqs = serve.requests_from_jobs(jobs)
    cfg = P.NetConfig.from_ansatz(W.SERVING_ANSATZ, P.BF16_MIXED)
    srv = serve.Server(serve.LibraryBackend(cfg), memory_budget=120 << 30, slots=6)
    res = srv.run(reqs)
    assert len(res) == 12
    assert srv.peak_footprint <= 120 << 30
    assert all(np.isfinite(r.energy) for r in res)
    summ = serve.summarize(res, max(r.done_s for r in res))
    assert summ["latency_ms"]["p99"] >= summ["latency_ms"]["p50"] > 0
