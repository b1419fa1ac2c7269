"""Failure detection without a fault: a kernel's bounded barrier wait expires, fn_sync reports
FN_ERR_TIMEOUT and clears the status, and the same context keeps computing the same results.
This file is collected last, so a run stopping at the first failure has run every other test."""
import time

import pytest
import torch

import workloads as W
from gpu_helpers import make_pair, need_gpu

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_and_the_context_survives():
    need_gpu()
    import paper_2401_10287_gb300 as P
    net, gpu = make_pair(W.lih(1), W.Ansatz(2, 32, 8, 2, "aniso"), 1)
    p = gpu.init_params(0)
    w, _ = gpu.init_walkers(64, 1, 0.5)
    lp0, sg0 = gpu.log_psi(p, w)
    gpu.sync()
    t0 = time.perf_counter()
    gpu.selftest_expired_wait(2000)                 # 2 ms barrier wait that nothing completes
    with pytest.raises(P.FnError) as err:
        gpu.sync()
    assert err.value.code == 4 and "expired" in str(err.value)
    assert time.perf_counter() - t0 < 5.0
    gpu.sync()                                      # the status word was cleared
    lp1, sg1 = gpu.log_psi(p, w)
    gpu.sync()
    torch.testing.assert_close(lp1, lp0, rtol=0, atol=1e-6)
    assert torch.equal(sg1, sg0)
    with pytest.raises(P.FnError) as err:
        gpu.selftest_expired_wait(0)
    assert err.value.code == 1
