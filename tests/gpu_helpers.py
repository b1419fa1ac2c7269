"""Shared set-up of the GPU parity tests: one system built twice, as an oracle
``Net`` and as a library ``System``, from the same workload description."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import ansatz


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def make_pair(sysm, ans, precision):
    import paper_2401_10287_gb300 as P
    net = ansatz.Net(sysm.nuclei.shape[0], sysm.n_up, sysm.n_down, ans.n_layers, ans.h1, ans.h2, ans.n_dets,
                     ans.envelope)
    gpu = P.System(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down, P.NetConfig.from_ansatz(ans, precision))
    return net, gpu


def oracle_params(net, seed, perturb=0.0):
    p = ansatz.init_params(net, seed)
    if perturb:
        p = p + perturb * np.random.default_rng(seed + 100).standard_normal(p.shape)
    return p


def to_dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype).cuda().contiguous()
