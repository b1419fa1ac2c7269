"""VMC training loop: parameters, persistent walkers and optimiser state, advanced by one
``fn_vmc_iteration`` per step (log|psi|, Metropolis, local energies, clipping, the Eq. 6
gradient and the Adam or gradient-descent update, all in libfnvmc.so)."""
from __future__ import annotations

from typing import List, Optional

import torch

from .api import System, TrainConfig


class Trainer:
    """Owns the device buffers of the loop; ``params`` and ``walkers`` are updated in place."""

    def __init__(self, system: System, params: torch.Tensor, walkers: torch.Tensor, cfg: TrainConfig):
        self.system = system
        self.cfg = cfg
        self.params = params
        self.walkers = walkers
        dev, B, P = walkers.device, walkers.shape[0], system.param_count
        self.opt_state = (torch.zeros(2 * P, dtype=system.dtype, device=dev) if cfg.optimizer == "adam" else None)
        self.grad = torch.empty(P, dtype=system.dtype, device=dev)
        self.log_psi = torch.empty(B, dtype=torch.float64, device=dev)
        self.e_local = torch.empty(B, dtype=torch.float64, device=dev)
        self.e_mean = torch.empty(1, dtype=torch.float64, device=dev)
        self.accepted = torch.zeros(1, dtype=torch.int64, device=dev)
        self.iteration = 0
        # the zero fills above run on the current stream; iterations may be enqueued on another
        torch.cuda.current_stream(dev).synchronize()

    def step(self, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        """Enqueues one iteration; returns the device tensor holding the mean (clipped) energy."""
        self.system.vmc_iteration(self.cfg, self.params, self.walkers, self.iteration, self.opt_state, self.grad,
                                  self.log_psi, self.e_local, self.e_mean, self.accepted, stream)
        self.iteration += 1
        return self.e_mean

    def run(self, n_iterations: int, stream: Optional[torch.cuda.Stream] = None) -> List[float]:
        """n iterations; the mean energies are gathered on the device (on the same stream as the
        iterations) and read back once."""
        stream = stream if stream is not None else torch.cuda.current_stream(self.walkers.device)
        means = torch.empty(n_iterations, dtype=torch.float64, device=self.walkers.device)
        with torch.cuda.stream(stream):
            for k in range(n_iterations):
                means[k : k + 1].copy_(self.step(stream))
        self.system.sync(stream=stream)
        return means.cpu().tolist()
