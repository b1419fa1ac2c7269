"""Torch-facing wrappers of the C ABI.  PyTorch provides device memory and streams only;
every step of the path runs in libfnvmc.so."""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from . import _lib

FP64, FP32, BF16_MIXED = 0, 1, 2
ISO, ANISO = 0, 1
_STATUS = {0: "FN_OK", 1: "FN_ERR_ARG", 2: "FN_ERR_OOM", 3: "FN_ERR_CUDA", 4: "FN_ERR_TIMEOUT",
           5: "FN_ERR_NUMERIC", 6: "FN_ERR_EMPTY", 7: "FN_ERR_UNSUPPORTED"}


class FnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return _lib.LIB_PATH


def load_library():
    return _lib.load()


def _check(code: int):
    if code != 0:
        raise FnError(code, _lib.load().fn_last_error().decode())


@dataclass(frozen=True)
class NetConfig:
    n_layers: int
    h1: int
    h2: int
    n_dets: int
    envelope: int = ISO
    precision: int = FP64

    @staticmethod
    def from_ansatz(ansatz, precision: int) -> "NetConfig":
        env = ANISO if ansatz.envelope == "aniso" else ISO
        return NetConfig(ansatz.n_layers, ansatz.h1, ansatz.h2, ansatz.n_dets, env, precision)


OPT_ADAM, OPT_SGD = 0, 1


@dataclass(frozen=True)
class TrainConfig:
    """Settings of one VMC training iteration (fn_train_config)."""
    n_mcmc_steps: int = 10
    step_size: float = 0.02
    seed: int = 0
    clip_width: float = 0.0
    optimizer: str = "adam"          # "adam" or "sgd"
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8

    def c_struct(self) -> _lib.TrainConfigC:
        opt = {"adam": OPT_ADAM, "sgd": OPT_SGD}[self.optimizer]
        return _lib.TrainConfigC(int(self.n_mcmc_steps), float(self.step_size), int(self.seed),
                                 float(self.clip_width), opt, float(self.lr), float(self.beta1),
                                 float(self.beta2), float(self.eps))


def _check_f64(t: torch.Tensor, n: int, name: str):
    if t.dtype != torch.float64 or t.numel() != n or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 tensor of {n} elements")


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def mulliken_charges(nuclei, charges, n_up: int, n_down: int) -> Tuple[np.ndarray, float]:
    """(Mulliken partial charges [M], UHF energy) in STO-6G for nuclei of H..Ne: the partial
    charges Algorithm 1 takes (fn_mulliken_charges, computed on the host)."""
    lib = _lib.load()
    nuc = np.ascontiguousarray(np.asarray(nuclei, dtype=np.float64).reshape(-1, 3))
    z = np.ascontiguousarray(np.asarray(charges, dtype=np.float64))
    q = np.zeros(z.shape[0])
    e = np.zeros(1)
    _check(lib.fn_mulliken_charges(nuc.ctypes.data_as(_lib._D), z.ctypes.data_as(_lib._D), int(z.shape[0]),
                                   int(n_up), int(n_down), q.ctypes.data_as(_lib._D), e.ctypes.data_as(_lib._D)))
    return q, float(e[0])


class System:
    """A molecule (nuclei, charges, spins) plus a network configuration on the current device."""

    def __init__(self, nuclei, charges, n_up: int, n_down: int, cfg: NetConfig):
        lib = _lib.load()
        self._lib = lib
        self.nuclei = np.ascontiguousarray(np.asarray(nuclei, dtype=np.float64).reshape(-1, 3))
        self.charges = np.ascontiguousarray(np.asarray(charges, dtype=np.float64).reshape(-1))
        self.n_up, self.n_down, self.cfg = int(n_up), int(n_down), cfg
        self.n_el = self.n_up + self.n_down
        c = _lib.NetConfigC(cfg.n_layers, cfg.h1, cfg.h2, cfg.n_dets, cfg.envelope, cfg.precision)
        h = C.c_void_p()
        _check(lib.fn_create_system(self.nuclei.ctypes.data_as(_lib._D), self.charges.ctypes.data_as(_lib._D),
                                    self.nuclei.shape[0], self.n_up, self.n_down, C.byref(c), C.byref(h)))
        self._h = h
        self.param_count = int(lib.fn_param_count(h))
        self.dtype = torch.float64 if cfg.precision == FP64 else torch.float32

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fn_destroy_system(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- host-side -------------------------------------------------------------------
    def workspace_bytes(self, n_walkers: int) -> int:
        return int(self._lib.fn_workspace_bytes(self._h, int(n_walkers)))

    def set_walker_offset(self, offset: int):
        _check(self._lib.fn_set_walker_offset(self._h, int(offset)))

    def mulliken_partial_charges(self) -> np.ndarray:
        """STO-6G UHF Mulliken charges of this molecule (H..Ne), the input Algorithm 1 takes."""
        return mulliken_charges(self.nuclei, self.charges, self.n_up, self.n_down)[0]

    def assign_electrons(self, partial_charges: Optional[Sequence[float]] = None):
        counts = (C.c_int * self.nuclei.shape[0])()
        atoms = (C.c_int * self.n_el)()
        pc = None
        if partial_charges is not None:
            arr = np.ascontiguousarray(np.asarray(partial_charges, dtype=np.float64))
            pc = arr.ctypes.data_as(_lib._D)
        _check(self._lib.fn_assign_electrons(self._h, pc, counts, atoms))
        return list(counts), list(atoms)

    # -- device-side -----------------------------------------------------------------
    def init_params(self, seed: int, device="cuda", stream=None) -> torch.Tensor:
        p = torch.empty(self.param_count, dtype=self.dtype, device=device)
        _check(self._lib.fn_init_params(self._h, int(seed), _ptr(p), _stream(stream)))
        return p

    def init_walkers(self, n_walkers: int, seed: int, init_std: float,
                     partial_charges: Optional[Sequence[float]] = None, device="cuda", stream=None):
        r = torch.empty((n_walkers, self.n_el, 3), dtype=self.dtype, device=device)
        counts = (C.c_int * self.nuclei.shape[0])()
        pc = None
        if partial_charges is not None:
            arr = np.ascontiguousarray(np.asarray(partial_charges, dtype=np.float64))
            pc = arr.ctypes.data_as(_lib._D)
        _check(self._lib.fn_init_walkers(self._h, int(n_walkers), int(seed), float(init_std), pc, _ptr(r), counts,
                                         _stream(stream)))
        return r, list(counts)

    def _check_walkers(self, params: torch.Tensor, walkers: torch.Tensor):
        if params.dtype != self.dtype or walkers.dtype != self.dtype:
            raise FnError(1, f"params and walkers must be {self.dtype}")
        if not (params.is_cuda and walkers.is_cuda and params.is_contiguous() and walkers.is_contiguous()):
            raise FnError(1, "params and walkers must be contiguous CUDA tensors")
        if params.numel() != self.param_count or walkers.shape[1:] != (self.n_el, 3):
            raise FnError(1, "parameter or walker shape mismatch")

    def log_psi(self, params, walkers, stream=None) -> Tuple[torch.Tensor, torch.Tensor]:
        self._check_walkers(params, walkers)
        B = walkers.shape[0]
        lp = torch.empty(B, dtype=torch.float64, device=walkers.device)
        sg = torch.empty(B, dtype=torch.int8, device=walkers.device)
        _check(self._lib.fn_log_psi(self._h, _ptr(params), _ptr(walkers), B, _ptr(lp), _ptr(sg), _stream(stream)))
        return lp, sg

    def log_psi_noalloc(self, params, walkers, stream=None) -> Tuple[torch.Tensor, torch.Tensor]:
        """log|psi| with the library's static scratch (no device allocation inside the call);
        the output tensors are allocated here, by the caller side."""
        self._check_walkers(params, walkers)
        B = walkers.shape[0]
        lp = torch.empty(B, dtype=torch.float64, device=walkers.device)
        sg = torch.empty(B, dtype=torch.int8, device=walkers.device)
        _check(self._lib.fn_log_psi_noalloc(self._h, _ptr(params), _ptr(walkers), B, _ptr(lp), _ptr(sg),
                                            _stream(stream)))
        return lp, sg

    def mcmc_steps(self, params, walkers, log_psi, n_steps: int, step_size: float, seed: int,
                   step_offset: int = 0, accept_count: Optional[torch.Tensor] = None, stream=None):
        self._check_walkers(params, walkers)
        B = walkers.shape[0]
        _check(self._lib.fn_mcmc_steps(self._h, _ptr(params), _ptr(walkers), _ptr(log_psi), B, int(n_steps),
                                       float(step_size), int(seed), int(step_offset), _ptr(accept_count),
                                       _stream(stream)))

    def local_energy(self, params, walkers, stream=None):
        self._check_walkers(params, walkers)
        B = walkers.shape[0]
        e = torch.empty(B, dtype=torch.float64, device=walkers.device)
        lp = torch.empty(B, dtype=torch.float64, device=walkers.device)
        sg = torch.empty(B, dtype=torch.int8, device=walkers.device)
        _check(self._lib.fn_local_energy(self._h, _ptr(params), _ptr(walkers), B, _ptr(e), _ptr(lp), _ptr(sg),
                                         _stream(stream)))
        return e, lp, sg

    def energy_grad(self, params, walkers, e_local, stream=None):
        self._check_walkers(params, walkers)
        B = walkers.shape[0]
        g = torch.empty(self.param_count, dtype=self.dtype, device=walkers.device)
        mean = torch.empty(1, dtype=torch.float64, device=walkers.device)
        e_local = e_local.to(torch.float64).contiguous()
        _check(self._lib.fn_energy_grad(self._h, _ptr(params), _ptr(walkers), _ptr(e_local), B, _ptr(g), _ptr(mean),
                                        _stream(stream)))
        return g, mean

    def log_psi_vjp(self, params, walkers, weights, stream=None):
        """sum_w weights[w] d log|psi_w| / d theta (blob order, blob dtype)."""
        self._check_walkers(params, walkers)
        B = walkers.shape[0]
        g = torch.empty(self.param_count, dtype=self.dtype, device=walkers.device)
        weights = weights.to(torch.float64).contiguous()
        _check(self._lib.fn_log_psi_vjp(self._h, _ptr(params), _ptr(walkers), _ptr(weights), B, _ptr(g),
                                        _stream(stream)))
        return g

    def pretrain_setup(self) -> float:
        """UHF/STO-6G of this molecule on the host; its occupied orbitals become the Eq. 5
        targets of pretrain_grad.  Returns the UHF energy."""
        e = np.zeros(1)
        _check(self._lib.fn_pretrain_setup(self._h, e.ctypes.data_as(_lib._D)))
        return float(e[0])

    def pretrain_grad(self, params, walkers, stream=None):
        """(gradient of the Eq. 5 loss [param_count] blob dtype, loss [1] float64)."""
        self._check_walkers(params, walkers)
        B = walkers.shape[0]
        g = torch.empty(self.param_count, dtype=self.dtype, device=walkers.device)
        loss = torch.empty(1, dtype=torch.float64, device=walkers.device)
        _check(self._lib.fn_pretrain_grad(self._h, _ptr(params), _ptr(walkers), B, _ptr(g), _ptr(loss),
                                          _stream(stream)))
        return g, loss

    def energy_moments(self, e_local, stream=None) -> torch.Tensor:
        """[count, sum E_L, sum E_L^2] (float64, on the device); sums over batches and devices."""
        _check_f64(e_local, e_local.numel(), "e_local")
        mom = torch.empty(3, dtype=torch.float64, device=e_local.device)
        _check(self._lib.fn_energy_moments(self._h, _ptr(e_local), int(e_local.numel()), _ptr(mom), _stream(stream)))
        return mom

    def energy_stats(self, moments, stream=None) -> torch.Tensor:
        """[count, mean, variance] of the local energies (Eq. 1) from (possibly summed) moments."""
        _check_f64(moments, 3, "moments")
        st = torch.empty(3, dtype=torch.float64, device=moments.device)
        _check(self._lib.fn_energy_stats(self._h, _ptr(moments), _ptr(st), _stream(stream)))
        return st

    def energy_weights(self, e_local, moments, stream=None) -> torch.Tensor:
        """Eq. 6 weights 2 (E_L - mean) / count with the mean and count of `moments`."""
        _check_f64(e_local, e_local.numel(), "e_local")
        _check_f64(moments, 3, "moments")
        w = torch.empty_like(e_local)
        _check(self._lib.fn_energy_weights(self._h, _ptr(e_local), int(e_local.numel()), _ptr(moments), _ptr(w),
                                           _stream(stream)))
        return w

    def _check_blob(self, *tensors):
        for t in tensors:
            if t.dtype != self.dtype or t.numel() != self.param_count or not t.is_contiguous():
                raise ValueError(f"expected a contiguous {self.dtype} blob of {self.param_count} elements")

    def adam_step(self, params, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-8, stream=None):
        """In-place Adam update of params (and of its moments m, v); step counts from 1."""
        self._check_blob(params, grad, m, v)
        _check(self._lib.fn_adam_step(self._h, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr),
                                      float(beta1), float(beta2), float(eps), _stream(stream)))

    def sgd_step(self, params, grad, lr: float, stream=None):
        self._check_blob(params, grad)
        _check(self._lib.fn_sgd_step(self._h, _ptr(params), _ptr(grad), float(lr), _stream(stream)))

    def clip_local_energy(self, e_local, width: float, out=None, stream=None):
        """(clipped energies, [centre, spread]); out may be e_local itself."""
        if e_local.dtype != torch.float64 or not e_local.is_contiguous():
            raise ValueError("e_local must be a contiguous float64 tensor")
        B = e_local.shape[0]
        out = torch.empty_like(e_local) if out is None else out
        _check_f64(out, B, "out")
        stats = torch.empty(2, dtype=torch.float64, device=e_local.device)
        _check(self._lib.fn_clip_local_energy(self._h, _ptr(e_local), B, float(width), _ptr(out), _ptr(stats),
                                              _stream(stream)))
        return out, stats

    def vmc_iteration(self, cfg: TrainConfig, params, walkers, iteration: int, opt_state, grad, log_psi, e_local,
                      e_mean=None, accept_count=None, stream=None):
        """One training iteration (fn_vmc_iteration); every tensor argument is updated in place."""
        self._check_walkers(params, walkers)
        self._check_blob(params, grad)
        if opt_state is not None and (opt_state.dtype != self.dtype or opt_state.numel() != 2 * self.param_count):
            raise ValueError("opt_state must hold 2 * param_count elements of the blob dtype")
        B = walkers.shape[0]
        _check_f64(log_psi, B, "log_psi")
        _check_f64(e_local, B, "e_local")
        if e_mean is not None:
            _check_f64(e_mean, 1, "e_mean")
        if accept_count is not None and (accept_count.dtype != torch.int64 or accept_count.numel() != 1):
            raise ValueError("accept_count must be a one-element int64 tensor")
        c = cfg.c_struct()
        _check(self._lib.fn_vmc_iteration(self._h, C.byref(c), _ptr(params), _ptr(walkers), B, int(iteration),
                                          _ptr(opt_state), _ptr(grad), _ptr(log_psi), _ptr(e_local), _ptr(e_mean),
                                          _ptr(accept_count), _stream(stream)))

    def selftest_expired_wait(self, wait_us: int = 2000, stream=None):
        """Enqueues a kernel whose bounded barrier wait expires (fn_selftest_expired_wait);
        the next sync() raises FnError with FN_ERR_TIMEOUT."""
        _check(self._lib.fn_selftest_expired_wait(self._h, int(wait_us), _stream(stream)))

    def profile_enable(self, enable: bool = True):
        _check(self._lib.fn_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        """{kernel class: (launches, total device ms)} since the last enable."""
        out = {}
        n = self._lib.fn_profile_read(self._h, -1, None, None, None)
        for i in range(n):
            name = C.c_char_p()
            cnt = C.c_int64()
            ms = C.c_double()
            self._lib.fn_profile_read(self._h, i, C.byref(name), C.byref(cnt), C.byref(ms))
            if cnt.value:
                out[name.value.decode()] = (int(cnt.value), float(ms.value))
        return out

    def sync(self, timeout_ms: int = 60000, stream=None):
        _check(self._lib.fn_sync(self._h, _stream(stream), int(timeout_ms)))


class EnergyGrad(torch.autograd.Function):
    """Surrogate loss whose gradient with respect to the parameters is Eq. 6.

    forward(params, walkers, e_local, system) returns mean E_L (a scalar); backward
    multiplies the library's VMC gradient by the incoming scalar.  The value-only
    forward is recomputed inside the library, no activations are kept.
    """

    @staticmethod
    def forward(ctx, params, walkers, e_local, system: System):
        g, mean = system.energy_grad(params.detach(), walkers, e_local)
        ctx.save_for_backward(g)
        return mean.to(params.dtype).reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return g * grad_out, None, None, None
