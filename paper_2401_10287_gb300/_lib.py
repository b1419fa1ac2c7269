"""ctypes declarations of the C ABI in include/fnvmc.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfnvmc.so")


class NetConfigC(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("h1", C.c_int), ("h2", C.c_int), ("n_dets", C.c_int),
                ("envelope", C.c_int), ("precision", C.c_int)]


class TrainConfigC(C.Structure):
    _fields_ = [("n_mcmc_steps", C.c_int), ("step_size", C.c_double), ("seed", C.c_uint64),
                ("clip_width", C.c_double), ("optimizer", C.c_int), ("lr", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)

SIGNATURES = {
    "fn_create_system": (C.c_int, [_D, _D, C.c_int, C.c_int, C.c_int, C.POINTER(NetConfigC), C.POINTER(_P)]),
    "fn_destroy_system": (C.c_int, [_P]),
    "fn_param_count": (C.c_int64, [_P]),
    "fn_workspace_bytes": (C.c_int64, [_P, C.c_int]),
    "fn_set_walker_offset": (C.c_int, [_P, C.c_uint64]),
    "fn_assign_electrons": (C.c_int, [_P, _D, _I, _I]),
    "fn_init_params": (C.c_int, [_P, C.c_uint64, _P, _P]),
    "fn_init_walkers": (C.c_int, [_P, C.c_int, C.c_uint64, C.c_double, _D, _P, _I, _P]),
    "fn_log_psi": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, _P]),
    "fn_mcmc_steps": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_int, C.c_double, C.c_uint64, C.c_uint64, _P, _P]),
    "fn_local_energy": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, _P, _P]),
    "fn_energy_grad": (C.c_int, [_P, _P, _P, _P, C.c_int, _P, _P, _P]),
    "fn_log_psi_noalloc": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, _P]),
    "fn_log_psi_vjp": (C.c_int, [_P, _P, _P, _P, C.c_int, _P, _P]),
    "fn_pretrain_setup": (C.c_int, [_P, _D]),
    "fn_pretrain_grad": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, _P]),
    "fn_energy_moments": (C.c_int, [_P, _P, C.c_int, _P, _P]),
    "fn_energy_stats": (C.c_int, [_P, _P, _P, _P]),
    "fn_energy_weights": (C.c_int, [_P, _P, C.c_int, _P, _P, _P]),
    "fn_adam_step": (C.c_int, [_P, _P, _P, _P, _P, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double, _P]),
    "fn_sgd_step": (C.c_int, [_P, _P, _P, C.c_double, _P]),
    "fn_clip_local_energy": (C.c_int, [_P, _P, C.c_int, C.c_double, _P, _P, _P]),
    "fn_vmc_iteration": (C.c_int, [_P, C.POINTER(TrainConfigC), _P, _P, C.c_int, C.c_int64, _P, _P, _P, _P, _P, _P,
                                   _P]),
    "fn_mulliken_charges": (C.c_int, [_D, _D, C.c_int, C.c_int, C.c_int, _D, _D]),
    "fn_selftest_expired_wait": (C.c_int, [_P, C.c_int, _P]),
    "fn_profile_enable": (C.c_int, [_P, C.c_int]),
    "fn_profile_read": (C.c_int, [_P, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "fn_sync": (C.c_int, [_P, _P, C.c_int]),
    "fn_last_error": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads the shared library and declares every exported entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
                           " (there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
