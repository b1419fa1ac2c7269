"""The C-ABI library builds and exports every entry point include/fnvmc.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "fnvmc.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:fn_status|int64_t|int|const char\*)\s+(fn_\w+)\s*\(", text, re.M)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("fn_create_system", "fn_init_walkers", "fn_mcmc_steps", "fn_local_energy", "fn_energy_grad",
              "fn_log_psi_noalloc", "fn_adam_step", "fn_sgd_step", "fn_clip_local_energy", "fn_vmc_iteration",
              "fn_mulliken_charges"
              ):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2401_10287_gb300 import build as B
    lib_path = B.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_2401_10287_gb300 import _lib
    assert set(_declared()) <= set(_lib.SIGNATURES)
