"""GB300 (sm_103a) variational Monte Carlo hot path for a FermiNet-style wavefunction.

The computation runs in ``libfnvmc.so`` (CUDA kernels behind the C ABI of
``include/fnvmc.h``); this package only marshals arguments (``_lib``, ``api``) and
builds the library (``build``).  Importing the package does not load the library;
the first call that needs it does, and fails loudly if it is missing.
"""
from .api import (FP32, FP64, BF16_MIXED, ISO, ANISO, NetConfig, FnError, System, EnergyGrad, TrainConfig,
                  library_path, load_library, mulliken_charges)
from .train import Trainer

__all__ = ["FP32", "FP64", "BF16_MIXED", "ISO", "ANISO", "NetConfig", "FnError", "System", "EnergyGrad",
           "TrainConfig", "Trainer", "library_path", "load_library", "mulliken_charges"]
