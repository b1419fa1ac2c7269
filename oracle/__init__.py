"""FP64 CPU oracle of the variational Monte Carlo hot path (TEST INFRASTRUCTURE ONLY).

This package is the plain, slow reference that the CUDA path is checked
against.  It is written from the method's definitions (Eqs. 1-6, Algorithm 1,
the electron-sampler and FermiNet-model sections) in float64 NumPy and shares
no code with the CUDA library: no kernels, headers, helpers, tables or
constant generators.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product path never does.

Modules
  rng       Philox4x32-10 counter-based generator, Box-Muller normals and the
            streams used for walker initialisation, proposals, acceptance and
            parameter initialisation.
  ionic     Algorithm 1 (ionic charge initialisation) and the spin split.
  ansatz    parameter layout, value-only log|psi|, forward-Laplacian jets,
            local energy (Eqs. 2-3), finite-difference Laplacian.
  mcmc      Metropolis-Hastings on |psi|^2.
  grad      VMC energy gradient (Eq. 6) by central finite differences.
  optim     Adam, gradient descent, local-energy clipping and the training iteration.
  scf       STO-6G (fitted here) UHF and Mulliken charges, the partial charges of
            Algorithm 1.

Parity status: every function is pinned by tests under ``tests/`` (closed
forms, invariants, brute force, finite differences, library routines).  The
LiH ionisation potential of Table 1 and the H2 curve of Fig. 1 need trained
networks and external data and are not reproduced (parity unpinned there).
"""
