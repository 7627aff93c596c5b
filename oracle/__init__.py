"""FP64 CPU oracle for the mixed-state multislice ptychography forward model
and its adjoint (arXiv 2505.14372, "phaser", §3 and §3.1-§3.2).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA path: it has its own
dense DFT (no ``numpy.fft``), its own frequency grids, propagators, loss and
adjoint, all in complex128 / float64.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants and brute-force finite differences (no worked example is printed
in the paper).  What no test can decide is bit-level agreement with the
paper's own package, whose conventions (DFT sign, normalisation, band-limit
shape, epsilon placement) are not printed; the readings taken here are
listed in ``ptycho.py``'s module docstring.
"""
from .ptycho import *  # noqa: F401,F403
