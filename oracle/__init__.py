"""Plain FP64 CPU oracle of the space-time reduced-order model.

TEST INFRASTRUCTURE ONLY.  This package is a slow, direct restatement of the
method (full-order march, POD, block assembly of the space-time reduced
operators, reduced solve, reconstruction) used to check the CUDA path.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product library never calls it and shares no
code with it.  Every function cites the section / equation of the paper it
follows.

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, an identity the paper states, a library routine used as an
independent solver, or brute force on tiny inputs, except where a docstring
says "parity unpinned".
"""
from . import fom, mlp, pod, strom  # noqa: F401
