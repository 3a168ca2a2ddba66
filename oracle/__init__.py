"""FP64 CPU oracle for COLATUS (arXiv 1208.3444): comoving all-pairs gravity,
Friedmann expansion and the Hubble-drag leapfrog.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_1208_3444_b300``) and imports nothing from it.

Every function states the passage of the paper it follows.  The O(N^2) pair
sums live in ``colatus_oracle.c`` (plain double loops); the integrators, the
Friedmann solver, diagnostics, the discrete adjoint and the tangent model are
plain NumPy written in the paper's order.

Parity status of each function is listed in ``PINS`` below; every entry is
pinned by a ``-m "not gpu"`` test against something other than the oracle
itself (closed forms, invariants, finite differences, brute force).
"""
from .core import *  # noqa: F401,F403
from .core import PINS  # noqa: F401
