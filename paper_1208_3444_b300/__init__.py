"""COLATUS hot path on B300 (sm_103a): comoving all-pairs gravity (arXiv
1208.3444, Eq. 1) fused with the Hubble-drag leapfrog (Eqs. 3-5) and FP64
Friedmann expansion (Eq. 2).

``binding`` is the ctypes layer over the C ABI ``include/colatus.h``
(libcolatus.so, built by ``build``); ``inputs`` draws seeded synthetic
initial conditions.  Importing the package does not load the CUDA library;
the first binding call does, and fails loudly if it is missing.
"""
__all__ = ["binding", "inputs", "build"]
