"""GB300 (sm_103a) IgA Helmholtz solver: deflated, CSLP-multigrid-preconditioned
GMRES on B-spline discretisations (arXiv 2010.10232).

The compute path is the CUDA library ``lib/libiga_helmholtz.so`` (C ABI in
``include/iga_helmholtz.h``); this package only marshals arguments.  Import
is lazy: the library is loaded on first use and its absence raises.
"""
from .solver import Helmholtz, IgaError  # noqa: F401

__all__ = ["Helmholtz", "IgaError"]
