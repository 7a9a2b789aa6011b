"""GB300 (sm_103a) library for the Krylov step of the PCEXP exponential
integrator on DG Euler (Li, Luo, Wang & Ju).

The compute path is the CUDA library ``libpcexp.so`` behind the C interface of
``include/pcexp.h``; this package only builds it (``build``) and marshals
arguments to it (``capi``).  There is no CPU fallback: importing ``capi``
without the built library raises.
"""
from .build import build  # noqa: F401
