"""GB300 (sm_103a) implementation of the staggered-grid real-valued P_N
operator and the Krylov solves built on it (Koerner, Portsmouth and Jakob,
"P_N-Method for Multiple Scattering in Participating Media", EGSR 2018).

The compute path is the CUDA library libpn_gb300.so (C ABI in
include/pn_gb300.h); `pn.System` is a thin ctypes binding over it.
"""
from .pn import (PN_F32, PN_F64, Batch, Layout, Net, PnError, System, load_library)  # noqa: F401

__all__ = ["System", "Batch", "Net", "Layout", "PnError", "load_library", "PN_F32", "PN_F64"]
