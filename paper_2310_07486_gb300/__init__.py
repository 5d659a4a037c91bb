"""GB300 (sm_103a) Monte Carlo of the Trotter-Suzuki 2D +-1 Ising spin glass in
a transverse field, with parallel tempering and the imaginary-time correlators
C(tau), Q2(tau) (arXiv 2310.07486).  See ``qsg.py`` for the binding of the C ABI
declared in ``include/qsg.h``."""
from .qsg import (APBC, HEATBATH, METROPOLIS, PBC, Context, QSGError, Shape, load_library, pack_spins,
                  qsg_workspace_bytes, unpack_spins)

__all__ = ["APBC", "HEATBATH", "METROPOLIS", "PBC", "Context", "QSGError", "Shape", "load_library", "pack_spins",
           "qsg_workspace_bytes", "unpack_spins"]
