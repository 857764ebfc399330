"""GB300 (sm_103a) implementation of CoNCPD-APG and lraCoNCPD-APG
(coupled nonnegative CP decomposition by alternating proximal gradient,
arXiv 2302.05119) behind the C ABI of include/cncpd.h.

    from paper_2302_05119_gb300 import CoupledNCP
    m = CoupledNCP(tensors, R=10, L=[3, 3, 0])
    m.set_factors(U0)
    stats = m.fit()

The CUDA library must be built first (``__graft_entry__.build()`` or
``python -m paper_2302_05119_gb300.build``); the first call into it raises
ImportError if it is missing (there is no fallback implementation).
"""

from . import _lib  # noqa: F401
from ._lib import CncpdError, lib  # noqa: F401
from .api import CoupledCPLoss, CoupledNCP, default_opts, lipschitz  # noqa: F401
