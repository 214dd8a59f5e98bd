"""GB300 (sm_103a) observer-siting hot path: vix, findmax, viewshed and site
kernels, the learned candidate proposal, behind the C ABI of
include/vshed.h, with a thin ctypes binding (vshed.py)."""
from . import vshed as _vshed
from .vshed import *  # noqa: F401,F403

__all__ = [n for n in dir(_vshed) if not n.startswith("_") and n not in ("ctypes", "os", "torch")]
