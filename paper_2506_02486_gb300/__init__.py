"""GB300 (sm_103a) Minimod acoustic-isotropic library.

The CUDA library ``libgbwave.so`` (C ABI in ``include/gbwave.h``) holds the
whole time step; :mod:`.gbwave` binds it with ctypes and :mod:`.runtime`
adds a PyTorch-owned global segment and a small shot helper.
"""

from .buildlib import build  # noqa: F401

__all__ = ["build"]
