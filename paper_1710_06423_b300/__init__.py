"""SAC-family 2D ideal-MHD step on one B300 GPU (arXiv 1710.06423, section 2).

The hot path lives in ``libsac.so`` (CUDA for sm_103a, C ABI in
``include/sac.h``); :mod:`.sac` is its ctypes binding and :mod:`.inputs` the
seeded initial states.  Importing the package does not load the library;
``Solver`` does, and fails loudly if it has not been built.
"""
from . import inputs  # noqa: F401


def __getattr__(name):
    if name in ("Solver", "SacError", "load"):
        from . import sac
        return getattr(sac, name)
    raise AttributeError(name)
