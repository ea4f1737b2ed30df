"""GB300 (sm_103a) library for joint reconstruction of initial pressure and
speed of sound in 2-D photoacoustic tomography (arXiv 2505.08482).

The compute runs in hand-written CUDA kernels behind the C ABI of
``include/pat.h`` (``libpat.so``, built in-tree by :func:`build`); this
package marshals arguments from PyTorch tensors.
"""
from ._build import build, LIB  # noqa: F401

__all__ = ["build", "LIB", "Plan", "GridSpec", "pml_auto"]


def __getattr__(name):
    if name in ("Plan", "GridSpec", "pml_auto"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
