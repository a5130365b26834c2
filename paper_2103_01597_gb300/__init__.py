"""GB300-native RK3 substep of sixth-order non-ideal MHD (arXiv:2103.01597).

The compute path is the C-ABI library ``libac.so`` (hand-written sm_103a CUDA
kernels, declared in ``include/ac.h``).  ``paper_2103_01597_gb300.ac`` is the
thin ctypes binding with the same names; PyTorch supplies device memory and
streams only.  ``synthetic`` draws seeded inputs.

The binding is imported lazily so that ``synthetic`` can be used without the
compiled library.
"""
import importlib

__all__ = ["ac", "closure", "synthetic"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
