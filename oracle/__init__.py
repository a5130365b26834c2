"""FP64 CPU oracle of the RK3 substep of non-ideal MHD (arXiv:2103.01597).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU
baseline leg of ``bench.py`` are the only callers allowed.  Nothing here is
shared with, or imported by, the CUDA path, and the CUDA path never falls back
to it.

Parts:
  * ``core``    -- ctypes wrappers of ``ac_oracle.c`` (stencils of Eq. 13,
                   Eqs. B.1-B.4, Williamson RK3, periodic map of Sec. 3.3,
                   forcing draw, restriction) plus FP64 NumPy reductions;
  * ``brute``   -- an independent dense-matrix (circulant Kronecker) NumPy
                   formulation of the same operators and RHS for tiny grids;
  * ``closure`` -- the learned-closure conv net forward/backward and Adam in
                   FP64 NumPy.
"""
from .build import build_oracle, library_path  # noqa: F401
from . import core  # noqa: F401
