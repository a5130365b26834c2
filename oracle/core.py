"""ctypes wrappers of the C oracle plus FP64 NumPy reductions.

Test infrastructure only (see the package docstring).  Arrays are NumPy
float64 with shape (8, nz, ny, nx) for a state (field order of Table B.1:
ln rho, u_x, u_y, u_z, s, A_x, A_y, A_z) and (nz, ny, nx) for one field, C
order, so x is the fastest index.
"""
import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

from .build import build_oracle

NFIELDS = 8
LNRHO, UX, UY, UZ, SS, AX, AY, AZ = range(8)

_i64 = ctypes.c_int64
_f64 = ctypes.c_double
_pf64 = ctypes.POINTER(ctypes.c_double)


class _CParams(ctypes.Structure):
    _fields_ = [("n", _i64 * 3), ("dx", _f64 * 3), ("nu", _f64), ("eta", _f64),
                ("cs0", _f64), ("gamma", _f64), ("cp", _f64), ("lnrho0", _f64),
                ("force_on", _i64), ("force_amp", _f64), ("force_k", _i64 * 3),
                ("force_e", _f64 * 3), ("force_phi", _f64), ("radius", _i64),
                ("K", _f64), ("zeta", _f64), ("heat", _f64), ("cool", _f64)]


@dataclass
class Forcing:
    """One step's forcing f0 e cos(k . x + phi) (a reading: not in the paper)."""
    k: tuple
    e: tuple
    phi: float
    amp: float


@dataclass
class Params:
    """Grid and physical parameters (Tables B.1, B.2; readings for values)."""
    n: tuple                       # (nx, ny, nz)
    L: tuple = (2 * math.pi, 2 * math.pi, 2 * math.pi)
    nu: float = 5e-3
    eta: float = 5e-3
    cs0: float = 1.0
    gamma: float = 5.0 / 3.0
    cp: float = 1.0
    lnrho0: float = 0.0
    forcing: Forcing = field(default=None)
    order: int = 6                 # stencil order 2r (Sec. 4 uses 6; 2, 4, 8 widen it)
    K: float = 0.0                 # thermal conductivity (Eq. B.3)
    zeta: float = 0.0              # bulk viscosity (Eqs. B.2, B.3)
    heat: float = 0.0              # explicit heating H (uniform rate)
    cool: float = 0.0              # explicit cooling C (uniform rate)

    @property
    def dx(self):
        return tuple(self.L[a] / self.n[a] for a in range(3))

    def c(self):
        cp = _CParams()
        for a in range(3):
            cp.n[a] = int(self.n[a])
            cp.dx[a] = float(self.dx[a])
        cp.nu, cp.eta, cp.cs0 = self.nu, self.eta, self.cs0
        cp.gamma, cp.cp, cp.lnrho0 = self.gamma, self.cp, self.lnrho0
        if self.order not in (2, 4, 6, 8):
            raise ValueError("stencil order must be 2, 4, 6 or 8")
        cp.radius = self.order // 2
        cp.K, cp.zeta, cp.heat, cp.cool = self.K, self.zeta, self.heat, self.cool
        if self.forcing is not None:
            cp.force_on = 1
            cp.force_amp = self.forcing.amp
            for a in range(3):
                cp.force_k[a] = int(self.forcing.k[a])
                cp.force_e[a] = float(self.forcing.e[a])
            cp.force_phi = self.forcing.phi
        return cp


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_oracle())
        PP = ctypes.POINTER(_pf64)
        P = ctypes.POINTER(_CParams)
        L.oracle_rhs_grid.argtypes = [PP, P, PP, _i64]
        L.oracle_substep.argtypes = [PP, PP, PP, P, _f64, _i64, _i64]
        L.oracle_substep.restype = _i64
        L.oracle_substep_cells.argtypes = [PP, PP, P, _f64, _i64, _i64,
                                           ctypes.POINTER(_i64), _pf64, _pf64, _i64]
        L.oracle_deriv.argtypes = [_pf64, P, _i64, _i64, _i64, _pf64]
        L.oracle_curl.argtypes = [PP, P, PP]
        L.oracle_periodic_halo.argtypes = [_pf64, ctypes.POINTER(_i64), _i64]
        L.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_splitmix64.restype = ctypes.c_uint64
        L.oracle_forcing_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.POINTER(_i64), _pf64, _pf64]
        L.oracle_forcing_field.argtypes = [P, PP]
        L.oracle_restrict.argtypes = [_pf64, ctypes.POINTER(_i64), _pf64]
        L.oracle_rk_alpha.argtypes = [_i64]
        L.oracle_rk_alpha.restype = _f64
        L.oracle_rk_beta.argtypes = [_i64]
        L.oracle_rk_beta.restype = _f64
        _lib = L
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_pf64)


def _ptrs(arrs):
    return (_pf64 * len(arrs))(*[_ptr(a) for a in arrs])


def _check_state(f, p):
    nx, ny, nz = p.n
    assert f.shape == (NFIELDS, nz, ny, nx), (f.shape, p.n)
    return np.ascontiguousarray(f, dtype=np.float64)


def default_threads():
    return os.cpu_count() or 1


def rhs(f, p, nthreads=0):
    """RHS of Eqs. B.1-B.4 (plus forcing if set) at every cell."""
    f = _check_state(f, p)
    out = np.empty_like(f)
    lib().oracle_rhs_grid(_ptrs(list(f)), ctypes.byref(p.c()), _ptrs(list(out)), nthreads)
    return out


def substep(f, w, p, dt, s, nthreads=0):
    """One Williamson RK3 substep s in {0, 1, 2}: returns (f_out, w_out).
    At s = 0, w is not read (may be None)."""
    f = _check_state(f, p)
    if w is None:
        assert s == 0
        w = np.zeros_like(f)
    w = np.array(w, dtype=np.float64, order="C", copy=True)
    fo = np.empty_like(f)
    lib().oracle_substep(_ptrs(list(f)), _ptrs(list(w)), _ptrs(list(fo)),
                         ctypes.byref(p.c()), float(dt), int(s), nthreads)
    return fo, w


def step(f, p, dt, nthreads=0):
    """One full RK3 step (substeps 0, 1, 2 with the same dt and forcing)."""
    w = None
    for s in range(3):
        f, w = substep(f, w, p, dt, s, nthreads)
    return f


def substep_cells(f, w, p, dt, s, cells, nthreads=0):
    """Substep s at the listed cells only.  cells: int array (m, 3) of (i, j, k).
    Returns (f_out, w_out), each (8, m)."""
    f = _check_state(f, p)
    if w is None:
        assert s == 0
        w = np.zeros_like(f)
    w = _check_state(w, p)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    m = cells.shape[0]
    fo = np.empty((NFIELDS, m))
    wo = np.empty((NFIELDS, m))
    lib().oracle_substep_cells(_ptrs(list(f)), _ptrs(list(w)), ctypes.byref(p.c()),
                               float(dt), int(s), m,
                               cells.ctypes.data_as(ctypes.POINTER(_i64)),
                               _ptr(fo), _ptr(wo), nthreads)
    return fo, wo


def deriv(f1, p, kind, a, b=None):
    """kind 'd1': first derivative along a; kind 'd2': d^2/dx_a dx_b."""
    f1 = np.ascontiguousarray(f1, dtype=np.float64)
    out = np.empty_like(f1)
    k = 0 if kind == "d1" else 1
    lib().oracle_deriv(_ptr(f1), ctypes.byref(p.c()), k, a, a if b is None else b, _ptr(out))
    return out


def curl(A, p):
    """B = curl A with the first-derivative operator (A: (3, nz, ny, nx))."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.empty_like(A)
    lib().oracle_curl(_ptrs(list(A)), ctypes.byref(p.c()), _ptrs(list(B)))
    return B


def periodic_halo(fp, n, r=3):
    """Fill the halo of a padded field (nz+2r, ny+2r, nx+2r), map of Sec. 3.3."""
    fp = np.array(fp, dtype=np.float64, order="C", copy=True)
    nn = (_i64 * 3)(*[int(v) for v in n])
    lib().oracle_periodic_halo(_ptr(fp), nn, r)
    return fp


def splitmix64(seed, counter):
    return int(lib().oracle_splitmix64(seed & (2**64 - 1), counter & (2**64 - 1)))


def forcing_draw(seed, step_index, amp):
    k = (_i64 * 3)()
    e = (_f64 * 3)()
    phi = _f64()
    lib().oracle_forcing_draw(seed & (2**64 - 1), step_index, k, e, ctypes.byref(phi))
    return Forcing(k=tuple(k), e=tuple(e), phi=phi.value, amp=amp)


def forcing_field(p):
    nx, ny, nz = p.n
    out = np.empty((3, nz, ny, nx))
    lib().oracle_forcing_field(ctypes.byref(p.c()), _ptrs(list(out)))
    return out


def restrict(fine):
    """Full-weighting restriction of one periodic field (sizes must be even)."""
    fine = np.ascontiguousarray(fine, dtype=np.float64)
    nz, ny, nx = fine.shape
    coarse = np.empty((nz // 2, ny // 2, nx // 2))
    nf = (_i64 * 3)(nx, ny, nz)
    lib().oracle_restrict(_ptr(fine), nf, _ptr(coarse))
    return coarse


def rk_coefficients():
    L = lib()
    return ([L.oracle_rk_alpha(s) for s in range(3)], [L.oracle_rk_beta(s) for s in range(3)])


# --------------------------------------------------------------------------
# Reductions (FP64).  Quantities: a field index 0..7, "umag" = |u|,
# "ekin" = rho |u|^2 / 2, "emag" = |curl A|^2 / 2, "cfl" = |u| + sqrt(c_s^2 +
# v_A^2) with v_A^2 = |B|^2 / rho (mu0 = 1).  Ops: max, min, sum, rms.
# Not in the paper (its timestep is constant, Sec. 5): readings.
# --------------------------------------------------------------------------

def quantity(f, p, q):
    f = _check_state(f, p)
    if isinstance(q, int):
        return f[q]
    u2 = f[UX] ** 2 + f[UY] ** 2 + f[UZ] ** 2
    if q == "umag":
        return np.sqrt(u2)
    rho = np.exp(f[LNRHO])
    if q == "ekin":
        return 0.5 * rho * u2
    B = curl(f[AX:AZ + 1], p)
    b2 = B[0] ** 2 + B[1] ** 2 + B[2] ** 2
    if q == "emag":
        return 0.5 * b2
    if q == "cfl":
        cs2 = p.cs0 ** 2 * np.exp(p.gamma * f[SS] / p.cp + (p.gamma - 1.0) * (f[LNRHO] - p.lnrho0))
        return np.sqrt(u2) + np.sqrt(cs2 + b2 / rho)
    raise ValueError(q)


def reduce(f, p, op, q):
    v = quantity(f, p, q).ravel()
    if op == "max":
        return float(v.max())
    if op == "min":
        return float(v.min())
    if op == "sum":
        return math.fsum(v)
    if op == "rms":
        return math.sqrt(math.fsum(v * v) / v.size)
    raise ValueError(op)
