"""Pins of the oracle's derivative operators (Sec. 4, Eq. 13; r = 3, sixth order).

Each pin comes from the mathematics, not from the oracle's own formula:
  * polynomial exactness: a sixth-order central first derivative on 7 points
    is exact for degree <= 6 and not for 7; the second derivative is exact
    through degree 7 (symmetry) and not 8; the face-diagonal mixed derivative
    is exact for x^a y^b with a + b <= 7 and not for a + b = 8 with a, b odd;
  * the measured convergence order on sinusoids is 6;
  * an independent dense-matrix formulation agrees on an 8^3 grid;
  * discrete identities that hold for any periodic field: div(curl A) = 0 and
    sum_i (D1 f)_i = 0.
A wrong coefficient, sign, axis or wrap index fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import core, brute
from paper_2103_01597_gb300 import synthetic


def _poly_grid(axes, n=16, dx=0.125):
    """Coordinates x_i = (i - n/2) dx on an n-cell periodic line per listed axis
    (other axes have 1 cell); dyadic dx keeps the sampling exact."""
    shape = [1, 1, 1]
    for a in axes:
        shape[a] = n
    nx, ny, nz = shape
    p = core.Params(n=(nx, ny, nz), L=tuple(shape[a] * dx for a in range(3)))
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = [(i - nx // 2) * dx, (j - ny // 2) * dx, (k - nz // 2) * dx]
    return p, coords


def _interior(n=16, r=3):
    return slice(r, n - r)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_d1_polynomial_exactness(oracle_lib, axis):
    p, X = _poly_grid([axis])
    x = X[axis]
    sl = [slice(None)] * 3
    sl[2 - axis] = _interior()
    sl = tuple(sl)
    for deg in range(0, 8):
        d = core.deriv(x ** deg, p, "d1", axis)
        exact = deg * x ** (deg - 1) if deg > 0 else np.zeros_like(x)
        err = np.max(np.abs(d[sl] - exact[sl]))
        if deg <= 6:
            assert err < 1e-10, (deg, err)
        else:
            assert err > 1e-6, (deg, err)  # degree 7 is not exact: order is exactly 6


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_d2_polynomial_exactness(oracle_lib, axis):
    p, X = _poly_grid([axis])
    x = X[axis]
    sl = [slice(None)] * 3
    sl[2 - axis] = _interior()
    sl = tuple(sl)
    for deg in range(0, 9):
        d = core.deriv(x ** deg, p, "d2", axis, axis)
        exact = deg * (deg - 1) * x ** (deg - 2) if deg > 1 else np.zeros_like(x)
        err = np.max(np.abs(d[sl] - exact[sl]))
        if deg <= 7:
            assert err < 1e-9, (deg, err)
        else:
            assert err > 1e-6, (deg, err)


@pytest.mark.parametrize("a,b", [(0, 1), (1, 0), (0, 2), (1, 2), (2, 1)])
def test_dab_polynomial_exactness(oracle_lib, a, b):
    p, X = _poly_grid([a, b])
    x, y = X[a], X[b]
    sl = [slice(None)] * 3
    sl[2 - a] = _interior()
    sl[2 - b] = _interior()
    sl = tuple(sl)
    for pa in range(0, 8):
        for pb in range(0, 8 - pa):
            f = x ** pa * y ** pb
            d = core.deriv(f, p, "d2", a, b)
            exact = (pa * pb * x ** max(pa - 1, 0) * y ** max(pb - 1, 0)
                     if pa > 0 and pb > 0 else np.zeros_like(x))
            err = np.max(np.abs(d[sl] - exact[sl]))
            assert err < 1e-9, (pa, pb, err)
    # total degree 8 with both powers odd is not reproduced
    f = x ** 3 * y ** 5
    d = core.deriv(f, p, "d2", a, b)
    exact = 15 * x ** 2 * y ** 4
    assert np.max(np.abs(d[sl] - exact[sl])) > 1e-6


def _sin_grid(n, axis):
    shape = [1, 1, 1]
    shape[axis] = n
    p = core.Params(n=tuple(shape))
    k, j, i = np.meshgrid(np.arange(shape[2]), np.arange(shape[1]), np.arange(shape[0]),
                          indexing="ij")
    idx = [i, j, k][axis]
    return p, idx * (2 * math.pi / n)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sinusoid_modified_wavenumbers(oracle_lib, axis):
    """Across the periodic wrap: D1 sin(mx) = kappa cos(mx), D2 sin(mx) = -k2 sin(mx)
    with the modified wavenumbers of the stencil weights."""
    n = 16
    p, x = _sin_grid(n, axis)
    dx = 2 * math.pi / n
    for m in range(1, 8):
        th = m * dx
        kappa = (1.5 * math.sin(th) - 0.3 * math.sin(2 * th) + math.sin(3 * th) / 30.0) / dx
        k2 = (49.0 / 18 - 3 * math.cos(th) + 0.3 * math.cos(2 * th)
              - math.cos(3 * th) / 45.0) / dx ** 2
        f = np.sin(m * x)
        np.testing.assert_allclose(core.deriv(f, p, "d1", axis), kappa * np.cos(m * x),
                                   atol=1e-13)
        np.testing.assert_allclose(core.deriv(f, p, "d2", axis, axis), -k2 * f, atol=1e-12)


def test_convergence_order_six(oracle_lib):
    errs1, errs2, errsx = [], [], []
    for n in (16, 32, 64):
        p = core.Params(n=(n, n, 1))
        dx = 2 * math.pi / n
        k, j, i = np.meshgrid(np.arange(1), np.arange(n), np.arange(n), indexing="ij")
        x, y = i * dx, j * dx
        f = np.sin(x) * np.cos(2 * y)
        errs1.append(np.max(np.abs(core.deriv(f, p, "d1", 0) - np.cos(x) * np.cos(2 * y))))
        errs2.append(np.max(np.abs(core.deriv(f, p, "d2", 1, 1) + 4 * f)))
        errsx.append(np.max(np.abs(core.deriv(f, p, "d2", 0, 1)
                                   + 2 * np.cos(x) * np.sin(2 * y))))
    for errs in (errs1, errs2, errsx):
        orders = [math.log2(errs[t] / errs[t + 1]) for t in range(2)]
        assert all(5.7 < o < 6.3 for o in orders), (errs, orders)


def test_brute_force_operators_8cube(oracle_lib):
    """C loops vs dense circulant-Kronecker matrices, non-cubic 8x6x7 grid with
    unequal spacings."""
    n = (8, 6, 7)
    p = core.Params(n=n, L=(1.0, 2.0, 3.5))
    ops = brute.Operators(p.n, p.dx)
    rng = np.random.default_rng(5)
    f = rng.standard_normal((n[2], n[1], n[0]))
    for a in range(3):
        np.testing.assert_allclose(core.deriv(f, p, "d1", a).ravel(), ops.D1[a] @ f.ravel(),
                                   rtol=0, atol=1e-12 * np.max(np.abs(ops.D1[a] @ f.ravel())))
        for b in range(3):
            ref = ops.D2[a, b] @ f.ravel()
            np.testing.assert_allclose(core.deriv(f, p, "d2", a, b).ravel(), ref,
                                       rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_div_curl_and_telescoping(oracle_lib):
    n = (12, 10, 9)
    p = core.Params(n=n, L=(1.0, 1.3, 0.7))
    rng = np.random.default_rng(7)
    A = rng.standard_normal((3, n[2], n[1], n[0]))
    B = core.curl(A, p)
    div = sum(core.deriv(np.ascontiguousarray(B[a]), p, "d1", a) for a in range(3))
    scale = max(np.max(np.abs(core.deriv(np.ascontiguousarray(B[a]), p, "d1", a)))
                for a in range(3))
    assert np.max(np.abs(div)) < 1e-12 * scale
    f = rng.standard_normal((n[2], n[1], n[0]))
    for a in range(3):
        d = core.deriv(f, p, "d1", a)
        assert abs(math.fsum(d.ravel())) < 1e-12 * np.sum(np.abs(d))


def test_noise_input_recipe():
    f = synthetic.noise_state((8, 8, 8), seed=1)
    assert f.shape == (8, 8, 8, 8)
    assert np.all(f[0] == 0) and np.all(f[4] == 0)
    assert 0.5e-5 < f[1].std() < 2e-5
