"""Pins of the oracle's stencils of order 2, 4 and 8 (radius r = 1, 2, 4 on the
point set of Sec. 4 Eq. 13 widened to radius r; the paper itself uses r = 3).

Each pin comes from the mathematics, not from the oracle's closed-form weights:
  * polynomial exactness: the order-2r first derivative is exact for degree
    <= 2r and not for 2r + 1, the second derivative through 2r + 1 and not
    2r + 2, the face-diagonal mixed derivative for x^a y^b with a + b <= 2r + 1
    and not for an odd-odd pair with a + b = 2r + 2;
  * modified wavenumbers across the periodic wrap from weights solved exactly
    (rational arithmetic) from the defining moment conditions;
  * the measured convergence order on sinusoids is 2r;
  * the dense-matrix formulation, built from those exact weights, agrees on
    the operators and on the whole RHS of Eqs. B.1-B.4;
  * sum_i (D1 f)_i = 0 for any periodic field.
"""
import math

import numpy as np
import pytest

from oracle import brute, core
from paper_2103_01597_gb300 import synthetic

ORDERS = [2, 4, 8]
PHYS = dict(nu=0.011, eta=0.007, cs0=1.3, gamma=1.4, cp=1.7, lnrho0=0.2)


def _poly_grid(axes, order, n=20, dx=0.125):
    shape = [1, 1, 1]
    for a in axes:
        shape[a] = n
    nx, ny, nz = shape
    p = core.Params(n=(nx, ny, nz), L=tuple(shape[a] * dx for a in range(3)), order=order)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = [(i - nx // 2) * dx, (j - ny // 2) * dx, (k - nz // 2) * dx]
    return p, coords


def _slices(axes, r, n=20):
    sl = [slice(None)] * 3
    for a in axes:
        sl[2 - a] = slice(r, n - r)
    return tuple(sl)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("axis", [0, 2])
def test_d1_d2_polynomial_exactness(oracle_lib, order, axis):
    r = order // 2
    p, X = _poly_grid([axis], order)
    x = X[axis]
    sl = _slices([axis], r)
    for deg in range(0, 2 * r + 3):
        d1 = core.deriv(x ** deg, p, "d1", axis)
        e1 = deg * x ** (deg - 1) if deg > 0 else np.zeros_like(x)
        err1 = np.max(np.abs(d1[sl] - e1[sl]))
        if deg <= 2 * r:
            assert err1 < 1e-9, (order, deg, err1)
        elif deg == 2 * r + 1:
            assert err1 > 1e-7, (order, deg, err1)  # the order is exactly 2r
        d2 = core.deriv(x ** deg, p, "d2", axis, axis)
        e2 = deg * (deg - 1) * x ** (deg - 2) if deg > 1 else np.zeros_like(x)
        err2 = np.max(np.abs(d2[sl] - e2[sl]))
        if deg <= 2 * r + 1:
            assert err2 < 1e-8, (order, deg, err2)
        else:
            assert err2 > 1e-7, (order, deg, err2)


@pytest.mark.parametrize("order", ORDERS)
def test_dab_polynomial_exactness(oracle_lib, order):
    r = order // 2
    a, b = 0, 1
    p, X = _poly_grid([a, b], order)
    x, y = X[a], X[b]
    sl = _slices([a, b], r)
    for pa in range(0, 2 * r + 2):
        for pb in range(0, 2 * r + 2 - pa):
            d = core.deriv(x ** pa * y ** pb, p, "d2", a, b)
            exact = (pa * pb * x ** max(pa - 1, 0) * y ** max(pb - 1, 0)
                     if pa > 0 and pb > 0 else np.zeros_like(x))
            assert np.max(np.abs(d[sl] - exact[sl])) < 1e-8, (order, pa, pb)
    # total degree 2r + 2 with both powers odd is not reproduced
    pa, pb = 1, 2 * r + 1
    d = core.deriv(x ** pa * y ** pb, p, "d2", a, b)
    exact = pa * pb * y ** (pb - 1)
    assert np.max(np.abs(d[sl] - exact[sl])) > 1e-7, order


@pytest.mark.parametrize("order", ORDERS)
def test_modified_wavenumbers_from_exact_weights(oracle_lib, order):
    r = order // 2
    w, aw = brute.central_weights(r)
    n = 16
    p = core.Params(n=(n, 1, 1), order=order)
    dx = 2 * math.pi / n
    x = (np.arange(n) * dx).reshape(1, 1, n)
    for m in range(1, 8):
        th = m * dx
        kappa = sum(2 * float(w[q - 1]) * math.sin(q * th) for q in range(1, r + 1)) / dx
        k2 = -(float(-2 * sum(aw)) + sum(2 * float(aw[q - 1]) * math.cos(q * th)
                                         for q in range(1, r + 1))) / dx ** 2
        f = np.sin(m * x)
        np.testing.assert_allclose(core.deriv(f, p, "d1", 0), kappa * np.cos(m * x), atol=1e-12)
        np.testing.assert_allclose(core.deriv(f, p, "d2", 0, 0), -k2 * f, atol=1e-11)


@pytest.mark.parametrize("order", ORDERS)
def test_convergence_order(oracle_lib, order):
    errs1, errs2, errsx = [], [], []
    ns = (16, 32, 64) if order < 8 else (32, 64, 128)  # asymptotic range for order 8
    for n in ns:
        p = core.Params(n=(n, n, 1), order=order)
        dx = 2 * math.pi / n
        k, j, i = np.meshgrid(np.arange(1), np.arange(n), np.arange(n), indexing="ij")
        x, y = i * dx, j * dx
        f = np.sin(x) * np.cos(2 * y)
        errs1.append(np.max(np.abs(core.deriv(f, p, "d1", 0) - np.cos(x) * np.cos(2 * y))))
        errs2.append(np.max(np.abs(core.deriv(f, p, "d2", 1, 1) + 4 * f)))
        errsx.append(np.max(np.abs(core.deriv(f, p, "d2", 0, 1) + 2 * np.cos(x) * np.sin(2 * y))))
    for errs in (errs1, errs2, errsx):
        orders = [math.log2(errs[t] / errs[t + 1]) for t in range(2)]
        assert all(order - 0.3 < o < order + 0.3 for o in orders), (order, errs, orders)


@pytest.mark.parametrize("order", ORDERS)
def test_brute_force_operators(oracle_lib, order):
    n = (9, 8, 10)
    p = core.Params(n=n, L=(1.0, 2.0, 3.5), order=order)
    ops = brute.Operators(p.n, p.dx, order)
    f = np.random.default_rng(15 + order).standard_normal((n[2], n[1], n[0]))
    for a in range(3):
        ref = ops.D1[a] @ f.ravel()
        np.testing.assert_allclose(core.deriv(f, p, "d1", a).ravel(), ref, rtol=0,
                                   atol=1e-12 * np.max(np.abs(ref)))
        for b in range(3):
            ref = ops.D2[a, b] @ f.ravel()
            np.testing.assert_allclose(core.deriv(f, p, "d2", a, b).ravel(), ref, rtol=0,
                                       atol=1e-12 * np.max(np.abs(ref)))


@pytest.mark.parametrize("order", ORDERS)
def test_rhs_brute_force(oracle_lib, order):
    n = (9, 8, 10)
    frc = core.Forcing(k=(1, -2, 1), e=(0.6, 0.0, -0.8), phi=0.4, amp=0.05)
    p = core.Params(n=n, L=(5.0, 4.0, 6.0), forcing=frc, order=order, **PHYS)
    f = synthetic.smooth_state(n, seed=9, amp=0.3)
    f += 0.02 * np.random.default_rng(10).standard_normal(f.shape)
    r = core.rhs(f, p)
    rb = brute.rhs(f, p)
    for q in range(8):
        scale = np.max(np.abs(rb[q]))
        assert np.max(np.abs(r[q] - rb[q])) <= 1e-12 * scale, (order, q)


@pytest.mark.parametrize("order", ORDERS)
def test_telescoping(oracle_lib, order):
    n = (12, 10, 9)
    p = core.Params(n=n, L=(1.0, 1.3, 0.7), order=order)
    f = np.random.default_rng(3).standard_normal((n[2], n[1], n[0]))
    for a in range(3):
        d = core.deriv(f, p, "d1", a)
        assert abs(math.fsum(d.ravel())) < 1e-12 * np.sum(np.abs(d))


def test_order_is_validated():
    with pytest.raises(ValueError):
        core.Params(n=(4, 4, 4), order=5).c()
