"""Pins of the oracle's RHS (Eqs. B.1-B.4) and RK3 integrator (Sec. 4).

Closed forms: for single-mode states every derivative of the stencils is a
known multiple of a sinusoid -- D1 sin = kappa cos, D2 sin = -k2 sin, and the
face-diagonal mixed derivative of sin(A) sin(B) is mu cos(A) cos(B) with
mu = 4 [270 s1 t1 - 27 s2 t2 + 2 s3 t3] / (720 dx dy) (s_m = sin m theta_x,
t_m = sin m theta_y), which differs from the tensor product kappa_x kappa_y.
Each case below writes the RHS of such a state out by hand from Eqs. B.1-B.4,
so a dropped term, a wrong sign, coefficient or operand in the oracle fails it.
"""
import math

import numpy as np
import pytest

from oracle import core, brute
from paper_2103_01597_gb300 import synthetic


def _kappa(m, n, L=2 * math.pi):
    dx = L / n
    th = 2 * math.pi * m / n
    return (1.5 * math.sin(th) - 0.3 * math.sin(2 * th) + math.sin(3 * th) / 30.0) / dx


def _k2(m, n, L=2 * math.pi):
    dx = L / n
    th = 2 * math.pi * m / n
    return (49.0 / 18 - 3 * math.cos(th) + 0.3 * math.cos(2 * th) - math.cos(3 * th) / 45.0) / dx ** 2


def _mu(m1, n1, m2, n2, L=2 * math.pi):
    dx, dy = L / n1, L / n2
    t1, t2 = 2 * math.pi * m1 / n1, 2 * math.pi * m2 / n2
    return 4 * (270 * math.sin(t1) * math.sin(t2) - 27 * math.sin(2 * t1) * math.sin(2 * t2)
                + 2 * math.sin(3 * t1) * math.sin(3 * t2)) / (720 * dx * dy)


def _coords(n):
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (i * 2 * math.pi / nx, j * 2 * math.pi / ny, k * 2 * math.pi / nz)


PHYS = dict(nu=0.3, eta=0.2, cs0=1.3, gamma=1.4, cp=2.0, lnrho0=0.1)


def _check(rhs, expected, tol=1e-11):
    scale = max(1.0, max(np.max(np.abs(e)) for e in expected.values() if not np.isscalar(e)))
    for q in range(8):
        e = expected.get(q, 0.0)
        err = np.max(np.abs(rhs[q] - e))
        assert err < tol * scale, (q, err)


def test_rhs_compressive_viscous_mode(oracle_lib):
    n = (16, 1, 1)
    p = core.Params(n=n, **PHYS)
    x, _, _ = _coords(n)
    m, eps = 2, 0.07
    kap, k2 = _kappa(m, 16), _k2(m, 16)
    f = np.zeros((8,) + x.shape)
    f[1] = eps * np.sin(m * x)
    r = core.rhs(f, p)
    cs2 = p.cs0 ** 2 * math.exp((p.gamma - 1) * (0 - p.lnrho0))
    T = cs2 / (p.cp * (p.gamma - 1))
    c, s = np.cos(m * x), np.sin(m * x)
    SS = (2.0 / 3.0) * eps ** 2 * kap ** 2 * c ** 2
    _check(r, {0: -eps * kap * c,
               1: -eps ** 2 * kap * s * c - (4.0 / 3.0) * p.nu * k2 * eps * s,
               4: 2 * p.nu * SS / T})


def test_rhs_pressure_gradient(oracle_lib):
    n = (16, 12, 1)
    p = core.Params(n=n, **PHYS)
    x, y, _ = _coords(n)
    m1, m2, d, sg = 1, 2, 0.2, 0.3
    f = np.zeros((8,) + x.shape)
    f[0] = d * np.sin(m1 * x)
    f[4] = sg * np.cos(m2 * y)
    r = core.rhs(f, p)
    cs2 = p.cs0 ** 2 * np.exp(p.gamma * f[4] / p.cp + (p.gamma - 1) * (f[0] - p.lnrho0))
    _check(r, {1: -cs2 * d * _kappa(m1, 16) * np.cos(m1 * x),
               2: -cs2 * (-sg * _kappa(m2, 12) * np.sin(m2 * y)) / p.cp})


def test_rhs_lorentz_induction_ohmic(oracle_lib):
    n = (16, 1, 1)
    p = core.Params(n=n, **PHYS)
    x, _, _ = _coords(n)
    m, eps, W, lam = 3, 0.05, 0.4, 0.3
    kap, k2 = _kappa(m, 16), _k2(m, 16)
    f = np.zeros((8,) + x.shape)
    f[0] = lam
    f[3] = W
    f[7] = eps * np.sin(m * x)
    r = core.rhs(f, p)
    c, s = np.cos(m * x), np.sin(m * x)
    cs2 = p.cs0 ** 2 * math.exp((p.gamma - 1) * (lam - p.lnrho0))
    T = cs2 / (p.cp * (p.gamma - 1))
    # B = (0, -eps kappa cos, 0), j = (0, 0, eps k2 sin), j x B = (eps^2 k2 kappa sin cos, 0, 0)
    _check(r, {1: k2 * kap * eps ** 2 * s * c * math.exp(-lam),
               4: p.eta * (k2 * eps * s) ** 2 / (math.exp(lam) * T),
               5: W * eps * kap * c,
               7: -p.eta * k2 * eps * s})


def test_rhs_shear_density_gradient_advection(oracle_lib):
    n = (16, 1, 1)
    p = core.Params(n=n, **PHYS)
    x, _, _ = _coords(n)
    m, eps, d, U0 = 2, 0.06, 0.15, 0.25
    kap, k2 = _kappa(m, 16), _k2(m, 16)
    f = np.zeros((8,) + x.shape)
    f[0] = d * np.sin(m * x)
    f[1] = U0
    f[2] = eps * np.sin(m * x)
    r = core.rhs(f, p)
    c, s = np.cos(m * x), np.sin(m * x)
    cs2 = p.cs0 ** 2 * np.exp((p.gamma - 1) * (f[0] - p.lnrho0))
    T = cs2 / (p.cp * (p.gamma - 1))
    _check(r, {0: -U0 * d * kap * c,
               1: -cs2 * d * kap * c,
               2: -U0 * eps * kap * c - p.nu * k2 * eps * s + p.nu * eps * d * kap ** 2 * c ** 2,
               4: p.nu * eps ** 2 * kap ** 2 * c ** 2 / T})


def test_rhs_graddiv_uses_diagonal_cross_derivative(oracle_lib):
    """u_y = eps sin(A) sin(B), A = m1 x, B = m2 y: grad(div u)_x = D_xy u_y is
    mu cos A cos B (face-diagonal stencil), not kappa_x kappa_y cos A cos B."""
    n = (16, 12, 1)
    p = core.Params(n=n, **PHYS)
    x, y, _ = _coords(n)
    m1, m2, eps = 1, 2, 0.08
    A, B = m1 * x, m2 * y
    k1, k2x, k2y = _kappa(m1, 16), _k2(m1, 16), _k2(m2, 12)
    kp2 = _kappa(m2, 12)
    mu = _mu(m1, 16, m2, 12)
    assert abs(mu - k1 * kp2) > 1e-3 * abs(mu)
    f = np.zeros((8,) + x.shape)
    f[2] = eps * np.sin(A) * np.sin(B)
    r = core.rhs(f, p)
    div = eps * kp2 * np.sin(A) * np.cos(B)
    cs2 = p.cs0 ** 2 * math.exp((p.gamma - 1) * (0 - p.lnrho0))
    T = cs2 / (p.cp * (p.gamma - 1))
    SS = (2.0 / 3.0) * div ** 2 + 0.5 * (eps * k1 * np.cos(A) * np.sin(B)) ** 2
    _check(r, {0: -div,
               1: p.nu / 3.0 * eps * mu * np.cos(A) * np.cos(B),
               2: (-f[2] * eps * kp2 * np.sin(A) * np.cos(B)
                   + p.nu * (-(k2x + k2y) * f[2] - k2y * f[2] / 3.0)),
               4: 2 * p.nu * SS / T})


def test_rhs_current_uses_diagonal_cross_derivative(oracle_lib):
    """A_y = eps sin(A) sin(B): j = grad(div A) - lap A = (mu cos A cos B, k2x A_y, 0),
    B = (0, 0, eps kappa_x cos A sin B)."""
    n = (16, 12, 1)
    p = core.Params(n=n, **PHYS)
    x, y, _ = _coords(n)
    m1, m2, eps = 2, 1, 0.09
    A, B = m1 * x, m2 * y
    k1, k2x, k2y = _kappa(m1, 16), _k2(m1, 16), _k2(m2, 12)
    mu = _mu(m1, 16, m2, 12)
    f = np.zeros((8,) + x.shape)
    f[6] = eps * np.sin(A) * np.sin(B)
    r = core.rhs(f, p)
    jx = eps * mu * np.cos(A) * np.cos(B)
    jy = k2x * f[6]
    Bz = eps * k1 * np.cos(A) * np.sin(B)
    cs2 = p.cs0 ** 2 * math.exp((p.gamma - 1) * (0 - p.lnrho0))
    T = cs2 / (p.cp * (p.gamma - 1))
    _check(r, {1: jy * Bz, 2: -jx * Bz,
               4: p.eta * (jx ** 2 + jy ** 2) / T,
               6: -p.eta * (k2x + k2y) * f[6]})


def test_rhs_forcing_term(oracle_lib):
    n = (8, 6, 4)
    frc = core.Forcing(k=(1, -2, 1), e=(0.6, 0.0, -0.8), phi=0.7, amp=0.05)
    p = core.Params(n=n, forcing=frc)
    x, y, z = _coords(n)
    r = core.rhs(np.zeros((8,) + x.shape), p)
    ph = x * 1 - 2 * y + z + 0.7
    _check(r, {1: 0.05 * 0.6 * np.cos(ph), 3: -0.05 * 0.8 * np.cos(ph)}, tol=1e-13)


def test_rhs_brute_force_8cube(oracle_lib):
    """Whole RHS: C oracle vs the dense-matrix formulation, random smooth state,
    non-cubic grid, unequal spacings, forcing on."""
    n = (8, 6, 7)
    frc = core.Forcing(k=(2, 0, -1), e=(0.0, 1.0, 0.0), phi=1.1, amp=0.05)
    p = core.Params(n=n, L=(5.0, 4.0, 6.0), forcing=frc, **PHYS)
    f = synthetic.smooth_state(n, seed=3, amp=0.3)
    f += 0.02 * np.random.default_rng(4).standard_normal(f.shape)
    r = core.rhs(f, p)
    rb = brute.rhs(f, p)
    for q in range(8):
        scale = np.max(np.abs(rb[q]))
        assert np.max(np.abs(r[q] - rb[q])) <= 1e-12 * scale, q


def _cyclic(f):
    """Rotate the state by (x, y, z) -> (y, z, x): new field at (x, y, z) is the old
    one at (z, x, y); vector components follow (new_x = old_z, ...)."""
    g = np.empty_like(f)
    # array axes are (z, y, x); new[z', y', x'] = old[z = y', y = x', x = z']
    def rot(a):
        return np.transpose(a, (1, 2, 0))
    g[0], g[4] = rot(f[0]), rot(f[4])
    g[1], g[2], g[3] = rot(f[3]), rot(f[1]), rot(f[2])
    g[5], g[6], g[7] = rot(f[7]), rot(f[5]), rot(f[6])
    return g


def test_rhs_rotation_equivariance(oracle_lib):
    n = (8, 8, 8)
    p = core.Params(n=n, **PHYS)
    f = synthetic.smooth_state(n, seed=9, amp=0.2)
    f += 0.01 * np.random.default_rng(10).standard_normal(f.shape)
    r1 = core.rhs(_cyclic(f), p)
    r2 = _cyclic(core.rhs(f, p))
    assert np.max(np.abs(r1 - r2)) < 1e-12 * np.max(np.abs(r2))


def test_mass_like_invariants(oracle_lib):
    """From uniform ln rho the first substep conserves sum(ln rho) to roundoff
    (its RHS is -div u, which telescopes); sum(div u) = 0 for any u."""
    n = (12, 10, 8)
    p = core.Params(n=n, L=(2.0, 3.0, 4.0), **PHYS)
    f = synthetic.noise_state(n, seed=11, sigma=1e-2)
    f[0] = 0.3
    fo, _ = core.substep(f, None, p, 1e-2, 0)
    assert abs(math.fsum(fo[0].ravel()) - math.fsum(f[0].ravel())) < 1e-13 * f[0].size
    div = sum(core.deriv(np.ascontiguousarray(f[1 + a]), p, "d1", a) for a in range(3))
    assert abs(math.fsum(div.ravel())) < 1e-12 * np.sum(np.abs(div))


def _beltrami(n, m, eps):
    x, _, _ = _coords(n)
    f = np.zeros((8,) + x.shape)
    f[6] = eps * np.sin(m * x)
    f[7] = eps * np.cos(m * x)
    return f


def test_rk3_amplification_polynomial(oracle_lib):
    """Beltrami field A = eps (0, sin mx, cos mx), u = 0: its RHS is exactly linear,
    dA/dt = -eta k2 A, so one step multiplies A by 1 + z + z^2/2 + z^3/6, z = -eta k2 dt
    (the stability polynomial of every 3-stage third-order Runge-Kutta scheme)."""
    n = (16, 1, 1)
    p = core.Params(n=n, eta=0.5, nu=0.1, cs0=1.0, gamma=5.0 / 3.0, cp=1.0)
    m, eps, dt = 2, 1e-3, 0.3
    f = _beltrami(n, m, eps)
    fo = core.step(f, p, dt)
    z = -p.eta * _k2(m, 16) * dt
    P = 1 + z + z * z / 2 + z ** 3 / 6
    np.testing.assert_allclose(fo[6:8], P * f[6:8], atol=1e-16, rtol=1e-13)
    assert np.max(np.abs(fo[1:4])) < 1e-18  # j x B = 0 and u x B = 0: u stays 0
    assert np.max(np.abs(fo[0])) < 1e-18  # only roundoff reaches ln rho


def test_rk3_third_order_and_beltrami_entropy(oracle_lib):
    """Beltrami decay with Ohmic heating, gamma = 5/3, c_s0 = c_p = 1, rho = 1:
    a(t) = a0 exp(-eta k2 t) and exp(gamma s) = 1 + gamma (gamma-1) k2 a0^2
    (1 - exp(-2 eta k2 t)) / 2 in closed form.  The oracle's global error at
    T = 1 falls as dt^3."""
    n = (16, 1, 1)
    g = 5.0 / 3.0
    p = core.Params(n=n, eta=0.4, nu=0.1, cs0=1.0, gamma=g, cp=1.0)
    m, a0 = 1, 0.5
    k2 = _k2(m, 16)
    Tend = 1.0
    exact_a = a0 * math.exp(-p.eta * k2 * Tend)
    exact_s = math.log(1 + g * (g - 1) * k2 * a0 ** 2 * (1 - math.exp(-2 * p.eta * k2 * Tend)) / 2) / g
    errs = []
    for N in (8, 16, 32):
        f = _beltrami(n, m, a0)
        for _ in range(N):
            f = core.step(f, p, Tend / N)
        a = np.sqrt(f[6] ** 2 + f[7] ** 2)
        assert np.ptp(a) < 1e-14 and np.ptp(f[4]) < 1e-14
        errs.append((abs(a.mean() - exact_a), abs(f[4].mean() - exact_s)))
    for c in range(2):
        orders = [math.log2(errs[t][c] / errs[t + 1][c]) for t in range(2)]
        assert all(2.8 < o < 3.3 for o in orders), (c, errs, orders)


def test_substep_w_not_read_at_s0(oracle_lib):
    n = (6, 5, 4)
    p = core.Params(n=n)
    f = synthetic.noise_state(n, seed=2, sigma=1e-3)
    w_nan = np.full_like(f, np.nan)
    fo1, w1 = core.substep(f, w_nan, p, 1e-3, 0)
    fo2, w2 = core.substep(f, None, p, 1e-3, 0)
    assert np.array_equal(fo1, fo2) and np.array_equal(w1, w2)


def test_substep_cells_matches_grid(oracle_lib):
    n = (10, 9, 8)
    p = core.Params(n=n, **PHYS)
    f = synthetic.smooth_state(n, seed=5, amp=0.2)
    w = synthetic.smooth_state(n, seed=6, amp=0.01)
    fo, wo = core.substep(f, w, p, 1e-3, 1)
    cells = np.array([[0, 0, 0], [9, 8, 7], [3, 4, 5], [9, 0, 7]])
    fc, wc = core.substep_cells(f, w, p, 1e-3, 1, cells)
    for m, (i, j, k) in enumerate(cells):
        assert np.array_equal(fc[:, m], fo[:, k, j, i])
        assert np.array_equal(wc[:, m], wo[:, k, j, i])
