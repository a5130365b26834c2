"""Pins of the terms of Eqs. B.2-B.3 beyond the base configuration: bulk
viscosity zeta, conduction div(K grad T), heating H and cooling C.

  * a uniform state: every derivative vanishes and Ds/Dt = (H - C) / (rho T);
  * single sinusoids: the zeta and K contributions in closed form through the
    modified wavenumbers of the sixth-order stencils;
  * the conduction reading (chain rule through xi = gamma s / c_p +
    (gamma - 1)(ln rho - ln rho0)) converges at sixth order to K lap T / (rho T)
    computed spectrally from T itself, i.e. to the definition div(K grad T);
  * the dense-matrix formulation agrees with every term on, at orders 6 and 4.
"""
import math

import numpy as np
import pytest

from oracle import brute, core
from paper_2103_01597_gb300 import synthetic

BASE = dict(nu=0.0, eta=0.0, cs0=1.2, gamma=1.4, cp=1.7, lnrho0=0.1)


def _state(n, lnrho=0.3, s=0.2):
    f = np.zeros((8, n[2], n[1], n[0]))
    f[0] = lnrho
    f[4] = s
    return f


def _thermo(p, lnrho, s):
    rho = math.exp(lnrho)
    cs2 = p.cs0 ** 2 * math.exp(p.gamma * s / p.cp + (p.gamma - 1) * (lnrho - p.lnrho0))
    T = cs2 / (p.cp * (p.gamma - 1))
    return rho, T


def _kappa(th, dx):
    return (1.5 * math.sin(th) - 0.3 * math.sin(2 * th) + math.sin(3 * th) / 30.0) / dx


def _k2(th, dx):
    return (49.0 / 18 - 3 * math.cos(th) + 0.3 * math.cos(2 * th) - math.cos(3 * th) / 45.0) / dx ** 2


def test_uniform_state_heating_cooling(oracle_lib):
    n = (4, 5, 6)
    p = core.Params(n=n, heat=0.7, cool=0.25, K=0.3, zeta=0.2, **BASE)
    r = core.rhs(_state(n), p)
    rho, T = _thermo(p, 0.3, 0.2)
    assert np.allclose(r[4], (0.7 - 0.25) / (rho * T), rtol=1e-14, atol=0)
    for q in (0, 1, 2, 3, 5, 6, 7):
        assert np.all(r[q] == 0.0), q


def test_bulk_viscosity_compressive_mode(oracle_lib):
    n = (16, 1, 1)
    dx = 2 * math.pi / n[0]
    x = (np.arange(n[0]) * dx).reshape(1, 1, -1)
    a, m, zeta = 0.01, 3, 0.05
    f = _state(n)
    f[1] = a * np.sin(m * x)
    p0 = core.Params(n=n, **BASE)
    p1 = core.Params(n=n, zeta=zeta, **BASE)
    d = core.rhs(f, p1) - core.rhs(f, p0)
    th = m * dx
    rho, T = _thermo(p0, 0.3, 0.2)
    divu = a * _kappa(th, dx) * np.cos(m * x)
    np.testing.assert_allclose(d[1], -zeta * _k2(th, dx) * a * np.sin(m * x), rtol=0, atol=1e-14)
    np.testing.assert_allclose(d[4], zeta * divu ** 2 / T, rtol=0, atol=1e-15)
    for q in (0, 2, 3, 5, 6, 7):
        assert np.max(np.abs(d[q])) < 1e-15, q


def test_conduction_single_modes(oracle_lib):
    n = (1, 12, 10)
    dy, dz = 2 * math.pi / n[1], 2 * math.pi / n[2]
    k, j, _ = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(1), indexing="ij")
    y, z = j * dy, k * dz
    s0, l1, my, mz, K = 0.05, 0.04, 2, 1, 0.3
    f = _state(n)
    f[4] = 0.2 + s0 * np.sin(my * y)
    f[0] = 0.3 + l1 * np.cos(mz * z)
    p = core.Params(n=n, K=K, **BASE)
    r = core.rhs(f, p)
    g, gm1 = p.gamma / p.cp, p.gamma - 1
    gxi_y = g * s0 * _kappa(my * dy, dy) * np.cos(my * y)
    gxi_z = -gm1 * l1 * _kappa(mz * dz, dz) * np.sin(mz * z)
    lapxi = -g * _k2(my * dy, dy) * s0 * np.sin(my * y) - gm1 * _k2(mz * dz, dz) * l1 * np.cos(mz * z)
    rho = np.exp(f[0])
    expected = K * (lapxi + gxi_y ** 2 + gxi_z ** 2) / rho  # K T (...) / (rho T)
    np.testing.assert_allclose(r[4], expected, rtol=1e-12, atol=0)  # stencils cancel the 0.2, 0.3 offsets


def test_conduction_converges_to_spectral_divergence(oracle_lib):
    """The chain-rule discretisation converges at sixth order to K lap T / (rho T)
    with lap T from the Fourier transform of T itself (spectrally exact here)."""
    K = 0.2
    errs = []
    for nn in (16, 32, 64):
        n = (nn, nn, 1)
        h = 2 * math.pi / nn
        _, j, i = np.meshgrid(np.arange(1), np.arange(nn), np.arange(nn), indexing="ij")
        x, y = i * h, j * h
        f = _state(n)
        f[4] = 0.2 + 0.1 * np.sin(x) * np.cos(2 * y)
        f[0] = 0.3 + 0.05 * np.cos(x + y)
        p = core.Params(n=n, K=K, **BASE)
        r = core.rhs(f, p)
        cs2 = p.cs0 ** 2 * np.exp(p.gamma * f[4] / p.cp + (p.gamma - 1) * (f[0] - p.lnrho0))
        T = cs2 / (p.cp * (p.gamma - 1))
        kx = np.fft.fftfreq(nn, 1.0 / nn)
        KX, KY = np.meshgrid(kx, kx, indexing="xy")
        lapT = np.real(np.fft.ifft2(-(KX ** 2 + KY ** 2) * np.fft.fft2(T[0])))[None]
        ref = K * lapT / (np.exp(f[0]) * T)
        errs.append(np.max(np.abs(r[4] - ref)))
    orders = [math.log2(errs[t] / errs[t + 1]) for t in range(2)]
    assert all(5.6 < o < 6.4 for o in orders), (errs, orders)


@pytest.mark.parametrize("order", [6, 4])
def test_brute_force_all_terms(oracle_lib, order):
    n = (9, 8, 10)
    frc = core.Forcing(k=(1, 0, -2), e=(0.0, 0.8, 0.6), phi=0.9, amp=0.05)
    p = core.Params(n=n, L=(5.0, 4.0, 6.0), forcing=frc, order=order, nu=0.011, eta=0.007,
                    cs0=1.3, gamma=1.4, cp=1.7, lnrho0=0.2, K=0.03, zeta=0.02, heat=0.4,
                    cool=0.15)
    f = synthetic.smooth_state(n, seed=21, amp=0.3)
    f += 0.02 * np.random.default_rng(22).standard_normal(f.shape)
    r = core.rhs(f, p)
    rb = brute.rhs(f, p)
    for q in range(8):
        scale = np.max(np.abs(rb[q]))
        assert np.max(np.abs(r[q] - rb[q])) <= 1e-12 * scale, (order, q)
