"""Pins of the oracle's halo map, forcing draw, restriction and reductions.

  * periodic halo (Sec. 3.3): equals NumPy's wrap padding, an independent
    library routine;
  * SplitMix64: published reference outputs (tests/golden/splitmix64.txt);
  * forcing draw (a reading; not in the paper): k in the shell 2 <= |k| <= 3,
    e unit and perpendicular to k, phi in [0, 2 pi), and the k draws cover the
    shell uniformly (chi-square);
  * restriction (a reading): full weighting of a separable sinusoid is the
    sinusoid at the coarse nodes times prod_a (1 + cos theta_a) / 2;
  * reductions: sum sin^2 over a periodic grid is N / 2 exactly, a planted
    spike is the max, closed forms of the energies and the CFL speed.
"""
import math
import os

import numpy as np
import pytest

from oracle import core

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_periodic_halo_matches_numpy_wrap(oracle_lib):
    n = (7, 5, 9)
    r = 3
    rng = np.random.default_rng(1)
    interior = rng.standard_normal((n[2], n[1], n[0]))
    padded = np.zeros((n[2] + 2 * r, n[1] + 2 * r, n[0] + 2 * r))
    padded[r:-r, r:-r, r:-r] = interior
    got = core.periodic_halo(padded, n, r)
    assert np.array_equal(got, np.pad(interior, r, mode="wrap"))


def test_splitmix64_reference_vectors(oracle_lib):
    rows = [line.split() for line in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if line.strip() and not line.startswith("#")]
    assert rows
    for seed, idx, out in rows:
        assert core.splitmix64(int(seed), int(idx)) == int(out)


def _shell():
    return [(a, b, c) for a in range(-3, 4) for b in range(-3, 4) for c in range(-3, 4)
            if 4 <= a * a + b * b + c * c <= 9]


def test_forcing_draw_properties(oracle_lib):
    shell = _shell()
    counts = {k: 0 for k in shell}
    steps = 20 * len(shell)
    for t in range(steps):
        fr = core.forcing_draw(2, t, 0.05)
        k = np.array(fr.k, dtype=float)
        e = np.array(fr.e)
        assert tuple(fr.k) in counts
        assert abs(np.dot(e, e) - 1) < 1e-15
        assert abs(np.dot(k, e)) < 1e-14 * np.linalg.norm(k)
        assert 0 <= fr.phi < 2 * math.pi
        counts[tuple(fr.k)] += 1
    obs = np.array(list(counts.values()), dtype=float)
    chi2 = np.sum((obs - 20) ** 2 / 20)
    dof = len(shell) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), chi2
    # deterministic in (seed, step)
    assert core.forcing_draw(7, 3, 1.0) == core.forcing_draw(7, 3, 1.0)
    assert core.forcing_draw(7, 3, 1.0) != core.forcing_draw(7, 4, 1.0)


def test_restriction_closed_form(oracle_lib):
    nf = (16, 12, 8)
    k, j, i = np.meshgrid(np.arange(nf[2]), np.arange(nf[1]), np.arange(nf[0]), indexing="ij")
    m = (2, 1, 3)
    th = [2 * math.pi * m[a] / nf[a] for a in range(3)]
    f = (np.sin(th[0] * i + 0.3) * np.cos(th[1] * j) * np.sin(th[2] * k + 1.0))
    c = core.restrict(f)
    K, J, I = np.meshgrid(np.arange(nf[2] // 2), np.arange(nf[1] // 2), np.arange(nf[0] // 2),
                          indexing="ij")
    fac = np.prod([(1 + math.cos(t)) / 2 for t in th])
    ref = fac * np.sin(th[0] * 2 * I + 0.3) * np.cos(th[1] * 2 * J) * np.sin(th[2] * 2 * K + 1.0)
    np.testing.assert_allclose(c, ref, atol=1e-14)
    assert np.allclose(core.restrict(np.full(nf[::-1], 2.5)), 2.5, atol=0, rtol=1e-15)


def test_reductions_closed_forms(oracle_lib):
    n = (16, 8, 4)
    p = core.Params(n=n, cs0=1.2, gamma=1.5, cp=1.0)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    f = np.zeros((8, n[2], n[1], n[0]))
    f[1] = np.sin(2 * math.pi * 3 * i / n[0])
    N = f[0].size
    assert core.reduce(f, p, "sum", 1) == pytest.approx(0.0, abs=1e-13)
    assert math.fsum((f[1] ** 2).ravel()) == pytest.approx(N / 2, rel=1e-15)
    assert core.reduce(f, p, "rms", 1) == pytest.approx(math.sqrt(0.5), rel=1e-15)
    g = np.zeros_like(f)
    g[4][2, 3, 5] = 7.0
    g[4][1, 1, 1] = -9.0
    assert core.reduce(g, p, "max", 4) == 7.0 and core.reduce(g, p, "min", 4) == -9.0
    # uniform flow, uniform density: ekin = rho |u|^2 / 2 everywhere
    h = np.zeros_like(f)
    h[0] = 0.4
    h[1:4] = np.array([0.3, -0.2, 0.1])[:, None, None, None]
    assert core.reduce(h, p, "sum", "ekin") == pytest.approx(
        N * 0.5 * math.exp(0.4) * 0.14, rel=1e-14)
    # Beltrami A: |curl A|^2 = kappa^2 eps^2 everywhere
    m, eps = 2, 0.3
    th = 2 * math.pi * m / n[0]
    dx = 2 * math.pi / n[0]
    kap = (1.5 * math.sin(th) - 0.3 * math.sin(2 * th) + math.sin(3 * th) / 30.0) / dx
    b = np.zeros_like(f)
    b[6] = eps * np.sin(2 * math.pi * m * i / n[0])
    b[7] = eps * np.cos(2 * math.pi * m * i / n[0])
    assert core.reduce(b, p, "max", "emag") == pytest.approx(0.5 * kap ** 2 * eps ** 2, rel=1e-13)
    # CFL speed with rho = 1, s = 0: |u| + sqrt(cs0^2 + |B|^2)
    b[1] = 0.25
    assert core.reduce(b, p, "max", "cfl") == pytest.approx(
        0.25 + math.sqrt(1.44 + kap ** 2 * eps ** 2), rel=1e-13)
    assert core.reduce(b, p, "max", "umag") == pytest.approx(0.25, rel=1e-15)


def test_rk_coefficients_sum_rules(oracle_lib):
    """2N-storage weights: the effective weights of the three RHS evaluations in
    the final state add to 1 (consistency)."""
    al, be = core.rk_coefficients()
    # weight of k_s in the final state: sum over later betas with alpha products
    w0 = be[0] + be[1] * al[1] + be[2] * al[2] * al[1]
    w1 = be[1] + be[2] * al[2]
    w2 = be[2]
    assert w0 + w1 + w2 == pytest.approx(1.0, rel=1e-15)
