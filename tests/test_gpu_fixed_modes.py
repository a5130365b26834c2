"""The integer-sum binary64 stencil path on states that stress its fixed point.

Each field is quantised about its own offset with a scale set by its own range;
the device picks group scales (FX_GROUP), per-field scales (FX_FIELD) or plain
binary64 stencils (FX_PLAIN, non-finite states).  Every case runs through the C
ABI on the default (AUTO) stencil path and is compared, substep by substep, with
the FP64 oracle at 1e-12 relative per field in the max norm (the bound the
method is held to; see test_gpu_substep.py).  The mode the device chose is
checked against the rule stated in include/ac.h, evaluated here on the host
from the same state.
"""
import math

import numpy as np
import pytest
import torch

from oracle import core
from paper_2103_01597_gb300 import ac, build, synthetic

from gpu_util import rel_err

pytestmark = pytest.mark.gpu

PHYS = dict(nu=2e-2, eta=3e-2, cs0=1.1, gamma=1.4, cp=1.3, lnrho0=0.2)
N = (24, 24, 24)
GROUPS = [(0,), (1, 2, 3), (4,), (5, 6, 7)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    ac.load_library()
    torch.cuda.init()


def expected_mode(f):
    """The mode rule of the integer-sum path, from the state's extremes."""
    if not np.all(np.isfinite(f)):
        return ac.AC_STENCIL_MODE_PLAIN
    e = {}
    for q in range(8):
        lo, hi = float(f[q].min()), float(f[q].max())
        c = 0.5 * lo + 0.5 * hi
        r = max(hi - c, c - lo)
        if r == 0.0:
            continue
        if not (2.0 ** -960 <= r < 2.0 ** 960):
            return ac.AC_STENCIL_MODE_PLAIN
        e[q] = math.frexp(r)[1]  # smallest E with r < 2^E
    for g in GROUPS:
        es = [e[q] for q in g if q in e]
        if es and min(es) < max(es) - 1:  # more than one binade apart
            return ac.AC_STENCIL_MODE_FIELD
    return ac.AC_STENCIL_MODE_GROUP


def pin_range(a, m):
    """Set two cells so that the field's extremes are exactly +m and -m."""
    assert np.max(np.abs(a)) <= m
    a[0, 0, 0] = m
    a[1, 2, 3] = -m
    return a


def run_substeps(f, force_amp=0.0, seed=2, steps=3):
    """Substeps 0..steps-1 from f on the AUTO path (each from the GPU's own
    previous state) against the oracle; returns the per-substep errors and the
    mode counts."""
    sim = ac.Simulation(N, force_amp=force_amp, seed=seed, **PHYS)
    assert ac.ac_get_stencil_path(sim.h)
    sim.load(f)
    dt = 1e-3
    w = None
    modes, errs = [], []
    forcing = core.forcing_draw(seed, 0, force_amp) if force_amp else None
    p = core.Params(n=N, forcing=forcing, **PHYS)
    for s in range(steps):
        modes.append(expected_mode(f))
        fo, wo = core.substep(f, w, p, dt, s)
        sim.substep(dt, s)
        fg, wg = sim.store(), sim.store_w()
        errs.append((rel_err(fg, fo), rel_err(wg, wo)))
        f, w = fg, wg
    counts = ac.ac_get_stencil_modes(sim.h)
    sim.close()
    want = tuple(modes.count(m) for m in range(3))
    return errs, counts, want


def assert_parity(errs):
    for s, (ef, ew) in enumerate(errs):
        assert np.all(ef <= 1e-12), (s, ef)
        assert np.all(ew <= 1e-12), (s, ew)


def test_weak_field_component():
    """u = 0 and A_z / A_x = 1e-8: pure diffusion of a tiny A_z beside O(0.1)
    components.  With one scale per group A_z would be resolved only to
    2^-50 of |A_x| (1e-8 relative); per-field scales keep 2^-50 of its own."""
    f = synthetic.smooth_state(N, seed=31, amp=0.2) + synthetic.noise_state(N, seed=32, sigma=1e-3)
    f[0] = 0.0
    f[1:5] = 0.0
    weak = synthetic.smooth_state(N, seed=33, amp=0.2) + synthetic.noise_state(N, seed=34,
                                                                               sigma=1e-3)
    f[7] = 1e-8 * weak[7]
    errs, counts, want = run_substeps(f, force_amp=0.05)
    assert counts == want, (counts, want)
    assert counts[ac.AC_STENCIL_MODE_FIELD] >= 1, counts
    assert_parity(errs)


def test_near_two_dimensional_flow():
    """u_z / u_x = 1e-8 with uniform (non-zero) ln rho and s: advection of u_z and
    its viscous terms need u_z resolved on its own scale."""
    f = synthetic.smooth_state(N, seed=41, amp=0.2) + synthetic.noise_state(N, seed=42, sigma=1e-3)
    f[0] = 0.3
    f[4] = -0.2
    small = synthetic.smooth_state(N, seed=43, amp=0.2) + synthetic.noise_state(N, seed=44,
                                                                                sigma=1e-3)
    f[3] = 1e-8 * small[3]
    errs, counts, want = run_substeps(f)
    assert counts == want, (counts, want)
    assert counts[ac.AC_STENCIL_MODE_FIELD] >= 1, counts
    assert_parity(errs)


def test_offset_background():
    """ln rho = 0.7 + 1e-7 noise, s = 1.3 + 1e-7 noise: the fluctuations, not the
    background, set each field's scale (the offset is the range's midpoint), so
    the pressure gradient keeps full relative precision.  The components of u
    and of A are pinned to equal ranges, so the group-scale mode runs."""
    g = np.random.Generator(np.random.PCG64(51))
    f = synthetic.smooth_state(N, seed=52, amp=0.02) + synthetic.noise_state(N, seed=53,
                                                                             sigma=1e-3)
    f[0] = 0.7 + 1e-7 * g.standard_normal(f[0].shape)
    f[4] = 1.3 + 1e-7 * g.standard_normal(f[4].shape)
    for q in (1, 2, 3):
        pin_range(f[q], 0.09)
    for q in (5, 6, 7):
        pin_range(f[q], 0.09)
    errs, counts, want = run_substeps(f, steps=1)
    assert counts == want == (1, 0, 0), (counts, want)
    assert_parity(errs)


@pytest.mark.parametrize("at_power", [False, True])
def test_range_at_binade_edge(at_power):
    """Every field's half-range just below a power of two (|F| reaches 2^50, the
    headroom the exact sums are sized for; a Nyquist checkerboard makes the
    second-derivative numerators reach 1088 |F|) or exactly at one."""
    m = 0.125 if at_power else np.nextafter(0.125, 0.0)
    f = synthetic.smooth_state(N, seed=61, amp=0.02)
    k, j, i = np.meshgrid(np.arange(N[2]), np.arange(N[1]), np.arange(N[0]), indexing="ij")
    checker = np.where((i + j + k) % 2 == 0, 1.0, -1.0)
    for q in (1, 2, 3):
        f[q] = m * checker * (1.0 if q != 2 else -1.0)
    for q in (0, 4, 5, 6, 7):
        f[q] = pin_range(0.5 * m * f[q] / np.max(np.abs(f[q])), m)
    errs, counts, want = run_substeps(f)
    assert counts == want, (counts, want)
    assert counts[ac.AC_STENCIL_MODE_GROUP] >= 1, counts
    assert_parity(errs)


@pytest.mark.parametrize("mz,mode", [(0.04, 0), (0.02, 1)])
def test_one_binade_of_slack(mz, mode):
    """u_x spans +-0.1 (E = -3), u_y +-0.05 (E = -4): one binade apart, so the
    components share u_x's scale.  u_z at +-0.04 (E = -4) keeps group scales;
    at +-0.02 (E = -5, two binades below u_x) it takes per-field scales."""
    f = synthetic.smooth_state(N, seed=91, amp=0.005)
    for q, m in ((1, 0.1), (2, 0.05), (3, mz), (5, 0.1), (6, 0.1), (7, 0.1)):
        f[q] = pin_range(f[q], m)
    assert expected_mode(f) == (ac.AC_STENCIL_MODE_GROUP if mode == 0 else
                                ac.AC_STENCIL_MODE_FIELD)
    errs, counts, want = run_substeps(f, steps=1)
    assert counts == want, (counts, want)
    assert_parity(errs)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_state_takes_plain_stencils(bad):
    """One NaN (or infinity) in u_y: the plan selects plain binary64 stencils, so
    the non-finite values spread over exactly the stencil neighbourhoods the
    definition spreads them to, every finite value still matches, and the
    step's CFL word reports the state as non-finite."""
    f = synthetic.smooth_state(N, seed=71, amp=0.2) + synthetic.noise_state(N, seed=72, sigma=1e-3)
    f[2][5, 6, 7] = bad
    sim = ac.Simulation(N, **PHYS)
    sim.load(f)
    p = core.Params(n=N, **PHYS)
    w = None
    for s in range(3):
        fo, wo = core.substep(f, w, p, 1e-3, s)
        sim.substep(1e-3, s)
        fg, wg = sim.store(), sim.store_w()
        for g, o in ((fg, fo), (wg, wo)):
            bad_o = ~np.isfinite(o)
            assert np.array_equal(~np.isfinite(g), bad_o), s
            assert np.any(bad_o)
            for q in range(8):
                fin = ~bad_o[q]
                den = np.max(np.abs(o[q][fin]))
                err = np.max(np.abs(g[q][fin] - o[q][fin]))
                assert err <= 1e-12 * den if den > 0 else err == 0, (s, q, err, den)
        f, w = fg, wg
    assert ac.ac_get_stencil_modes(sim.h) == (0, 0, 3)
    with pytest.raises(ac.AcError) as ei:
        ac.ac_last_cfl(sim.h)
    assert ei.value.code == ac.AC_ERR_NONFINITE
    sim.close()


def test_benchmark_noise_state_runs_group_scales():
    """The configuration's own initial state (noise of amplitude 1e-5 on u and
    A, ln rho = s = 0) and its forced step: the modes follow the rule."""
    f = synthetic.noise_state(N, seed=2)
    errs, counts, want = run_substeps(f, force_amp=0.05)
    assert counts == want, (counts, want)
    assert_parity(errs)


def test_constant_fields():
    """Constant fields quantise to zero (every stencil of a constant is zero)."""
    f = synthetic.smooth_state(N, seed=81, amp=0.2)
    f[0] = 0.25
    f[3] = -0.5
    f[4] = 0.0
    f[6] = 1.0
    errs, counts, want = run_substeps(f)
    assert counts == want, (counts, want)
    assert_parity(errs)


@pytest.mark.parametrize("dt", [0.0, 1e-120, -1e-120])
def test_zero_or_tiny_dt_takes_plain_stencils(dt):
    """The integer-sum kernels fold dt into their coefficients (1 / dt^2 must stay
    in range for the CFL speed), so a step of zero or of magnitude below 1e-100
    runs the plain binary64 stencils: no mode is counted, the state moves by
    at most dt times its right-hand side, and the CFL speed of the input state
    matches the one the integer-sum path reports for it."""
    f = synthetic.smooth_state(N, 21, amp=0.3) + synthetic.noise_state(N, 22, 1e-3)
    sim = ac.Simulation(N, force_amp=0.0, seed=1, **PHYS)
    sim.load(f)
    sim.step(dt)
    assert tuple(ac.ac_get_stencil_modes(sim.h)) == (0, 0, 0)
    g = sim.store()
    if dt == 0.0:
        assert np.array_equal(g, f)
    else:
        assert np.max(np.abs(g - f)) <= 1e-110
    cfl_plain = ac.ac_last_cfl(sim.h)
    ref = ac.Simulation(N, force_amp=0.0, seed=1, **PHYS)
    ref.load(f)
    ref.step(1e-3)
    assert sum(ac.ac_get_stencil_modes(ref.h)) == 3
    assert abs(ac.ac_last_cfl(ref.h) - cfl_plain) <= 1e-12 * cfl_plain
    sim.close()
    ref.close()
