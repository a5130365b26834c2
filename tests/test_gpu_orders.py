"""GPU parity of the substep at stencil orders 2, 4 and 8 (radius 1, 2, 4 on
the point set of Eq. 13 widened to radius r) against the FP64 oracle at the
same order, through the C ABI.

Tolerances as for the sixth-order path: FP64 1e-12 relative per field (max
norm) for f and w; binary32 f <= 2e-6 and w <= 2e-4 relative on inputs already
rounded to binary32; reductions 1e-12.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    ac.load_library()
    torch.cuda.init()


def _state(n, seed, amp=0.2):
    f = synthetic.smooth_state(n, seed, amp=amp)
    f += synthetic.noise_state(n, seed + 100, sigma=1e-3)
    f[0] += 0.1 * synthetic.uniform_state(n, seed + 200)[0]
    return f


def _run(n, order, layout, precision, L, phys, seed, steps=3):
    """Three substeps on the GPU and in the oracle; yields the per-substep
    relative errors of f and w."""
    sim = ac.Simulation(n, L=L, layout=layout, precision=precision, force_amp=0.05, seed=seed,
                        order=order, **phys)
    assert ac.ac_get_stencil_order(sim.h) == order
    f = _state(n, seed=sum(n) + order)
    sim.load(f)
    fcur = f if precision == ac.AC_FP64 else f.astype(np.float32).astype(np.float64)
    w = None
    dt = 1e-3
    errs = []
    for s in range(steps):
        p = core.Params(n=n, L=L, forcing=core.forcing_draw(seed, 0, 0.05), order=order, **phys)
        fo, wo = core.substep(fcur, w, p, dt, s)
        sim.substep(dt, s)
        fg, wg = sim.store(), sim.store_w()
        errs.append((rel_err(fg, fo), rel_err(wg, wo)))
        fcur, w = fg, wg
    sim.close()
    return errs


# ragged against the 32x4 CTA; axes shorter than the stencil width
SIZES = [(16, 12, 10), (37, 21, 13), (5, 3, 7)]


@pytest.mark.parametrize("order", [2, 4, 8])
@pytest.mark.parametrize("n", SIZES)
def test_fp64_orders_match_oracle_periodic(order, n):
    for s, (ef, ew) in enumerate(_run(n, order, ac.AC_LAYOUT_PERIODIC, ac.AC_FP64,
                                      (2 * math.pi, 3.0, 5.5), PHYS, seed=2)):
        assert np.all(ef <= 1e-12), (order, s, ef)
        assert np.all(ew <= 1e-12), (order, s, ew)


@pytest.mark.parametrize("order", [2, 4])
def test_fp64_orders_match_oracle_padded(order):
    n = (16, 12, 10)
    for s, (ef, ew) in enumerate(_run(n, order, ac.AC_LAYOUT_PADDED, ac.AC_FP64,
                                      (2 * math.pi, 3.0, 5.5), PHYS, seed=2)):
        assert np.all(ef <= 1e-12), (order, s, ef)
        assert np.all(ew <= 1e-12), (order, s, ew)


@pytest.mark.parametrize("order", [2, 4, 8])
@pytest.mark.parametrize("precision", [ac.AC_FP32, ac.AC_FP32_W64])
def test_fp32_orders_within_bound(order, precision):
    n = (20, 16, 12)
    phys = dict(nu=5e-3, eta=5e-3, cs0=1.0, gamma=5.0 / 3.0, cp=1.0, lnrho0=0.0)
    for s, (ef, ew) in enumerate(_run(n, order, ac.AC_LAYOUT_PERIODIC, precision,
                                      (2 * math.pi,) * 3, phys, seed=3)):
        print("order %d fp32 s=%d max rel err f %.2e w %.2e" % (order, s, ef.max(), ew.max()))
        assert np.all(ef <= 2e-6), (order, s, ef)
        assert np.all(ew <= 2e-4), (order, s, ew)


@pytest.mark.parametrize("order", [2, 4, 8])
def test_reductions_at_order(order):
    n = (20, 16, 12)
    sim = ac.Simulation(n, order=order, **PHYS)
    f = _state(n, seed=9)
    sim.load(f)
    p = core.Params(n=n, order=order, **PHYS)
    for quantity, oq in [(ac.AC_Q_EMAG, "emag"), (ac.AC_Q_CFL, "cfl")]:
        for op, oname in [(ac.AC_MAX, "max"), (ac.AC_SUM, "sum")]:
            g = sim.reduce(op, quantity)
            o = core.reduce(f, p, oname, oq)
            scale = np.sum(np.abs(core.quantity(f, p, oq))) if oname == "sum" else abs(o)
            assert abs(g - o) <= 1e-12 * scale, (order, quantity, oname, g, o)
    sim.close()


def test_order_api():
    n = (8, 8, 8)
    sim = ac.Simulation(n, L=(1.0, 1.0, 1.0))
    assert ac.ac_get_stencil_order(sim.h) == 6
    assert ac.ac_get_stencil_path(sim.h)            # integer sums at order 6
    ac.ac_set_stencil_order(sim.h, 4)
    assert not ac.ac_get_stencil_path(sim.h)        # only order 6 has them
    for bad in (0, 3, 5, 10):
        with pytest.raises(ac.AcError):
            ac.ac_set_stencil_order(sim.h, bad)
    ac.ac_set_stencil_order(sim.h, 6)
    ac.ac_set_stencil_mode(sim.h, ac.AC_STENCIL_FIXED)
    with pytest.raises(ac.AcError):                 # FIXED needs order 6
        ac.ac_set_stencil_order(sim.h, 2)
    assert ac.ac_get_stencil_order(sim.h) == 6
    ac.ac_set_stencil_mode(sim.h, ac.AC_STENCIL_AUTO)
    sim.load(_state(n, seed=1))
    sim.substep(1e-3, 0)
    with pytest.raises(ac.AcError):                 # not inside a step
        ac.ac_set_stencil_order(sim.h, 4)
    sim.close()
    pad = ac.Simulation(n, layout=ac.AC_LAYOUT_PADDED)
    with pytest.raises(ac.AcError):                 # the padded halo is 3 cells
        ac.ac_set_stencil_order(pad.h, 8)
    pad.close()
