"""GPU parity of the full Eqs. B.2-B.3 terms (conduction K, bulk viscosity
zeta, heating H, cooling C) against the FP64 oracle, on every kernel path:
plain binary64 (padded layout, unequal spacings), the integer-sum binary64
path (cubic periodic grid), the binary32 tiled kernel (order 6) and the
binary32 direct-load kernel (order 4).

Tolerances as for the base terms: binary64 1e-12 relative per field; binary32
f <= 2e-6 and w <= 2e-4 relative on inputs already rounded to binary32.
"""
import math

import numpy as np
import pytest
import torch

from oracle import core
from paper_2103_01597_gb300 import ac, build, synthetic

from gpu_util import rel_err

pytestmark = pytest.mark.gpu

TERMS = dict(K=0.03, zeta=0.02, heat=0.4, cool=0.15)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    ac.load_library()
    torch.cuda.init()


def _state(n, seed, amp=0.2):
    f = synthetic.smooth_state(n, seed, amp=amp)
    f += synthetic.noise_state(n, seed + 100, sigma=1e-3)
    f[0] += 0.1 * synthetic.uniform_state(n, seed + 200)[0]
    f[4] += 0.05 * synthetic.uniform_state(n, seed + 300)[4]
    return f


def _run(n, L, layout, precision, phys, order=6, mode=None, seed=4):
    sim = ac.Simulation(n, L=L, layout=layout, precision=precision, force_amp=0.05, seed=seed,
                        order=order, **phys, **TERMS)
    if mode is not None:
        ac.ac_set_stencil_mode(sim.h, mode)
    f = _state(n, seed=sum(n))
    sim.load(f)
    fcur = f if precision == ac.AC_FP64 else f.astype(np.float32).astype(np.float64)
    w = None
    errs = []
    for s in range(3):
        p = core.Params(n=n, L=L, forcing=core.forcing_draw(seed, 0, 0.05), order=order, **phys,
                        **TERMS)
        fo, wo = core.substep(fcur, w, p, 1e-3, s)
        sim.substep(1e-3, s)
        fg, wg = sim.store(), sim.store_w()
        errs.append((rel_err(fg, fo), rel_err(wg, wo)))
        fcur, w = fg, wg
    path = ac.ac_get_stencil_path(sim.h)
    sim.close()
    return errs, path


PHYS = dict(nu=2e-2, eta=3e-2, cs0=1.1, gamma=1.4, cp=1.3, lnrho0=0.2)


@pytest.mark.parametrize("layout", [ac.AC_LAYOUT_PADDED, ac.AC_LAYOUT_PERIODIC])
@pytest.mark.parametrize("n", [(16, 12, 10), (37, 21, 13)])
def test_fp64_full_entropy_unequal_spacing(n, layout):
    errs, fixed = _run(n, (2 * math.pi, 3.0, 5.5), layout, ac.AC_FP64, PHYS)
    assert not fixed
    for s, (ef, ew) in enumerate(errs):
        assert np.all(ef <= 1e-12), (s, ef)
        assert np.all(ew <= 1e-12), (s, ew)


@pytest.mark.parametrize("n", [(16, 12, 20), (24, 24, 24)])
def test_fp64_full_entropy_integer_sums(n):
    h = 0.3
    errs, fixed = _run(n, tuple(h * v for v in n), ac.AC_LAYOUT_PERIODIC, ac.AC_FP64, PHYS,
                       mode=ac.AC_STENCIL_FIXED)
    assert fixed
    for s, (ef, ew) in enumerate(errs):
        assert np.all(ef <= 1e-12), (s, ef)
        assert np.all(ew <= 1e-12), (s, ew)


@pytest.mark.parametrize("order", [6, 4])
@pytest.mark.parametrize("precision", [ac.AC_FP32, ac.AC_FP32_W64])
def test_fp32_full_entropy_within_bound(order, precision):
    n = (20, 16, 12)
    phys = dict(nu=5e-3, eta=5e-3, cs0=1.0, gamma=5.0 / 3.0, cp=1.0, lnrho0=0.0)
    errs, _ = _run(n, (2 * math.pi,) * 3, ac.AC_LAYOUT_PERIODIC, precision, phys, order=order)
    for s, (ef, ew) in enumerate(errs):
        print("order %d fp32 full entropy s=%d f %.2e w %.2e" % (order, s, ef.max(), ew.max()))
        assert np.all(ef <= 2e-6), (s, ef)
        assert np.all(ew <= 2e-4), (s, ew)


def test_entropy_terms_validated():
    sim = ac.Simulation((8, 8, 8))
    for bad in [dict(K=-1.0), dict(zeta=-0.1), dict(heat=float("nan")), dict(cool=-2.0),
                dict(K=float("inf"))]:
        with pytest.raises(ac.AcError):
            ac.ac_set_entropy_terms(sim.h, **bad)
    ac.ac_set_entropy_terms(sim.h, K=0.0, zeta=0.0, heat=0.3, cool=0.3)  # H - C = 0: base kernels
    sim.close()
