"""Domain decomposition with halo exchange (Sec. 3.2-3.3) on one GPU.

The grid is split into subdomains with radius-3 halos; each substep packs the
outbound sides and edges, delivers them, unpacks them into the neighbours'
halos and updates the outer segments while the inner segment is updated
concurrently.  The result must equal the undecomposed substep bitwise: the
per-cell arithmetic is the same code as the padded-layout substep, and the
halos hold exactly the values the periodic map gives (a wrong segment box,
direction or neighbour would change some cell).
"""
import math

import numpy as np
import pytest
import torch

from paper_2103_01597_gb300 import ac, build, synthetic

pytestmark = pytest.mark.gpu

PHYS = dict(nu=2e-2, eta=3e-2, cs0=1.1, gamma=1.4, cp=1.3, lnrho0=0.2)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    ac.load_library()
    torch.cuda.init()


def _state(n, seed):
    f = synthetic.smooth_state(n, seed, amp=0.2) + synthetic.noise_state(n, seed + 1, sigma=1e-3)
    return f


def _compare(n, p, precision, overlap, steps=2, L=(2 * math.pi, 3.0, 5.5), force_amp=0.05):
    f = _state(n, seed=sum(p) + 3 * precision)
    ref = ac.Simulation(n, L=L, layout=ac.AC_LAYOUT_PADDED, precision=precision,
                        force_amp=force_amp, seed=4, **PHYS)
    dec = ac.Decomp(n, p, L=L, precision=precision, force_amp=force_amp, seed=4,
                    overlap=overlap, **PHYS)
    ref.load(f)
    dec.load(f)
    for _ in range(steps):
        for s in range(3):
            ref.substep(1e-3, s)
            dec.substep(1e-3, s)
            if s == 1:  # mid-step: the accumulator too
                assert np.array_equal(dec.store_w(), ref.store_w())
        assert np.array_equal(dec.store(), ref.store())
    info = dec.info()
    dec.close()
    ref.close()
    return info


@pytest.mark.parametrize("p", [(2, 1, 1), (2, 2, 2), (1, 1, 8), (1, 3, 2)])
@pytest.mark.parametrize("overlap", [True, False])
def test_decomposed_fp64_bitwise(p, overlap):
    n = (48, 36, 64) if p != (1, 3, 2) else (40, 36, 24)
    info = _compare(n, p, ac.AC_FP64, overlap)
    assert info["p"] == p and info["messages"] == 18 * p[0] * p[1] * p[2]


@pytest.mark.parametrize("precision", [ac.AC_FP32, ac.AC_FP32_W64])
def test_decomposed_fp32_bitwise(precision):
    _compare((48, 36, 64), (2, 2, 2), precision, True)


def test_decomposed_matches_periodic_binary64_stencils():
    """The decomposed binary64 run also equals the periodic-layout handle on
    plain binary64 stencils (AC_STENCIL_FP64) bitwise."""
    n = (32, 32, 32)
    f = _state(n, seed=5)
    ref = ac.Simulation(n, force_amp=0.05, seed=6, **PHYS)
    ac.ac_set_stencil_mode(ref.h, ac.AC_STENCIL_FP64)
    dec = ac.Decomp(n, ac.ac_decomp_partition(4), force_amp=0.05, seed=6, **PHYS)
    ref.load(f)
    dec.load(f)
    ref.step(1e-3)
    dec.step(1e-3)
    assert np.array_equal(dec.store(), ref.store())
    dec.close()
    ref.close()


def test_decomposed_256_fp64():
    """The timed grid size, 2 x 2 x 2 subdomains of 128^3, one forced step."""
    n = (256, 256, 256)
    f = synthetic.noise_state(n, seed=2)
    ref = ac.Simulation(n, layout=ac.AC_LAYOUT_PADDED, force_amp=0.05, seed=2)
    dec = ac.Decomp(n, (2, 2, 2), force_amp=0.05, seed=2)
    ref.load(f)
    dec.load(f)
    ref.step(1e-3)
    dec.step(1e-3)
    assert np.array_equal(dec.store(), ref.store())
    dec.close()
    ref.close()


def test_decomposed_rejects_bad_partitions():
    for n, p in [((32, 32, 30), (1, 1, 4)), ((32, 32, 32), (1, 1, 8)), ((32, 32, 32), (0, 1, 1))]:
        with pytest.raises(ac.AcError) as ei:
            ac.Decomp(n, p)
        assert ei.value.code == ac.AC_ERR_ARG
