"""The float32 host format of the state (ac_load_f32 / ac_store_f32).

Binary32 states take and give their values unchanged (periodic layout: the
state's own bytes; padded layout: through the staging buffer); a binary64 state
takes binary32 values exactly and is rounded to nearest on store.  Loading the
binary32 values must leave the handle exactly as loading the same values in
binary64 does, so a step after either is bitwise the same.
"""
import numpy as np
import pytest

from paper_2103_01597_gb300 import ac, build, synthetic

pytestmark = pytest.mark.gpu

N = (20, 12, 9)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    ac.load_library()


def _state32():
    f = synthetic.smooth_state(N, 3, amp=0.3) + synthetic.noise_state(N, 4, 1e-3)
    return np.ascontiguousarray(f.astype(np.float32))


CASES = [(ac.AC_FP32, ac.AC_LAYOUT_PERIODIC), (ac.AC_FP32, ac.AC_LAYOUT_PADDED),
         (ac.AC_FP32_W64, ac.AC_LAYOUT_PERIODIC), (ac.AC_FP64, ac.AC_LAYOUT_PERIODIC),
         (ac.AC_FP64, ac.AC_LAYOUT_PADDED)]


@pytest.mark.parametrize("precision,layout", CASES)
def test_round_trip(precision, layout):
    x = _state32()
    sim = ac.Simulation(N, precision=precision, layout=layout)
    ac.ac_load_f32(sim.h, ac.AC_ALL, x)
    y = np.empty_like(x)
    ac.ac_store_f32(sim.h, ac.AC_ALL, y)
    assert np.array_equal(y, x)
    assert np.array_equal(sim.store(), x.astype(np.float64))  # the values themselves
    # one field on its own
    z = x.copy()
    z[3] *= 2.0
    ac.ac_load_f32(sim.h, 3, np.ascontiguousarray(z[3]))
    one = np.empty_like(z[3])
    ac.ac_store_f32(sim.h, 3, one)
    assert np.array_equal(one, z[3])
    sim.close()


@pytest.mark.parametrize("precision,layout", CASES)
def test_step_after_f32_load_equals_f64_load(precision, layout):
    x = _state32()
    out = []
    for f32 in (True, False):
        sim = ac.Simulation(N, precision=precision, layout=layout, force_amp=0.05, seed=3)
        if f32:
            ac.ac_load_f32(sim.h, ac.AC_ALL, x)
        else:
            sim.load(x.astype(np.float64))
        sim.step(1e-3)
        out.append(sim.store())
        sim.close()
    assert np.array_equal(out[0], out[1])


def test_f64_state_rounds_on_store():
    x = synthetic.smooth_state(N, 5, amp=0.3) + synthetic.noise_state(N, 6, 1e-3)
    sim = ac.Simulation(N, precision=ac.AC_FP64)
    sim.load(x)
    y = np.empty(x.shape, dtype=np.float32)
    ac.ac_store_f32(sim.h, ac.AC_ALL, y)
    assert np.array_equal(y, x.astype(np.float32))  # round to nearest
    sim.close()


def test_argument_errors():
    sim = ac.Simulation(N, precision=ac.AC_FP32)
    with pytest.raises(ac.AcError):
        ac.ac_load_f32(sim.h, ac.AC_ALL, 0)
    with pytest.raises(ac.AcError):
        ac.ac_store_f32(sim.h, 8, np.empty(N[::-1], dtype=np.float32))
    sim.close()
