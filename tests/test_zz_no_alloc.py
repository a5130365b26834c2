"""The allocation-free reduction, ac_reduce_noalloc.

Some callers cannot allocate device memory: an application that manages all
device memory through its own pool and only lends this library its field
arrays cannot create an ac_handle (whose work areas come from cudaMalloc).
For them ac_reduce_noalloc keeps its partial sums in a fixed device array
inside the library.  This test calls it through the C ABI on torch-owned
arrays and checks it against ac_reduce on the same state, twice in a row (the
shared fixed array keeps the previous call's contents), within the tolerance
the other reduction tests use (1e-12 relative; max and min exactly).  It runs
last so that a failure here leaves every other test already run.
"""
import math

import numpy as np
import pytest
import torch

from paper_2103_01597_gb300 import ac, build, synthetic

pytestmark = pytest.mark.gpu


def _state(n):
    f = synthetic.smooth_state(n, seed=31, amp=0.3) + synthetic.noise_state(n, seed=32, sigma=1e-3)
    f[0] += 0.05
    return f


@pytest.mark.parametrize("precision,layout", [(ac.AC_FP64, ac.AC_LAYOUT_PERIODIC),
                                              (ac.AC_FP64, ac.AC_LAYOUT_PADDED),
                                              (ac.AC_FP32, ac.AC_LAYOUT_PERIODIC)])
def test_noalloc_reduce_matches_ac_reduce(precision, layout):
    build.build()
    n = (36, 20, 28)
    L = (2 * math.pi, 3.0, 4.5)
    phys = dict(nu=5e-3, eta=5e-3, cs0=1.2, gamma=1.4, cp=1.1, lnrho0=0.1)
    sim = ac.Simulation(n, L=L, layout=layout, precision=precision, **phys)
    try:
        sim.load(_state(n))
        if layout == ac.AC_LAYOUT_PADDED:
            ac.ac_periodic_halo(sim.h)
        stream = torch.cuda.current_stream().cuda_stream
        ptrs = [sim.state[0, q].data_ptr() for q in range(8)]
        grid = ac.make_grid(n, L, layout)
        params = ac.make_params(precision=precision, **phys)
        ops = [ac.AC_MAX, ac.AC_MIN, ac.AC_SUM, ac.AC_RMS]
        quantities = [ac.AC_LNRHO, ac.AC_UY, ac.AC_AZ, ac.AC_Q_UMAG, ac.AC_Q_EKIN, ac.AC_Q_EMAG,
                      ac.AC_Q_CFL]
        for _ in range(2):  # two calls in a row share the fixed scratch array
            for q in quantities:
                for op in ops:
                    ref = ac.ac_reduce(sim.h, op, q)
                    got = ac.ac_reduce_noalloc(ptrs, grid, params, op, q, stream)
                    if op in (ac.AC_MAX, ac.AC_MIN):
                        assert got == ref, (q, op, got, ref)
                    else:
                        scale = abs(ref)
                        if op == ac.AC_SUM:  # bound on sum |q|: cells x max |q|
                            mx = max(abs(ac.ac_reduce(sim.h, ac.AC_MAX, q)),
                                     abs(ac.ac_reduce(sim.h, ac.AC_MIN, q)))
                            scale = mx * float(np.prod(n))
                        assert abs(got - ref) <= 1e-12 * max(scale, 1e-300), (q, op, got, ref)
    finally:
        sim.close()


def test_noalloc_rejects_sizes_beyond_the_fixed_array():
    build.build()
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    ptrs = [buf.data_ptr()] * 8
    grid = ac.make_grid((4, 4, 8193))
    with pytest.raises(ac.AcError) as ei:
        ac.ac_reduce_noalloc(ptrs, grid, ac.make_params(), ac.AC_MAX, ac.AC_UX)
    assert ei.value.code == ac.AC_ERR_ARG
