"""Runs every checked kernel path of the library built with AC_BOUNDS_CHECK
(libac_bc.so) on small and ragged grids and prints, as one JSON object, the
first recorded out-of-range index word of each group (0: none) and the
self-test of the checks.  Used by tests/test_gpu_bounds.py in a process of its
own (the checked library replaces the normal one for the whole process)."""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2103_01597_gb300 import ac, build, closure as cl, synthetic  # noqa: E402

ac.load_library(path=build.build(bounds_check=True))
torch.cuda.init()
out = {}


def take(name):
    rc, w = ac.ac_bounds_check_take()
    assert rc == ac.AC_OK, rc
    out[name] = w


def state(n, seed):
    return synthetic.smooth_state(n, seed, amp=0.2) + synthetic.noise_state(n, seed + 7, 1e-3)


def run_sim(n, steps=1, **kw):
    mode = kw.pop("mode", None)
    sim = ac.Simulation(n, **kw)
    if mode is not None:
        ac.ac_set_stencil_mode(sim.h, mode)
    sim.load(state(n, sum(n)))
    for _ in range(steps):
        sim.step(1e-3)
    for q in (ac.AC_LNRHO, ac.AC_UX, ac.AC_AZ, ac.AC_Q_UMAG, ac.AC_Q_EKIN, ac.AC_Q_EMAG,
              ac.AC_Q_CFL):
        for op in (ac.AC_MAX, ac.AC_SUM, ac.AC_RMS):
            sim.reduce(op, q)
    assert np.all(np.isfinite(sim.store()))
    sim.close()


SIZES = [(16, 16, 16), (37, 21, 13), (5, 3, 7), (1, 12, 10), (33, 9, 4)]
TERMS = dict(K=0.02, zeta=0.01, heat=0.3, cool=0.1)
cube = [(16, 16, 16), (24, 24, 24), (9, 9, 9)]

# binary64 on integer sums (cubic periodic grids, equal spacing), with and without the full entropy terms
for n in cube:
    run_sim(n, steps=2, precision=ac.AC_FP64, mode=ac.AC_STENCIL_FIXED)
    run_sim(n, precision=ac.AC_FP64, mode=ac.AC_STENCIL_FIXED, **TERMS)
take("fp64_integer_sums")
# plain binary64: unequal spacings, both layouts, every order (8: periodic only)
for n in SIZES:
    for layout in (ac.AC_LAYOUT_PERIODIC, ac.AC_LAYOUT_PADDED):
        run_sim(n, L=(2 * math.pi, 3.0, 5.5), layout=layout, precision=ac.AC_FP64)
    for order in (2, 4, 8):
        run_sim(n, precision=ac.AC_FP64, order=order)
run_sim((16, 12, 10), L=(2 * math.pi, 3.0, 5.5), precision=ac.AC_FP64, **TERMS)
take("fp64_plain")
# binary32 and binary32 with a binary64 accumulator: tiled (order 6) and direct kernels
for prec in (ac.AC_FP32, ac.AC_FP32_W64):
    for n in SIZES + [(64, 40, 12)]:
        run_sim(n, steps=2, precision=prec)
        run_sim(n, precision=prec, layout=ac.AC_LAYOUT_PADDED)
        for order in (2, 4, 8):
            run_sim(n, precision=prec, order=order)
    run_sim((20, 16, 12), precision=prec, **TERMS)
take("fp32")
# batched ensemble of uneven boxes
boxes = [((32, 48, 64), (2 * math.pi,) * 3, 3e-3, 7e-3), ((48, 16, 24), (2 * math.pi, 3.0, 4.0), 1e-2, 1e-3),
         ((36, 12, 40), (5.0, 2.0, 6.0), 5e-3, 5e-3), ((4, 8, 3), (1.0, 1.0, 1.0), 2e-3, 4e-3)]
for prec in (ac.AC_FP32, ac.AC_FP32_W64):
    b = ac.Batch(boxes, precision=prec)
    for i, spec in enumerate(boxes):
        b.load(i, state(spec[0], 40 + i))
    for _ in range(2):
        b.step(1e-3)
    b.close()
take("batch")
# closure convolutions on all three paths
for n in [(130, 3, 4), (7, 5, 3), (40, 8, 29), (300, 1, 29), (1, 1, 1)]:
    x = torch.from_numpy(synthetic.turbulent_state(n, 3, kmax=3, amp=0.5).astype(np.float32)).cuda()
    for path in (ac.AC_CONV_TCGEN05, ac.AC_CONV_TCGEN05_PAIR, ac.AC_CONV_MMA_SYNC):
        c = cl.Closure(n, seed=1, conv_path=path)
        y = c.correction(x)
        assert torch.isfinite(y).all()
        c.status()
        c.close()
take("closure")
rc, vals = ac.ac_bounds_check_selftest()
out["selftest_status"] = rc
out["selftest_values"] = vals
rc, w = ac.ac_bounds_check_take()
out["selftest_word"] = w
print(json.dumps(out))
