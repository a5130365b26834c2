"""Handles on separate streams keep separate state.

Two handles stepping at once on two streams (their kernels free to overlap on
the GPU, or ordered by events as the end-to-end loop orders them) give bitwise
the result of one handle stepping alone: no work area, plan, forcing table or
CFL slot is shared between handles.  Covered for the integer-sum binary64 path
(per-substep extremes, plan and int64 copies), the binary32 tiled kernel and
the ensemble kernel.
"""
import numpy as np
import pytest
import torch

from paper_2103_01597_gb300 import ac, build, synthetic

pytestmark = pytest.mark.gpu

N = (40, 40, 40)  # cubic, equal spacing: the integer-sum path applies
STEPS = 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    ac.load_library()
    torch.cuda.init()


def _state(seed):
    f = synthetic.smooth_state(N, seed, amp=0.2) + synthetic.noise_state(N, seed + 1, 1e-3)
    return np.ascontiguousarray(f)


def _alone(precision, f, dt):
    sim = ac.Simulation(N, precision=precision, force_amp=0.05, seed=11)
    sim.load(f)
    if precision == ac.AC_FP64:
        assert ac.ac_get_stencil_path(sim.h)  # the integer-sum path
    cfl = []
    for _ in range(STEPS):
        sim.step(dt)
        cfl.append(ac.ac_last_cfl(sim.h))
    out = sim.store()
    sim.close()
    return out, cfl


@pytest.mark.parametrize("precision", [ac.AC_FP64, ac.AC_FP32])
@pytest.mark.parametrize("ordered", [False, True])
def test_two_handles_on_two_streams_bitwise(precision, ordered):
    dt = 1e-3
    fa, fb = _state(3), _state(5)
    ref_a, cfl_a = _alone(precision, fa, dt)
    ref_b, cfl_b = _alone(precision, fb, dt)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    sims = [ac.Simulation(N, precision=precision, force_amp=0.05, seed=11,
                          stream=s.cuda_stream) for s in streams]
    sims[0].load(fa)
    sims[1].load(fb)
    torch.cuda.synchronize()
    done = [torch.cuda.Event(), torch.cuda.Event()]
    cfl = [[], []]
    for _ in range(STEPS):
        for k in range(2):
            if ordered:
                streams[k].wait_event(done[1 - k])
            ac.ac_integrate_step(sims[k].h, dt)
            done[k].record(streams[k])
        for k in range(2):
            cfl[k].append(ac.ac_last_cfl(sims[k].h))
    outs = [s.store() for s in sims]
    for s in sims:
        s.close()
    assert np.array_equal(outs[0], ref_a)
    assert np.array_equal(outs[1], ref_b)
    assert cfl[0] == cfl_a and cfl[1] == cfl_b


def test_two_ensembles_on_two_streams_bitwise():
    spec = synthetic.ensemble(4)[:6]
    boxes = [(n, (2 * np.pi,) * 3, nu, eta) for n, nu, eta in spec]
    states = [[synthetic.noise_state(n, 100 * r + i) for i, (n, _, _, _) in enumerate(boxes)]
              for r in range(2)]
    dt = 1e-3

    def run(batches):
        for r, b in enumerate(batches):
            for i, f in enumerate(states[r]):
                b.load(i, f)
        torch.cuda.synchronize()
        for _ in range(STEPS):
            for b in batches:
                b.step(dt)
        return [[b.store(i) for i in range(len(boxes))] for b in batches]

    alone = []
    for r in range(2):
        b = ac.Batch(boxes)
        for i, f in enumerate(states[r]):
            b.load(i, f)
        for _ in range(STEPS):
            b.step(dt)
        alone.append([b.store(i) for i in range(len(boxes))])
        b.close()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    batches = [ac.Batch(boxes, stream=s.cuda_stream) for s in streams]
    together = run(batches)
    for b in batches:
        b.close()
    for r in range(2):
        for i in range(len(boxes)):
            assert np.array_equal(together[r][i], alone[r][i]), (r, i)
