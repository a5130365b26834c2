"""GPU tests of the batched ensemble (persistent launch over uneven boxes).

Each box of the batch must equal, bitwise, the same box advanced alone by the
single-box binary32 kernel (the batch runs the same tile body on every work
item), whatever the work split (autotuned z extent) and with or without the
CUDA graph; boxes are also checked against the FP64 oracle within the binary32
bound of the single-box tests (f 2e-6, w 2e-4 relative per field).
"""
import json
import math

import numpy as np
import pytest
import torch

from oracle import core
from paper_2103_01597_gb300 import ac, build, synthetic

from gpu_util import rel_err, sample_cells

pytestmark = pytest.mark.gpu

BOXES = [((32, 48, 64), (2 * math.pi,) * 3, 3e-3, 7e-3),
         ((48, 16, 24), (2 * math.pi, 3.0, 4.0), 1e-2, 1e-3),
         ((36, 12, 40), (5.0, 2.0, 6.0), 5e-3, 5e-3),
         ((4, 8, 3), (1.0, 1.0, 1.0), 2e-3, 4e-3)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    ac.load_library()


def _state(n, seed):
    return synthetic.smooth_state(n, seed, amp=0.2) + synthetic.noise_state(n, seed + 50, 1e-3)


def _single(spec, f, dt, steps, precision=ac.AC_FP32):
    n, L, nu, eta = spec
    sim = ac.Simulation(n, L=L, precision=precision, nu=nu, eta=eta)
    sim.load(f)
    for _ in range(steps):
        sim.step(dt)
    out, w = sim.store(), sim.store_w()
    sim.close()
    return out, w


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("precision", [ac.AC_FP32, ac.AC_FP32_W64])
def test_batch_equals_single_boxes_bitwise(graph, precision):
    b = ac.Batch(BOXES, precision=precision)
    states = [_state(spec[0], 10 + i) for i, spec in enumerate(BOXES)]
    for i, f in enumerate(states):
        b.load(i, f)
    ac.ac_batch_set_graph(b.b, graph)
    for _ in range(2):
        b.step(1e-3)
    for i, spec in enumerate(BOXES):
        ref, refw = _single(spec, states[i], 1e-3, 2, precision)
        assert np.array_equal(b.store(i), ref), i
        assert np.array_equal(b.store_w(i), refw), i
    b.close()


def test_tuner_and_work_split_do_not_change_results(tmp_path):
    states = [_state(spec[0], 20 + i) for i, spec in enumerate(BOXES)]
    outs = []
    cache = str(tmp_path / "tune.json")
    for tune in (False, True):
        b = ac.Batch(BOXES)
        for i, f in enumerate(states):
            b.load(i, f)
        if tune:
            zc = ac.ac_batch_tune(b.b, 1e-3, cache)
            assert zc in (8, 16, 32, 64, 128)
            zc1, shapes, ms = ac.ac_batch_get_tiling(b.b, len(BOXES))
            assert zc1 == zc and set(shapes) <= {ac.AC_TILE_32X8, ac.AC_TILE_16X16}
            assert ms[0] > 0 and 0 < ms[1] <= ms[0]  # the default split is a candidate
            cls = {}
            for (n, _, _, _), sh in zip(BOXES, shapes):  # one shape per (nx, ny) class
                assert cls.setdefault(n[:2], sh) == sh
            assert ac.ac_batch_tune(b.b, 1e-3, cache) == zc  # read back from the cache
            assert ac.ac_batch_get_tiling(b.b, len(BOXES))[1] == shapes
            assert ac.ac_batch_info(b.b)["zc"] == zc
            for i, f in enumerate(states):  # tuning leaves the state untouched
                assert np.array_equal(b.store(i), f.astype(np.float32).astype(np.float64))
        b.step(1e-3)
        outs.append([b.store(i) for i in range(len(BOXES))])
        b.close()
    for x, y in zip(*outs):
        assert np.array_equal(x, y)
    with open(cache) as fh:  # the cache is a JSON object
        entries = json.load(fh)
    (entry,) = entries.values()
    assert entry["zc"] == zc and len(entry["tiles"]) == len(BOXES)
    assert [int(c) for c in entry["tiles"]] == shapes


def test_cache_file_of_other_content_is_not_rewritten(tmp_path):
    cache = tmp_path / "other.json"
    cache.write_text('{"something": [1, 2, 3]}\n')
    b = ac.Batch(BOXES[:2])
    ac.ac_batch_tune(b.b, 1e-3, str(cache))
    b.close()
    assert cache.read_text() == '{"something": [1, 2, 3]}\n'


@pytest.mark.parametrize("shapes", [[0, 0, 0, 0], [1, 1, 1, 1], [1, 0, 1, 0], [0, 1, 0, 1]])
@pytest.mark.parametrize("zc", [5, 64])
def test_tile_shapes_bitwise(shapes, zc):
    """Either tile shape, for any box (ragged in x at nx = 36, in y at ny = 12,
    smaller than a tile at (4, 8, 3)), gives the single-box result bitwise."""
    b = ac.Batch(BOXES, precision=ac.AC_FP32_W64)
    states = [_state(spec[0], 40 + i) for i, spec in enumerate(BOXES)]
    for i, f in enumerate(states):
        b.load(i, f)
    ac.ac_batch_set_tiling(b.b, zc, shapes)
    assert ac.ac_batch_get_tiling(b.b, len(BOXES))[:2] == (zc, shapes)
    for s in range(3):
        b.substep(1e-3, s)
    for i, spec in enumerate(BOXES):
        ref, refw = _single(spec, states[i], 1e-3, 1, ac.AC_FP32_W64)
        assert np.array_equal(b.store(i), ref), i
        assert np.array_equal(b.store_w(i), refw), i
    with pytest.raises(ac.AcError):
        ac.ac_batch_set_tiling(b.b, zc, [0, 1, 2, 0])
    b.close()


def test_batch_f32_host_copies():
    """Binary32 host copies of a box move its state unchanged, and a step after
    them equals a step after the binary64 load of the same values."""
    states = [_state(spec[0], 60 + i).astype(np.float32) for i, spec in enumerate(BOXES)]
    res = []
    for f32 in (True, False):
        b = ac.Batch(BOXES)
        for i, f in enumerate(states):
            if f32:
                ac.ac_batch_load_f32(b.b, i, ac.AC_ALL, np.ascontiguousarray(f))
            else:
                b.load(i, f.astype(np.float64))
        if f32:
            for i, f in enumerate(states):
                back = np.empty_like(f)
                ac.ac_batch_store_f32(b.b, i, ac.AC_ALL, back)
                assert np.array_equal(back, f)
                one = np.empty_like(f[2])
                ac.ac_batch_store_f32(b.b, i, 2, one)
                assert np.array_equal(one, f[2])
        b.step(1e-3)
        res.append([b.store(i) for i in range(len(BOXES))])
        b.close()
    for x, y in zip(*res):
        assert np.array_equal(x, y)


def test_batch_boxes_match_oracle():
    b = ac.Batch(BOXES)
    states = [_state(spec[0], 30 + i) for i, spec in enumerate(BOXES)]
    for i, f in enumerate(states):
        b.load(i, f)
    fo = [s.astype(np.float32).astype(np.float64) for s in states]
    wo = [None] * len(BOXES)
    for s in range(3):
        b.substep(1e-3, s)
        for i, (n, L, nu, eta) in enumerate(BOXES):
            p = core.Params(n=n, L=L, nu=nu, eta=eta)
            of, ow = core.substep(fo[i], wo[i], p, 1e-3, s)
            gf, gw = b.store(i), b.store_w(i)
            assert np.all(rel_err(gf, of) <= 2e-6), (i, s, rel_err(gf, of))
            assert np.all(rel_err(gw, ow) <= 2e-4), (i, s, rel_err(gw, ow))
            fo[i], wo[i] = gf, gw
    b.close()


def test_batch_reduce_equals_single():
    b = ac.Batch(BOXES)
    f = _state(BOXES[1][0], 41)
    b.load(1, f)
    n, L, nu, eta = BOXES[1]
    sim = ac.Simulation(n, L=L, precision=ac.AC_FP32, nu=nu, eta=eta)
    sim.load(f)
    for q in (ac.AC_UX, ac.AC_Q_EKIN, ac.AC_Q_EMAG, ac.AC_Q_CFL):
        for op in (ac.AC_MAX, ac.AC_SUM, ac.AC_RMS):
            assert ac.ac_batch_reduce(b.b, 1, op, q) == sim.reduce(op, q)
    sim.close()
    b.close()


def test_batch_argument_errors():
    common = ac.make_params(precision=ac.AC_FP32)
    good = ac.ac_box(8, 8, 8, 1.0, 1.0, 1.0, 1e-3, 1e-3)
    for boxes, params in [([good], ac.make_params(precision=ac.AC_FP64)),
                          ([ac.ac_box(6, 8, 8, 1.0, 1.0, 1.0, 1e-3, 1e-3)], common),
                          ([good] * 129, common),
                          ([good], ac.make_params(precision=ac.AC_FP32, force_amp=0.1))]:
        with pytest.raises(ac.AcError) as ei:
            ac.ac_batch_init(boxes, params)
        assert ei.value.code == ac.AC_ERR_ARG
    b = ac.Batch([((8, 8, 8), (1.0,) * 3, 1e-3, 1e-3)])
    with pytest.raises(ac.AcError) as ei:
        b.substep(1e-3, 2)
    assert ei.value.code == ac.AC_ERR_STATE
    b.close()


def test_ensemble_64_boxes_sampled():
    """The 64-box ensemble (per-axis sizes from {32, 48, 64, 96, 128}, nu and eta
    log-uniform in [1e-3, 1e-2], seed 4), tuned and graph-captured: one step,
    sampled cells of four boxes against the oracle (FP32 bound)."""
    spec = synthetic.ensemble(4)
    boxes = [(n, (2 * math.pi,) * 3, nu, eta) for n, nu, eta in spec]
    b = ac.Batch(boxes)
    states = {}
    for i, (n, _, _, _) in enumerate(boxes):
        f = synthetic.noise_state(n, 100 + i)
        b.load(i, f)
        if i in (0, 17, 40, 63):
            states[i] = f
    ac.ac_batch_tune(b.b, 1e-3)
    ac.ac_batch_set_graph(b.b, True)
    b.step(1e-3)
    for i, f in states.items():
        n, L, nu, eta = boxes[i]
        p = core.Params(n=n, L=L, nu=nu, eta=eta)
        ref = core.step(f.astype(np.float32).astype(np.float64), p, 1e-3)
        got = b.store(i)
        cells = sample_cells(n, 500, seed=i)
        idx = (cells[:, 2], cells[:, 1], cells[:, 0])
        assert np.all(rel_err(np.stack([got[q][idx] for q in range(8)]),
                              np.stack([ref[q][idx] for q in range(8)])) <= 2e-6), i
    info = ac.ac_batch_info(b.b)
    assert info["cells"] == sum(n[0] * n[1] * n[2] for n, _, _, _ in boxes)
    b.close()
