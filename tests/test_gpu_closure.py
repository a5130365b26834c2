"""GPU tests of the learned closure (restriction, conv net forward, backward,
Adam, guarded application) against the FP64 oracle, and of what training buys.

The oracle evaluates the net at the precision the configuration fixes
(bfloat16 weights and network input, everything else binary64).  The kernels
also store the hidden activations, the output gradient and the masked input
gradients as bfloat16 MMA operands; the difference that makes is bfloat16
rounding noise, whose spread sigma per element the oracle estimates (Monte
Carlo over random rounding errors at those points, the probabilistic model of
Higham and Mary).  Each tensor must lie within 4 sigma in the L2 norm and 6
sigma in the max norm of the configuration-precision oracle (the oracle's own
kernel-point rounding, a deterministic instance, measures at most 1.7 and 2.8:
test_oracle_closure.py).  As a diagnostic, each tensor is also compared with
the oracle evaluated with bfloat16 at the kernel's rounding points, 2e-2
relative in the max norm (binary32 vs binary64 accumulation).  Restriction:
1e-6 relative (binary32 output of a binary64 sum); Adam 1e-4 of the update.
"""
import math

import numpy as np
import pytest
import torch

from oracle import closure as oc
from oracle import core
from paper_2103_01597_gb300 import ac, build, synthetic
from paper_2103_01597_gb300 import closure as cl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    ac.load_library()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(8, -1)).cuda()


def _rows(t):
    return [t[q].data_ptr() for q in range(8)]


def _maxrel(g, o):
    return float(np.max(np.abs(g - o)) / np.max(np.abs(o)))


def _within_spread(g, o, sigma, what):
    """g against the configuration-precision oracle o, in units of the bfloat16
    rounding spread sigma: L2 ratio <= 4 and max-norm ratio <= 6."""
    d = np.asarray(g, dtype=np.float64) - o
    l2 = float(np.linalg.norm(d) / np.linalg.norm(sigma))
    mx = float(np.max(np.abs(d)) / np.max(sigma))
    print("%s: deviation / rounding spread: L2 %.2f, max %.2f" % (what, l2, mx))
    assert l2 <= 4.0 and mx <= 6.0, (what, l2, mx)


def test_restriction_matches_oracle():
    nf = (16, 12, 20)
    f = synthetic.smooth_state(nf, 3, amp=0.4) + synthetic.noise_state(nf, 4, 1e-2)
    sim = ac.Simulation(nf, precision=ac.AC_FP64)
    sim.load(f)
    nc = (8, 6, 10)
    out = torch.empty((8, 8 * 6 * 10), dtype=torch.float32, device="cuda")
    ptrs, _, _, _ = ac.ac_get_state(sim.h)
    ac.ac_restrict(ptrs, ac.AC_FP64, nf, _rows(out))
    got = out.double().cpu().numpy().reshape(8, nc[2], nc[1], nc[0])
    for q in range(8):
        assert _maxrel(got[q], core.restrict(f[q])) <= 1e-6, q
    sim.close()


def _setup(n, seed):
    net = oc.Net.init(seed)
    params = net.flat().astype(np.float32)
    net = oc.Net.unflat(params.astype(np.float64))  # the binary32 values the GPU holds
    rng = np.random.default_rng(seed)
    x = synthetic.turbulent_state(n, seed, kmax=3, amp=0.5).astype(np.float32).astype(np.float64)
    in_scale = (0.5 + rng.random(8)).astype(np.float32)
    out_scale = (0.01 + 0.1 * rng.random(8)).astype(np.float32)
    return net, params, x, in_scale, out_scale


PATHS = [ac.AC_CONV_TCGEN05, ac.AC_CONV_MMA_SYNC, ac.AC_CONV_TCGEN05_PAIR]


# one x-row tile, ragged tiles, several tiles per row, odd sizes, a single cell;
# nz = 29 and 26 split into z-chunks whose last one overlaps the one before on
# the paired path, (7, 5, 3) and (300, 1, 29) have an odd number of columns
@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n", [(16, 12, 10), (40, 8, 6), (130, 3, 4), (300, 2, 3), (7, 5, 3),
                               (1, 1, 1), (24, 6, 29), (300, 1, 29), (129, 3, 26)])
def test_forward_matches_oracle(n, path):
    net, params, x, ins, outs = _setup(n, 5)
    c = cl.Closure(n, params=params, conv_path=path)
    c.set_scales(ins, outs)
    got = c.correction(_dev(x)).double().cpu().numpy().reshape((8,) + x.shape[1:])
    c.status()
    xn = x / ins.astype(np.float64)[:, None, None, None]
    sc = outs.astype(np.float64)[:, None, None, None]
    y, _ = net.forward(xn, bf16="config")
    _within_spread(got, y * sc, net.rounding_spread(xn) * sc, "forward %s" % (n,))
    yk, _ = net.forward(xn, bf16="kernel")  # diagnostic: the kernel's rounding points
    assert _maxrel(got, yk * sc) <= 2e-2, _maxrel(got, yk * sc)
    c.close()


def _patch(x, z, y, xi, r):
    """The (8, 2r+1, 2r+1, 2r+1) periodic neighbourhood of cell (z, y, xi)."""
    nz, ny, nx = x.shape[1:]
    iz = np.arange(z - r, z + r + 1) % nz
    iy = np.arange(y - r, y + r + 1) % ny
    ix = np.arange(xi - r, xi + r + 1) % nx
    return x[:, iz][:, :, iy][:, :, :, ix]


@pytest.mark.parametrize("n", [(128, 128, 128), (256, 256, 256)])
def test_forward_sampled_at_full_size(n):
    """The inference sizes (the 128^3 coarse grid of the closure workload, the
    256^3 inference workload) on the default path, in the bench's launch
    configuration: 48 sampled cells against the oracle.  A cell's output depends
    on its 7^3 neighbourhood (three 3x3x3 layers), so the oracle evaluates each
    on a 9^3 periodic patch around it (the patch's own wrap reaches the centre
    after no fewer than four layers)."""
    net = oc.Net.init(11)
    params = net.flat().astype(np.float32)
    net = oc.Net.unflat(params.astype(np.float64))
    x = synthetic.noise_state(n, 12, 0.5).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(13)
    ins = (0.5 + rng.random(8)).astype(np.float32)
    outs = (0.01 + 0.1 * rng.random(8)).astype(np.float32)
    c = cl.Closure(n, params=params)
    c.set_scales(ins, outs)
    got = c.correction(_dev(x)).double().cpu().numpy().reshape((8,) + x.shape[1:])
    c.status()
    c.close()
    isc = ins.astype(np.float64)[:, None, None, None]
    sc = outs.astype(np.float64)
    cells = [(int(rng.integers(n[2])), int(rng.integers(n[1])), int(rng.integers(n[0])))
             for _ in range(48)]
    g, want, sig, wk = [], [], [], []
    for (z, y, xi) in cells:
        p = _patch(x, z, y, xi, 4) / isc
        yo, _ = net.forward(p, bf16="config")
        yk, _ = net.forward(p, bf16="kernel")
        sp = net.rounding_spread(p, samples=8)
        g.append(got[:, z, y, xi])
        want.append(yo[:, 4, 4, 4] * sc)
        wk.append(yk[:, 4, 4, 4] * sc)
        sig.append(sp[:, 4, 4, 4] * sc)
    g, want, sig, wk = map(np.array, (g, want, sig, wk))
    _within_spread(g, want, sig, "forward %s, 48 sampled cells" % (n,))
    assert _maxrel(g, wk) <= 2e-2, _maxrel(g, wk)


def test_forward_paths_agree_at_64_cubed():
    """The tcgen05 (one CTA and paired) and mma.sync forward passes on a 64^3
    grid (4 096 tiles of a row each on the persistent grids): same bfloat16
    operands, different accumulation order, so agreement to bfloat16 rounding
    of the hidden activations."""
    n = (64, 64, 64)
    net, params, x, ins, outs = _setup(n, 9)
    xs = _dev(x)
    outs_ = []
    for path in PATHS:
        c = cl.Closure(n, params=params, conv_path=path)
        c.set_scales(ins, outs)
        outs_.append(c.correction(xs).double().cpu().numpy())
        c.status()
        c.close()
    for o in outs_[1:]:
        assert _maxrel(outs_[0], o) <= 1e-2, _maxrel(outs_[0], o)
    # every cell against the oracle
    xn = x / ins.astype(np.float64)[:, None, None, None]
    y, _ = net.forward(xn, bf16="kernel")  # diagnostic: the kernel's rounding points
    ref = (y * outs.astype(np.float64)[:, None, None, None]).reshape(8, -1)
    assert _maxrel(outs_[0], ref) <= 2e-2, _maxrel(outs_[0], ref)


def test_conv_path_selection():
    c = cl.Closure((8, 8, 8))
    assert ac.ac_closure_get_conv_path(c.c) == ac.AC_CONV_TCGEN05
    ac.ac_closure_set_conv_path(c.c, ac.AC_CONV_MMA_SYNC)
    assert ac.ac_closure_get_conv_path(c.c) == ac.AC_CONV_MMA_SYNC
    ac.ac_closure_set_conv_path(c.c, ac.AC_CONV_TCGEN05_PAIR)
    assert ac.ac_closure_get_conv_path(c.c) == ac.AC_CONV_TCGEN05_PAIR
    with pytest.raises(ac.AcError):
        ac.ac_closure_set_conv_path(c.c, 7)
    c.close()


# all paths on one ragged x-tile (16 cells: one K-step of the weight gradient);
# the tcgen05 backward also on two x-segments (the second 8 cells), several rows
# and two z-chunks, and on a partial K-step (nx = 20) with three z-chunks, the
# last of one tile
GRAD_CASES = [(p, (16, 12, 10)) for p in PATHS] + [
    (ac.AC_CONV_TCGEN05, (136, 9, 18)),
    (ac.AC_CONV_TCGEN05_PAIR, (136, 9, 18)),
    (ac.AC_CONV_TCGEN05, (20, 7, 33)),
]


@pytest.mark.parametrize("path,n", GRAD_CASES)
def test_gradients_and_adam_match_oracle(path, n):
    net, params, x, ins, outs = _setup(n, 6)
    rng = np.random.default_rng(7)
    tgt = (outs.astype(np.float64)[:, None, None, None]
           * rng.standard_normal(x.shape)).astype(np.float32).astype(np.float64)
    c = cl.Closure(n, params=params, conv_path=path)
    c.set_scales(ins, outs)
    loss = c.loss(_dev(x), _dev(tgt))
    g = ac.ac_closure_get_grads(c.c).astype(np.float64)
    xn = x / ins.astype(np.float64)[:, None, None, None]
    tn = tgt / outs.astype(np.float64)[:, None, None, None]
    lo, go = net.loss_and_grads(xn, tn, bf16="config")
    assert abs(loss - lo) <= 1e-3 * lo, (loss, lo)
    spread = net.rounding_spread(xn, tn)
    _, gk = net.loss_and_grads(xn, tn, bf16="kernel")  # diagnostic
    off = 0
    for li in range(3):
        for a in range(2):
            sz = go[li][a].size
            gg = g[off:off + sz]
            _within_spread(gg, go[li][a].ravel(), spread[li][a].ravel(),
                           "gradient layer %d %s" % (li + 1, "Wb"[a]))
            err = _maxrel(gg, gk[li][a].ravel())
            assert err <= 2e-2, (li, a, err)
            off += sz
    # one Adam step on the GPU's own gradients
    ac.ac_closure_adam_step(c.c, 1e-3)
    new = ac.ac_closure_get_params(c.c).astype(np.float64)
    ad = oc.Adam([params.shape], lr=1e-3)
    ref = ad.step([params.astype(np.float64)], [g])[0]
    upd_g = new - params.astype(np.float64)
    upd_o = ref - params.astype(np.float64)
    assert np.max(np.abs(upd_g - upd_o)) <= 1e-4 * np.max(np.abs(upd_o))
    c.close()


@pytest.mark.parametrize("path", PATHS)
def test_apply_guard(path):
    n = (16, 8, 12)
    net, params, x, ins, outs = _setup(n, 8)
    sim = ac.Simulation(n, precision=ac.AC_FP32)
    sim.load(x)
    before = cl.current_state(sim).clone()
    c = cl.Closure(n, params=params, conv_path=path)
    c.set_scales(ins, outs)
    corr = c.correction(before.clone()).clone()
    assert not c.apply(sim, limit=1e-9)  # larger than the limit: left unchanged
    assert torch.equal(cl.current_state(sim), before)
    assert c.apply(sim, limit=1e3)
    after = cl.current_state(sim)
    assert torch.allclose(after, before + corr, rtol=0, atol=1e-6)
    sim.close()
    c.close()


def test_training_reduces_coarse_error():
    """Fine 32^3 binary64 run restricted to 16^3: the trained closure predicts
    the coarse step's defect on held-out pairs far better than zero (what the
    plain coarse step without closure implies)."""
    nf = (32, 32, 32)
    f0 = synthetic.turbulent_state(nf, 21, kmax=6, amp=0.4)
    pairs = cl.make_pairs(f0, nf, 48, 2e-3, seed=3, force_amp=0.05)
    train, held = pairs[:40], pairs[40:]
    ins = cl.channel_rms([p[0] for p in train])
    outs = cl.channel_rms([p[1] for p in train])
    c = cl.Closure((16, 16, 16), seed=1)
    c.set_scales(ins, outs)
    base = np.mean([c.loss(x, t) for x, t in held])
    for it in range(600):
        x, t = train[it % len(train)]
        c.train_step(x, t, lr=2e-3 if it < 400 else 5e-4)
    after = np.mean([c.loss(x, t) for x, t in held])
    # relative defect left after the correction vs the defect itself
    rel = []
    for x, t in held:
        corr = c.correction(x)
        rel.append(float(torch.linalg.vector_norm(t - corr) / torch.linalg.vector_norm(t)))
    print("closure: held-out loss %.3e -> %.3e, relative defect %.3f" % (base, after,
                                                                         float(np.mean(rel))))
    assert after < 0.5 * base
    assert np.mean(rel) < 0.75
    c.close()
