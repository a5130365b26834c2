"""The table-driven binary64 exp of the binary64 substep kernels (Tang's method,
256-entry table) against CUDA's exp on the device and against the host's exp,
through `ac_diag_exp_table`: within one unit in the last place of CUDA's exp on
|x| < 700, the paired exp(x) equal to the single one and exp(-x) within two
units of the host's, and CUDA's exp itself wherever the table does not apply
(|x| >= 700, infinities, NaN)."""
import numpy as np
import pytest
import torch

from paper_2103_01597_gb300 import ac

pytestmark = pytest.mark.gpu


def _run(x):
    xd = torch.from_numpy(x).cuda()
    y = torch.empty(4 * x.size, dtype=torch.float64, device="cuda")
    assert ac.ac_diag_exp_table(xd, y) == ac.AC_OK
    return y.cpu().numpy().reshape(4, x.size)


def _ulps(a, b):
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def test_table_exp_against_cuda_and_host():
    rng = np.random.default_rng(11)
    x = np.concatenate([
        rng.uniform(-700, 700, 1 << 20),
        rng.uniform(-40, 40, 1 << 20),
        rng.uniform(-1e-3, 1e-3, 1 << 16),                 # near 0: reduction with N = 0
        np.arange(-300, 301) * (np.log(2) / 256),         # on and next to reduction nodes
        np.nextafter(np.arange(-300, 301) * (np.log(2) / 256), np.inf),
        np.array([0.0, -0.0, 1.0, -1.0, 699.999, -699.999]),
    ])
    y = _run(x)
    tab, cuda, pair_p, pair_m = y
    assert _ulps(tab, cuda).max() <= 1
    assert np.array_equal(pair_p, tab)
    # the host's exp is itself within an ulp of the exact value
    host_p, host_m = np.exp(x), np.exp(-x)
    assert _ulps(tab, host_p).max() <= 2
    assert _ulps(pair_m, host_m).max() <= 2
    assert np.all(tab[x == 0.0] == 1.0) and np.all(pair_m[x == 0.0] == 1.0)


def test_fallback_outside_the_table_range():
    x = np.array([700.0, -700.0, 705.5, -705.5, 709.7, 710.0, -745.0, -800.0,
                  np.inf, -np.inf, np.nan])
    tab, cuda, pair_p, pair_m = _run(x)
    with np.errstate(over="ignore"):
        host_m = np.exp(-x)  # the fallback's exp(-x) is CUDA's; compare with the host's by class
    for i, v in enumerate(x):
        if np.isnan(v):
            assert np.isnan(tab[i]) and np.isnan(pair_p[i]) and np.isnan(pair_m[i])
            continue
        assert tab[i] == cuda[i] and pair_p[i] == cuda[i]
        assert (pair_m[i] == 0.0) == (host_m[i] == 0.0)
        assert np.isinf(pair_m[i]) == np.isinf(host_m[i])
