"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_err(g, o):
    """Per-field max-norm relative error max|g - o| / max|o| (absolute when o == 0)."""
    out = []
    for q in range(g.shape[0]):
        den = np.max(np.abs(o[q]))
        num = np.max(np.abs(g[q] - o[q]))
        out.append(num / den if den > 0 else num)
    return np.array(out)


def ulp_err(g, o):
    """The paper's error metric (Sec. 5, Eqs. 14-15): |m - c| / 2^(floor(log2|m|) - 52)
    for binary64 model values m != 0."""
    m = np.asarray(o, dtype=np.float64)
    c = np.asarray(g, dtype=np.float64)
    nz = m != 0
    eps = np.ldexp(1.0, (np.floor(np.log2(np.abs(m[nz]))) - 52).astype(int))
    return np.abs(m[nz] - c[nz]) / eps


def sample_cells(n, count, seed):
    """Random cells plus every corner and face-adjacent boundary cell pattern."""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    cells = [rng.integers(0, nx, count), rng.integers(0, ny, count), rng.integers(0, nz, count)]
    cells = np.stack(cells, axis=1)
    edge = []
    for i in (0, 1, 2, nx - 3, nx - 2, nx - 1):
        for j in (0, 2, ny - 1):
            for k in (0, 1, nz - 2, nz - 1):
                edge.append((i % nx, j % ny, k % nz))
    return np.concatenate([cells, np.array(edge)], axis=0).astype(np.int64)
