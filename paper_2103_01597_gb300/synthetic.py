"""Seeded synthetic inputs for the MHD substep (NumPy PCG64, FP64 on the host).

This module holds none of the method's arithmetic: it only draws initial
states and ensemble parameters.  The same bytes feed the CUDA path (through
``ac_load``) and the CPU oracle.  States are float64 arrays of shape
(8, nz, ny, nx), fields ordered as Table B.1 (ln rho, u_x, u_y, u_z, s, A_x,
A_y, A_z), x fastest.

Recipes:
  * ``noise_state``:   ln rho = s = 0, u and A i.i.d. Gaussian N(0, sigma^2)
                       (sigma = 1e-5 unless given), per cell and component;
  * ``uniform_state``: every field i.i.d. uniform in [0, 1) -- the paper's own
                       benchmark initial condition (Sec. 5);
  * ``ensemble``:      box sizes drawn per axis from {32, 48, 64, 96, 128} and
                       nu, eta log-uniform in [1e-3, 1e-2].
"""
import numpy as np

NFIELDS = 8


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def noise_state(n, seed, sigma=1e-5):
    nx, ny, nz = n
    g = _rng(seed)
    f = np.zeros((NFIELDS, nz, ny, nx))
    for q in (1, 2, 3, 5, 6, 7):
        f[q] = g.normal(0.0, sigma, size=(nz, ny, nx))
    return f


def uniform_state(n, seed):
    nx, ny, nz = n
    g = _rng(seed)
    return g.random(size=(NFIELDS, nz, ny, nx))


def smooth_state(n, seed, amp=0.1):
    """A smooth random state: a few low Fourier modes per field (test use)."""
    nx, ny, nz = n
    g = _rng(seed)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = np.zeros((NFIELDS, nz, ny, nx))
    for q in range(NFIELDS):
        for _ in range(3):
            m = g.integers(-2, 3, size=3)
            ph = g.random() * 2 * np.pi
            a = amp * g.random()
            f[q] += a * np.cos(2 * np.pi * (m[0] * i / nx + m[1] * j / ny + m[2] * k / nz) + ph)
    return f


def ensemble(seed, count=64, sizes=(32, 48, 64, 96, 128), lo=1e-3, hi=1e-2):
    """List of (n, nu, eta) for a batched ensemble: n per axis from `sizes`."""
    g = _rng(seed)
    out = []
    for _ in range(count):
        n = tuple(int(sizes[g.integers(0, len(sizes))]) for _ in range(3))
        nu = float(np.exp(g.uniform(np.log(lo), np.log(hi))))
        eta = float(np.exp(g.uniform(np.log(lo), np.log(hi))))
        out.append((n, nu, eta))
    return out
