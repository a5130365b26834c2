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
                       nu, eta log-uniform in [1e-3, 1e-2];
  * ``turbulent_state``: random-phase modes up to |k| = kmax with a power-law
                       spectrum (learned-closure training data).
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


def turbulent_state(n, seed, kmax=6, amp=0.3, slope=-5.0 / 3.0):
    """Random-phase Fourier modes with 1 <= |k| <= kmax, mode amplitudes
    ~ |k|^(slope / 2 - 1) (a shell energy spectrum ~ k^slope).  u has rms `amp`;
    A is drawn with an extra 1/|k| so that B = curl A (evaluated spectrally
    here, for the normalisation only) has rms `amp`; ln rho and s have rms
    amp / 4.  Used for the learned-closure data: energy up to the scales the
    coarse grid resolves, signal speeds O(1)."""
    nx, ny, nz = n
    g = _rng(seed)
    kx = np.fft.fftfreq(nx, 1.0 / nx)
    ky = np.fft.fftfreq(ny, 1.0 / ny)
    kz = np.fft.fftfreq(nz, 1.0 / nz)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    shell = (kk >= 1) & (kk <= kmax)
    weight = np.where(shell, np.maximum(kk, 1.0) ** (slope / 2 - 1.0), 0.0)
    f = np.zeros((NFIELDS, nz, ny, nx))
    spectra = {}
    for q in range(NFIELDS):
        spec = weight * np.exp(2j * np.pi * g.random(kk.shape)) * g.normal(1.0, 0.3, kk.shape)
        if q >= 5:
            spec = spec / np.maximum(kk, 1.0)
        spectra[q] = spec
        field = np.real(np.fft.ifftn(spec))
        if q < 5:
            rms = np.sqrt(np.mean(field ** 2))
            a = amp if q in (1, 2, 3) else amp / 4
            f[q] = field * (a / rms if rms > 0 else 0.0)
        else:
            f[q] = field
    Ah = [np.fft.fftn(f[5 + a]) for a in range(3)]
    B = [np.real(np.fft.ifftn(1j * (KY * Ah[2] - KZ * Ah[1]))),
         np.real(np.fft.ifftn(1j * (KZ * Ah[0] - KX * Ah[2]))),
         np.real(np.fft.ifftn(1j * (KX * Ah[1] - KY * Ah[0])))]
    brms = np.sqrt(np.mean(B[0] ** 2 + B[1] ** 2 + B[2] ** 2) / 3)
    if brms > 0:
        f[5:8] *= amp / brms
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
