"""Dense-matrix NumPy formulation of the operators and RHS, for tiny grids.

Test infrastructure only.  This is a second, independent writing of the same
definitions as ``ac_oracle.c``: every derivative operator is an explicit
N x N matrix (N = nx ny nz) built from periodic shift matrices with Kronecker
products (x fastest, so the x factor is the last one), and the RHS of
Eqs. B.1-B.4 is assembled from whole-grid vectors.  It shares no code with the
C oracle; the two are compared on grids of 8^3 cells or fewer.
"""
from fractions import Fraction

import numpy as np

NF = 8


def _solve_exact(A, b):
    """Solve the square system A x = b exactly (Fractions, Gauss-Jordan)."""
    n = len(b)
    M = [[Fraction(v) for v in row] + [Fraction(b[i])] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        M[c] = [v / M[c][c] for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                M[r] = [vr - M[r][c] * vc for vr, vc in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


def central_weights(r):
    """Weights of the order-2r central differences from their defining moment
    conditions (Taylor expansion of f(x +- m h)), solved exactly:
      first derivative  sum_m w_m (f_m - f_-m) / h:  2 sum_m w_m m = 1 and
                        sum_m w_m m^k = 0 for odd k = 3 .. 2r-1;
      second derivative sum_m a_m (f_m + f_-m - 2 f_0) / h^2:  sum_m a_m m^2 = 1
                        and sum_m a_m m^k = 0 for even k = 4 .. 2r.
    Returns (w, a) as lists of Fractions indexed by m - 1."""
    ms = range(1, r + 1)
    A1 = [[m ** k for m in ms] for k in range(1, 2 * r, 2)]
    b1 = [Fraction(1, 2)] + [0] * (r - 1)
    A2 = [[m ** k for m in ms] for k in range(2, 2 * r + 1, 2)]
    b2 = [1] + [0] * (r - 1)
    return _solve_exact(A1, b1), _solve_exact(A2, b2)


def _shift(n, m):
    """n x n periodic shift: (T f)_i = f_{(i + m) mod n}."""
    T = np.zeros((n, n))
    for i in range(n):
        T[i, (i + m) % n] = 1.0
    return T


def _axis_op(n3, a, M1):
    """Embed a 1-D operator M1 acting along axis a (0 = x) into the 3-D grid."""
    nx, ny, nz = n3
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    fac = [Ix, Iy, Iz]
    fac[a] = M1
    # vector index = (k * ny + j) * nx + i  ->  kron(Z, kron(Y, X))
    return np.kron(fac[2], np.kron(fac[1], fac[0]))


class Operators:
    """Derivative matrices of order 2r (default: sixth, r = 3) on an
    (nx, ny, nz) periodic grid; the mixed derivative uses the face diagonals,
    sum_m a_m S_m / (4 dx_a dx_b), S_m expanding like 4 m^2 dx_a dx_b d_a d_b
    plus the same higher moments as the axis second difference."""

    def __init__(self, n3, dx3, order=6):
        self.n3 = tuple(n3)
        self.dx = tuple(dx3)
        r = order // 2
        w, aw = central_weights(r)
        c1 = {m: float(w[m - 1]) for m in range(1, r + 1)}
        c2 = {m: float(aw[m - 1]) for m in range(1, r + 1)}
        c0 = float(-2 * sum(aw))
        T = {}
        for a in range(3):
            for m in range(-r, r + 1):
                T[a, m] = _axis_op(self.n3, a, _shift(self.n3[a], m))
        self.T = T
        self.D1 = []
        for a in range(3):
            M = sum(c1[m] * (T[a, m] - T[a, -m]) for m in range(1, r + 1))
            self.D1.append(M / self.dx[a])
        N = T[0, 0].shape[0]
        self.D2 = {}
        for a in range(3):
            M = c0 * np.eye(N) + sum(c2[m] * (T[a, m] + T[a, -m]) for m in range(1, r + 1))
            self.D2[a, a] = M / self.dx[a] ** 2
        for a in range(3):
            for b in range(3):
                if a == b:
                    continue
                M = np.zeros((N, N))
                for m in range(1, r + 1):
                    S = (T[a, m] @ T[b, m] + T[a, -m] @ T[b, -m]
                         - T[a, m] @ T[b, -m] - T[a, -m] @ T[b, m])
                    M += c2[m] * S
                self.D2[a, b] = M / (4.0 * self.dx[a] * self.dx[b])


def rhs(f, p, ops=None):
    """RHS of Eqs. B.1-B.4 with whole-grid vectors; f: (8, nz, ny, nx)."""
    if ops is None:
        ops = Operators(p.n, p.dx, getattr(p, "order", 6))
    shape = f.shape[1:]
    v = [f[q].ravel() for q in range(NF)]
    lnrho, s = v[0], v[4]
    u = v[1:4]
    A = v[5:8]
    g = [[ops.D1[a] @ v[q] for a in range(3)] for q in range(NF)]
    Hu = [[[ops.D2[a, b] @ u[m] for b in range(3)] for a in range(3)] for m in range(3)]
    Ha = [[[ops.D2[a, b] @ A[m] for b in range(3)] for a in range(3)] for m in range(3)]
    rho = np.exp(lnrho)
    cs2 = p.cs0 ** 2 * np.exp(p.gamma * s / p.cp + (p.gamma - 1.0) * (lnrho - p.lnrho0))
    T = cs2 / (p.cp * (p.gamma - 1.0))
    divu = g[1][0] + g[2][1] + g[3][2]
    lapu = [Hu[m][0][0] + Hu[m][1][1] + Hu[m][2][2] for m in range(3)]
    lapa = [Ha[m][0][0] + Ha[m][1][1] + Ha[m][2][2] for m in range(3)]
    gdu = [Hu[0][m][0] + Hu[1][m][1] + Hu[2][m][2] for m in range(3)]
    gda = [Ha[0][m][0] + Ha[1][m][1] + Ha[2][m][2] for m in range(3)]
    gA = g[5:8]
    B = np.array([gA[2][1] - gA[1][2], gA[0][2] - gA[2][0], gA[1][0] - gA[0][1]])
    J = np.array([gda[m] - lapa[m] for m in range(3)])
    U = np.array(u)
    gu = [g[1 + m] for m in range(3)]
    S = [[0.5 * (gu[m][n] + gu[n][m]) - (divu / 3.0 if m == n else 0.0) for n in range(3)]
         for m in range(3)]
    SS2 = sum(S[m][n] ** 2 for m in range(3) for n in range(3))
    JxB = np.cross(J, B, axis=0)
    UxB = np.cross(U, B, axis=0)
    J2 = (J ** 2).sum(axis=0)

    def adv(q):
        return U[0] * g[q][0] + U[1] * g[q][1] + U[2] * g[q][2]

    out = np.empty((NF, v[0].size))
    K = getattr(p, "K", 0.0)
    zeta = getattr(p, "zeta", 0.0)
    heat, cool = getattr(p, "heat", 0.0), getattr(p, "cool", 0.0)
    out[0] = -adv(0) - divu
    force = np.zeros((3, v[0].size))
    if p.forcing is not None:
        nx, ny, nz = p.n
        kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        ph = p.forcing.phi + 2 * np.pi * (p.forcing.k[0] * ii / nx + p.forcing.k[1] * jj / ny
                                          + p.forcing.k[2] * kk / nz)
        for a in range(3):
            force[a] = (p.forcing.amp * p.forcing.e[a] * np.cos(ph)).ravel()
    for m in range(3):
        sgl = S[m][0] * g[0][0] + S[m][1] * g[0][1] + S[m][2] * g[0][2]
        out[1 + m] = (-adv(1 + m) - cs2 * (g[4][m] / p.cp + g[0][m]) + JxB[m] / rho
                      + p.nu * (lapu[m] + gdu[m] / 3.0 + 2.0 * sgl) + zeta * gdu[m] + force[m])
    # conduction div(K grad T) = K T (lap xi + |grad xi|^2), xi = gamma s / c_p + (gamma-1) ln rho
    gxi = [p.gamma / p.cp * g[4][a] + (p.gamma - 1.0) * g[0][a] for a in range(3)]
    lapxi = sum(p.gamma / p.cp * (ops.D2[a, a] @ s) + (p.gamma - 1.0) * (ops.D2[a, a] @ lnrho)
                for a in range(3))
    cond = K * T * (lapxi + sum(x * x for x in gxi))
    out[4] = -adv(4) + (heat - cool + cond + p.eta * J2 + 2.0 * rho * p.nu * SS2
                        + zeta * rho * divu ** 2) / (rho * T)
    for m in range(3):
        out[5 + m] = UxB[m] + p.eta * lapa[m]
    return out.reshape((NF,) + shape)
