/*
 * ac_oracle.c -- plain, slow FP64 CPU oracle of one third-order Runge-Kutta
 * substep of compressible non-ideal MHD on a periodic grid (Pekkila et al.,
 * "Scalable communication for high-order stencil computations using
 * CUDA-aware MPI", arXiv:2103.01597).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path and must never be used by it.
 *
 * Everything here is written for a reader checking it against the paper:
 *   - the stencil point set is Sec. 4, Eq. 13 (axes and face diagonals,
 *     radius r = 3, i.e. sixth order, Sec. 4); radii 1, 2 and 4 (orders 2, 4,
 *     8) use the same kind of point set (a widening beyond the paper);
 *   - the equations are Appendix B, Eqs. B.1-B.4 with the symbols of
 *     Tables B.1 and B.2;
 *   - time integration is the third-order 2N-storage Runge-Kutta scheme of
 *     Williamson (1980) that Sec. 4 names;
 *   - the periodic halo map is the one of Sec. 3.3: s' = ((s - r) mod n) + r.
 * Readings of what the paper leaves unstated (coefficients, constants,
 * forcing) are listed in the design notes of the repository; each is marked
 * "reading" below.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math), so
 * every operation is a separately rounded IEEE binary64 operation.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Field order, Table B.1: ln rho, u (3), s, A (3). */
enum { LNRHO = 0, UX = 1, UY = 2, UZ = 3, SS = 4, AX = 5, AY = 6, AZ = 7, NFIELDS = 8 };

/* All members are 8 bytes wide so the Python side can mirror this layout
 * without padding rules. */
typedef struct {
    int64_t n[3];          /* cells per axis (computational domain N, Sec. 2) */
    double dx[3];          /* grid spacing per axis                            */
    double nu, eta;        /* kinematic viscosity, magnetic diffusivity       */
    double cs0, gamma, cp; /* reference sound speed, adiabatic index, c_p     */
    double lnrho0;         /* reference log density                            */
    int64_t force_on;      /* 1: add the forcing term to du/dt                 */
    double force_amp;      /* forcing amplitude f0                             */
    int64_t force_k[3];    /* integer wave vector of this step's forcing      */
    double force_e[3];     /* unit polarisation vector, perpendicular to k    */
    double force_phi;      /* phase of this step's forcing                     */
    int64_t radius;        /* stencil radius r (order 2r): 1, 2, 3 or 4       */
    double K;              /* radiative thermal conductivity (constant)        */
    double zeta;           /* bulk viscosity (kinematic, as in Eq. B.2)        */
    double heat, cool;     /* explicit heating H and cooling C (uniform rates) */
} oracle_params;

/* ------------------------------------------------------------------------ */
/* Grid access with the periodic map of Sec. 3.3.                             */
/* ------------------------------------------------------------------------ */

static int64_t wrap(int64_t i, int64_t n)
{
    int64_t m = i % n;
    return m < 0 ? m + n : m;
}

/* Value of field f at cell (i, j, k) + offset, x fastest. */
static double at(const double *f, const oracle_params *p,
                 int64_t i, int64_t j, int64_t k)
{
    int64_t ii = wrap(i, p->n[0]);
    int64_t jj = wrap(j, p->n[1]);
    int64_t kk = wrap(k, p->n[2]);
    return f[(kk * p->n[1] + jj) * p->n[0] + ii];
}

/* Value of f at c + m * e_a (one step of m cells along axis a). */
static double axis_pt(const double *f, const oracle_params *p, const int64_t c[3],
                      int a, int64_t m)
{
    int64_t q[3] = {c[0], c[1], c[2]};
    q[a] += m;
    return at(f, p, q[0], q[1], q[2]);
}

/* Value of f at c + m_a e_a + m_b e_b (a face-diagonal point of Eq. 13). */
static double diag_pt(const double *f, const oracle_params *p, const int64_t c[3],
                      int a, int64_t ma, int b, int64_t mb)
{
    int64_t q[3] = {c[0], c[1], c[2]};
    q[a] += ma;
    q[b] += mb;
    return at(f, p, q[0], q[1], q[2]);
}

/* ------------------------------------------------------------------------ */
/* Central differences of order 2r on the point set of Eq. 13 (r = 3: sixth   */
/* order, Sec. 4).  Reading: the paper prints no coefficients; these are the */
/* standard central ones, the unique weights on the points 0, +-1 .. +-r     */
/* exact for polynomials of degree 2r (first derivative) and 2r + 1 (second  */
/* derivative).  Closed form (Fornberg 1988), with w_m on (f_m - f_-m) and   */
/* a_m on (f_m + f_-m):                                                      */
/*   w_m = (-1)^(m+1) (r!)^2 / (m (r-m)! (r+m)!),   a_m = 2 w_m / m,         */
/*   a_0 = -2 (a_1 + ... + a_r).                                             */
/* For r = 3: w = (3/4, -3/20, 1/60) = (45, -9, 1)/60 and                    */
/* a = (3/2, -3/20, 1/90), a_0 = -49/18.                                     */
/* ------------------------------------------------------------------------ */

static double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i)
        f *= i; /* exact: k <= 8 */
    return f;
}

/* w_m of the first derivative (one rounding: numerator and denominator are
 * exact integers). */
static double w_first(int r, int m)
{
    double num = factorial(r) * factorial(r);
    double den = (double)m * factorial(r - m) * factorial(r + m);
    return (m % 2 ? num : -num) / den;
}

/* a_m (m >= 1) of the second derivative. */
static double w_second(int r, int m)
{
    double num = 2.0 * factorial(r) * factorial(r);
    double den = (double)m * (double)m * factorial(r - m) * factorial(r + m);
    return (m % 2 ? num : -num) / den;
}

/* First derivative along axis a: sum_m w_m (f_m - f_-m) / dx_a. */
static double d1(const double *f, const oracle_params *p, const int64_t c[3], int a)
{
    const int r = (int)p->radius;
    double sum = 0.0;
    for (int m = 1; m <= r; ++m)
        sum += w_first(r, m) * (axis_pt(f, p, c, a, m) - axis_pt(f, p, c, a, -m));
    return sum / p->dx[a];
}

/* Second derivative along axis a: [a_0 f_0 + sum_m a_m (f_m + f_-m)] / dx_a^2. */
static double d2(const double *f, const oracle_params *p, const int64_t c[3], int a)
{
    const int r = (int)p->radius;
    double a0 = 0.0, sum = 0.0;
    for (int m = 1; m <= r; ++m) {
        a0 -= 2.0 * w_second(r, m);
        sum += w_second(r, m) * (axis_pt(f, p, c, a, m) + axis_pt(f, p, c, a, -m));
    }
    return (a0 * axis_pt(f, p, c, a, 0) + sum) / (p->dx[a] * p->dx[a]);
}

/* Mixed derivative d^2 f / (dx_a dx_b), a != b, from the face diagonals only
 * (Eq. 13 holds no other off-axis points):
 *   sum_m a_m S_m / (4 dx_a dx_b),
 *   S_m = f(+m,+m) + f(-m,-m) - f(+m,-m) - f(-m,+m) in the (a, b) plane.
 * Along the two diagonals S_m = 2 sum_k m^2k / (2k)! (D+^2k - D-^2k) f with
 * D+- = dx_a d_a +- dx_b d_b, and D+^2 - D-^2 = 4 dx_a dx_b d_a d_b: the same
 * moment conditions as the second derivative, hence the weights a_m
 * (r = 3: [270 S_1 - 27 S_2 + 2 S_3] / (720 dx_a dx_b)). */
static double dab(const double *f, const oracle_params *p, const int64_t c[3], int a, int b)
{
    const int r = (int)p->radius;
    double sum = 0.0;
    for (int64_t m = 1; m <= r; ++m) {
        double S = diag_pt(f, p, c, a, m, b, m) + diag_pt(f, p, c, a, -m, b, -m)
                 - diag_pt(f, p, c, a, m, b, -m) - diag_pt(f, p, c, a, -m, b, m);
        sum += w_second(r, (int)m) * S;
    }
    return sum / (4.0 * p->dx[a] * p->dx[b]);
}

/* Second derivative d^2 f / (dx_a dx_b) for any pair (a, b). */
static double dd(const double *f, const oracle_params *p, const int64_t c[3], int a, int b)
{
    return a == b ? d2(f, p, c, a) : dab(f, p, c, a, b);
}

/* ------------------------------------------------------------------------ */
/* Forcing term (not in the paper; reading): f0 e cos(k . x + phi) with      */
/* x_a = i_a dx_a and k in units of 2 pi / L_a, so k . x = sum 2 pi k_a i_a / n_a. */
/* ------------------------------------------------------------------------ */

static void forcing_at(const oracle_params *p, const int64_t c[3], double out[3])
{
    const double two_pi = 6.283185307179586476925286766559;
    double phase = p->force_phi;
    for (int a = 0; a < 3; ++a)
        phase += two_pi * (double)p->force_k[a] * (double)c[a] / (double)p->n[a];
    double cphase = cos(phase);
    for (int a = 0; a < 3; ++a)
        out[a] = p->force_amp * p->force_e[a] * cphase;
}

/* ------------------------------------------------------------------------ */
/* Right-hand side of Eqs. B.1-B.4 at one cell.                              */
/* Readings: mu0 = 1 (mu0 enters only through j = mu0^-1 curl B and the      */
/* mu0 j^2 heating term); H = C = K = zeta = 0; c_s^2 is the ideal-gas       */
/* adiabatic sound speed c_s0^2 exp(gamma s / c_p + (gamma-1)(ln rho -       */
/* ln rho0)) and T = c_s^2 / (c_p (gamma - 1)).                              */
/* ------------------------------------------------------------------------ */

void oracle_rhs(const double *const f[NFIELDS], const oracle_params *p,
                int64_t i, int64_t j, int64_t k, double out[NFIELDS])
{
    const int64_t c[3] = {i, j, k};
    const int U[3] = {UX, UY, UZ};
    const int A[3] = {AX, AY, AZ};

    /* Values at the cell. */
    double v[NFIELDS];
    for (int q = 0; q < NFIELDS; ++q)
        v[q] = at(f[q], p, i, j, k);
    const double lnrho = v[LNRHO];
    const double s = v[SS];
    double u[3];
    for (int a = 0; a < 3; ++a)
        u[a] = v[U[a]];

    /* First derivatives of every field: g[q][a] = d f_q / d x_a. */
    double g[NFIELDS][3];
    for (int q = 0; q < NFIELDS; ++q)
        for (int a = 0; a < 3; ++a)
            g[q][a] = d1(f[q], p, c, a);

    /* Second derivatives of u and A: hu[m][a][b] = d^2 u_m / dx_a dx_b. */
    double hu[3][3][3], ha[3][3][3];
    for (int m = 0; m < 3; ++m)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                hu[m][a][b] = dd(f[U[m]], p, c, a, b);
                ha[m][a][b] = dd(f[A[m]], p, c, a, b);
            }

    /* Thermodynamics. */
    const double rho = exp(lnrho);
    const double cs2 = p->cs0 * p->cs0
                     * exp(p->gamma * s / p->cp + (p->gamma - 1.0) * (lnrho - p->lnrho0));
    const double T = cs2 / (p->cp * (p->gamma - 1.0));

    /* div u, Laplacians, grad div (Table B.2 operators). */
    const double divu = g[UX][0] + g[UY][1] + g[UZ][2];
    double lapu[3], lapa[3], graddivu[3], graddiva[3];
    for (int m = 0; m < 3; ++m) {
        lapu[m] = hu[m][0][0] + hu[m][1][1] + hu[m][2][2];
        lapa[m] = ha[m][0][0] + ha[m][1][1] + ha[m][2][2];
        graddivu[m] = hu[0][m][0] + hu[1][m][1] + hu[2][m][2];
        graddiva[m] = ha[0][m][0] + ha[1][m][1] + ha[2][m][2];
    }

    /* B = curl A;  j = mu0^-1 curl B = grad(div A) - lap A  (mu0 = 1). */
    double B[3], J[3];
    B[0] = g[AZ][1] - g[AY][2];
    B[1] = g[AX][2] - g[AZ][0];
    B[2] = g[AY][0] - g[AX][1];
    for (int m = 0; m < 3; ++m)
        J[m] = graddiva[m] - lapa[m];

    /* Traceless rate-of-strain tensor S_mn = (d_n u_m + d_m u_n)/2 - delta_mn div u / 3. */
    double S[3][3];
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n)
            S[m][n] = 0.5 * (g[U[m]][n] + g[U[n]][m]) - (m == n ? divu / 3.0 : 0.0);
    double SS2 = 0.0;
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n)
            SS2 += S[m][n] * S[m][n];

    /* j x B, u x B, j^2. */
    double JxB[3], UxB[3];
    JxB[0] = J[1] * B[2] - J[2] * B[1];
    JxB[1] = J[2] * B[0] - J[0] * B[2];
    JxB[2] = J[0] * B[1] - J[1] * B[0];
    UxB[0] = u[1] * B[2] - u[2] * B[1];
    UxB[1] = u[2] * B[0] - u[0] * B[2];
    UxB[2] = u[0] * B[1] - u[1] * B[0];
    const double J2 = J[0] * J[0] + J[1] * J[1] + J[2] * J[2];

    /* u . grad of a scalar field q. */
#define ADV(q) (u[0] * g[(q)][0] + u[1] * g[(q)][1] + u[2] * g[(q)][2])

    /* Eq. B.1: D ln rho / Dt = -div u. */
    out[LNRHO] = -ADV(LNRHO) - divu;

    /* Eq. B.2:
     * Du/Dt = -c_s^2 grad(s/c_p + ln rho) + j x B / rho
     *         + nu [lap u + grad(div u)/3 + 2 S . grad ln rho]
     *         + zeta grad(div u)  (+ forcing). */
    double fr[3] = {0.0, 0.0, 0.0};
    if (p->force_on)
        forcing_at(p, c, fr);
    for (int m = 0; m < 3; ++m) {
        double sgl = 0.0; /* (S . grad ln rho)_m */
        for (int n = 0; n < 3; ++n)
            sgl += S[m][n] * g[LNRHO][n];
        out[U[m]] = -ADV(U[m])
                  - cs2 * (g[SS][m] / p->cp + g[LNRHO][m])
                  + JxB[m] / rho
                  + p->nu * (lapu[m] + graddivu[m] / 3.0 + 2.0 * sgl)
                  + p->zeta * graddivu[m]
                  + fr[m];
    }

    /* Eq. B.3 (mu0 = 1):
     * rho T Ds/Dt = H - C + div(K grad T) + eta j^2 + 2 rho nu S:S + zeta rho (div u)^2.
     * Reading (the paper fixes no discretisation of the conduction term): with
     * T = T_0 exp(xi), xi = gamma s / c_p + (gamma - 1)(ln rho - ln rho0),
     * grad T = T grad xi and, K constant, div(K grad T) = K T (lap xi + |grad xi|^2),
     * with grad xi and lap xi from the stencils of s and ln rho.  H and C are
     * uniform rates (the paper gives no form). */
    double cond = 0.0;
    if (p->K != 0.0) {
        double gxi2 = 0.0, lapxi = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double gxi = p->gamma / p->cp * g[SS][a] + (p->gamma - 1.0) * g[LNRHO][a];
            gxi2 += gxi * gxi;
            lapxi += p->gamma / p->cp * d2(f[SS], p, c, a) + (p->gamma - 1.0) * d2(f[LNRHO], p, c, a);
        }
        cond = p->K * T * (lapxi + gxi2);
    }
    out[SS] = -ADV(SS) + (p->heat - p->cool + cond + p->eta * J2 + 2.0 * rho * p->nu * SS2
                          + p->zeta * rho * divu * divu) / (rho * T);

    /* Eq. B.4: dA/dt = u x B + eta lap A. */
    for (int m = 0; m < 3; ++m)
        out[A[m]] = UxB[m] + p->eta * lapa[m];
#undef ADV
}

/* ------------------------------------------------------------------------ */
/* Williamson (1980) third-order 2N-storage Runge-Kutta, Sec. 4.             */
/* Reading: the paper prints no coefficients; Williamson's low-storage       */
/* third-order set is alpha = (0, -5/9, -153/128), beta = (1/3, 15/16, 8/15). */
/* Substep s:  w <- alpha_s w + dt RHS(f);  f <- f + beta_s w.               */
/* At s = 0, alpha_0 = 0 and w is not read at all.                           */
/* ------------------------------------------------------------------------ */

static const double RK_ALPHA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double RK_BETA[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

double oracle_rk_alpha(int64_t s) { return RK_ALPHA[s]; }
double oracle_rk_beta(int64_t s) { return RK_BETA[s]; }

static void substep_cell(const double *const fin[NFIELDS], const double *const win[NFIELDS],
                         const oracle_params *p, double dt, int64_t s,
                         int64_t i, int64_t j, int64_t k,
                         double fout_v[NFIELDS], double wout_v[NFIELDS])
{
    double rhs[NFIELDS];
    oracle_rhs(fin, p, i, j, k, rhs);
    const int64_t lin = (k * p->n[1] + j) * p->n[0] + i;
    for (int q = 0; q < NFIELDS; ++q) {
        double wn = dt * rhs[q];
        if (s > 0)
            wn = RK_ALPHA[s] * win[q][lin] + wn;
        wout_v[q] = wn;
        fout_v[q] = fin[q][lin] + RK_BETA[s] * wn;
    }
}

static int set_threads(int64_t nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads((int)nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* One substep over the whole grid.  fin is read only; w is read (s > 0) and
 * overwritten; fout receives the new state.  fout must not alias fin.
 * Returns the number of threads used. */
int64_t oracle_substep(const double *const fin[NFIELDS], double *const w[NFIELDS],
                       double *const fout[NFIELDS], const oracle_params *p,
                       double dt, int64_t s, int64_t nthreads)
{
    const int used = set_threads(nthreads);
    const int64_t nx = p->n[0], ny = p->n[1], nz = p->n[2];
#pragma omp parallel for schedule(static) collapse(2)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                double fo[NFIELDS], wo[NFIELDS];
                substep_cell(fin, (const double *const *)w, p, dt, s, i, j, k, fo, wo);
                const int64_t lin = (k * ny + j) * nx + i;
                for (int q = 0; q < NFIELDS; ++q)
                    fout[q][lin] = fo[q];
                /* w is read at this cell only, so overwriting it here is safe. */
                for (int q = 0; q < NFIELDS; ++q)
                    w[q][lin] = wo[q];
            }
    return used;
}

/* One substep evaluated only at the listed cells (cells[3m..3m+2] = i, j, k);
 * outputs are field-major: fout[q * ncells + m], wout[q * ncells + m]. */
void oracle_substep_cells(const double *const fin[NFIELDS], const double *const win[NFIELDS],
                          const oracle_params *p, double dt, int64_t s,
                          int64_t ncells, const int64_t *cells,
                          double *fout, double *wout, int64_t nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < ncells; ++m) {
        double fo[NFIELDS], wo[NFIELDS];
        substep_cell(fin, win, p, dt, s, cells[3 * m], cells[3 * m + 1], cells[3 * m + 2], fo, wo);
        for (int q = 0; q < NFIELDS; ++q) {
            fout[q * ncells + m] = fo[q];
            wout[q * ncells + m] = wo[q];
        }
    }
}

/* RHS over the whole grid (out[q] has n[0] n[1] n[2] entries). */
void oracle_rhs_grid(const double *const f[NFIELDS], const oracle_params *p,
                     double *const out[NFIELDS], int64_t nthreads)
{
    set_threads(nthreads);
    const int64_t nx = p->n[0], ny = p->n[1], nz = p->n[2];
#pragma omp parallel for schedule(static) collapse(2)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                double r[NFIELDS];
                oracle_rhs(f, p, i, j, k, r);
                const int64_t lin = (k * ny + j) * nx + i;
                for (int q = 0; q < NFIELDS; ++q)
                    out[q][lin] = r[q];
            }
}

/* A single derivative operator over the whole grid, for the operator pins:
 * kind 0 = first derivative along a; kind 1 = second derivative d^2/dx_a dx_b
 * (b == a: the pure second derivative, b != a: the mixed one). */
void oracle_deriv(const double *f, const oracle_params *p, int64_t kind,
                  int64_t a, int64_t b, double *out)
{
    const int64_t nx = p->n[0], ny = p->n[1], nz = p->n[2];
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                const int64_t c[3] = {i, j, k};
                out[(k * ny + j) * nx + i] =
                    kind == 0 ? d1(f, p, c, (int)a) : dd(f, p, c, (int)a, (int)b);
            }
}

/* B = curl A over the whole grid with the first-derivative operator above. */
void oracle_curl(const double *const A[3], const oracle_params *p, double *const B[3])
{
    const int64_t nx = p->n[0], ny = p->n[1], nz = p->n[2];
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                const int64_t c[3] = {i, j, k};
                const int64_t lin = (k * ny + j) * nx + i;
                B[0][lin] = d1(A[2], p, c, 1) - d1(A[1], p, c, 2);
                B[1][lin] = d1(A[0], p, c, 2) - d1(A[2], p, c, 0);
                B[2][lin] = d1(A[1], p, c, 0) - d1(A[0], p, c, 1);
            }
}

/* ------------------------------------------------------------------------ */
/* Periodic halo of a padded array, Sec. 3.3: a halo cell at padded index s  */
/* holds the computational-domain cell ((s - r) mod n) + r, per axis.  The   */
/* padded array has (n_a + 2r) cells per axis, x fastest.  Every halo cell   */
/* (sides, edges and corners) is filled.                                     */
/* ------------------------------------------------------------------------ */

void oracle_periodic_halo(double *fp, const int64_t n[3], int64_t r)
{
    const int64_t mx = n[0] + 2 * r, my = n[1] + 2 * r, mz = n[2] + 2 * r;
    for (int64_t k = 0; k < mz; ++k)
        for (int64_t j = 0; j < my; ++j)
            for (int64_t i = 0; i < mx; ++i) {
                const int inside = i >= r && i < n[0] + r && j >= r && j < n[1] + r
                                && k >= r && k < n[2] + r;
                if (inside)
                    continue;
                const int64_t si = wrap(i - r, n[0]) + r;
                const int64_t sj = wrap(j - r, n[1]) + r;
                const int64_t sk = wrap(k - r, n[2]) + r;
                fp[(k * my + j) * mx + i] = fp[(sk * my + sj) * mx + si];
            }
}

/* ------------------------------------------------------------------------ */
/* Forcing draw (not in the paper; reading).  One counter-based generator,  */
/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the n-th output of the   */
/* stream with seed x is mix(x + (n + 1) * 0x9E3779B97F4A7C15), where mix is */
/* the published finaliser.                                                  */
/* ------------------------------------------------------------------------ */

uint64_t oracle_splitmix64(uint64_t seed, uint64_t counter)
{
    uint64_t z = seed + (counter + 1u) * UINT64_C(0x9E3779B97F4A7C15);
    z = (z ^ (z >> 30)) * UINT64_C(0xBF58476D1CE4E5B9);
    z = (z ^ (z >> 27)) * UINT64_C(0x94D049BB133111EB);
    return z ^ (z >> 31);
}

/* Uniform double in [0, 1) from the top 53 bits. */
static double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

/* Draw the forcing of step `step`:
 *   draw 0:      k, uniformly from the wave vectors with 2 <= |k| <= 3, in the
 *                order kx, ky, kz ascending from -3 to 3 (index = draw mod count);
 *   draws 1-12:  up to four candidate vectors e, each component uniform in
 *                [-1, 1); the first with |k x e|^2 >= |k|^2 |e|^2 / 4 and
 *                |e|^2 >= 1/16 is kept; if none is, e is the unit vector of
 *                the first axis with the smallest |k_a|;
 *   draw 13:     phi uniform in [0, 2 pi).
 * The polarisation is (k x e) / |k x e| (perpendicular to k: non-helical). The
 * counters of step t are 16 t .. 16 t + 13. */
void oracle_forcing_draw(uint64_t seed, uint64_t step, int64_t k_out[3], double e_out[3],
                         double *phi_out)
{
    const uint64_t base = 16u * step;
    int64_t count = 0;
    for (int64_t kx = -3; kx <= 3; ++kx)
        for (int64_t ky = -3; ky <= 3; ++ky)
            for (int64_t kz = -3; kz <= 3; ++kz) {
                int64_t k2 = kx * kx + ky * ky + kz * kz;
                if (k2 >= 4 && k2 <= 9)
                    ++count;
            }
    uint64_t pick = oracle_splitmix64(seed, base + 0) % (uint64_t)count;
    int64_t k[3] = {0, 0, 0};
    int64_t idx = 0;
    for (int64_t kx = -3; kx <= 3; ++kx)
        for (int64_t ky = -3; ky <= 3; ++ky)
            for (int64_t kz = -3; kz <= 3; ++kz) {
                int64_t k2 = kx * kx + ky * ky + kz * kz;
                if (k2 >= 4 && k2 <= 9) {
                    if ((uint64_t)idx == pick) {
                        k[0] = kx;
                        k[1] = ky;
                        k[2] = kz;
                    }
                    ++idx;
                }
            }
    const double kk[3] = {(double)k[0], (double)k[1], (double)k[2]};
    const double k2 = kk[0] * kk[0] + kk[1] * kk[1] + kk[2] * kk[2];

    double e[3] = {0.0, 0.0, 0.0};
    int found = 0;
    for (int tries = 0; tries < 4 && !found; ++tries) {
        double c[3];
        for (int a = 0; a < 3; ++a)
            c[a] = 2.0 * u01(oracle_splitmix64(seed, base + 1 + 3 * tries + a)) - 1.0;
        double x[3];
        x[0] = kk[1] * c[2] - kk[2] * c[1];
        x[1] = kk[2] * c[0] - kk[0] * c[2];
        x[2] = kk[0] * c[1] - kk[1] * c[0];
        const double x2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        const double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        if (c2 >= 1.0 / 16.0 && x2 >= 0.25 * k2 * c2) {
            for (int a = 0; a < 3; ++a)
                e[a] = c[a];
            found = 1;
        }
    }
    if (!found) {
        int best = 0;
        for (int a = 1; a < 3; ++a)
            if (llabs(k[a]) < llabs(k[best]))
                best = a;
        e[best] = 1.0;
    }
    double x[3];
    x[0] = kk[1] * e[2] - kk[2] * e[1];
    x[1] = kk[2] * e[0] - kk[0] * e[2];
    x[2] = kk[0] * e[1] - kk[1] * e[0];
    const double xn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    for (int a = 0; a < 3; ++a) {
        k_out[a] = k[a];
        e_out[a] = x[a] / xn;
    }
    *phi_out = 6.283185307179586476925286766559 * u01(oracle_splitmix64(seed, base + 13));
}

/* Forcing field of the current parameters over the whole grid (3 arrays). */
void oracle_forcing_field(const oracle_params *p, double *const out[3])
{
    const int64_t nx = p->n[0], ny = p->n[1], nz = p->n[2];
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                const int64_t c[3] = {i, j, k};
                double fr[3];
                forcing_at(p, c, fr);
                const int64_t lin = (k * ny + j) * nx + i;
                for (int a = 0; a < 3; ++a)
                    out[a][lin] = fr[a];
            }
}

/* ------------------------------------------------------------------------ */
/* Restriction fine -> coarse (learned-closure data path; reading): full     */
/* weighting with weights [1, 2, 1] / 4 per axis centred on the even fine    */
/* cells, so coarse cell I sits on fine cell 2 I.  Fine sizes must be even.  */
/* ------------------------------------------------------------------------ */

void oracle_restrict(const double *fine, const int64_t nf[3], double *coarse)
{
    const int64_t nc[3] = {nf[0] / 2, nf[1] / 2, nf[2] / 2};
    const double w[3] = {0.25, 0.5, 0.25};
    for (int64_t K = 0; K < nc[2]; ++K)
        for (int64_t J = 0; J < nc[1]; ++J)
            for (int64_t I = 0; I < nc[0]; ++I) {
                double acc = 0.0;
                for (int dk = -1; dk <= 1; ++dk)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int di = -1; di <= 1; ++di) {
                            const int64_t fi = wrap(2 * I + di, nf[0]);
                            const int64_t fj = wrap(2 * J + dj, nf[1]);
                            const int64_t fk = wrap(2 * K + dk, nf[2]);
                            acc += w[di + 1] * w[dj + 1] * w[dk + 1]
                                 * fine[(fk * nf[1] + fj) * nf[0] + fi];
                        }
                coarse[(K * nc[1] + J) * nc[0] + I] = acc;
            }
}
