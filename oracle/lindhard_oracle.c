/*
 * Lindhard susceptibility oracle: plain FP64 CPU code.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The GPU library never
 * links, includes or calls it, and it shares no code with the GPU library.
 *
 * What it computes (Wang et al., "Lindhard and RPA susceptibility
 * computations in extended momentum space in electron doped cuprates"):
 *
 *   Sec. 2, Eq. 9:  Im chi(q,w) = - Int_{-w}^{0} de/(2 pi) Int d^dp/(2 pi)^d
 *                                   A(p,e) A(p+q, e+w)
 *   Sec. 3 (2D reduction, k_z dispersion neglected): d = 2.
 *   Sec. 2, Eqs. 4-5: A(p,e) = |M(p)|^2 * gamma / (pi [(e - xi_p)^2 + gamma^2]),
 *                     a Lorentzian of unit weight centred on the band energy.
 *   Sec. 3 (rigid band): mu shifted to hold the requested electron count.
 *
 * Discretisation (each choice is a reading of where the paper is silent):
 *   lattice constant 1, zone width 2 pi, N = zones * npz points per axis,
 *   p_i = (i - N/2) * dp, dp = 2 pi / npz;
 *   cell-centred energies e_j = -E + (j + 1/2) de, de = 2E / n_eps;
 *   the T = 0 occupation split of Sec. 3 / Appendix A (Eq. A3): the integral
 *   over e in [-w, 0] becomes the sum over cells j with e_j < 0 and
 *   e_{j+m} >= 0, i.e. 2j+1 < n_eps <= 2(j+m)+1;
 *   w_m = m de; lags q_l = (l - Q/2) dp;
 *   d^2p/(2 pi)^2 -> dp^2/(2 pi)^2 = 1/npz^2 per grid point;
 *   zones == 1: the grid is one period and p+q wraps (reduced zone);
 *   zones  > 1: A = 0 outside the grid (extended zone, truncation).
 *
 * Everything is a plain loop in the order the formula is written.  OpenMP
 * splits independent outputs across threads; no sum is reordered within one
 * output.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double LO_PI = 3.14159265358979323846264338327950288;

/* Single-band dispersion eps0(p) in eV.
 * kind 0: square-lattice tight binding with hoppings t, t', t'' (the band
 *         that stands in for the paper's KKR CuO2 band of Sec. 3):
 *         -2t (cos px + cos py) - 4t' cos px cos py - 2t'' (cos 2px + cos 2py)
 * kind 1: free electrons, |p|^2 / 2 (the "free fermion form" of Sec. 2). */
double lo_band(int kind, double t, double tp, double tpp, double px, double py)
{
    if (kind == 1)
        return 0.5 * (px * px + py * py);
    return -2.0 * t * (cos(px) + cos(py)) - 4.0 * tp * cos(px) * cos(py)
           - 2.0 * tpp * (cos(2.0 * px) + cos(2.0 * py));
}

/* Electron count per site including spin at chemical potential mu
 * (rigid band, Sec. 3).  Each first-zone state carries the weight of its
 * Lorentzian (Eq. 5) below the Fermi level:
 *   Int_{-inf}^{0} gamma / (pi [(e - xi)^2 + gamma^2]) de = 1/2 - atan(xi/gamma)/pi,
 * summed over the npz x npz first-zone grid with measure 2/npz^2. */
double lo_filling(int kind, double t, double tp, double tpp, double gamma,
                  int npz, double mu)
{
    double dp = 2.0 * LO_PI / npz, sum = 0.0;
    for (int ix = 0; ix < npz; ++ix)
        for (int iy = 0; iy < npz; ++iy) {
            double px = (ix - npz / 2) * dp, py = (iy - npz / 2) * dp;
            double xi = lo_band(kind, t, tp, tpp, px, py) - mu;
            sum += 0.5 - atan(xi / gamma) / LO_PI;
        }
    return 2.0 * sum / ((double)npz * (double)npz);
}

/* mu such that lo_filling(mu) == filling, by bisection on [-20, 20] eV.
 * lo_filling is strictly increasing in mu, so the root is unique.
 * Returns 0 on success, 1 if the filling lies outside (0, 2). */
int lo_mu(int kind, double t, double tp, double tpp, double gamma, int npz,
          double filling, double *mu_out)
{
    double lo = -20.0, hi = 20.0;
    if (!(filling > lo_filling(kind, t, tp, tpp, gamma, npz, lo)) ||
        !(filling < lo_filling(kind, t, tp, tpp, gamma, npz, hi)))
        return 1;
    for (int it = 0; it < 200 && hi - lo > 1e-14; ++it) {
        double mid = 0.5 * (lo + hi);
        if (lo_filling(kind, t, tp, tpp, gamma, npz, mid) < filling)
            lo = mid;
        else
            hi = mid;
    }
    *mu_out = 0.5 * (lo + hi);
    return 0;
}

/* Derivatives of mu at fixed filling (the rigid band of Sec. 3): the filling
 * n(mu; t, t', t'', gamma) of lo_filling is held constant, so by the implicit
 * function theorem dmu/dtheta = -(dn/dtheta) / (dn/dmu), with, per state,
 *   d/dmu    [1/2 - atan(xi/gamma)/pi] =  gamma / (pi (xi^2 + gamma^2)),
 *   d/dtheta [ ... ]                   = -gamma / (pi (xi^2 + gamma^2)) dxi/dtheta,
 *   d/dgamma [ ... ]                   =  xi / (pi (xi^2 + gamma^2)),
 * dxi/d(t, t', t'') = (-2 (cos px + cos py), -4 cos px cos py,
 * -2 (cos 2px + cos 2py)) for the tight-binding band, 0 for free electrons.
 * out[0..3] = dmu/d(t, t', t'', gamma). */
void lo_dmu_dparams(int kind, double t, double tp, double tpp, double gamma, int npz, double mu, double *out)
{
    double dp = 2.0 * LO_PI / npz, dn_dmu = 0.0, dn[4] = {0.0, 0.0, 0.0, 0.0};
    for (int ix = 0; ix < npz; ++ix)
        for (int iy = 0; iy < npz; ++iy) {
            double px = (ix - npz / 2) * dp, py = (iy - npz / 2) * dp;
            double xi = lo_band(kind, t, tp, tpp, px, py) - mu;
            double D = xi * xi + gamma * gamma;
            double w = gamma / (LO_PI * D);
            dn_dmu += w;
            if (kind == 0) {
                dn[0] -= w * (-2.0 * (cos(px) + cos(py)));
                dn[1] -= w * (-4.0 * cos(px) * cos(py));
                dn[2] -= w * (-2.0 * (cos(2.0 * px) + cos(2.0 * py)));
            }
            dn[3] += xi / (LO_PI * D);
        }
    for (int r = 0; r < 4; ++r) out[r] = -dn[r] / dn_dmu;   /* the measure 2/npz^2 cancels */
}

/* Spectral function A(p_i, e_j) on the grid (Eqs. 4-5), layout [N][N][n_eps]
 * with the energy index fastest.  |M(p)|^2 = exp(-|p|^2 ff_a^2 / 8) stands in
 * for the Bloch momentum density of Eq. 7; ff_a == 0 means |M|^2 = 1. */
void lo_spectral(int kind, double t, double tp, double tpp, double mu,
                 double gamma, double ff_a, int zones, int npz, int n_eps,
                 double e_max, double *A)
{
    int N = zones * npz;
    double dp = 2.0 * LO_PI / npz, de = 2.0 * e_max / n_eps;
#pragma omp parallel for schedule(static)
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy) {
            double px = (ix - N / 2) * dp, py = (iy - N / 2) * dp;
            double xi = lo_band(kind, t, tp, tpp, px, py) - mu;
            double m2 = (ff_a == 0.0) ? 1.0
                        : exp(-(px * px + py * py) * ff_a * ff_a / 8.0);
            for (int j = 0; j < n_eps; ++j) {
                double e = -e_max + (j + 0.5) * de;
                A[((size_t)ix * N + iy) * n_eps + j] =
                    m2 * gamma / (LO_PI * ((e - xi) * (e - xi) + gamma * gamma));
            }
        }
}

/* Index of momentum i + s on the grid, or -1 if it falls outside
 * (extended zone).  In the reduced zone (zones == 1) it wraps. */
static long lo_shift(long i, long s, long N, int periodic)
{
    long k = i + s;
    if (periodic) {
        k %= N;
        if (k < 0) k += N;
        return k;
    }
    return (k >= 0 && k < N) ? k : -1;
}

/* The discrete Eq. 9 at n sample outputs (lx[k], ly[k], m[k]):
 *   out[k] = -(de / 2 pi) (1 / npz^2) *
 *            sum_{j: e_j < 0 <= e_{j+m}} sum_{p, p+q on grid} A(p, e_j) A(p+q, e_{j+m})
 * with q = ((lx - Q/2) dp, (ly - Q/2) dp), Q = q_extent, w = m de. */
void lo_imchi_samples(int zones, int npz, int n_eps, double e_max,
                      const double *A, int q_extent, long n, const int *lx,
                      const int *ly, const int *m, double *out)
{
    long N = (long)zones * npz;
    int periodic = (zones == 1);
    double de = 2.0 * e_max / n_eps;
    double c = de / (2.0 * LO_PI) / ((double)npz * (double)npz);
#pragma omp parallel for schedule(dynamic, 1)
    for (long k = 0; k < n; ++k) {
        long sx = lx[k] - q_extent / 2, sy = ly[k] - q_extent / 2;
        int mm = m[k];
        double sum = 0.0;
        for (long ix = 0; ix < N; ++ix) {
            long jx = lo_shift(ix, sx, N, periodic);
            if (jx < 0) continue;
            for (long iy = 0; iy < N; ++iy) {
                long jy = lo_shift(iy, sy, N, periodic);
                if (jy < 0) continue;
                const double *a = A + ((size_t)ix * N + iy) * n_eps;
                const double *b = A + ((size_t)jx * N + jy) * n_eps;
                for (int j = 0; j + mm < n_eps; ++j) {
                    /* occupied at e_j (e_j < 0), empty at e_{j+m} (>= 0) */
                    if (2 * j + 1 < n_eps && 2 * (j + mm) + 1 >= n_eps)
                        sum += a[j] * b[j + mm];
                }
            }
        }
        out[k] = -c * sum;
    }
}

/* Finite temperature (Sec. 2 Eq. 1, Appendix A Eq. A1).  The Fermi function
 * of the grid energy (measured from mu) at temperature kT > 0:
 *   f(e) = 1 / (exp(e / kT) + 1),   1 - f(e) = 1 / (exp(-e / kT) + 1).
 * With the matrix element F of Eq. A1, the occupation difference
 * f(e) - f(e + w) replaces the T = 0 window [-w, 0] of Eq. A3:
 *   quantity 1: Im chi_T(q, w_m) = -c sum_{j, p} A(p, e_j) A(p+q, e_{j+m})
 *                                      [f(e_j) - f(e_{j+m})]
 *   quantity 2: S(q, w_m) = -(1/pi) Im chi_T(q, w_m) / (1 - exp(-w_m / kT))
 * (the fluctuation-dissipation relation, Eq. 1), summed here in the form
 * that also holds at w = 0:
 *   S(q, w_m) = (c/pi) sum_{j, p} A(p, e_j) A(p+q, e_{j+m}) f(e_j) [1 - f(e_{j+m})]
 * (f(e) [1 - f(e + w)] (1 - exp(-w/kT)) = f(e) - f(e + w) for every e, w).
 * The sums run over cells with 0 <= j, j + m < n_eps; m may be negative.
 * Same grid, lags and prefactor c = (de / 2 pi) / npz^2 as lo_imchi_samples. */
void lo_thermal_samples(int zones, int npz, int n_eps, double e_max,
                        const double *A, int q_extent, double kT, int quantity,
                        long n, const int *lx, const int *ly, const int *m, double *out)
{
    long N = (long)zones * npz;
    int periodic = (zones == 1);
    double de = 2.0 * e_max / n_eps;
    double c = de / (2.0 * LO_PI) / ((double)npz * (double)npz);
    double *f = (double *)malloc(sizeof(double) * 2 * (size_t)n_eps);
    double *fe = f + n_eps;            /* 1 - f */
    for (int j = 0; j < n_eps; ++j) {
        double e = -e_max + (j + 0.5) * de;
        f[j] = 1.0 / (exp(e / kT) + 1.0);
        fe[j] = 1.0 / (exp(-e / kT) + 1.0);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (long k = 0; k < n; ++k) {
        long sx = lx[k] - q_extent / 2, sy = ly[k] - q_extent / 2;
        int mm = m[k];
        double sum = 0.0;
        for (long ix = 0; ix < N; ++ix) {
            long jx = lo_shift(ix, sx, N, periodic);
            if (jx < 0) continue;
            for (long iy = 0; iy < N; ++iy) {
                long jy = lo_shift(iy, sy, N, periodic);
                if (jy < 0) continue;
                const double *a = A + ((size_t)ix * N + iy) * n_eps;
                const double *b = A + ((size_t)jx * N + jy) * n_eps;
                for (int j = 0; j < n_eps; ++j) {
                    if (j + mm < 0 || j + mm >= n_eps) continue;
                    double wgt = quantity == 1 ? f[j] - f[j + mm] : f[j] * fe[j + mm];
                    sum += a[j] * b[j + mm] * wgt;
                }
            }
        }
        out[k] = quantity == 1 ? -c * sum : c / LO_PI * sum;
    }
    free(f);
}

/* Gradient of L = sum_{l,m} w[l_x][l_y][m] Im chi(q_l, w_m) with respect to
 * A(p_i, e_j), at n sample points (ix[k], iy[k], j[k]).  Eq. 9 is bilinear in
 * the occupied part a = A [e < 0] and the empty part b = A [e >= 0]:
 *   dL/da(p, e_j)   = -c sum_{l,m} w(l,m) b(p + q_l, e_{j+m})
 *   dL/db(p', e_j') = -c sum_{l,m} w(l,m) a(p' - q_l, e_{j'-m})
 * w has layout [Q][Q][n_omega]. */
void lo_grad_A_samples(int zones, int npz, int n_eps, double e_max,
                       const double *A, int q_extent, int n_omega,
                       const double *w, long n, const int *ix, const int *iy,
                       const int *jj, double *out)
{
    long N = (long)zones * npz;
    int periodic = (zones == 1), Q = q_extent;
    double de = 2.0 * e_max / n_eps;
    double c = de / (2.0 * LO_PI) / ((double)npz * (double)npz);
#pragma omp parallel for schedule(dynamic, 1)
    for (long k = 0; k < n; ++k) {
        int j = jj[k];
        int occupied = (2 * j + 1 < n_eps);
        double sum = 0.0;
        for (int lx = 0; lx < Q; ++lx) {
            long sx = lx - Q / 2;
            long kx = lo_shift(ix[k], occupied ? sx : -sx, N, periodic);
            if (kx < 0) continue;
            for (int ly = 0; ly < Q; ++ly) {
                long sy = ly - Q / 2;
                long ky = lo_shift(iy[k], occupied ? sy : -sy, N, periodic);
                if (ky < 0) continue;
                const double *row = A + ((size_t)kx * N + ky) * n_eps;
                const double *wr = w + ((size_t)lx * Q + ly) * n_omega;
                for (int mm = 0; mm < n_omega; ++mm) {
                    if (occupied) {
                        /* partner e_{j+m} must be on the grid and empty */
                        int jp = j + mm;
                        if (jp < n_eps && 2 * jp + 1 >= n_eps)
                            sum += wr[mm] * row[jp];
                    } else {
                        /* partner e_{j-m} must be on the grid and occupied */
                        int jp = j - mm;
                        if (jp >= 0 && 2 * jp + 1 < n_eps)
                            sum += wr[mm] * row[jp];
                    }
                }
            }
        }
        out[k] = -c * sum;
    }
}

/* Gradient of L = sum_{l,m} w[l_x][l_y][m] X(q_l, w_m) with respect to
 * A(p_i, e_j) at finite temperature, X = Im chi_T (quantity 1) or S(q, w)
 * (quantity 2) as lo_thermal_samples sums them (Eq. 1, Appendix A Eq. A1):
 *   X(q, m) = kappa sum_{p, j} A(p, e_j) A(p + q, e_{j+m}) W(j, m),
 *   W(j, m) = f_j - f_{j+m} (kappa = -c)  or  f_j (1 - f_{j+m}) (kappa = c/pi).
 * A(p0, e_j0) enters as the first factor (p = p0, j = j0) and as the second
 * (p = p0 - q, j = j0 - m), so
 *   dL/dA(p0, e_j0) = kappa sum_{l,m} w(l,m) [W(j0, m) A(p0 + q_l, e_{j0+m})
 *                                            + W(j0 - m, m) A(p0 - q_l, e_{j0-m})],
 * every partner on the grid (the same shifts and edges as the forward sum). */
void lo_thermal_grad_A_samples(int zones, int npz, int n_eps, double e_max,
                               const double *A, int q_extent, int n_omega,
                               double kT, int quantity, const double *w,
                               long n, const int *ix, const int *iy,
                               const int *jj, double *out)
{
    long N = (long)zones * npz;
    int periodic = (zones == 1), Q = q_extent;
    double de = 2.0 * e_max / n_eps;
    double c = de / (2.0 * LO_PI) / ((double)npz * (double)npz);
    double kappa = quantity == 1 ? -c : c / LO_PI;
    double *f = (double *)malloc(sizeof(double) * 2 * (size_t)n_eps);
    double *fe = f + n_eps;            /* 1 - f */
    for (int j = 0; j < n_eps; ++j) {
        double e = -e_max + (j + 0.5) * de;
        f[j] = 1.0 / (exp(e / kT) + 1.0);
        fe[j] = 1.0 / (exp(-e / kT) + 1.0);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (long k = 0; k < n; ++k) {
        int j0 = jj[k];
        double sum = 0.0;
        for (int lx = 0; lx < Q; ++lx) {
            long sx = lx - Q / 2;
            long ax = lo_shift(ix[k], sx, N, periodic), bx = lo_shift(ix[k], -sx, N, periodic);
            for (int ly = 0; ly < Q; ++ly) {
                long sy = ly - Q / 2;
                long ay = lo_shift(iy[k], sy, N, periodic), by = lo_shift(iy[k], -sy, N, periodic);
                const double *wr = w + ((size_t)lx * Q + ly) * n_omega;
                if (ax >= 0 && ay >= 0) {           /* A(p0, e_j0) first: partner at p0 + q, e_{j0+m} */
                    const double *row = A + ((size_t)ax * N + ay) * n_eps;
                    for (int mm = 0; mm < n_omega && j0 + mm < n_eps; ++mm) {
                        double wgt = quantity == 1 ? f[j0] - f[j0 + mm] : f[j0] * fe[j0 + mm];
                        sum += wr[mm] * wgt * row[j0 + mm];
                    }
                }
                if (bx >= 0 && by >= 0) {           /* A(p0, e_j0) second: partner at p0 - q, e_{j0-m} */
                    const double *row = A + ((size_t)bx * N + by) * n_eps;
                    for (int mm = 0; mm < n_omega && j0 - mm >= 0; ++mm) {
                        int jq = j0 - mm;
                        double wgt = quantity == 1 ? f[jq] - f[j0] : f[jq] * fe[j0];
                        sum += wr[mm] * wgt * row[jq];
                    }
                }
            }
        }
        out[k] = kappa * sum;
    }
    free(f);
}

/* Derivatives of A(p, e) (Eqs. 4-5 with the band above) with respect to the
 * five band parameters theta = (t, t', t'', mu, gamma), written into
 * dA[5][N][N][n_eps].  With D = (e - xi)^2 + gamma^2:
 *   dA/dxi    = |M|^2 (gamma/pi) 2 (e - xi) / D^2
 *   dA/dgamma = |M|^2 ((e - xi)^2 - gamma^2) / (pi D^2)
 *   dxi/d(t, t', t'', mu) = (-2(cx+cy), -4 cx cy, -2(c2x+c2y), -1). */
void lo_spectral_dtheta(double t, double tp, double tpp, double mu,
                        double gamma, double ff_a, int zones, int npz,
                        int n_eps, double e_max, double *dA)
{
    long N = (long)zones * npz;
    size_t plane = (size_t)N * N * n_eps;
    double dp = 2.0 * LO_PI / npz, de = 2.0 * e_max / n_eps;
#pragma omp parallel for schedule(static)
    for (long ix = 0; ix < N; ++ix)
        for (long iy = 0; iy < N; ++iy) {
            double px = (ix - N / 2) * dp, py = (iy - N / 2) * dp;
            double xi = lo_band(0, t, tp, tpp, px, py) - mu;
            double m2 = (ff_a == 0.0) ? 1.0
                        : exp(-(px * px + py * py) * ff_a * ff_a / 8.0);
            double dxi[4] = {-2.0 * (cos(px) + cos(py)),
                             -4.0 * cos(px) * cos(py),
                             -2.0 * (cos(2.0 * px) + cos(2.0 * py)), -1.0};
            for (int j = 0; j < n_eps; ++j) {
                double e = -e_max + (j + 0.5) * de;
                double d = (e - xi) * (e - xi) + gamma * gamma;
                double dA_dxi = m2 * (gamma / LO_PI) * 2.0 * (e - xi) / (d * d);
                double dA_dg = m2 * ((e - xi) * (e - xi) - gamma * gamma) / (LO_PI * d * d);
                size_t at = ((size_t)ix * N + iy) * n_eps + j;
                for (int r = 0; r < 4; ++r)
                    dA[r * plane + at] = dA_dxi * dxi[r];
                dA[4 * plane + at] = dA_dg;
            }
        }
}

/* Real part of chi by the Kramers-Kronig relation (Sec. 4: "the real part of
 * the Lindhard susceptibility ... by applying Kramers-Kronig relation"):
 *   Re chi(w) = (1/pi) P Int Im chi(w') / (w' - w) dw'
 * over the whole line, with Im chi(q, -w) = -Im chi(q, w) (the bands of this
 * problem have A(-p, e) = A(p, e), so chi(-q) = chi(q)), on the transfer grid
 * w_k = k de, k < n_omega (Im chi taken as zero beyond the computed window).
 * The principal value is Maclaurin's rule on a uniform grid:
 *   P Int g(t) / (t - x_m) dt ~ 2 h sum_{k - m odd} g(t_k) / (t_k - x_m),
 * and folding the negative transfers onto the positive ones gives
 *   Re chi_m = (4/pi) sum_{k >= 1, k - m odd} k Im chi_k / (k^2 - m^2).
 * im, re: [n_lines][n_omega]. */
void lo_kk_real(long n_lines, int n_omega, const double *im, double *re)
{
#pragma omp parallel for schedule(static)
    for (long l = 0; l < n_lines; ++l) {
        const double *x = im + l * n_omega;
        for (int m = 0; m < n_omega; ++m) {
            double s = 0.0;
            for (int k = 1; k < n_omega; ++k)
                if ((k - m) % 2 != 0)
                    s += (double)k * x[k] / ((double)k * k - (double)m * m);
            re[l * n_omega + m] = 4.0 / LO_PI * s;
        }
    }
}

/* RPA susceptibility (Sec. 4): chi_RPA = chi / (1 - V_q chi), with the Coulomb
 * interaction V_q = v0 / |q|^2 (the paper gives only its 1/q^2 decay; v0 in
 * eV a^2, lattice constant a = 1).  chi = re + i im at lag (l_x, l_y),
 * q = ((l_x - Q/2) dp, (l_y - Q/2) dp).  At q = 0, V is infinite and chi_RPA
 * takes its limit 0 (v0 = 0: no interaction, chi_RPA = chi everywhere).
 * out: [Q][Q][n_omega][2] (re, im). */
void lo_rpa(int Q, int n_omega, double dp, double v0, const double *re, const double *im, double *out)
{
#pragma omp parallel for schedule(static)
    for (long l = 0; l < (long)Q * Q; ++l) {
        const double qx = (double)(l / Q - Q / 2) * dp, qy = (double)(l % Q - Q / 2) * dp;
        const double q2 = qx * qx + qy * qy;
        for (int m = 0; m < n_omega; ++m) {
            const long at = l * n_omega + m;
            if (q2 == 0.0 && v0 != 0.0) {
                out[2 * at] = 0.0;
                out[2 * at + 1] = 0.0;
                continue;
            }
            const double V = v0 == 0.0 ? 0.0 : v0 / q2;
            const double a = re[at], b = im[at];
            /* (a + i b) / (1 - V a - i V b) */
            const double dr = 1.0 - V * a, di = -V * b;
            const double den = dr * dr + di * di;
            out[2 * at] = (a * dr + b * di) / den;
            out[2 * at + 1] = (b * dr - a * di) / den;
        }
    }
}

int lo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
