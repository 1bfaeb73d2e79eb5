/*
 * sm_oracle.c -- plain, slow, FP64 CPU oracle for the Second Moment (SM)
 * thermal-radiative-transfer hot path of Olivier, Warsa & Park,
 * "Efficient, Nonlinear Second Moment Methods for Multigroup Thermal
 * Radiative Transfer" (arXiv 2504.21784).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this file.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py use it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Every routine restates one passage of the paper (cited per function by
 * section / equation) in the most direct form: generic finite-element
 * assembly with basis functions evaluated at quadrature points, partial-pivot
 * Gaussian elimination for the per-cell systems, compensated sums for the
 * angular moments.  No blocking, fusion or closed-form shortcut is used.
 *
 * Conventions (shared with the library only as a documented interface):
 *   cells      cell = iy*nx + ix  (1D: ny = 1)
 *   nodes      2D: n = a + 2*b, a = x-side (0 = low x), b = y-side;
 *              1D: n = a.  Nodes are the Gauss-Lobatto (corner) points.
 *   directions 1D: ascending Gauss-Legendre mu.
 *              2D: quadrant-major q = 0..3 with signs (+,+), (-,+), (-,-),
 *              (+,-) of (Omega_x, Omega_y); inside a quadrant polar-major
 *              (ascending polar cosine xi), then azimuth.
 *   arrays     I[d][g][cell][node], q[g][cell][node], sigma[g][cell].
 *   sides      0 = low x (left), 1 = high x (right), 2 = low y (bottom),
 *              3 = high y (top).
 *
 * Parity status per function is listed in the file header of oracle/__init__.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* O1. Angular quadrature (Sec. 2: discrete ordinates {Omega_d, w_d}; the   */
/* paper's sets are Gauss-Legendre in 1D (Sec. 6.1) and square             */
/* Chebyshev-Legendre in 2D (Sec. 6.3, 6.4)).                              */
/* ------------------------------------------------------------------------ */

/* n-point Gauss-Legendre rule on [-1,1]: Newton iteration on P_n using the
 * three-term recurrence (k+1)P_{k+1} = (2k+1) x P_k - k P_{k-1}.  Nodes are
 * returned ascending. */
int orc_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1) return -1;
    for (int i = 0; i < n; ++i) {
        /* initial guess for the i-th largest root */
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        double pn = 0.0, pnm1 = 0.0, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            /* P_n(z) and P_{n-1}(z) by the recurrence */
            pnm1 = 1.0;
            pn = z;
            for (int k = 1; k < n; ++k) {
                double pkp1 = ((2.0 * k + 1.0) * z * pn - k * pnm1) / (k + 1.0);
                pnm1 = pn;
                pn = pkp1;
            }
            /* P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1) */
            dp = n * (z * pn - pnm1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        pnm1 = 1.0;
        pn = z;
        for (int k = 1; k < n; ++k) {
            double pkp1 = ((2.0 * k + 1.0) * z * pn - k * pnm1) / (k + 1.0);
            pnm1 = pn;
            pn = pkp1;
        }
        dp = n * (z * pn - pnm1) / (z * z - 1.0);
        /* roots come out descending; store ascending */
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* 1D set: mu_d = Gauss-Legendre nodes, w_d = 2*pi * GL weight so that the
 * weights sum to 4*pi (the normalisation that makes E = (1/c) sum w I equal
 * 4*pi*I/c for isotropic I, Sec. 2 definitions of E_g and B_g/4pi). */
int orc_quadrature_1d(int n, double *mu, double *w)
{
    if (orc_gauss_legendre(n, mu, w)) return -1;
    for (int i = 0; i < n; ++i) w[i] *= 2.0 * ORC_PI;
    return n;
}

/* 2D product set in x-y geometry: the four upper-hemisphere octants (the
 * lower hemisphere folds onto them by the xi -> -xi symmetry, so each weight
 * is doubled).  Per octant n_polar polar cosines (the positive nodes of the
 * 2*n_polar-point GL rule) times n_azim equal-weight azimuths at the
 * midpoints phi_j = (j + 1/2) (pi/2) / n_azim.  Projection onto the plane:
 * Omega = (sqrt(1-xi^2) cos phi, sqrt(1-xi^2) sin phi). */
int orc_quadrature_2d(int n_polar, int n_azim, double *omx, double *omy, double *w)
{
    if (n_polar < 1 || n_azim < 1) return -1;
    int m = 2 * n_polar;
    double *gx = (double *)malloc(sizeof(double) * m);
    double *gw = (double *)malloc(sizeof(double) * m);
    orc_gauss_legendre(m, gx, gw);
    static const int sgx[4] = {+1, -1, -1, +1};
    static const int sgy[4] = {+1, +1, -1, -1};
    int d = 0;
    for (int q = 0; q < 4; ++q) {
        for (int p = 0; p < n_polar; ++p) {
            double xi = gx[n_polar + p]; /* ascending positive nodes */
            double wp = gw[n_polar + p];
            double s = sqrt(1.0 - xi * xi);
            for (int a = 0; a < n_azim; ++a) {
                double phi = (a + 0.5) * (0.5 * ORC_PI) / n_azim;
                omx[d] = sgx[q] * s * cos(phi);
                omy[d] = sgy[q] * s * sin(phi);
                w[d] = 2.0 * wp * (0.5 * ORC_PI) / n_azim;
                ++d;
            }
        }
    }
    free(gx);
    free(gw);
    return d;
}

/* ------------------------------------------------------------------------ */
/* O2. Planck and Rosseland group integrals (Sec. 2, Eqs. planck,           */
/* black_body and the definitions of b_g and r_g; series after Clark).      */
/* ------------------------------------------------------------------------ */

/* B_{2k}/(2k)! for k = 0..ORC_NB-1 from the identity
 *   sum_{j=0}^{m} (B_j/j!) / (m+1-j)! = 0  (m >= 1),  B_0 = 1,
 * i.e. the product of x/(e^x-1) and (e^x-1)/x is 1. */
#define ORC_NBJ 64
static double orc_bern_over_fact[ORC_NBJ]; /* B_j / j!, all j */
static int orc_bern_ready = 0;

static void orc_bern_init(void)
{
    if (orc_bern_ready) return;
    double inv_fact[ORC_NBJ + 2];
    inv_fact[0] = 1.0;
    for (int k = 1; k < ORC_NBJ + 2; ++k) inv_fact[k] = inv_fact[k - 1] / k;
    orc_bern_over_fact[0] = 1.0;
    for (int m = 1; m < ORC_NBJ; ++m) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += orc_bern_over_fact[j] * inv_fact[m + 1 - j];
        /* coefficient of b_m is 1/1! = 1 */
        orc_bern_over_fact[m] = -s;
    }
    orc_bern_ready = 1;
}

/* exported for the pin that compares with 2*(-1)^(k+1) zeta(2k)/(2 pi)^(2k) */
double orc_bernoulli_over_factorial(int j)
{
    orc_bern_init();
    if (j < 0 || j >= ORC_NBJ) return NAN;
    return orc_bern_over_fact[j];
}

#define ORC_PLANCK_SWITCH 2.0
#define ORC_15_PI4 (15.0 / (ORC_PI * ORC_PI * ORC_PI * ORC_PI))

/* sum_{n>=1} e^{-n x} (x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4)
 * = integral_x^inf t^3/(e^t - 1) dt   (x > 0). */
static double orc_planck_tail_sum(double x)
{
    double s = 0.0;
    for (int n = 1; n < 100000; ++n) {
        double e = exp(-n * x);
        double dn = (double)n;
        double t = e * (x * x * x / dn + 3.0 * x * x / (dn * dn) + 6.0 * x / (dn * dn * dn) +
                        6.0 / (dn * dn * dn * dn));
        s += t;
        if (t <= 1e-18 * s) break;
        if (e == 0.0) break;
    }
    return s;
}

/* integral_0^x t^3/(e^t-1) dt = x^3/3 - x^4/8 + sum_k B_2k x^(2k+3)/((2k)!(2k+3)) */
static double orc_planck_head_sum(double x)
{
    orc_bern_init();
    double s = x * x * x / 3.0 - x * x * x * x / 8.0;
    double x2 = x * x;
    double xp = x * x * x; /* x^(2k+3) built up */
    for (int k = 1; 2 * k < ORC_NBJ; ++k) {
        xp *= x2;
        double t = orc_bern_over_fact[2 * k] * xp / (2.0 * k + 3.0);
        s += t;
        if (fabs(t) <= 1e-18 * fabs(s)) break;
    }
    return s;
}

/* P(x) = (15/pi^4) integral_0^x t^3/(e^t-1) dt : cumulative normalised Planck. */
double orc_planck_P(double x)
{
    if (!(x > 0.0)) return 0.0;
    if (isinf(x)) return 1.0;
    if (x < ORC_PLANCK_SWITCH) return ORC_15_PI4 * orc_planck_head_sum(x);
    return 1.0 - ORC_15_PI4 * orc_planck_tail_sum(x);
}

/* Q(x) = 1 - P(x), evaluated without cancellation for large x. */
double orc_planck_Q(double x)
{
    if (!(x > 0.0)) return 1.0;
    if (isinf(x)) return 0.0;
    if (x < ORC_PLANCK_SWITCH) return 1.0 - ORC_15_PI4 * orc_planck_head_sum(x);
    return ORC_15_PI4 * orc_planck_tail_sum(x);
}

/* exported so a pin can compare the two branches at the switch point */
double orc_planck_P_head(double x) { return ORC_15_PI4 * orc_planck_head_sum(x); }
double orc_planck_P_tail(double x) { return 1.0 - ORC_15_PI4 * orc_planck_tail_sum(x); }

/* x^4/(e^x - 1), with its x -> 0 limit 0 and its x -> inf limit 0. */
static double orc_x4_over_expm1(double x)
{
    if (!(x > 0.0) || isinf(x)) return 0.0;
    if (x > 700.0) return 0.0;
    return x * x * x * x / expm1(x);
}

/* R(x) = (15/4pi^4) integral_0^x t^4 e^t/(e^t-1)^2 dt.  Integrating by parts,
 * integral t^4 e^t/(e^t-1)^2 = -t^4/(e^t-1) + 4 integral t^3/(e^t-1), so
 * R(x) = P(x) - (15/(4 pi^4)) x^4/(e^x-1). */
double orc_rosseland_R(double x)
{
    if (!(x > 0.0)) return 0.0;
    if (isinf(x)) return 1.0;
    return orc_planck_P(x) - 0.25 * ORC_15_PI4 * orc_x4_over_expm1(x);
}

double orc_rosseland_RQ(double x) /* 1 - R(x) */
{
    if (!(x > 0.0)) return 1.0;
    if (isinf(x)) return 0.0;
    return orc_planck_Q(x) + 0.25 * ORC_15_PI4 * orc_x4_over_expm1(x);
}

/* b_g(T), r_g(T) for all groups.  The lowest edge is taken to 0 and the
 * highest to infinity so that sum_g b_g = sum_g r_g = 1 (the normalisation
 * stated with the definition of b_g in Sec. 2).  A group whose lower reduced
 * edge lies in the tail branch is evaluated as a difference of tails (Q), all
 * others as a difference of P: the same integral, without cancellation. */
void orc_group_spectra(int G, const double *edges, double T, double *b, double *r)
{
    for (int g = 0; g < G; ++g) {
        double lo = (g == 0) ? 0.0 : edges[g] / T;
        double hi = (g == G - 1) ? INFINITY : edges[g + 1] / T;
        if (lo >= ORC_PLANCK_SWITCH) {
            if (b) b[g] = orc_planck_Q(lo) - orc_planck_Q(hi);
            if (r) r[g] = orc_rosseland_RQ(lo) - orc_rosseland_RQ(hi);
        } else {
            if (b) b[g] = orc_planck_P(hi) - orc_planck_P(lo);
            if (r) r[g] = orc_rosseland_R(hi) - orc_rosseland_R(lo);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* O3. Opacity (Sec. 3, Rem. opacity: sigma_g piecewise constant from the   */
/* element-average temperature; Sec. 6.2 form alpha/nu^3 (1 - e^{-nu/T}))   */
/* ------------------------------------------------------------------------ */

/* kind 0: sigma_{g,K} = s_K * Tbar_K^{-3}                (gray power law)
 * kind 1: sigma_{g,K} = s_K * alpha (1 - exp(-E_g/Tbar_K)) / E_g^3 with E_g
 *         the geometric mean of the finite group edges.
 * Tbar_K is the mean of the nodal values (exact cell average for Y_1). */
void orc_opacity(int kind, double alpha, int G, const double *edges, int ncell, int nnode,
                 const double *T_nodal, const double *scale, double *sigma)
{
    for (int k = 0; k < ncell; ++k) {
        double tb = 0.0;
        for (int n = 0; n < nnode; ++n) tb += T_nodal[k * nnode + n];
        tb /= nnode;
        for (int g = 0; g < G; ++g) {
            double s;
            if (kind == 0) {
                s = scale[k] / (tb * tb * tb);
            } else {
                double eg = sqrt(edges[g] * edges[g + 1]);
                s = scale[k] * alpha * (1.0 - exp(-eg / tb)) / (eg * eg * eg);
            }
            sigma[(size_t)g * ncell + k] = s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* a1. Emission source (Eq. smm_be_transport right-hand side):              */
/*   q_{g,n} = sigma_g B_g(T_n) / 4pi,  B_g = a c T^4 b_g(T)  (Eq. planck)  */
/* evaluated at the nodes (lumped, Sec. 6 opening).                          */
/* ------------------------------------------------------------------------ */
void orc_emission(int G, const double *edges, double a, double c, int ncell, int nnode,
                  const double *T_nodal, const double *sigma, double *q)
{
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
    double *b = (double *)malloc(sizeof(double) * (G > 0 ? G : 1));
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
    for (int k = 0; k < ncell; ++k) {
        for (int n = 0; n < nnode; ++n) {
            double T = T_nodal[k * nnode + n];
            orc_group_spectra(G, edges, T, b, NULL);
            double B = a * c * T * T * T * T;
            for (int g = 0; g < G; ++g)
                q[((size_t)g * ncell + k) * nnode + n] =
                    sigma[(size_t)g * ncell + k] * B * b[g] / (4.0 * ORC_PI);
        }
    }
    free(b);
    }
}

/* Isotropic boundary inflow B_g(T_bdr)/4pi per side (Eq. transport BC);
 * T_bdr <= 0 means vacuum (zero inflow). */
void orc_inflow(int G, const double *edges, double a, double c, const double *T_bdr,
                double *inflow)
{
    double *b = (double *)malloc(sizeof(double) * (G > 0 ? G : 1));
    for (int s = 0; s < 4; ++s) {
        double T = T_bdr[s];
        if (!(T > 0.0)) {
            for (int g = 0; g < G; ++g) inflow[s * G + g] = 0.0;
            continue;
        }
        orc_group_spectra(G, edges, T, b, NULL);
        for (int g = 0; g < G; ++g)
            inflow[s * G + g] = a * c * T * T * T * T * b[g] / (4.0 * ORC_PI);
    }
    free(b);
}

/* ------------------------------------------------------------------------ */
/* a2. Upwind DG transport sweep (Sec. 3, Eqs. upwind and dgsn_transport),  */
/* all forms lumped with the tensor 2-point Gauss-Lobatto rule (Sec. 6).    */
/* ------------------------------------------------------------------------ */

/* 1D linear Lagrange basis on the reference interval [0,1] */
static double orc_phi(int a, double s) { return a ? s : 1.0 - s; }
static double orc_dphi(int a) { return a ? 1.0 : -1.0; }

/* Solve the n x n system A x = b in place by Gaussian elimination with
 * partial pivoting.  Returns 0, or -1 on a zero pivot. */
static int orc_solve_dense(int n, double *A, double *b)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
        if (A[p * n + k] == 0.0) return -1;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[k * n + j];
                A[k * n + j] = A[p * n + j];
                A[p * n + j] = t;
            }
            double t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double f = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * b[j];
        b[k] = s / A[k * n + k];
    }
    return 0;
}

typedef struct {
    int dim, nx, ny;
    double hx, hy;
} orc_mesh;

/* value of the DG expansion of cell (ix,iy) at reference point (s,t) */
static double orc_eval_cell(const orc_mesh *m, const double *Icell, double s, double t)
{
    double v = 0.0;
    if (m->dim == 1) {
        for (int a = 0; a < 2; ++a) v += Icell[a] * orc_phi(a, s);
    } else {
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) v += Icell[a + 2 * b] * orc_phi(a, s) * orc_phi(b, t);
    }
    return v;
}

/* One (d,g) sweep.  Ox, Oy: direction; sig_t: total sigma~ per cell;
 * src: lumped nodal right-hand side density q + I^k/(c dt) per cell/node;
 * inflow[4]: boundary inflow per side; out: I[cell][node]. */
static int orc_sweep_one(const orc_mesh *m, double Ox, double Oy, const double *sig_t,
                         const double *src, const double *inflow, double *out)
{
    const int nn = (m->dim == 1) ? 2 : 4;
    const int nx = m->nx, ny = m->ny;
    const double hx = m->hx, hy = m->hy;
    /* cells are visited in an upwind topological order */
    const int xs = (Ox > 0.0) ? 1 : -1;
    const int ys = (m->dim == 2 && Oy < 0.0) ? -1 : 1;
    double A[16], rhs[4];
    for (int jj = 0; jj < ny; ++jj) {
        int iy = (ys > 0) ? jj : ny - 1 - jj;
        for (int ii = 0; ii < nx; ++ii) {
            int ix = (xs > 0) ? ii : nx - 1 - ii;
            int k = iy * nx + ix;
            memset(A, 0, sizeof(A));
            memset(rhs, 0, sizeof(rhs));
            if (m->dim == 1) {
                /* volume terms at the two Lobatto points, weight h/2 */
                for (int qp = 0; qp < 2; ++qp) {
                    double s = (double)qp, W = 0.5 * hx;
                    for (int i = 0; i < 2; ++i) {
                        double ui = orc_phi(i, s), dui = orc_dphi(i) / hx;
                        rhs[i] += W * ui * orc_eval_cell(m, src + k * nn, s, 0.0);
                        for (int j = 0; j < 2; ++j) {
                            double uj = orc_phi(j, s);
                            A[i * 2 + j] += W * (-(Ox * dui) * uj + sig_t[k] * ui * uj);
                        }
                    }
                }
                /* faces: left (s=0, n=-1) and right (s=1, n=+1) */
                for (int f = 0; f < 2; ++f) {
                    double s = (double)f, nrm = f ? 1.0 : -1.0;
                    double On = Ox * nrm;
                    if (On > 0.0) {
                        for (int i = 0; i < 2; ++i)
                            for (int j = 0; j < 2; ++j)
                                A[i * 2 + j] += On * orc_phi(i, s) * orc_phi(j, s);
                    } else {
                        double Iup;
                        int nb = ix + (f ? 1 : -1);
                        if (nb < 0 || nb >= nx)
                            Iup = inflow[f ? 1 : 0];
                        else
                            Iup = orc_eval_cell(m, out + (iy * nx + nb) * nn, f ? 0.0 : 1.0, 0.0);
                        for (int i = 0; i < 2; ++i) rhs[i] -= On * orc_phi(i, s) * Iup;
                    }
                }
                if (orc_solve_dense(2, A, rhs)) return -1;
            } else {
                /* volume terms at the four Lobatto (corner) points, weight hx hy/4 */
                for (int qb = 0; qb < 2; ++qb)
                    for (int qa = 0; qa < 2; ++qa) {
                        double s = (double)qa, t = (double)qb, W = 0.25 * hx * hy;
                        double srcv = orc_eval_cell(m, src + k * nn, s, t);
                        for (int i = 0; i < 4; ++i) {
                            int ia = i & 1, ib = i >> 1;
                            double ui = orc_phi(ia, s) * orc_phi(ib, t);
                            double gx = orc_dphi(ia) * orc_phi(ib, t) / hx;
                            double gy = orc_phi(ia, s) * orc_dphi(ib) / hy;
                            rhs[i] += W * ui * srcv;
                            for (int j = 0; j < 4; ++j) {
                                double uj = orc_phi(j & 1, s) * orc_phi(j >> 1, t);
                                A[i * 4 + j] += W * (-(Ox * gx + Oy * gy) * uj + sig_t[k] * ui * uj);
                            }
                        }
                    }
                /* four faces, each with the 2-point Lobatto rule (weight len/2) */
                for (int f = 0; f < 4; ++f) {
                    double nxv = 0.0, nyv = 0.0, len;
                    if (f == 0) { nxv = -1.0; len = hy; }
                    else if (f == 1) { nxv = 1.0; len = hy; }
                    else if (f == 2) { nyv = -1.0; len = hx; }
                    else { nyv = 1.0; len = hx; }
                    double On = Ox * nxv + Oy * nyv;
                    for (int fp = 0; fp < 2; ++fp) {
                        double s, t;
                        if (f < 2) { s = (f == 1) ? 1.0 : 0.0; t = (double)fp; }
                        else { s = (double)fp; t = (f == 3) ? 1.0 : 0.0; }
                        double Wf = 0.5 * len;
                        if (On > 0.0) {
                            for (int i = 0; i < 4; ++i) {
                                double ui = orc_phi(i & 1, s) * orc_phi(i >> 1, t);
                                for (int j = 0; j < 4; ++j) {
                                    double uj = orc_phi(j & 1, s) * orc_phi(j >> 1, t);
                                    A[i * 4 + j] += Wf * On * ui * uj;
                                }
                            }
                        } else {
                            /* upwind neighbour trace at the same physical point */
                            int nbx = ix, nby = iy;
                            double ns = s, nt = t;
                            if (f == 0) { nbx = ix - 1; ns = 1.0; }
                            else if (f == 1) { nbx = ix + 1; ns = 0.0; }
                            else if (f == 2) { nby = iy - 1; nt = 1.0; }
                            else { nby = iy + 1; nt = 0.0; }
                            double Iup;
                            if (nbx < 0 || nbx >= nx || nby < 0 || nby >= ny)
                                Iup = inflow[f];
                            else
                                Iup = orc_eval_cell(m, out + (nby * nx + nbx) * nn, ns, nt);
                            for (int i = 0; i < 4; ++i) {
                                double ui = orc_phi(i & 1, s) * orc_phi(i >> 1, t);
                                rhs[i] -= Wf * On * ui * Iup;
                            }
                        }
                    }
                }
                if (orc_solve_dense(4, A, rhs)) return -1;
            }
            for (int n = 0; n < nn; ++n) out[k * nn + n] = rhs[n];
        }
    }
    return 0;
}

/* Sweep a list of (d,g) pairs (pairs[2*i] = d, pairs[2*i+1] = g), or all
 * pairs in order d-major when pairs == NULL (then npairs is ignored).
 *   sigma[g][cell]       multigroup opacity sigma_g (not sigma~)
 *   inv_cdt              1/(c dt); 0 gives the steady-state operator
 *   q[g][cell][node]     emission density
 *   I_prev               previous-time intensity I^k (NULL: zero), laid out
 *                        [d][g][cell][node], or [pair][cell][node] when
 *                        prev_per_pair is non-zero
 *   inflow[4][G]         boundary inflow per side and group
 *   out[pair][cell][node]
 * The time-edge source I^k/(c dt) and sigma~ = sigma + 1/(c dt) follow
 * Eq. smm_be_transport.  Returns 0, or -1 on a singular local system. */
int orc_sweep_pairs(int dim, int nx, int ny, double x0, double x1, double y0, double y1,
                    int ndir, const double *omx, const double *omy, int G, const double *sigma,
                    double inv_cdt, const double *q, const double *I_prev, int prev_per_pair,
                    const double *inflow, int npairs, const int *pairs, double *out, int nthreads)
{
    orc_mesh m;
    m.dim = dim;
    m.nx = nx;
    m.ny = (dim == 1) ? 1 : ny;
    m.hx = (x1 - x0) / nx;
    m.hy = (dim == 1) ? 1.0 : (y1 - y0) / ny;
    const int nn = (dim == 1) ? 2 : 4;
    const size_t ncell = (size_t)m.nx * m.ny;
    const int np = pairs ? npairs : ndir * G;
    int err = 0;
#ifdef _OPENMP
    /* nthreads > 0 limits this call only (num_threads clause) */
    const int nth = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err) num_threads(nth)
#endif
    for (int pi = 0; pi < np; ++pi) {
        int d = pairs ? pairs[2 * pi] : pi / G;
        int g = pairs ? pairs[2 * pi + 1] : pi % G;
        double *sig_t = (double *)malloc(sizeof(double) * ncell);
        double *src = (double *)malloc(sizeof(double) * ncell * nn);
        for (size_t k = 0; k < ncell; ++k) {
            sig_t[k] = sigma[(size_t)g * ncell + k] + inv_cdt;
            for (int n = 0; n < nn; ++n) {
                double ip = 0.0;
                if (I_prev && prev_per_pair)
                    ip = I_prev[((size_t)pi * ncell + k) * nn + n];
                else if (I_prev)
                    ip = I_prev[(((size_t)d * G + g) * ncell + k) * nn + n];
                src[k * nn + n] = q[((size_t)g * ncell + k) * nn + n] + inv_cdt * ip;
            }
        }
        double infl[4];
        for (int s = 0; s < 4; ++s) infl[s] = inflow[s * G + g];
        err |= orc_sweep_one(&m, omx[d], (dim == 1) ? 0.0 : omy[d], sig_t, src, infl,
                             out + (size_t)pi * ncell * nn) ? 1 : 0;
        free(sig_t);
        free(src);
    }
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* a3. Angular moments (Sec. 2: E, F, the SM tensor T, and the collapse      */
/* numerators sum_g sigma_g E_g, sum_g sigma_g F_g of Eqs. sigmaE and        */
/* additive_mg_correction), with compensated (Kahan) sums.                   */
/*   2D, per node: [phi, Fx, Fy, Txx, Txy, Tyy, SE, SFx, SFy]               */
/*   1D, per node: [phi, F, T, SE, SF]                                       */
/* phi = sum w I = c E;  T = sum w (Omega Omega - I/3) I (in-plane block);   */
/* SE = sum_g sigma_g sum_d w I;  SF = sum_g sigma_g sum_d w Omega I.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    double s, c;
} orc_kahan;
static void orc_kadd(orc_kahan *k, double v)
{
    double y = v - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

void orc_moments(int dim, int ncell, int ndir, const double *omx, const double *omy,
                 const double *w, int G, const double *sigma, const double *I, double *mom)
{
    const int nn = (dim == 1) ? 2 : 4;
    const int nm = (dim == 1) ? 5 : 9;
    /* cells are independent: the threads split them, each sum keeps its order */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int k = 0; k < ncell; ++k) {
        for (int n = 0; n < nn; ++n) {
            orc_kahan acc[9];
            memset(acc, 0, sizeof(acc));
            for (int g = 0; g < G; ++g) {
                double sg = sigma[(size_t)g * ncell + k];
                for (int d = 0; d < ndir; ++d) {
                    double v = I[(((size_t)d * G + g) * ncell + k) * nn + n];
                    double wi = w[d] * v;
                    double ox = omx[d];
                    if (dim == 1) {
                        orc_kadd(&acc[0], wi);
                        orc_kadd(&acc[1], wi * ox);
                        orc_kadd(&acc[2], wi * (ox * ox - 1.0 / 3.0));
                        orc_kadd(&acc[3], sg * wi);
                        orc_kadd(&acc[4], sg * wi * ox);
                    } else {
                        double oy = omy[d];
                        orc_kadd(&acc[0], wi);
                        orc_kadd(&acc[1], wi * ox);
                        orc_kadd(&acc[2], wi * oy);
                        orc_kadd(&acc[3], wi * (ox * ox - 1.0 / 3.0));
                        orc_kadd(&acc[4], wi * ox * oy);
                        orc_kadd(&acc[5], wi * (oy * oy - 1.0 / 3.0));
                        orc_kadd(&acc[6], sg * wi);
                        orc_kadd(&acc[7], sg * wi * ox);
                        orc_kadd(&acc[8], sg * wi * oy);
                    }
                }
            }
            for (int i = 0; i < nm; ++i) mom[((size_t)k * nn + n) * nm + i] = acc[i].s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* a4. Closures for the gray low-order system (Sec. 2: Eqs. sigmaE, sigmaF,  */
/* the Planck-collapsed sigma_P, the additive correction                     */
/* sum_g (sigma_F - sigma_g) F_g, the tensor T; Eq. alpha).  Gray opacities  */
/* are nodal (Rem. opacity); the spectra use the nodal temperature.          */
/*   2D out per node: [E, Fx, Fy, Txx, Txy, Tyy, sigE, sigF, sigP, Cx, Cy]   */
/*   1D out per node: [E, F, T, sigE, sigF, sigP, C]                         */
/* sigma_E = SE/phi is a mean of the positive group opacities weighted by   */
/* the group energies; where phi <= 0 or SE <= 0 (the lumped DG intensity,  */
/* with no positivity fix-up, can dip below zero) it is not defined and     */
/* falls back to sigma_P.                                                   */
/* ------------------------------------------------------------------------ */
void orc_closures(int dim, int ncell, int G, const double *edges, double c, const double *sigma,
                  const double *T_nodal, const double *mom, double *out)
{
    const int nn = (dim == 1) ? 2 : 4;
    const int nm = (dim == 1) ? 5 : 9;
    const int no = (dim == 1) ? 7 : 11;
    double *b = (double *)malloc(sizeof(double) * (G > 0 ? G : 1));
    double *r = (double *)malloc(sizeof(double) * (G > 0 ? G : 1));
    for (int k = 0; k < ncell; ++k) {
        for (int n = 0; n < nn; ++n) {
            const double *mm = mom + ((size_t)k * nn + n) * nm;
            double *o = out + ((size_t)k * nn + n) * no;
            double T = T_nodal[k * nn + n];
            orc_group_spectra(G, edges, T, b, r);
            double nb = 0.0, db = 0.0, nr = 0.0, dr = 0.0;
            for (int g = 0; g < G; ++g) {
                double sg = sigma[(size_t)g * ncell + k];
                nb += b[g] * sg;
                db += b[g];
                nr += r[g] * sg;
                dr += r[g];
            }
            double sP = nb / db, sF = nr / dr;
            double phi = mm[0];
            double SE = mm[dim == 1 ? 3 : 6];
            double sE = (phi > 0.0 && SE > 0.0) ? SE / phi : sP;
            if (dim == 1) {
                o[0] = phi / c;
                o[1] = mm[1];
                o[2] = mm[2];
                o[3] = sE;
                o[4] = sF;
                o[5] = sP;
                o[6] = sF * mm[1] - mm[4];
            } else {
                o[0] = phi / c;
                o[1] = mm[1];
                o[2] = mm[2];
                o[3] = mm[3];
                o[4] = mm[4];
                o[5] = mm[5];
                o[6] = sE;
                o[7] = sF;
                o[8] = sP;
                o[9] = sF * mm[1] - mm[7];
                o[10] = sF * mm[2] - mm[8];
            }
        }
    }
    free(b);
    free(r);
}

/* alpha = sum_d w_d |Omega_d . n| / sum_d w_d (Eq. alpha) for n = x-hat. */
double orc_alpha(int ndir, const double *omx, const double *w)
{
    double s = 0.0, sw = 0.0;
    for (int d = 0; d < ndir; ++d) {
        s += w[d] * fabs(omx[d]);
        sw += w[d];
    }
    return s / sw;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
