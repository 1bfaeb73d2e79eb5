// FP64 Planck / Rosseland group integrals and the kernels built on them:
// multigroup opacity, emission source (row a1), boundary inflow and the
// closures recomputed from a temperature (row a4 standalone).
//
// P(x) = (15/pi^4) int_0^x t^3/(e^t-1) dt is evaluated with the two series
// used by Clark (Sec. 2, Eq. planck and the b_g definition):
//   x <  2: x^3/3 - x^4/8 + sum_k B_2k x^(2k+3) / ((2k)! (2k+3))
//   x >= 2: 1 - (15/pi^4) sum_n e^{-nx} (x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4)
// and the Rosseland integral by parts, R(x) = P(x) - (15/4pi^4) x^4/(e^x-1),
// which gives r_g with dB_g/dT = 4 a c T^3 r_g (Sec. 2); for x < 2 the factor
// x/(e^x-1) is the Bernoulli generating series itself.  A group whose lower
// reduced edge is in the tail branch is differenced in tails (1 - P) to keep
// relative accuracy; the lowest edge is 0 and the highest infinity so that
// sum_g b_g = 1.
#include <math.h>

#include "sm_internal.cuh"

namespace smk {

constexpr int NBERN = 18;   // head terms: (2/2pi)^36 < 1e-17
constexpr int NTAIL = 24;   // tail terms: e^{-2*24} ~ 1e-21
constexpr double XSWITCH = 2.0;
constexpr double PI_D = 3.14159265358979323846;
constexpr double C15 = 15.0 / (PI_D * PI_D * PI_D * PI_D);

// d_k = (B_2k/(2k)!) / (2k+3), k = 1..NBERN, from B_2k/(2k)! =
// (-1)^(k+1) 2 zeta(2k) / (2 pi)^(2k); zeta(2k) summed directly with an
// Euler-Maclaurin tail (k >= 2) and zeta(2) = pi^2/6.
__constant__ double c_head[NBERN];
__constant__ double c_bern[NBERN];   // B_2k/(2k)!, k = 1..NBERN
__constant__ double c_inv_n[NTAIL][4];

static bool g_tables_ready[128] = {false};

void planck_upload_tables(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return;
    if (g_tables_ready[dev]) return;
    double head[NBERN], bern[NBERN];
    for (int k = 1; k <= NBERN; ++k) {
        const int s = 2 * k;
        double zeta;
        if (k == 1) {
            zeta = PI_D * PI_D / 6.0;
        } else {
            const int N = 2000;
            double acc = 0.0;
            for (int n = N; n >= 1; --n) acc += pow((double)n, -s);
            // tail sum_{n>N} n^-s ~ N^(1-s)/(s-1) - N^-s/2 + s N^(-s-1)/12
            acc += pow((double)N, 1 - s) / (s - 1) - 0.5 * pow((double)N, -s) +
                   s * pow((double)N, -s - 1) / 12.0;
            zeta = acc;
        }
        double bk = 2.0 * zeta / pow(2.0 * PI_D, s);
        if (k % 2 == 0) bk = -bk;
        head[k - 1] = bk / (2.0 * k + 3.0);
        bern[k - 1] = bk;
    }
    double invn[NTAIL][4];
    for (int n = 1; n <= NTAIL; ++n) {
        double r = 1.0 / n;
        invn[n - 1][0] = r;
        invn[n - 1][1] = r * r;
        invn[n - 1][2] = r * r * r;
        invn[n - 1][3] = r * r * r * r;
    }
    if (cudaMemcpyToSymbol(c_head, head, sizeof(head)) == cudaSuccess &&
        cudaMemcpyToSymbol(c_bern, bern, sizeof(bern)) == cudaSuccess &&
        cudaMemcpyToSymbol(c_inv_n, invn, sizeof(invn)) == cudaSuccess)
        g_tables_ready[dev] = true;
}

// Values of the cumulative spectra at one reduced edge x = nu/T.
struct EdgeVals {
    double P, Q;   // P(x), 1 - P(x)
    double R, RQ;  // R(x), 1 - R(x)
    bool tail;     // x in the tail branch
};

__device__ __forceinline__ EdgeVals edge_vals(double x) {
    EdgeVals e;
    if (!(x > 0.0)) {
        e.P = 0.0; e.Q = 1.0; e.R = 0.0; e.RQ = 1.0; e.tail = false;
        return e;
    }
    if (isinf(x)) {
        e.P = 1.0; e.Q = 0.0; e.R = 1.0; e.RQ = 0.0; e.tail = true;
        return e;
    }
    if (x < XSWITCH) {
        const double y = x * x;
        double poly = c_head[NBERN - 1], pb = c_bern[NBERN - 1];
#pragma unroll
        for (int k = NBERN - 2; k >= 0; --k) {
            poly = fma(poly, y, c_head[k]);
            pb = fma(pb, y, c_bern[k]);
        }
        poly *= y;
        pb *= y;
        const double x3 = y * x;
        const double s = x3 * ((1.0 / 3.0) - 0.125 * x + poly);
        e.P = C15 * s;
        e.Q = 1.0 - e.P;
        // x^4/(e^x - 1) = x^3 * x/(e^x - 1), with x/(e^x - 1) = 1 - x/2 + sum B_2k x^2k/(2k)!
        const double rx = 0.25 * C15 * x3 * (1.0 - 0.5 * x + pb);
        e.R = e.P - rx;
        e.RQ = e.Q + rx;
        e.tail = false;
        return e;
    }
    const double e1 = exp(-x);
    const int nmax = min(NTAIL, (int)(40.0 / x) + 2);
    double en = 1.0, sum = 0.0;
    const double x2 = x * x, x3 = x2 * x, x2_3 = 3.0 * x2, x_6 = 6.0 * x;
    for (int n = 0; n < nmax; ++n) {
        en *= e1;
        const double t = fma(x3, c_inv_n[n][0],
                             fma(x2_3, c_inv_n[n][1], fma(x_6, c_inv_n[n][2], 6.0 * c_inv_n[n][3])));
        sum = fma(en, t, sum);
    }
    e.Q = C15 * sum;
    e.P = 1.0 - e.Q;
    const double rx = 0.25 * C15 * (x2 * x2) * e1 / (1.0 - e1);
    e.R = e.P - rx;
    e.RQ = e.Q + rx;
    e.tail = true;
    return e;
}

// b_g and r_g of the group between reduced edges lo < hi
__device__ __forceinline__ void group_br(const EdgeVals &lo, const EdgeVals &hi, double &b,
                                         double &r) {
    if (lo.tail) {
        b = lo.Q - hi.Q;
        r = lo.RQ - hi.RQ;
    } else {
        b = hi.P - lo.P;
        r = hi.R - lo.R;
    }
}

// ---------------------------------------------------------------------------
// Opacity: one thread per cell.
__global__ void opacity_kernel(int ncell, int nn, int G, int kind, double alpha,
                               const double *__restrict__ edges, const double *__restrict__ T,
                               const double *__restrict__ scale, double *__restrict__ sigma,
                               unsigned int *ctrl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncell) return;
    double tb = 0.0;
    for (int n = 0; n < nn; ++n) tb += T[(size_t)k * nn + n];
    tb /= nn;
    if (!(tb > 0.0) || !isfinite(tb)) atomicOr(ctrl + CTRL_STATUS, ST_NONPHYSICAL);
    const double s = scale[k];
    if (kind == SM_OPACITY_POWER) {
        const double v = s / (tb * tb * tb);
        for (int g = 0; g < G; ++g) sigma[(size_t)g * ncell + k] = v;
    } else {
        for (int g = 0; g < G; ++g) {
            const double eg = sqrt(edges[g] * edges[g + 1]);
            sigma[(size_t)g * ncell + k] = s * alpha * (-expm1(-eg / tb)) / (eg * eg * eg);
        }
    }
}

// ---------------------------------------------------------------------------
// Emission (row a1): one thread per (cell, node), walking the group edges once.
// Writes the sweep's source records src[cell][g][8] = {q at the nodes (unused
// node slots 0), sigma~, sigma, 0, 0} in the sweep precision; padding groups
// get no source and sigma~ = 1.
template <typename RT>
__global__ void emission_kernel(int ncell, int nn, int G, int Gp, const double *__restrict__ edges,
                                double acT4_scale, double inv_cdt, const double *__restrict__ T,
                                const double *__restrict__ sigma, RT *__restrict__ src,
                                double *__restrict__ gray, double *__restrict__ qcanon,
                                unsigned int *ctrl) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell * nn) return;
    const int cell = t / nn, node = t - cell * nn;
    double Tn = T[t];
    if (!(Tn > 0.0) || !isfinite(Tn)) {
        atomicOr(ctrl + CTRL_STATUS, ST_NONPHYSICAL);
    }
    const double B4 = acT4_scale * Tn * Tn * Tn * Tn;  // a c T^4 / 4 pi
    const double invT = 1.0 / Tn;
    EdgeVals lo = edge_vals(0.0);
    double nb = 0.0, db = 0.0, nr = 0.0, dr = 0.0;
    RT *rec0 = src + (size_t)cell * Gp * 8;
    for (int g = 0; g < G; ++g) {
        const double xhi = (g == G - 1) ? INFINITY : edges[g + 1] * invT;
        // beyond x ~ 745 the tails 1 - P and 1 - R underflow to exactly 0, so
        // every higher group has b = r = 0: skip their series
        const EdgeVals hi = (lo.tail && lo.Q == 0.0 && lo.RQ == 0.0) ? lo : edge_vals(xhi);
        double b, r;
        group_br(lo, hi, b, r);
        const double sg = sigma[(size_t)g * ncell + cell];
        nb = fma(b, sg, nb);
        db += b;
        nr = fma(r, sg, nr);
        dr += r;
        const double qv = sg * b * B4;
        RT *rec = rec0 + (size_t)g * 8;
        rec[node] = (RT)qv;
        if (qcanon) qcanon[((size_t)g * ncell + cell) * nn + node] = qv;
        if (node == 0) {
            for (int n = nn; n < 4; ++n) rec[n] = (RT)0;
            rec[4] = (RT)(sg + inv_cdt);
            rec[5] = (RT)sg;
            rec[6] = (RT)0;
            rec[7] = (RT)0;
        }
        lo = hi;
    }
    for (int g = G; g < Gp; ++g) {  // padding groups: no source, unit sigma~
        RT *rec = rec0 + (size_t)g * 8;
        rec[node] = (RT)0;
        if (node == 0) {
            for (int n = nn; n < 4; ++n) rec[n] = (RT)0;
            rec[4] = (RT)1;
            rec[5] = (RT)0;
            rec[6] = (RT)0;
            rec[7] = (RT)0;
        }
    }
    gray[(size_t)t * 2 + 0] = nb / db;
    gray[(size_t)t * 2 + 1] = nr / dr;
}

// Boundary inflow B_g(T_bdr)/4pi per side (Eq. transport boundary condition).
template <typename RT>
__global__ void inflow_kernel(int G, int Gp, const double *__restrict__ edges, double ac4pi,
                              double T0, double T1, double T2, double T3, RT *__restrict__ out) {
    const int s = threadIdx.x;
    if (s >= 4) return;
    const double Tb = (s == 0) ? T0 : (s == 1) ? T1 : (s == 2) ? T2 : T3;
    if (!(Tb > 0.0)) {
        for (int g = 0; g < Gp; ++g) out[s * Gp + g] = (RT)0;
        return;
    }
    const double B4 = ac4pi * Tb * Tb * Tb * Tb;
    EdgeVals lo = edge_vals(0.0);
    for (int g = 0; g < G; ++g) {
        const double xhi = (g == G - 1) ? INFINITY : edges[g + 1] / Tb;
        const EdgeVals hi = edge_vals(xhi);
        double b, r;
        group_br(lo, hi, b, r);
        out[s * Gp + g] = (RT)(B4 * b);
        lo = hi;
    }
    for (int g = G; g < Gp; ++g) out[s * Gp + g] = (RT)0;
}

// Closures from moments and a temperature (row a4, standalone form).
__global__ void closures_T_kernel(int dim, int ncell, int nn, int G, double inv_c,
                                  const double *__restrict__ edges, const double *__restrict__ mom,
                                  const double *__restrict__ T, const double *__restrict__ sigma,
                                  double *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell * nn) return;
    const int cell = t / nn;
    const double Tn = T[t];
    const double invT = 1.0 / Tn;
    EdgeVals lo = edge_vals(0.0);
    double nb = 0.0, db = 0.0, nr = 0.0, dr = 0.0;
    for (int g = 0; g < G; ++g) {
        const double xhi = (g == G - 1) ? INFINITY : edges[g + 1] * invT;
        const EdgeVals hi = edge_vals(xhi);
        double b, r;
        group_br(lo, hi, b, r);
        const double sg = sigma[(size_t)g * ncell + cell];
        nb = fma(b, sg, nb);
        db += b;
        nr = fma(r, sg, nr);
        dr += r;
        lo = hi;
    }
    const double sP = nb / db, sF = nr / dr;
    if (dim == 1) {
        const double *m = mom + (size_t)t * 5;
        double *o = out + (size_t)t * 7;
        const double phi = m[0];
        o[0] = phi * inv_c;
        o[1] = m[1];
        o[2] = m[2];
        o[3] = (phi != 0.0) ? m[3] / phi : sP;
        o[4] = sF;
        o[5] = sP;
        o[6] = sF * m[1] - m[4];
    } else {
        const double *m = mom + (size_t)t * 9;
        double *o = out + (size_t)t * 11;
        const double phi = m[0];
        o[0] = phi * inv_c;
        o[1] = m[1];
        o[2] = m[2];
        o[3] = m[3];
        o[4] = m[4];
        o[5] = m[5];
        o[6] = (phi != 0.0) ? m[6] / phi : sP;
        o[7] = sF;
        o[8] = sP;
        o[9] = sF * m[1] - m[7];
        o[10] = sF * m[2] - m[8];
    }
}

// ---------------------------------------------------------------------------
cudaError_t launch_opacity(const sm_problem *p, const double *T, const double *scale,
                           double *sigma, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (p->ncell + threads - 1) / threads;
    opacity_kernel<<<blocks, threads, 0, s>>>(p->ncell, p->nn, p->G, p->desc.opacity_kind,
                                              p->desc.opacity_alpha, p->d_edges, T, scale, sigma,
                                              p->d_ctrl);
    return cudaGetLastError();
}

cudaError_t launch_emission(const sm_problem *p, const double *T, const double *sigma,
                            double *q_canon, cudaStream_t s) {
    const int threads = 128;
    const int n = p->ncell * p->nn;
    const int blocks = (n + threads - 1) / threads;
    const double scale = p->desc.a * p->desc.c / (4.0 * PI_D);
    if (p->prec == 32)
        emission_kernel<float><<<blocks, threads, 0, s>>>(
            p->ncell, p->nn, p->G, p->Gp, p->d_edges, scale, p->inv_cdt, T, sigma,
            (float *)p->d_src, p->d_gray, q_canon, p->d_ctrl);
    else
        emission_kernel<double><<<blocks, threads, 0, s>>>(
            p->ncell, p->nn, p->G, p->Gp, p->d_edges, scale, p->inv_cdt, T, sigma,
            (double *)p->d_src, p->d_gray, q_canon, p->d_ctrl);
    return cudaGetLastError();
}

cudaError_t launch_inflow(const sm_problem *p, cudaStream_t s) {
    const double sc = p->desc.a * p->desc.c / (4.0 * PI_D);
    const double *Tb = p->desc.T_bdr;
    if (p->prec == 32)
        inflow_kernel<float><<<1, 32, 0, s>>>(p->G, p->Gp, p->d_edges, sc, Tb[0], Tb[1], Tb[2],
                                               Tb[3], (float *)p->d_inflow);
    else
        inflow_kernel<double><<<1, 32, 0, s>>>(p->G, p->Gp, p->d_edges, sc, Tb[0], Tb[1], Tb[2],
                                                Tb[3], (double *)p->d_inflow);
    return cudaGetLastError();
}

cudaError_t launch_closures_from_T(const sm_problem *p, const double *mom, const double *T,
                                   const double *sigma, double *out, cudaStream_t s) {
    const int threads = 128;
    const int n = p->ncell * p->nn;
    closures_T_kernel<<<(n + threads - 1) / threads, threads, 0, s>>>(
        p->dim, p->ncell, p->nn, p->G, 1.0 / p->desc.c, p->d_edges, mom, T, sigma, out);
    return cudaGetLastError();
}

}  // namespace smk
