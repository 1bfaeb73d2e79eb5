// FP64 Planck / Rosseland group integrals and the kernels built on them:
// multigroup opacity, emission source (row a1), boundary inflow and the
// closures recomputed from a temperature (row a4 standalone).
//
// P(x) = (15/pi^4) int_0^x t^3/(e^t-1) dt rests on the two series used by
// Clark (Sec. 2, Eq. planck and the b_g definition):
//   small x: x^3/3 - x^4/8 + sum_k B_2k x^(2k+3) / ((2k)! (2k+3))
//   large x: 1 - (15/pi^4) sum_n e^{-nx} (x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4)
// and the Rosseland integral by parts, R(x) = P(x) - (15/4pi^4) x^4/(e^x-1),
// which gives r_g with dB_g/dT = 4 a c T^3 r_g (Sec. 2); for small x the
// factor x/(e^x-1) is the Bernoulli generating series itself.  The GPU takes
// the first series for x < 1, the first term of the second for x >= 37 (the
// next is below double rounding), and in between, where both series need the
// most terms, degree-6 Taylor expansions about the nearest of the centres 1,
// 1 + 1/32, ..., 37 (|x - c| <= 1/64), whose coefficients the host derives
// once from P'(x) = (15/pi^4) x^3/(e^x - 1) in extended precision.  A group
// whose lower reduced edge is at or above the switch near x = 2 is differenced
// in tails (1 - P) to keep relative accuracy; the lowest edge is 0 and the
// highest infinity so that sum_g b_g = 1.
#include <math.h>

#include <atomic>

#include "sm_internal.cuh"

namespace smk {

constexpr int NBERN = 18;   // head terms: (2/2pi)^36 < 1e-17
// from x = 37 on, e^{-x} < 1e-16: the tail series keeps its first term only
constexpr double XCLOSED = 37.0;
constexpr double PI_D = 3.14159265358979323846;
constexpr double C15 = 15.0 / (PI_D * PI_D * PI_D * PI_D);

// d_k = (B_2k/(2k)!) / (2k+3), k = 1..NBERN, from B_2k/(2k)! =
// (-1)^(k+1) 2 zeta(2k) / (2 pi)^(2k); zeta(2k) summed directly with an
// Euler-Maclaurin tail (k >= 2) and zeta(2) = pi^2/6.
__constant__ double c_head[NBERN];
__constant__ double c_bern[NBERN];   // B_2k/(2k)!, k = 1..NBERN
// e^{-x} by the table-driven method of Tang (ACM TOMS 15, 1989): 64/ln2, and
// ln2/64 split into a 32-bit high part (exact products with the step index)
// and the rounded remainder; the table holds 2^{-j/64}, j = 0..63.
__constant__ double c_exp[3];
__device__ double g_exp2_tab[64];
// Taylor tables: centre j at c_j = XT0 + j/TSTEP; per centre two series of
// NTAY coefficients in h = x - c_j, (P, R) for c_j < 2 and (1 - P, 1 - R) for
// c_j >= 2 (so that the tails keep their relative accuracy).
constexpr double XT0 = 1.0, XT1 = 37.0;
constexpr int TSTEP = 32;  // centres per unit of x
constexpr int NCEN = 1153;  // (XT1 - XT0) * TSTEP + 1
constexpr int NTAY = 7;    // remainder (1/64 / 2pi)^7 < 1e-18 of the leading term
constexpr int JSW = 32;    // centres j < JSW lie below x = 2: P, R; from there on 1 - P, 1 - R
static_assert(XT1 == XCLOSED, "the Taylor tables end where the one-term tail takes over");
__device__ double g_ptab[NCEN][2][NTAY];
__device__ double g_pcen[NCEN];

// Taylor coefficients of the tables, in long double.  With E(h) = e^{c+h} - 1,
// g = 1/E, f = (c+h)^3 g and F4 = (c+h) f as power series in h:
// P(c+h) = P(c) + (15/pi^4) sum_k f_k h^{k+1}/(k+1), and
// R = P - (15/(4 pi^4)) F4; P(c) = 1 - Q(c) with Q(c) from the exponential
// series (all its terms, to e^{-200 c}).
static void planck_taylor_tables(double out[NCEN][2][NTAY]) {
    typedef long double LD;
    const LD PI = 3.141592653589793238462643383279502884L;
    const LD C = 15.0L / (PI * PI * PI * PI);
    for (int j = 0; j < NCEN; ++j) {
        const LD c = (LD)XT0 + (LD)j / TSTEP;
        LD Q = 0.0L;
        for (int n = 200; n >= 1; --n) {
            const LD m = n;
            Q += expl(-m * c) * (c * c * c / m + 3.0L * c * c / (m * m) + 6.0L * c / (m * m * m) +
                                 6.0L / (m * m * m * m));
        }
        Q *= C;
        LD E[NTAY + 1], g[NTAY + 1], f[NTAY + 1], F4[NTAY + 1];
        const LD ec = expl(c);
        LD fact = 1.0L;
        for (int k = 0; k <= NTAY; ++k) {
            if (k) fact *= k;
            E[k] = ec / fact;
        }
        E[0] = expm1l(c);
        for (int k = 0; k <= NTAY; ++k) {
            LD acc = (k == 0) ? 1.0L : 0.0L;
            for (int i = 1; i <= k; ++i) acc -= E[i] * g[k - i];
            g[k] = acc / E[0];
        }
        const LD a[4] = {c * c * c, 3.0L * c * c, 3.0L * c, 1.0L};
        for (int k = 0; k <= NTAY; ++k) {
            LD acc = 0.0L;
            for (int i = 0; i <= 3 && i <= k; ++i) acc += a[i] * g[k - i];
            f[k] = acc;
        }
        for (int k = 0; k <= NTAY; ++k) F4[k] = c * f[k] + (k ? f[k - 1] : 0.0L);
        LD pk[NTAY], rk[NTAY];
        pk[0] = 1.0L - Q;
        for (int k = 1; k < NTAY; ++k) pk[k] = C * f[k - 1] / k;
        for (int k = 0; k < NTAY; ++k) rk[k] = pk[k] - 0.25L * C * F4[k];
        const bool tail = j >= JSW;
        for (int k = 0; k < NTAY; ++k) {
            if (!tail) {
                out[j][0][k] = (double)pk[k];
                out[j][1][k] = (double)rk[k];
            } else if (k == 0) {
                out[j][0][0] = (double)Q;
                out[j][1][0] = (double)(Q + 0.25L * C * F4[0]);
            } else {
                out[j][0][k] = (double)-pk[k];
                out[j][1][k] = (double)-rk[k];
            }
        }
    }
}

// set once a device has its tables; two threads uploading at once write the same data
static std::atomic<bool> g_tables_ready[128];

void planck_upload_tables(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return;
    if (g_tables_ready[dev].load(std::memory_order_acquire)) return;
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
    const long double ln2 = 0.693147180559945309417232121458176568L;
    const long double l64 = ln2 / 64.0L;
    int ex = 0;
    frexp((double)l64, &ex);
    const double l64_hi = ldexp(floor(ldexp((double)l64, 32 - ex)), ex - 32);
    const double cexp[3] = {(double)(64.0L / ln2), l64_hi, (double)(l64 - (long double)l64_hi)};
    double tab[64];
    for (int j = 0; j < 64; ++j) tab[j] = (double)exp2l(-(long double)j / 64.0L);
    static double ptab[NCEN][2][NTAY];
    planck_taylor_tables(ptab);
    double pcen[NCEN];
    for (int j = 0; j < NCEN; ++j) pcen[j] = XT0 + (double)j / TSTEP;
    if (cudaMemcpyToSymbol(c_head, head, sizeof(head)) == cudaSuccess &&
        cudaMemcpyToSymbol(c_bern, bern, sizeof(bern)) == cudaSuccess &&
        cudaMemcpyToSymbol(c_exp, cexp, sizeof(cexp)) == cudaSuccess &&
        cudaMemcpyToSymbol(g_exp2_tab, tab, sizeof(tab)) == cudaSuccess &&
        cudaMemcpyToSymbol(g_ptab, ptab, sizeof(ptab)) == cudaSuccess &&
        cudaMemcpyToSymbol(g_pcen, pcen, sizeof(pcen)) == cudaSuccess)
        g_tables_ready[dev].store(true, std::memory_order_release);
}

// Values of the cumulative spectra at one reduced edge x = nu/T, in the form
// the group differences need: below the switch (tail false) v = P(x),
// rv = R(x); from the switch on (tail true) v = 1 - P(x), rv = 1 - R(x), which
// keeps the relative accuracy of the tails.  The switch sits at x = 2 (the
// first table centre at or above it takes the tail form, so inside the table
// it falls at 2 - 1/32); tail is non-decreasing in x.
struct EdgeVals {
    double v, rv;
    bool tail;
};

// Terms of the head series (x < 1) for a truncation error below 2^-56 of its
// leading term, decided in FP32 on xf (a count only needs to be large enough,
// and FP64 compares are scarce on this GPU).
__device__ __forceinline__ bool in_taylor(float xf) {
    return xf >= (float)XT0 && xf < (float)XT1;
}
__device__ __forceinline__ int head_terms(float xf) {
    return xf <= 0.25f ? 6 : xf <= 0.5f ? 7 : xf <= 1.0f ? 10 : xf <= 1.5f ? 14 : NBERN;
}

// e^{-x} for 0 <= x < 708 (normal results): x = N ln2/64 + r with
// N = round(64 x/ln2) and |r| <= ln2/128, so e^{-x} = 2^{-(N>>6)} 2^{-(N&63)/64}
// e^{-r}, with e^{-r} by its degree-6 Taylor polynomial (remainder below
// |r|^7/7! < 2e-20).  About two thirds of the FP64 work of exp() here.
__device__ __forceinline__ double exp_neg(double x) {
    const double Nd = rint(x * c_exp[0]);
    const double s = fma(Nd, c_exp[2], fma(Nd, c_exp[1], -x));  // -r
    const int n = (int)Nd;
    double p = fma(s, 1.0 / 720.0, 1.0 / 120.0);
    p = fma(p, s, 1.0 / 24.0);
    p = fma(p, s, 1.0 / 6.0);
    p = fma(p, s, 0.5);
    p = fma(p, s, 1.0);
    p = fma(p, s, 1.0);
    const double scale = __longlong_as_double((long long)(1023 - (n >> 6)) << 52);
    return __ldg(&g_exp2_tab[n & 63]) * p * scale;
}

// K: head-series terms to use (at least head_terms(xf)); callers that keep a
// warp converged pass the warp maximum, so that every lane reads the same
// coefficient at each step.  xf: x rounded to FP32 or computed in FP32 (it
// only steers branches and term counts, which have margin for its relative
// error below 1e-6).
__device__ __forceinline__ EdgeVals edge_vals(double x, float xf, int K) {
    EdgeVals e;
    if (!(xf > 0.0f)) {  // x = 0: P = R = 0
        e.v = 0.0; e.rv = 0.0; e.tail = false;
        return e;
    }
    if (isinf(xf)) {     // x = infinity: 1 - P = 1 - R = 0
        e.v = 0.0; e.rv = 0.0; e.tail = true;
        return e;
    }
    if (in_taylor(xf)) {
        const int j = __float2int_rn((xf - (float)XT0) * (float)TSTEP);  // nearest centre
        const double h = x - __ldg(&g_pcen[j]);
        const double *t = &g_ptab[j][0][0];
        double a = __ldg(t + NTAY - 1), b = __ldg(t + 2 * NTAY - 1);
#pragma unroll
        for (int k = NTAY - 2; k >= 0; --k) {
            a = fma(a, h, __ldg(t + k));
            b = fma(b, h, __ldg(t + NTAY + k));
        }
        e.v = a; e.rv = b; e.tail = j >= JSW;  // the table holds the same forms
        return e;
    }
    if (xf < (float)XT0) {
        // head series: P = (15/pi^4) (x^3/3 - x^4/8 + sum d_k x^(2k+3)), and
        // x^4/(e^x - 1) = x^3 (1 - x/2 + sum B_2k x^2k/(2k)!)
        const double y = x * x;
        double poly = c_head[K - 1], pb = c_bern[K - 1];
        for (int k = K - 2; k >= 0; --k) {
            poly = fma(poly, y, c_head[k]);
            pb = fma(pb, y, c_bern[k]);
        }
        poly *= y;
        pb *= y;
        const double x3 = y * x;
        const double P = C15 * (x3 * ((1.0 / 3.0) - 0.125 * x + poly));
        e.v = P;
        e.rv = P - 0.25 * C15 * x3 * (1.0 - 0.5 * x + pb);
        e.tail = false;
        return e;
    }
    // x >= 37: only the n = 1 term of the tail series is above double rounding,
    // 1 - P = (15/pi^4) e^{-x} (x^3 + 3x^2 + 6x + 6), and 1/(1 - e^{-x}) = 1
    const double e1 = xf < 708.0f ? exp_neg(x) : exp(-x);
    const double x2 = x * x;
    const double Q = C15 * e1 * fma(fma(x + 3.0, x, 6.0), x, 6.0);
    e.v = Q;
    e.rv = Q + 0.25 * C15 * (x2 * x2) * e1;
    e.tail = true;
    return e;
}

// Test hook kernel: e^{-x} by exp_neg where it applies (0 <= x < 708).
__global__ void exp_neg_kernel(const double *__restrict__ x, double *__restrict__ out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    out[i] = (v >= 0.0 && v < 708.0) ? exp_neg(v) : exp(-v);
}

__device__ __forceinline__ EdgeVals edge_vals(double x) {
    const float xf = (float)x;
    return edge_vals(x, xf, xf < (float)XT0 ? head_terms(xf) : 1);
}

// b_g and r_g of the group between reduced edges lo < hi (lo.tail implies
// hi.tail): differences of tails when the lower edge is in the tail form,
// else of P and R (converting the upper edge where it crosses the switch)
__device__ __forceinline__ void group_br(const EdgeVals &lo, const EdgeVals &hi, double &b,
                                         double &r) {
    if (lo.tail) {
        b = lo.v - hi.v;
        r = lo.rv - hi.rv;
    } else {
        double hv = hi.v, hr = hi.rv;
        if (hi.tail) {
            hv = 1.0 - hv;
            hr = 1.0 - hr;
        }
        b = hv - lo.v;
        r = hr - lo.rv;
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
// get no source and sigma~ = 1.  The Planck and Rosseland means take
// sum_g b_g = sum_g r_g = 1 (the lowest edge is 0, the highest infinity).
// Launched with one warp per block and (G + 1) floats of dynamic shared
// memory: the edges in FP32, for the branch decisions.
template <typename RT>
__global__ void emission_kernel(int ncell, int nn, int G, int Gp, const double *__restrict__ edges,
                                double acT4_scale, double inv_cdt, const double *__restrict__ T,
                                const double *__restrict__ sigma, RT *__restrict__ src,
                                double *__restrict__ gray, double *__restrict__ qcanon,
                                unsigned int *ctrl, const int *__restrict__ member_on) {
    if (member_on && *member_on == 0) return;  // a batch member that is not swept this pass
    extern __shared__ float s_edges[];
    for (int i = threadIdx.x; i <= G; i += 32) s_edges[i] = (float)edges[i];
    __syncwarp();
    // Lanes past the last node evaluate a copy of it and store nothing, so
    // that every warp stays converged through the edge loop (the series term
    // counts below are warp maxima).
    const int n_nodes = ncell * nn;
    const int t_raw = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t_raw < n_nodes;
    const int t = active ? t_raw : n_nodes - 1;
    const int cell = t / nn, node = t - cell * nn;
    double Tn = T[t];
    if (active && (!(Tn > 0.0) || !isfinite(Tn))) atomicOr(ctrl + CTRL_STATUS, ST_NONPHYSICAL);
    const double B4 = acT4_scale * Tn * Tn * Tn * Tn;  // a c T^4 / 4 pi
    const double invT = 1.0 / Tn;
    const float invTf = 1.0f / (float)Tn;
    EdgeVals lo = edge_vals(0.0);
    double nb = 0.0, nr = 0.0;
    RT *rec0 = src + (size_t)cell * Gp * 8;
    for (int g = 0; g < G; ++g) {
        const bool last = g == G - 1;
        const double xhi = last ? INFINITY : edges[g + 1] * invT;
        const float xf = last ? INFINITY : s_edges[g + 1] * invTf;
        // beyond x ~ 745 the tails 1 - P and 1 - R underflow to exactly 0, so
        // every higher group has b = r = 0: skip their series (tested on the
        // bits, both tails being +0 there)
        const bool skip = lo.tail && ((__double_as_longlong(lo.v) |
                                       __double_as_longlong(lo.rv)) == 0);
        const int K = __reduce_max_sync(0xffffffffu,
                                        (!skip && xf < (float)XT0) ? head_terms(xf) : 1);
        const EdgeVals hi = skip ? lo : edge_vals(xhi, xf, K);
        double b, r;
        group_br(lo, hi, b, r);
        const double sg = sigma[(size_t)g * ncell + cell];
        nb = fma(b, sg, nb);
        nr = fma(r, sg, nr);
        const double qv = sg * b * B4;
        if (active) {
            rec0[(size_t)g * 8 + node] = (RT)qv;
            if (qcanon) qcanon[((size_t)g * ncell + cell) * nn + node] = qv;
        }
        lo = hi;
    }
    if (!active) return;
    // the per-cell part of each record (unused node slots, sigma~, sigma), and
    // the padding groups (no source, unit sigma~), shared out among the nodes
    // of the cell so that each warp converts a quarter of the opacities
    for (int g = node; g < Gp; g += nn) {
        RT *rec = rec0 + (size_t)g * 8;
        if (g < G) {
            const double sg = sigma[(size_t)g * ncell + cell];
            rec[4] = (RT)(sg + inv_cdt);
            rec[5] = (RT)sg;
        } else {
            for (int n = 0; n < nn; ++n) rec[n] = (RT)0;
            rec[4] = (RT)1;
            rec[5] = (RT)0;
        }
        for (int n = nn; n < 4; ++n) rec[n] = (RT)0;
        rec[6] = (RT)0;
        rec[7] = (RT)0;
    }
    gray[(size_t)t * 2 + 0] = nb;
    gray[(size_t)t * 2 + 1] = nr;
}

// Group Planck functions and their temperature derivatives at the nodes,
// for the adjoint (one thread per node): B4[g][cell][node] = B_g(T)/4pi and
// cB[g][cell][node] = sigma_g dB_g/dT / 4pi with dB_g/dT = 4 a c T^3 r_g
// (Sec. 2), and sdB[cell][node] = sum_g sigma_g dB_g/dT.
__global__ void planck_parts_kernel(int ncell, int nn, int G, const double *__restrict__ edges,
                                    double ac, const double *__restrict__ T,
                                    const double *__restrict__ sigma, double *__restrict__ B4,
                                    double *__restrict__ cB, double *__restrict__ sdB) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell * nn) return;
    const int cell = t / nn, node = t - cell * nn;
    const double Tn = T[t];
    const double invT = 1.0 / Tn;
    const double inv4pi = 1.0 / (4.0 * PI_D);
    const double aT4 = ac * Tn * Tn * Tn * Tn, dT = 4.0 * ac * Tn * Tn * Tn;
    EdgeVals lo = edge_vals(0.0);
    double s = 0.0;
    for (int g = 0; g < G; ++g) {
        const double xhi = (g == G - 1) ? INFINITY : edges[g + 1] * invT;
        const EdgeVals hi = (lo.tail && lo.v == 0.0 && lo.rv == 0.0) ? lo : edge_vals(xhi);
        double b, r;
        group_br(lo, hi, b, r);
        const double sg = sigma[(size_t)g * ncell + cell];
        const size_t o = ((size_t)g * ncell + cell) * nn + node;
        B4[o] = aT4 * b * inv4pi;
        cB[o] = sg * dT * r * inv4pi;
        s += sg * dT * r;
        lo = hi;
    }
    sdB[t] = s;
}

// Opacity shape f_g(Tbar) = sigma_g / s and its derivative df_g/dTbar per
// [g][cell] (POWER: Tbar^-3; LARSEN: alpha (1 - e^{-E_g/Tbar})/E_g^3, E_g the
// geometric mean of the group's edges), Tbar the cell mean of the nodal T.
__global__ void opacity_shape_kernel(int ncell, int nn, int G, int kind, double alpha,
                                     const double *__restrict__ edges,
                                     const double *__restrict__ T, double *__restrict__ f,
                                     double *__restrict__ df) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncell) return;
    double tb = 0.0;
    for (int n = 0; n < nn; ++n) tb += T[(size_t)k * nn + n];
    tb /= nn;
    for (int g = 0; g < G; ++g) {
        double fv, dv;
        if (kind == SM_OPACITY_POWER) {
            fv = 1.0 / (tb * tb * tb);
            dv = -3.0 * fv / tb;
        } else {
            const double eg = sqrt(edges[g] * edges[g + 1]);
            fv = alpha * (-expm1(-eg / tb)) / (eg * eg * eg);
            dv = -alpha * exp(-eg / tb) / (eg * eg * tb * tb);
        }
        f[(size_t)g * ncell + k] = fv;
        df[(size_t)g * ncell + k] = dv;
    }
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
                            double *q_canon, cudaStream_t s, const int *active) {
    // one warp per block: node costs differ by up to ~2x (hot nodes have more
    // edges below the underflow point), and small blocks keep the last wave short
    const int threads = 32;
    const int n = p->ncell * p->nn;
    const int blocks = (n + threads - 1) / threads;
    const double scale = p->desc.a * p->desc.c / (4.0 * PI_D);
    if (p->prec == 32)
        emission_kernel<float><<<blocks, threads, (p->G + 1) * sizeof(float), s>>>(
            p->ncell, p->nn, p->G, p->Gp, p->d_edges, scale, p->inv_cdt, T, sigma,
            (float *)p->d_src, p->d_gray, q_canon, p->d_ctrl, active);
    else
        emission_kernel<double><<<blocks, threads, (p->G + 1) * sizeof(float), s>>>(
            p->ncell, p->nn, p->G, p->Gp, p->d_edges, scale, p->inv_cdt, T, sigma,
            (double *)p->d_src, p->d_gray, q_canon, p->d_ctrl, active);
    return cudaGetLastError();
}

cudaError_t launch_planck_parts(const sm_problem *p, const double *T, const double *sigma,
                                double *B4, double *cB, double *sdB, cudaStream_t s) {
    const int n = p->ncell * p->nn;
    planck_parts_kernel<<<(n + 127) / 128, 128, 0, s>>>(p->ncell, p->nn, p->G, p->d_edges,
                                                       p->desc.a * p->desc.c, T, sigma, B4, cB,
                                                       sdB);
    return cudaGetLastError();
}

cudaError_t launch_opacity_shape(const sm_problem *p, const double *T, double *f, double *df,
                                 cudaStream_t s) {
    opacity_shape_kernel<<<(p->ncell + 127) / 128, 128, 0, s>>>(
        p->ncell, p->nn, p->G, p->desc.opacity_kind, p->desc.opacity_alpha, p->d_edges, T, f, df);
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

extern "C" sm_status sm_debug_exp_neg(const double *x, double *out, int n, void *stream) {
    if (n < 0 || (n > 0 && (!x || !out))) {
        smk::set_last_error("sm_debug_exp_neg: n >= 0 and non-NULL arrays required");
        return SM_ERR_INVALID_ARG;
    }
    if (n == 0) return SM_OK;
    smk::planck_upload_tables();
    smk::exp_neg_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, out, n);
    if (cudaGetLastError() != cudaSuccess) {
        smk::set_last_error("sm_debug_exp_neg: launch failed");
        return SM_ERR_CUDA;
    }
    return SM_OK;
}
