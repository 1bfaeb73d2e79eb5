// Device code of the FP64 Planck / Rosseland group integrals and of the
// emission of one node (row a1), shared by the emission kernel
// (sm_planck.cu, tables in the module's constant and global memory) and the
// sweep kernel with fused emission (sm_sweep.cu, the same tables reached
// through a kernel parameter): every function takes a table accessor Tab with
//   head(k), bern(k)  -- d_k = (B_2k/(2k)!)/(2k+3) and B_2k/(2k)!, k = 1..NBERN
//   cexp(i)           -- 64/ln2 and ln2/64 split in a high and a low part
//   exp2(j)           -- 2^{-j/64}, j = 0..63
//   pcen(j), ptab(j)  -- Taylor centre j and its [2][NTAY] coefficients.
//
// P(x) = (15/pi^4) int_0^x t^3/(e^t-1) dt rests on the two series used by
// Clark (Sec. 2, Eq. planck and the b_g definition):
//   small x: x^3/3 - x^4/8 + sum_k B_2k x^(2k+3) / ((2k)! (2k+3))
//   large x: 1 - (15/pi^4) sum_n e^{-nx} (x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4)
// and the Rosseland integral by parts, R(x) = P(x) - (15/4pi^4) x^4/(e^x-1),
// which gives r_g with dB_g/dT = 4 a c T^3 r_g (Sec. 2); for small x the
// factor x/(e^x-1) is the Bernoulli generating series itself.  The GPU takes
// the first series for x < 1, the first term of the second for x >= 37 (the
// next is below double rounding), and in between degree-6 Taylor expansions
// about the nearest of the centres 1, 1 + 1/32, ..., 37 (|x - c| <= 1/64).
// A group whose lower reduced edge is at or above the switch near x = 2 is
// differenced in tails (1 - P) to keep relative accuracy; the lowest edge is 0
// and the highest infinity so that sum_g b_g = 1.
#pragma once

#include <math.h>
#include <stdint.h>

namespace smk {

constexpr int NBERN = 18;   // head terms: (2/2pi)^36 < 1e-17
// from x = 37 on, e^{-x} < 1e-16: the tail series keeps its first term only
constexpr double XCLOSED = 37.0;
constexpr double PI_D = 3.14159265358979323846;
constexpr double C15 = 15.0 / (PI_D * PI_D * PI_D * PI_D);
// Taylor tables: centre j at c_j = XT0 + j/TSTEP; per centre two series of
// NTAY coefficients in h = x - c_j, (P, R) for c_j < 2 and (1 - P, 1 - R) for
// c_j >= 2 (so that the tails keep their relative accuracy).
constexpr double XT0 = 1.0, XT1 = 37.0;
constexpr int TSTEP = 32;  // centres per unit of x
constexpr int NCEN = 1153;  // (XT1 - XT0) * TSTEP + 1
constexpr int NTAY = 7;    // remainder (1/64 / 2pi)^7 < 1e-18 of the leading term
constexpr int JSW = 32;    // centres j < JSW lie below x = 2: P, R; from there on 1 - P, 1 - R
static_assert(XT1 == XCLOSED, "the Taylor tables end where the one-term tail takes over");

// Host copies of the tables (head and Bernoulli coefficients, the exponential's
// constants and 2^{-j/64} table, the Taylor tables), derived in extended
// precision (sm_planck.cu).
void planck_host_tables(double head[NBERN], double bern[NBERN], double cexp[3], double exp2[64],
                        double (*ptab)[2][NTAY]);

// The tables as a kernel parameter: the series coefficients by value, the
// larger tables by device address.
struct PlanckTabs {
    double head[NBERN], bern[NBERN], cexp[3];
    const double *ptab;  // [NCEN][2][NTAY]
    const double *pcen;  // [NCEN]
    const double *exp2;  // [64]
};

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

// e^{-x} for 0 <= x < 708 (normal results) by the table-driven method of Tang
// (ACM TOMS 15, 1989): x = N ln2/64 + r with N = round(64 x/ln2) and
// |r| <= ln2/128, so e^{-x} = 2^{-(N>>6)} 2^{-(N&63)/64} e^{-r}, with e^{-r} by
// its degree-6 Taylor polynomial (remainder below |r|^7/7! < 2e-20).  About
// two thirds of the FP64 work of exp() here.
template <class Tab>
__device__ __forceinline__ double exp_neg(double x, const Tab &t) {
    const double Nd = rint(x * t.cexp(0));
    const double s = fma(Nd, t.cexp(2), fma(Nd, t.cexp(1), -x));  // -r
    const int n = (int)Nd;
    double p = fma(s, 1.0 / 720.0, 1.0 / 120.0);
    p = fma(p, s, 1.0 / 24.0);
    p = fma(p, s, 1.0 / 6.0);
    p = fma(p, s, 0.5);
    p = fma(p, s, 1.0);
    p = fma(p, s, 1.0);
    const double scale = __longlong_as_double((long long)(1023 - (n >> 6)) << 52);
    return t.exp2(n & 63) * p * scale;
}

// K: head-series terms to use (at least head_terms(xf)); callers that keep a
// warp converged pass the warp maximum, so that every lane reads the same
// coefficient at each step.  xf: x rounded to FP32 or computed in FP32 (it
// only steers branches and term counts, which have margin for its relative
// error below 1e-6).
template <class Tab>
__device__ __forceinline__ EdgeVals edge_vals(double x, float xf, int K, const Tab &tb) {
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
        const double h = x - tb.pcen(j);
        const double *t = tb.ptab(j);
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
        double poly = tb.head(K - 1), pb = tb.bern(K - 1);
        for (int k = K - 2; k >= 0; --k) {
            poly = fma(poly, y, tb.head(k));
            pb = fma(pb, y, tb.bern(k));
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
    const double e1 = xf < 708.0f ? exp_neg(x, tb) : exp(-x);
    const double x2 = x * x;
    const double Q = C15 * e1 * fma(fma(x + 3.0, x, 6.0), x, 6.0);
    e.v = Q;
    e.rv = Q + 0.25 * C15 * (x2 * x2) * e1;
    e.tail = true;
    return e;
}

template <class Tab>
__device__ __forceinline__ EdgeVals edge_vals(double x, const Tab &tb) {
    const float xf = (float)x;
    return edge_vals(x, xf, xf < (float)XT0 ? head_terms(xf) : 1, tb);
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

// Emission (row a1) of one node, walking the group edges once: q_{g,n} =
// sigma_g a c T^4 b_g(T) / 4pi into the sweep's source record
// src[cell][g][8] = {q at the nodes (unused node slots 0), sigma~, sigma, 0, 0}
// in the sweep precision (padding groups: no source, sigma~ = 1), and the
// nodal Planck- and Rosseland-collapsed numerators sum_g b_g sigma_g and
// sum_g r_g sigma_g into gray[t][2] (sum_g b_g = sum_g r_g = 1: the lowest edge
// is 0, the highest infinity).  Every lane of the warp must call it (the
// head-series term counts are warp maxima); an inactive lane evaluates a copy
// of an active node and stores nothing.  s_edges: the edges in FP32, for the
// branch decisions.
template <typename RT, class Tab>
__device__ __forceinline__ void emit_node(int cell, int node, bool active, int ncell, int nn, int G,
                                          int Gp, const double *__restrict__ edges,
                                          const float *s_edges, double acT4_scale, double inv_cdt,
                                          const double *__restrict__ T,
                                          const double *__restrict__ sigma, RT *__restrict__ src,
                                          double *__restrict__ gray, double *__restrict__ qcanon,
                                          unsigned int *ctrl, unsigned int nonphysical_bit,
                                          const Tab &tb) {
    const int t = cell * nn + node;
    const double Tn = T[t];
    if (active && (!(Tn > 0.0) || !isfinite(Tn))) atomicOr(ctrl, nonphysical_bit);
    const double B4 = acT4_scale * Tn * Tn * Tn * Tn;  // a c T^4 / 4 pi
    const double invT = 1.0 / Tn;
    const float invTf = 1.0f / (float)Tn;
    EdgeVals lo = edge_vals(0.0, tb);
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
        const EdgeVals hi = skip ? lo : edge_vals(xhi, xf, K, tb);
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
    // of the cell so that each lane converts a quarter of the opacities
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

}  // namespace smk
