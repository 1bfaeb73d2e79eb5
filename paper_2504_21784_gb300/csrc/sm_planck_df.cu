// Emission (row a1) of an FP32-sweep problem in double-FP32 arithmetic.
//
// The sweep of an FP32 problem reads FP32 source records, so its emission
// needs the Planck group integrals (Sec. 2, Eq. planck and the b_g
// definition) to FP32 precision.  The FP64 evaluation (sm_planck.cu, used by
// FP64 problems and by sm_emission) spends about 20 FP64 operations per (node,
// group edge), and this GPU issues FP64 at 1/64 of its FP32 rate.  Here the
// same series -- the head series below x = 1, the Taylor tables on [1, 37),
// the one-term tail series with its table-driven exponential from 37 on --
// run on unevaluated pairs hi + lo of FP32 numbers (about 48 significant bits)
// with error-free transformations on the FP32 pipes, the terms of high order
// (below 2^-24 of the leading term) in plain FP32.  The records come out as
// the FP64 evaluation rounded to FP32, up to a unit in the last place where
// the two round differently, and the nodal Planck and Rosseland numerators
// (FP64 outputs, for the closures) agree with it to about 1e-14.  Tails below
// FP32's range (e^{-x} for x beyond 87) are zero here; their records are below
// FP32's range anyway.  FP64 is used once per node (1/T, a c T^4) and for the
// two numerators' final sums.
#include <math.h>

#include <atomic>

#include "sm_internal.cuh"
#include "sm_planck.cuh"

namespace smk {
namespace pdf {

// ---------------------------------------------------------------------------
// pairs of FP32 numbers, every operation explicitly rounded (no contraction)

__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 add(float2 a, float2 b) {
    float2 s = two_sum(a.x, b.x);
    s.y = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
    return two_sum(s.x, s.y);
}
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return two_sum(p, e);
}
__device__ __forceinline__ float2 mul_f(float2 a, float b) {  // b an FP32 number
    const float p = __fmul_rn(a.x, b);
    float e = __fmaf_rn(a.x, b, -p);
    e = __fmaf_rn(a.y, b, e);
    return two_sum(p, e);
}
__device__ __forceinline__ float2 scale2(float2 a, float s) {  // s a power of two
    return make_float2(__fmul_rn(a.x, s), __fmul_rn(a.y, s));
}
__device__ __forceinline__ double join(float2 a) { return (double)a.x + (double)a.y; }

// The pair nearest to an FP64 x from its bits alone (integer and FP32
// operations): hi = x rounded to FP32 (to nearest, ties to even), lo = the
// remainder rounded to FP32.  |x| below 2^-102 gives (0, 0) and above FP32's
// range (+-inf, 0): neither occurs for the temperatures, edges and opacities
// of the emission.
__device__ __forceinline__ float2 split(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
    const int e = (int)((u >> 52) & 0x7ff);
    if (e < 921) return make_float2(__int_as_float((int)sign), __int_as_float((int)sign));
    if (e > 1150) return make_float2(__int_as_float((int)(sign | 0x7f800000u)), 0.f);
    const unsigned long long m = u & 0x000fffffffffffffull;
    unsigned hb = ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29);
    const int rem = (int)(m & 0x1fffffffull);
    const bool up = rem > 0x10000000 || (rem == 0x10000000 && (hb & 1u));
    hb += up ? 1u : 0u;  // a carry into the exponent is the right rounding
    const int d = up ? rem - 0x20000000 : rem;  // x - hi in units of 2^(e - 1075)
    float lo = __int2float_rn(d);
    const int k = e - 1075;
    if (k >= -126)
        lo = __fmul_rn(lo, __int_as_float((k + 127) << 23));
    else
        lo = __fmul_rn(__fmul_rn(lo, __int_as_float((-64 + 127) << 23)),
                       __int_as_float((k + 64 + 127) << 23));
    return make_float2(__int_as_float((int)(sign | hb)), sign ? -lo : lo);
}

// compensated sum of products a += x y (the Dot2 scheme of Ogita, Rump and
// Oishi): s the running FP32 sum, c the exact errors of its additions and
// products plus the low parts' terms
struct Acc {
    float s = 0.f, c = 0.f;
};
__device__ __forceinline__ void acc_mul(Acc &a, float2 x, float2 y) {
    const float p = __fmul_rn(x.x, y.x);
    float e = __fmaf_rn(x.x, y.x, -p);
    e = __fmaf_rn(x.x, y.y, e);
    e = __fmaf_rn(x.y, y.x, e);
    const float2 t = two_sum(a.s, p);
    a.s = t.x;
    a.c = __fadd_rn(a.c, __fadd_rn(t.y, e));
}

// ---------------------------------------------------------------------------
// tables (pairs of the FP64 tables, uploaded once per device)
__constant__ float2 c_head[NBERN];  // d_k = (B_2k/(2k)!)/(2k+3)
__constant__ float2 c_bern[NBERN];  // B_2k/(2k)!
__constant__ float2 c_exp2[64];     // 2^{-j/64}
__constant__ float2 c_c15, c_third; // 15/pi^4, 1/3
__constant__ float c_l64[3];        // ln2/64 = l1 + l2 + l3, l1 with 11 significant bits
__constant__ float c_i64;           // 64/ln2
__device__ float2 g_ptab[NCEN][2][NTAY];

static std::atomic<bool> g_ready[128];

static void split_host(double x, float2 &o) {
    o.x = (float)x;
    o.y = (float)(x - (double)o.x);
}

static bool upload_tables() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return false;
    if (g_ready[dev].load(std::memory_order_acquire)) return true;
    double head[NBERN], bern[NBERN], cexp[3], ex2[64];
    static double ptab[NCEN][2][NTAY];
    static float2 ptab_df[NCEN][2][NTAY];
    planck_host_tables(head, bern, cexp, ex2, ptab);
    float2 h[NBERN], b[NBERN], e2[64], c15, third;
    for (int k = 0; k < NBERN; ++k) {
        split_host(head[k], h[k]);
        split_host(bern[k], b[k]);
    }
    for (int j = 0; j < 64; ++j) split_host(ex2[j], e2[j]);
    for (int j = 0; j < NCEN; ++j)
        for (int s = 0; s < 2; ++s)
            for (int k = 0; k < NTAY; ++k) split_host(ptab[j][s][k], ptab_df[j][s][k]);
    split_host(C15, c15);
    split_host(1.0 / 3.0, third);
    // ln2/64 in three FP32 parts; the first with 11 significant bits, so that
    // its product with the step index (at most 2^13) is exact
    const long double l64 = 0.693147180559945309417232121458176568L / 64.0L;
    int ex = 0;
    frexp((double)l64, &ex);
    const float l1 = (float)ldexp(floor(ldexp((double)l64, 11 - ex)), ex - 11);
    const float l2 = (float)(l64 - (long double)l1);
    const float l3 = (float)(l64 - (long double)l1 - (long double)l2);
    const float l[3] = {l1, l2, l3};
    const float i64 = (float)(64.0L / 0.693147180559945309417232121458176568L);
    if (cudaMemcpyToSymbol(c_head, h, sizeof(h)) != cudaSuccess ||
        cudaMemcpyToSymbol(c_bern, b, sizeof(b)) != cudaSuccess ||
        cudaMemcpyToSymbol(c_exp2, e2, sizeof(e2)) != cudaSuccess ||
        cudaMemcpyToSymbol(c_c15, &c15, sizeof(c15)) != cudaSuccess ||
        cudaMemcpyToSymbol(c_third, &third, sizeof(third)) != cudaSuccess ||
        cudaMemcpyToSymbol(c_l64, l, sizeof(l)) != cudaSuccess ||
        cudaMemcpyToSymbol(c_i64, &i64, sizeof(i64)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_ptab, ptab_df, sizeof(ptab_df)) != cudaSuccess)
        return false;
    g_ready[dev].store(true, std::memory_order_release);
    return true;
}

// ---------------------------------------------------------------------------
// the cumulative spectra at one reduced edge, as in sm_planck.cuh (v = P, R
// below the switch near x = 2, v = 1 - P, 1 - R from it on)
struct EV {
    float2 v, rv;
    bool tail;
};

// e^{-x} for 37 <= x < 87 (Tang's table-driven method, as in sm_planck.cuh):
// x = N ln2/64 + r, |r| <= ln2/128, e^{-x} = 2^{-(N>>6)} 2^{-(N&63)/64} e^{-r}
__device__ __forceinline__ float2 exp_neg(float2 x) {
    const float N = rintf(__fmul_rn(x.x, c_i64));
    const int n = (int)N;
    // r = x - N (l1 + l2 + l3): x.x - N l1 exactly (N l1 is exact and close to x.x)
    const float r1 = __fsub_rn(x.x, __fmul_rn(N, c_l64[0]));
    const float p2 = __fmul_rn(N, c_l64[1]);
    const float e2 = __fmaf_rn(N, c_l64[1], -p2);
    float2 r = two_sum(r1, -p2);
    r.y = __fadd_rn(r.y, __fsub_rn(__fsub_rn(x.y, e2), __fmul_rn(N, c_l64[2])));
    r = two_sum(r.x, r.y);
    const float2 u = neg(r);  // e^{-r} = sum u^k / k!
    float s = __fmaf_rn(__fmaf_rn(1.0f / 720.0f, u.x, 1.0f / 120.0f), u.x, 1.0f / 24.0f);
    s = __fmaf_rn(s, u.x, 1.0f / 6.0f);  // |u|^3 / 6 < 2^-27: FP32 suffices from here on
    float2 p = add(mul_f(u, s), make_float2(0.5f, 0.f));
    p = add(mul(p, u), make_float2(1.f, 0.f));
    p = add(mul(p, u), make_float2(1.f, 0.f));
    p = mul(p, c_exp2[n & 63]);
    return scale2(p, __int_as_float((127 - (n >> 6)) << 23));
}

// K: head-series terms (warp maximum, as the FP64 evaluation takes them)
__device__ __forceinline__ EV edge_vals(float2 x, int K) {
    EV e;
    const float xf = x.x;
    if (!(xf > 0.0f)) {
        e.v = e.rv = make_float2(0.f, 0.f);
        e.tail = false;
        return e;
    }
    if (isinf(xf)) {
        e.v = e.rv = make_float2(0.f, 0.f);
        e.tail = true;
        return e;
    }
    if (in_taylor(xf)) {
        const int j = __float2int_rn((xf - (float)XT0) * (float)TSTEP);  // nearest centre
        const float c = (float)XT0 + (float)j / (float)TSTEP;             // exact
        const float2 h = two_sum(__fsub_rn(x.x, c), x.y);  // x.x - c is exact (Sterbenz)
        const float2 *t = &g_ptab[j][0][0];
        float2 r[2];
#pragma unroll
        for (int sidx = 0; sidx < 2; ++sidx) {
            const float2 *ts = t + sidx * NTAY;
            // terms of order 4 and higher (below 2^-30 of the leading one) in FP32
            float a = __ldg(&ts[NTAY - 1].x);
#pragma unroll
            for (int k = NTAY - 2; k >= 4; --k) a = __fmaf_rn(a, h.x, __ldg(&ts[k].x));
            float2 A = add(mul_f(h, a), ts[3]);
            A = add(mul(A, h), ts[2]);
            A = add(mul(A, h), ts[1]);
            A = add(mul(A, h), ts[0]);
            r[sidx] = A;
        }
        e.v = r[0];
        e.rv = r[1];
        e.tail = j >= JSW;
        return e;
    }
    if (xf < (float)XT0) {
        // P = C15 x^3 (1/3 - x/8 + y sum d_k y^(k-1)), R = P - C15/4 x^3 (1 - x/2 +
        // y sum B_2k/(2k)! y^(k-1)), y = x^2; terms from k = 4 on in FP32
        const float2 y = mul(x, x);
        float ph = c_head[K - 1].x, pb = c_bern[K - 1].x;
        for (int k = K - 2; k >= 3; --k) {
            ph = __fmaf_rn(ph, y.x, c_head[k].x);
            pb = __fmaf_rn(pb, y.x, c_bern[k].x);
        }
        float2 P1 = make_float2(ph, 0.f), P2 = make_float2(pb, 0.f);
        if (K > 3) {
            P1 = add(mul_f(y, ph), c_head[2]);
            P2 = add(mul_f(y, pb), c_bern[2]);
        } else if (K == 3) {
            P1 = c_head[2];
            P2 = c_bern[2];
        }
        for (int k = 1; k >= 0; --k) {
            if (k + 1 < K) {
                P1 = add(mul(P1, y), c_head[k]);
                P2 = add(mul(P2, y), c_bern[k]);
            } else if (k + 1 == K) {
                P1 = c_head[k];
                P2 = c_bern[k];
            }
        }
        P1 = mul(P1, y);
        P2 = mul(P2, y);
        const float2 x3 = mul(y, x);
        const float2 inner = add(add(c_third, scale2(neg(x), 0.125f)), P1);
        const float2 P = mul(c_c15, mul(x3, inner));
        const float2 rin = add(add(make_float2(1.f, 0.f), scale2(neg(x), 0.5f)), P2);
        e.v = P;
        e.rv = add(P, neg(scale2(mul(c_c15, mul(x3, rin)), 0.25f)));
        e.tail = false;
        return e;
    }
    // x >= 37: 1 - P = C15 e^{-x} (x^3 + 3x^2 + 6x + 6), 1 - R = 1 - P + C15/4 x^4 e^{-x}
    if (!(xf < 87.0f)) {  // below FP32's range
        e.v = e.rv = make_float2(0.f, 0.f);
        e.tail = true;
        return e;
    }
    const float2 e1 = exp_neg(x);
    float2 poly = add(x, make_float2(3.f, 0.f));
    poly = add(mul(poly, x), make_float2(6.f, 0.f));
    poly = add(mul(poly, x), make_float2(6.f, 0.f));
    const float2 ce = mul(c_c15, e1);
    const float2 Q = mul(ce, poly);
    const float2 x2 = mul(x, x);
    e.v = Q;
    e.rv = add(Q, scale2(mul(ce, mul(x2, x2)), 0.25f));
    e.tail = true;
    return e;
}

__device__ __forceinline__ void group_br(const EV &lo, const EV &hi, float2 &b, float2 &r) {
    if (lo.tail) {
        b = add(lo.v, neg(hi.v));
        r = add(lo.rv, neg(hi.rv));
    } else {
        float2 hv = hi.v, hr = hi.rv;
        if (hi.tail) {
            hv = add(make_float2(1.f, 0.f), neg(hv));
            hr = add(make_float2(1.f, 0.f), neg(hr));
        }
        b = add(hv, neg(lo.v));
        r = add(hr, neg(lo.rv));
    }
}

// One thread per (cell, node), one warp per block, as the FP64 emission
// kernel: the same records and numerators (in pairs, see above).
__global__ void emission_df_kernel(int ncell, int nn, int G, int Gp,
                                   const double *__restrict__ edges, double acT4_scale,
                                   double inv_cdt, const double *__restrict__ T,
                                   const double *__restrict__ sigma, float *__restrict__ src,
                                   double *__restrict__ gray, unsigned int *ctrl,
                                   const int *__restrict__ member_on) {
    if (member_on && *member_on == 0) return;  // a batch member that is not swept this pass
    extern __shared__ float2 s_e[];
    for (int i = threadIdx.x; i <= G; i += 32) s_e[i] = split(edges[i]);
    __syncwarp();
    const int n_nodes = ncell * nn;
    const int t_raw = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t_raw < n_nodes;
    const int t = active ? t_raw : n_nodes - 1;
    const int cell = t / nn, node = t - cell * nn;
    const double Tn = T[t];
    if (active && (!(Tn > 0.0) || !isfinite(Tn))) atomicOr(ctrl + CTRL_STATUS, ST_NONPHYSICAL);
    const float2 invT = split(1.0 / Tn);
    const float2 B4 = split(acT4_scale * Tn * Tn * Tn * Tn);  // a c T^4 / 4 pi
    EV lo = edge_vals(make_float2(0.f, 0.f), 1);
    Acc nb, nr;
    float *rec0 = src + (size_t)cell * Gp * 8;
    for (int g = 0; g < G; ++g) {
        const bool last = g == G - 1;
        const float2 x = last ? make_float2(INFINITY, 0.f) : mul(s_e[g + 1], invT);
        // once both tails are exactly 0, every higher group has b = r = 0
        const bool skip = lo.tail && lo.v.x == 0.f && lo.rv.x == 0.f && lo.v.y == 0.f &&
                          lo.rv.y == 0.f;
        const int K = __reduce_max_sync(0xffffffffu,
                                        (!skip && x.x < (float)XT0) ? head_terms(x.x) : 1);
        const EV hi = skip ? lo : edge_vals(x, K);
        float2 b, r;
        group_br(lo, hi, b, r);
        const float2 sg = split(sigma[(size_t)g * ncell + cell]);
        acc_mul(nb, b, sg);
        acc_mul(nr, r, sg);
        if (active) {
            const float2 q = mul(mul(sg, b), B4);
            rec0[(size_t)g * 8 + node] = __fadd_rn(q.x, q.y);
        }
        lo = hi;
    }
    if (!active) return;
    // the per-cell part of each record, shared out among the nodes of the cell
    const float2 icdt = split(inv_cdt);
    for (int g = node; g < Gp; g += nn) {
        float *rec = rec0 + (size_t)g * 8;
        if (g < G) {
            const float2 sg = split(sigma[(size_t)g * ncell + cell]);
            const float2 st = add(sg, icdt);
            rec[4] = __fadd_rn(st.x, st.y);
            rec[5] = __fadd_rn(sg.x, sg.y);
        } else {
            for (int n = 0; n < nn; ++n) rec[n] = 0.f;
            rec[4] = 1.f;
            rec[5] = 0.f;
        }
        for (int n = nn; n < 4; ++n) rec[n] = 0.f;
        rec[6] = 0.f;
        rec[7] = 0.f;
    }
    gray[(size_t)t * 2 + 0] = (double)nb.s + (double)nb.c;
    gray[(size_t)t * 2 + 1] = (double)nr.s + (double)nr.c;
}

}  // namespace pdf

bool planck_df_upload_tables(void) { return pdf::upload_tables(); }

cudaError_t launch_emission_df(const sm_problem *p, const double *T, const double *sigma,
                               cudaStream_t s, const int *active) {
    if (!pdf::upload_tables()) return cudaErrorUnknown;
    const int threads = 32;
    const int n = p->ncell * p->nn;
    const int blocks = (n + threads - 1) / threads;
    const double scale = p->desc.a * p->desc.c / (4.0 * PI_D);
    pdf::emission_df_kernel<<<blocks, threads, (p->G + 1) * sizeof(float2), s>>>(
        p->ncell, p->nn, p->G, p->Gp, p->d_edges, scale, p->inv_cdt, T, sigma,
        static_cast<float *>(p->d_src), p->d_gray, p->d_ctrl, active);
    return cudaGetLastError();
}

}  // namespace smk
