// FP64-accurate defect correction of the transport solve with FP32 sweeps
// (the FP32 sweep path refined to the FP64 solution inside the outer SM
// iteration).
//
// The caller's state -- the previous step's intensity I^k, the intensity of
// the step, the emission records -- is FP64 (a precision-64 problem).  Each
// outer iteration of Algorithm 1 replaces the FP64 sweep by corrections of
// an intensity iterate I (which starts at I^k), each
//   1. the residual of the lumped upwind-DG equations (Eq. dgsn_transport with
//      the time term of Eq. smm_be_transport) at I:
//      r = S + (upwind face terms of I) - M I per node, S = q + I^k/(c dt),
//      stored in FP32;
//   2. an FP32 sweep of the correction, M d = r + (upwind face terms of d)
//      with zero inflow (the sweep kernel with q = 0 and r in place of I^k,
//      1/(c dt) -> 1);
//   3. I += d (for the correction that ends the outer iteration, inside the
//      moments kernel, which reads the iterate anyway and writes I + d to a
//      second iterate buffer),
// until a correction is below 1e-8 of the iterate (at most MAX_CORR per outer
// iteration; max |d| from a pass over d alone).  From the second outer
// iteration of a step on, the iterate
// already solves the previous records' equations to that tolerance and only
// the emission has changed (the opacities are frozen for the step), so the
// first correction sweeps the change of q itself and skips the residual.  A
// correction leaves the FP32 solve's relative error of d, so
// the next one is that much smaller and the iterate reaches the solution of
// the transport equations for the outer iteration's temperature -- the FP64
// sweep's intensity, up to rounding.  One correction per outer iteration
// would not do: its FP32 error would enter the closures and, through the
// low-order solve, the next temperature, and the outer iteration carries
// such errors along.  Then the moments of the iterate, read from it directly
// (the sweep's fused FP32 moments of d would carry FP32 rounding of the large
// first corrections into every later moment).
//
// Double-FP32 arithmetic.  This GPU issues FP64 at 1/64 of its FP32 rate: an
// FP64 residual (about 30 FP64 operations per cell, direction and group) and
// FP64 updates and moment sums made the refined step slower than the FP64
// sweep path.  So the iterate, I^k and the records are held during the step
// as unevaluated sums hi + lo of two FP32 numbers (about 48 significant bits),
// and the residual, the update and the moment sums use error-free FP32
// transformations (TwoSum of Knuth, the FMA form of Dekker's product) in
// compensated sums on the FP32 pipes; FP64 is used only to split the FP64 inputs into pairs once per
// step (and the records once per outer iteration), to join the iterate back
// into FP64 at the end of the step, and for the 36 dot products per (cell,
// quadrant) of the moments.  The pairs keep their full precision for values
// above about 1e-30 (below that the low part loses bits to FP32's range);
// the residual's error is then about 2^-44 of the magnitude of its terms.
//
// The local cell system is the sweep kernel's (per node, divided by the nodal
// mass; u / d = upwind / downwind side, A = sigma~ + mu + eta, mu =
// |Omega_x|/h_x, eta = |Omega_y|/h_y):
//   [ A   mu  eta  0  ] [I_uu]   [S_uu + 2 mu X_u + 2 eta Y_u]
//   [-mu  A   0   eta ] [I_du] = [S_du + 2 eta Y_d          ]
//   [-eta 0   A   mu  ] [I_ud]   [S_ud + 2 mu X_d           ]
//   [ 0  -eta -mu  A  ] [I_dd]   [S_dd                      ]
// with X the x-outflow of the upwind cell (its downwind-x nodes) or the
// boundary inflow, Y the same along y.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sm_internal.cuh"

namespace smk {

constexpr int MAX_CORR = 4;         // corrections per outer iteration, at most
constexpr double CORR_TOL = 1e-8;   // stop once max |d| <= CORR_TOL max |I|

// ---------------------------------------------------------------------------
// double-FP32 numbers (x = hi + lo, |lo| <= ulp(hi)/2); every operation is an
// explicitly rounded FP32 operation, so the compiler neither contracts nor
// reorders them.

// a + b = s + e exactly (Knuth)
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
// a + b, absolute error within about 2^-44 (|a| + |b|) also where a and b
// cancel (the residual's case)
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float2 s = two_sum(a.x, b.x);
    s.y = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
    return two_sum(s.x, s.y);
}
// a + d for an FP32 d
__device__ __forceinline__ float2 df_add_f(float2 a, float d) {
    float2 s = two_sum(a.x, d);
    s.y = __fadd_rn(s.y, a.y);
    return two_sum(s.x, s.y);
}
// A sum of products and pairs accumulated with compensation (the Dot2 scheme
// of Ogita, Rump and Oishi, "Accurate sum and dot product", 2005): s carries
// the running FP32 sum, c the exact errors of its additions (TwoSum) and of
// the products' high parts (one FMA each) plus the pairs' low parts and cross
// terms.  The result s + c errs by about 2^-24 of itself plus 2^-44 of the
// terms' magnitudes, so a sum that cancels to a small residual keeps its
// accuracy relative to the terms.  About half the operations of summing
// products of pairs as pairs.
struct Acc {
    float s = 0.f, c = 0.f;
};
__device__ __forceinline__ void acc_add(Acc &a, float2 v) {  // a += v
    const float2 t = two_sum(a.s, v.x);
    a.s = t.x;
    a.c = __fadd_rn(a.c, __fadd_rn(t.y, v.y));
}
__device__ __forceinline__ void acc_mul(Acc &a, float2 x, float2 y) {  // a += x y
    const float p = __fmul_rn(x.x, y.x);
    float e = __fmaf_rn(x.x, y.x, -p);
    e = __fmaf_rn(x.x, y.y, e);
    e = __fmaf_rn(x.y, y.x, e);
    const float2 t = two_sum(a.s, p);
    a.s = t.x;
    a.c = __fadd_rn(a.c, __fadd_rn(t.y, e));
}
__device__ __forceinline__ float2 neg(float2 x) { return make_float2(-x.x, -x.y); }

// the pair nearest to an FP64 x (FP64 operations: used once per value and step)
__device__ __forceinline__ float2 df_split(double x) {
    const float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
}
__device__ __forceinline__ double df_join(float2 a) { return (double)a.x + (double)a.y; }

struct RefineArgs {
    int nx, ny, ncell, NQ, NWT, NGB, DB, LG, GW, Gp;
    float2 inv_cdt;
    const LaneConst *lanes;
    const float2 *mueta;    // [NQ*DB*32][2] mu, eta per lane as pairs
    const float2 *rec;      // [cell][Gp][6] q at the 4 nodes, sigma~, sigma as pairs
    const float2 *inflow;   // [4][Gp] pairs
    const float2 *I_k;      // packed I^k as pairs ([element][node])
    const float2 *I;        // packed iterate as pairs
    float *r;               // packed FP32 residual (out)
    size_t n_elems;         // packed elements (four nodes each; one thread each)
};

// The residual of one packed element (warp task wg of quadrant Q, cell,
// slot, lane): four nodes, each a compensated sum of its source and products
// of pairs.  The quadrant is a template parameter so that the
// upwind/downwind roles of the nodes are compile-time register indices.
// The residual of one packed element (warp task wg of quadrant Q, cell,
// slot, lane): four nodes, each a compensated sum of its source and products
// of pairs.  The quadrant is a template parameter so that the
// upwind/downwind roles of the nodes are compile-time register indices.
template <int Q>
__device__ __forceinline__ void residual_elem(const RefineArgs &R, const size_t e, const int lane,
                                              const int slot, const int cell, const int wt) {
    const int db = wt / R.NGB, gb = wt - db * R.NGB;
    const int li = (Q * R.DB + db) * 32 + lane;
    const LaneConst &L = R.lanes[li];
    float4 *ro = reinterpret_cast<float4 *>(R.r) + e;
    if (!L.valid) {
        *ro = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const int g = gb * R.GW * R.LG + slot * R.LG + L.g_lo;
    constexpr int sx = (Q == 0 || Q == 3) ? 1 : -1, sy = Q < 2 ? 1 : -1;
    constexpr int au = sx > 0 ? 0 : 1, bu = sy > 0 ? 0 : 1;
    constexpr int nuu = au + 2 * bu, ndu = (1 - au) + 2 * bu;
    constexpr int nud = au + 2 * (1 - bu), ndd = (1 - au) + 2 * (1 - bu);
    const int ix = cell % R.nx, iy = cell / R.nx;
    // the packed elements of the same (warp task, slot, lane) at another cell
    const ptrdiff_t cell_stride = (ptrdiff_t)R.GW * 32;
    const float2 *Ic = R.I + e * 4;
    float2 I[4];
    const float2 *rec = R.rec + ((size_t)cell * R.Gp + g) * 6;
    const float2 *ik = R.I_k + e * 4;
    // every node's equation starts from its source S = q + I^k/(c dt)
    Acc a[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        I[n] = Ic[n];
        acc_add(a[n], rec[n]);
        acc_mul(a[n], R.inv_cdt, ik[n]);
    }
    float2 Xu, Xd, Yu, Yd;
    if (ix - sx >= 0 && ix - sx < R.nx) {
        const float2 *nb = Ic - sx * cell_stride * 4;
        Xu = nb[ndu];
        Xd = nb[ndd];
    } else {
        Xu = Xd = R.inflow[(sx > 0 ? 0 : 1) * R.Gp + g];
    }
    if (iy - sy >= 0 && iy - sy < R.ny) {
        const float2 *nb = Ic - sy * (ptrdiff_t)R.nx * cell_stride * 4;
        Yu = nb[nud];
        Yd = nb[ndd];
    } else {
        Yu = Yd = R.inflow[(sy > 0 ? 2 : 3) * R.Gp + g];
    }
    const float2 mu = R.mueta[li * 2], eta = R.mueta[li * 2 + 1];
    const float2 mu2 = make_float2(2.f * mu.x, 2.f * mu.y);  // exact
    const float2 eta2 = make_float2(2.f * eta.x, 2.f * eta.y);
    const float2 mA = neg(df_add(df_add(rec[4], mu), eta));  // -A
    // r = S + inflow terms - M I, row by row of the cell system
    acc_mul(a[nuu], mu2, Xu);
    acc_mul(a[nuu], eta2, Yu);
    acc_mul(a[nuu], mA, I[nuu]);
    acc_mul(a[nuu], neg(mu), I[ndu]);
    acc_mul(a[nuu], neg(eta), I[nud]);
    acc_mul(a[ndu], eta2, Yd);
    acc_mul(a[ndu], mA, I[ndu]);
    acc_mul(a[ndu], mu, I[nuu]);
    acc_mul(a[ndu], neg(eta), I[ndd]);
    acc_mul(a[nud], mu2, Xd);
    acc_mul(a[nud], mA, I[nud]);
    acc_mul(a[nud], eta, I[nuu]);
    acc_mul(a[nud], neg(mu), I[ndd]);
    acc_mul(a[ndd], mA, I[ndd]);
    acc_mul(a[ndd], eta, I[ndu]);
    acc_mul(a[ndd], mu, I[nud]);
    float r[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) r[n] = __fadd_rn(a[n].s, a[n].c);
    *ro = make_float4(r[0], r[1], r[2], r[3]);
}

// One thread per (warp task, cell, slot, lane): the residual of its four
// nodes.  Padding lanes (no direction) get r = 0, so their correction is 0.
__global__ void __launch_bounds__(256) residual_kernel(const RefineArgs R) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= R.n_elems) return;
    const int lane = (int)(e & 31);
    // the (warp task, cell, slot) of the element in 32-bit unsigned
    // arithmetic: e / 32 counts 512-byte blocks of the packed FP32 residual,
    // so it stays below 2^32 on any device; a 64-bit division costs several
    // times the instructions, and this kernel is bound by instruction issue
    const unsigned rest = (unsigned)(e >> 5);
    const unsigned gw = (unsigned)R.GW, nc = (unsigned)R.ncell;
    const unsigned r1 = rest / gw;
    const int slot = (int)(rest - r1 * gw);
    const unsigned wgu = r1 / nc;
    const int cell = (int)(r1 - wgu * nc);
    const int wg = (int)wgu;
    const int q = wg / R.NWT, wt = wg - q * R.NWT;
    switch (q) {
        case 0: residual_elem<0>(R, e, lane, slot, cell, wt); break;
        case 1: residual_elem<1>(R, e, lane, slot, cell, wt); break;
        case 2: residual_elem<2>(R, e, lane, slot, cell, wt); break;
        default: residual_elem<3>(R, e, lane, slot, cell, wt); break;
    }
}

// I_out = I + d (the iterate as pairs, the FP32 correction in the same
// packed layout, one element of four nodes per thread; I_out may be I), with
// max |I_out| in *imax: non-negative FP32 numbers order like their bit
// patterns, so the maximum is an integer atomic on the bits.
__global__ void __launch_bounds__(256) update_kernel(const float2 *I, const float *__restrict__ d,
                                                     float2 *I_out, size_t n_elems,
                                                     unsigned int *__restrict__ imax) {
    unsigned mi = 0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_elems;
         e += (size_t)gridDim.x * blockDim.x) {
        const float4 dv = reinterpret_cast<const float4 *>(d)[e];
        const float4 *ip = reinterpret_cast<const float4 *>(I + e * 4);
        const float4 a = ip[0], b = ip[1];
        const float2 n0 = df_add_f(make_float2(a.x, a.y), dv.x);
        const float2 n1 = df_add_f(make_float2(a.z, a.w), dv.y);
        const float2 n2 = df_add_f(make_float2(b.x, b.y), dv.z);
        const float2 n3 = df_add_f(make_float2(b.z, b.w), dv.w);
        float4 *op = reinterpret_cast<float4 *>(I_out + e * 4);
        op[0] = make_float4(n0.x, n0.y, n1.x, n1.y);
        op[1] = make_float4(n2.x, n2.y, n3.x, n3.y);
        mi = max(mi, max(max(__float_as_uint(fabsf(n0.x)), __float_as_uint(fabsf(n1.x))),
                         max(__float_as_uint(fabsf(n2.x)), __float_as_uint(fabsf(n3.x)))));
    }
    mi = __reduce_max_sync(0xffffffffu, mi);
    if ((threadIdx.x & 31) == 0 && mi) atomicMax(imax, mi);
}

// max |d| of the correction (FP32 bits; NaN above every finite value)
__global__ void __launch_bounds__(256) dmax_kernel(const float4 *__restrict__ d, size_t n,
                                                   unsigned int *__restrict__ dmax) {
    unsigned m = 0u;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = d[i];
        m = max(m, max(max(__float_as_uint(fabsf(v.x)), __float_as_uint(fabsf(v.y))),
                       max(__float_as_uint(fabsf(v.z)), __float_as_uint(fabsf(v.w)))));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(dmax, m);
}

// Moments of the iterate, per node: one warp per (quadrant, direction block,
// cell); each lane sums its direction's intensities over all groups of the
// direction block as pairs, plain and sigma-weighted (sigma_g from the
// records), the sums pass through shared memory as pairs, and each lane
// forms one of the 36 moments (4 nodes x {phi, F, P} and sigma-weighted
// {phi, F}) as the compensated dot product (Acc) of the 32 lanes' sums with
// the pairs of their weights (wpair) -- on the FP32 pipes: in FP64 these dot
// products bounded the kernel where a direction block holds few groups (the
// gray problems); partial moments per (quadrant, direction block) go to
// part[qd][cell][36] for the fixed-order reduction.  Padding lanes have zero
// weights and padding groups zero intensity.
constexpr int MOM_WARPS = 4;
__global__ void __launch_bounds__(MOM_WARPS * 32)
moments_kernel(const float2 *__restrict__ I, const float *__restrict__ dI,
               float2 *__restrict__ I_new, unsigned int *__restrict__ imax,
               const LaneConst *__restrict__ lanes, const float2 *__restrict__ wpair,
               const float2 *__restrict__ rec, int ncell, int NQ, int DB, int NGB, int NWT,
               int GW, int LG, int Gp, double *__restrict__ part) {
    __shared__ float2 sh[MOM_WARPS][8][33];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const long long wglob = (long long)blockIdx.x * MOM_WARPS + wi;
    if (wglob >= (long long)NQ * DB * ncell) return;
    const int qd = (int)(wglob / ncell), cell = (int)(wglob - (long long)qd * ncell);
    const int q = qd / DB, db = qd - q * DB;
    const LaneConst &L = lanes[qd * 32 + lane];
    Acc s[4], ss[4];
    unsigned im = 0u;
    for (int gb = 0; gb < NGB; ++gb) {
        const int wt = db * NGB + gb;
        const size_t e0 = (((size_t)q * NWT + wt) * ncell + cell) * GW;
        for (int gw = 0; gw < GW; ++gw) {
            const int g = gb * GW * LG + gw * LG + L.g_lo;
            const float2 sg = rec[((size_t)cell * Gp + g) * 6 + 5];
            const size_t e = (e0 + gw) * 32 + lane;
            const float4 *ip = reinterpret_cast<const float4 *>(I + e * 4);
            const float4 a = ip[0], b = ip[1];
            float2 v[4] = {make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y),
                           make_float2(b.z, b.w)};
            if (dI) {
                // the pending correction: I + dI (update_kernel's operations),
                // written to the other iterate buffer
                const float4 dv = reinterpret_cast<const float4 *>(dI)[e];
                v[0] = df_add_f(v[0], dv.x);
                v[1] = df_add_f(v[1], dv.y);
                v[2] = df_add_f(v[2], dv.z);
                v[3] = df_add_f(v[3], dv.w);
                float4 *op = reinterpret_cast<float4 *>(I_new + e * 4);
                op[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
                op[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
                im = max(im, max(max(__float_as_uint(fabsf(v[0].x)), __float_as_uint(fabsf(v[1].x))),
                                 max(__float_as_uint(fabsf(v[2].x)), __float_as_uint(fabsf(v[3].x)))));
            }
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                acc_add(s[n], v[n]);
                acc_mul(ss[n], sg, v[n]);
            }
        }
    }
    if (dI) {
        im = __reduce_max_sync(0xffffffffu, im);
        if (lane == 0 && im) atomicMax(imax, im);
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        sh[wi][n][lane] = two_sum(s[n].s, s[n].c);
        sh[wi][4 + n][lane] = two_sum(ss[n].s, ss[n].c);
    }
    __syncwarp();
    const float2 *wq = wpair + (size_t)qd * 32 * 6;
    for (int m = lane; m < 36; m += 32) {
        const int n = m / 9, k = m - 9 * n;
        const int row = k < 6 ? n : 4 + n, wrow = k < 6 ? k : k - 6;
        Acc a;
        for (int j = 0; j < 32; ++j) acc_mul(a, wq[j * 6 + wrow], sh[wi][row][j]);
        part[((size_t)qd * ncell + cell) * 36 + m] = (double)a.s + (double)a.c;
    }
}

// Per (cell, group): the records as pairs (q at the nodes, sigma~, sigma) for
// the residual and the moments; the FP32 records of the correction sweep (no
// emission, the problem's sigma~ and sigma); and, when the pairs held the
// previous outer iteration's records (dq != NULL), FP32 records whose
// emission is the change of q since then.
__global__ void records_kernel(const double *__restrict__ rec, float2 *__restrict__ rec_df,
                               float *__restrict__ rec32, float *__restrict__ dq, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *a = rec + i * 8;
    float2 *o = rec_df + i * 6;
    float *f = rec32 + i * 8;
    const float s4 = __double2float_rn(a[4]), s5 = __double2float_rn(a[5]);
    if (dq) {
        float *h = dq + i * 8;
        for (int k = 0; k < 4; ++k) h[k] = __double2float_rn(a[k] - df_join(o[k]));
        h[4] = s4;
        h[5] = s5;
        h[6] = 0.0f;
        h[7] = 0.0f;
    }
    for (int k = 0; k < 6; ++k) o[k] = df_split(a[k]);
    for (int k = 0; k < 4; ++k) f[k] = 0.0f;
    f[4] = s4;
    f[5] = s5;
    f[6] = 0.0f;
    f[7] = 0.0f;
}

// FP64 values to pairs (n values), and back (in place: each thread reads its
// two FP32 numbers before it writes the FP64 number over them).
// y = pairs of x, and the bits of max |x| (high parts) into *xmax
__global__ void split_kernel(const double *__restrict__ x, float2 *__restrict__ y, size_t n,
                             unsigned int *__restrict__ xmax) {
    unsigned m = 0u;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = df_split(x[i]);
        y[i] = v;
        m = max(m, __float_as_uint(fabsf(v.x)));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(xmax, m);
}
// the pairs of xy (or of src, when given) joined into FP64 in xy; in place
// each thread reads its pair before writing its double over it
__global__ void join_kernel(void *xy, const float2 *src, size_t n) {
    const float2 *in = src ? src : static_cast<const float2 *>(xy);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = in[i];
        static_cast<double *>(xy)[i] = df_join(v);
    }
}

// mu, eta of every lane and the boundary inflow as pairs
__global__ void tables_kernel(const LaneConst *__restrict__ lanes, int nlanes,
                              const double *__restrict__ inflow, int ninflow,
                              float2 *__restrict__ mueta, float2 *__restrict__ inflow_df) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nlanes) {
        mueta[2 * i] = df_split(lanes[i].mu);
        mueta[2 * i + 1] = df_split(lanes[i].eta);
        // the moment weights of the lane as pairs, after the mu / eta table
        float2 *wp = mueta + 2 * (size_t)nlanes + 6 * (size_t)i;
#pragma unroll
        for (int k = 0; k < 6; ++k) wp[k] = df_split(lanes[i].wm[k]);
    }
    if (i < ninflow) inflow_df[i] = df_split(inflow[i]);
}

}  // namespace smk

struct sm_refine_state {
    float *r = nullptr, *d = nullptr;  // packed FP32 residual and correction
    float2 *ik = nullptr;              // packed I^k as pairs
    float2 *rec_df = nullptr;          // [cell][Gp][6] records as pairs
    float *rec32 = nullptr;            // [cell][Gp][8] FP32 records of the correction sweep
    float *rec_dq = nullptr;           // [cell][Gp][8] the same with the change of q as emission
    bool fresh = true;                 // no outer iteration of this step has run yet
    bool met = false;                  // the last solve's corrections met the tolerance
    float *inflow0 = nullptr;          // [4][Gp] zero inflow
    float2 *mueta = nullptr;           // [NQ*DB*32][2] mu, eta; then [NQ*DB*32][6] weights
    float2 *inflow_df = nullptr;       // [4][Gp]
    double *part = nullptr;            // [NQ*DB][cell][36] partial moments of the iterate
    float2 *alt = nullptr;             // the second iterate buffer (pairs)
    float2 *home = nullptr;            // the caller's buffer, the first (pairs during the step)
    const float2 *cur = nullptr;       // the iterate: ik at the step's start, then home / alt
    unsigned int *maxes = nullptr;     // max |d| of the last correction sweep, max |I| of
                                       // the iterate (FP32 bits)
    unsigned int *h_maxes = nullptr;   // pinned mirror
    int W = 0, S = 0, NS = 0;          // tiling of the FP32 correction sweep
    int resident = 0;                  // its CTAs that fit
    int corrections = 0;               // corrections of the running step
};

namespace smk {

void refine_free(sm_problem *p) {
    if (!p->refine) return;
    sm_refine_state &R = *p->refine;
    for (void *b : {(void *)R.r, (void *)R.d, (void *)R.ik, (void *)R.rec_df, (void *)R.rec32,
                    (void *)R.rec_dq,
                    (void *)R.inflow0, (void *)R.mueta, (void *)R.inflow_df, (void *)R.part,
                    (void *)R.maxes, (void *)R.alt})
        if (b) cudaFree(b);
    if (R.h_maxes) cudaFreeHost(R.h_maxes);
    delete p->refine;
    p->refine = nullptr;
}

sm_status refine_ensure(sm_problem *p) {
    if (p->refine) return SM_OK;
    if (p->dim != 2 || p->prec != 64) {
        set_last_error("FP64 defect correction needs a 2D problem with FP64 state (precision 64)");
        return SM_ERR_UNSUPPORTED;
    }
    p->refine = new sm_refine_state();
    sm_refine_state &R = *p->refine;
    const size_t ie = (size_t)p->NQ * p->NWT * p->ncell * p->GW * 32 * 4;
    const size_t nrec = (size_t)p->ncell * p->Gp;
    const size_t npart = (size_t)p->NQ * p->DB * p->ncell * 36;
    const int nlanes = p->NQ * p->DB * 32;
    if (cudaMalloc(&R.r, ie * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&R.d, ie * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&R.ik, ie * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&R.alt, ie * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&R.rec_df, nrec * 6 * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&R.rec32, nrec * 8 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&R.rec_dq, nrec * 8 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&R.inflow0, (size_t)4 * p->Gp * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&R.mueta, (size_t)nlanes * 8 * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&R.inflow_df, (size_t)4 * p->Gp * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&R.part, npart * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&R.maxes, 2 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMallocHost(&R.h_maxes, 2 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(R.inflow0, 0, (size_t)4 * p->Gp * sizeof(float)) != cudaSuccess) {
        refine_free(p);
        set_last_error("FP64 defect correction: device allocation failed");
        return SM_ERR_OOM;
    }
    const int ninfl = 4 * p->Gp, nt = std::max(nlanes, ninfl);
    tables_kernel<<<(nt + 127) / 128, 128, 0, p->stream>>>(
        p->d_lanes, nlanes, static_cast<const double *>(p->d_inflow), ninfl, R.mueta, R.inflow_df);
    if (cudaGetLastError() != cudaSuccess) {
        refine_free(p);
        set_last_error("FP64 defect correction: table launch failed");
        return SM_ERR_CUDA;
    }
    // the FP32 correction sweep's tiling: the widest strip (at most 16
    // columns) that fits with two prefetch stages and is no narrower than the
    // problem's own, so that its strips fit the face buffer and row flags
    for (int W : {16, 14, 12, 8, 6, 4, 2}) {
        if (W < p->W) break;
        const int r = sweep2d_max_resident_prec(32, p, W, 2, nullptr);
        if (r > 0) {
            R.W = W;
            R.S = 2;
            R.resident = r;
            break;
        }
    }
    if (R.resident <= 0) {
        R.W = p->W;
        R.S = p->S;
        R.resident = sweep2d_max_resident_prec(32, p, p->W, p->S, nullptr);
    }
    if (R.resident <= 0) {
        refine_free(p);
        set_last_error("FP64 defect correction: the FP32 sweep tiling does not fit");
        return SM_ERR_UNSUPPORTED;
    }
    R.NS = (p->nx + R.W - 1) / R.W;
    p->workspace_bytes += ie * 24 + nrec * 112 + (size_t)20 * p->Gp + (size_t)nlanes * 64 +
                          npart * 8 + 8;
    return SM_OK;
}

// Start of a refined step: I^k (FP64, packed) as pairs, and the iterate (held
// in the caller's FP64 buffer I, of the same size) set to them.
sm_status refine_begin(sm_problem *p, const double *I_k, void *I) {
    sm_refine_state &R = *p->refine;
    R.fresh = true;
    R.home = static_cast<float2 *>(I);
    R.cur = R.ik;  // the first update writes the iterate into the caller's buffer
    const size_t nv = (size_t)p->NQ * p->NWT * p->ncell * p->GW * 32 * 4;
    const unsigned blocks = (unsigned)std::min<size_t>((nv + 255) / 256, 152 * 16);
    if (cudaMemsetAsync(R.maxes, 0, 2 * sizeof(unsigned int), p->stream) != cudaSuccess) {
        set_last_error("FP64 defect correction: split launch failed");
        return SM_ERR_CUDA;
    }
    split_kernel<<<blocks, 256, 0, p->stream>>>(I_k, R.ik, nv, R.maxes + 1);
    if (cudaGetLastError() != cudaSuccess) {
        set_last_error("FP64 defect correction: split launch failed");
        return SM_ERR_CUDA;
    }
    p->launches++;
    return SM_OK;
}

// End of a refined step: the iterate joined back into FP64 in the caller's
// buffer (in place when it is there).
sm_status refine_end(sm_problem *p, void *I) {
    sm_refine_state &R = *p->refine;
    const size_t nv = (size_t)p->NQ * p->NWT * p->ncell * p->GW * 32 * 4;
    const unsigned blocks = (unsigned)std::min<size_t>((nv + 255) / 256, 152 * 16);
    const float2 *src = R.cur == static_cast<const float2 *>(I) ? nullptr : R.cur;
    join_kernel<<<blocks, 256, 0, p->stream>>>(I, src, nv);
    if (cudaGetLastError() != cudaSuccess) {
        set_last_error("FP64 defect correction: join launch failed");
        return SM_ERR_CUDA;
    }
    p->launches++;
    R.cur = static_cast<const float2 *>(I);
    return SM_OK;
}

// The transport solve of one outer iteration by defect correction of the
// iterate I (pairs, in the caller's buffer; the records hold the emission of
// the current temperature), then the moments of I into mom.  Synchronizes
// the stream after each correction (the stopping test reads the maxima).
sm_status refine_solve(sm_problem *p, void *I, double *mom) {
    if (p->refine->NS > p->NS) {
        // the problem's tiling changed since the workspace was made: the face
        // buffer and row flags hold p->NS strips, so pick the tiling again
        // (the step's pairs of I^k are kept)
        sm_refine_state &O = *p->refine;
        int W = 0, S = 0, res = 0;
        for (int w : {16, 14, 12, 8, 6, 4, 2}) {
            if (w < p->W) break;
            const int r = sweep2d_max_resident_prec(32, p, w, 2, nullptr);
            if (r > 0) {
                W = w;
                S = 2;
                res = r;
                break;
            }
        }
        if (res <= 0 || (p->nx + W - 1) / W > p->NS) {
            set_last_error("FP64 defect correction: no correction-sweep tiling fits the face buffer");
            return SM_ERR_UNSUPPORTED;
        }
        O.W = W;
        O.S = S;
        O.resident = res;
        O.NS = (p->nx + W - 1) / W;
    }
    sm_refine_state &R = *p->refine;
    cudaStream_t s = p->stream;
    const size_t ie = (size_t)p->NQ * p->NWT * p->ncell * p->GW * 32 * 4;
    const size_t nrec = (size_t)p->ncell * p->Gp;
    auto cuda_fail = [](const char *what) {
        set_last_error(what);
        return SM_ERR_CUDA;
    };
    // after the first outer iteration of the step the iterate solves the
    // previous records' equations to the stopping tolerance, and only the
    // emission q has changed since (sigma is frozen for the step), so the
    // residual is the change of q: the first correction sweeps it directly,
    // without the residual kernel
    const bool from_dq = !R.fresh && R.met;
    records_kernel<<<(unsigned)((nrec + 255) / 256), 256, 0, s>>>(
        static_cast<const double *>(p->d_src), R.rec_df, R.rec32, from_dq ? R.rec_dq : nullptr,
        nrec);
    R.fresh = false;
    if (cudaGetLastError() != cudaSuccess) return cuda_fail("FP64 defect correction: records launch failed");
    p->launches++;
    (void)I;  // the iterate is R.cur; the caller's buffer is R.home
    RefineArgs A;
    A.nx = p->nx;
    A.ny = p->ny;
    A.ncell = p->ncell;
    A.NQ = p->NQ;
    A.NWT = p->NWT;
    A.NGB = p->NGB;
    A.DB = p->DB;
    A.LG = p->LG;
    A.GW = p->GW;
    A.Gp = p->Gp;
    {
        const float hi = (float)p->inv_cdt;
        A.inv_cdt = make_float2(hi, (float)(p->inv_cdt - (double)hi));
    }
    A.lanes = p->d_lanes;
    A.mueta = R.mueta;
    A.rec = R.rec_df;
    A.inflow = R.inflow_df;
    A.I_k = R.ik;
    A.r = R.r;
    A.n_elems = ie / 4;
    const unsigned ublocks =
        (unsigned)std::max<size_t>(1, std::min<size_t>((ie / 4 + 255) / 256, 152 * 8));
    // The correction that meets the tolerance is added to the iterate by the
    // moments kernel (which reads the iterate anyway), writing the other
    // iterate buffer; the others by update_kernel, in place (out of place into
    // the caller's buffer while the iterate is still I^k's pairs).  So the
    // stopping test reads max |d| from a pass over d alone, and max |I| of the
    // iterate before the correction (split, update or moments kernel).
    bool pending = false;
    for (int c = 0; c < MAX_CORR; ++c) {
        const bool dq = from_dq && c == 0;
        if (pending) {
            float2 *out = R.cur == R.ik ? R.home : const_cast<float2 *>(R.cur);
            if (cudaMemsetAsync(R.maxes + 1, 0, sizeof(unsigned int), s) != cudaSuccess)
                return cuda_fail("FP64 defect correction: update launch failed");
            update_kernel<<<ublocks, 256, 0, s>>>(R.cur, R.d, out, ie / 4, R.maxes + 1);
            if (cudaGetLastError() != cudaSuccess)
                return cuda_fail("FP64 defect correction: update launch failed");
            p->launches++;
            R.cur = out;
            pending = false;
        }
        if (!dq) {
            A.I = R.cur;
            residual_kernel<<<(unsigned)((A.n_elems + 255) / 256), 256, 0, s>>>(A);
            if (cudaGetLastError() != cudaSuccess)
                return cuda_fail("FP64 defect correction: residual launch failed");
            p->launches++;
        }
        // the FP32 correction sweep: source r (or the change of q), no
        // emission, zero inflow, its own tiling, no moment stage
        ++p->epoch;
        SweepArgs a = make_sweep_args(p, dq ? nullptr : R.r, R.d);
        a.src = dq ? R.rec_dq : R.rec32;
        a.inflow = R.inflow0;
        a.inv_cdt = 1.0;
        a.W = R.W;
        a.S = R.S;
        a.NS = R.NS;
        a.strip_x0 = nullptr;  // uniform strips of R.W columns
        a.mom_acc = nullptr;   // no moments: those of the iterate are taken after
        a.n_tasks = R.NS * p->NQ * p->NWT;
        a.publish = publish_rows(a.n_tasks, R.resident);
        if (cudaMemsetAsync(p->d_ctrl, 0, 2 * sizeof(unsigned int), s) != cudaSuccess ||
            cudaMemsetAsync(R.maxes, 0, sizeof(unsigned int), s) != cudaSuccess ||
            launch_sweep2d_prec(32, p, a, std::min(a.n_tasks, R.resident), s) != cudaSuccess)
            return cuda_fail("FP64 defect correction: correction sweep launch failed");
        dmax_kernel<<<ublocks, 256, 0, s>>>(reinterpret_cast<const float4 *>(R.d), ie / 4,
                                            R.maxes);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(R.h_maxes, R.maxes, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost,
                            s) != cudaSuccess)
            return cuda_fail("FP64 defect correction: correction sweep launch failed");
        p->launches += 2;
        pending = true;
        ++R.corrections;
        const sm_status st = sm_synchronize(p);  // also reports a wavefront timeout
        if (st != SM_OK) return st;
        float dmax, imax;
        std::memcpy(&dmax, &R.h_maxes[0], sizeof(dmax));
        std::memcpy(&imax, &R.h_maxes[1], sizeof(imax));
        if (!std::isfinite(dmax) || !std::isfinite(imax)) {
            set_last_error("FP64 defect correction: the correction is not finite");
            return SM_ERR_NONPHYSICAL;
        }
        // max |I| of the iterate before this correction: the test's scale
        // (the correction is tiny next to I whenever the test can pass)
        R.met = (double)dmax <= CORR_TOL * (double)imax;
        if (R.met) break;
    }
    // the last correction's update with the moments of the updated iterate,
    // into the iterate buffer that is not being read
    float2 *out = R.cur == R.home ? R.alt : R.home;
    if (pending && cudaMemsetAsync(R.maxes + 1, 0, sizeof(unsigned int), s) != cudaSuccess)
        return cuda_fail("FP64 defect correction: moments launch failed");
    const long long warps = (long long)p->NQ * p->DB * p->ncell;
    moments_kernel<<<(unsigned)((warps + MOM_WARPS - 1) / MOM_WARPS), MOM_WARPS * 32, 0, s>>>(
        R.cur, pending ? R.d : nullptr, out, R.maxes + 1, p->d_lanes,
        R.mueta + 2 * (size_t)p->NQ * p->DB * 32, R.rec_df, p->ncell, p->NQ, p->DB, p->NGB,
        p->NWT, p->GW, p->LG, p->Gp, R.part);
    if (cudaGetLastError() != cudaSuccess ||
        launch_reduce_prec(64, p, R.part, p->NQ * p->DB, mom, nullptr, s) != cudaSuccess)
        return cuda_fail("FP64 defect correction: moments launch failed");
    p->launches += 2;
    if (pending) R.cur = out;
    return SM_OK;
}

int refine_take_corrections(sm_problem *p) {
    if (!p->refine) return 0;
    const int c = p->refine->corrections;
    p->refine->corrections = 0;
    return c;
}

}  // namespace smk
