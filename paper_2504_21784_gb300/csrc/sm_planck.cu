// FP64 Planck / Rosseland group integrals and the kernels built on them:
// multigroup opacity, emission source (row a1), boundary inflow and the
// closures recomputed from a temperature (row a4 standalone).  The series,
// the Taylor tables and the emission of one node are in sm_planck.cuh; this
// file holds the tables (derived on the host, uploaded once per device) and
// the kernels.
#include <math.h>

#include <atomic>

#include "sm_internal.cuh"
#include "sm_planck.cuh"

namespace smk {

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

// The host copies of every table (the double-FP32 emission derives its own
// from them).
void planck_host_tables(double head[NBERN], double bern[NBERN], double cexp_out[3],
                        double exp2_tab[64], double (*ptab)[2][NTAY]) {
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
    cexp_out[0] = (double)(64.0L / ln2);
    cexp_out[1] = l64_hi;
    cexp_out[2] = (double)(l64 - (long double)l64_hi);
    for (int j = 0; j < 64; ++j) exp2_tab[j] = (double)exp2l(-(long double)j / 64.0L);
    planck_taylor_tables(ptab);
}

void planck_upload_tables(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return;
    if (g_tables_ready[dev].load(std::memory_order_acquire)) return;
    double head[NBERN], bern[NBERN], cexp[3], tab[64];
    static double ptab[NCEN][2][NTAY];
    planck_host_tables(head, bern, cexp, tab, ptab);
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

// The tables as module globals (the emission, inflow and closure kernels).
struct GlobalTabs {
    __device__ __forceinline__ double head(int k) const { return c_head[k]; }
    __device__ __forceinline__ double bern(int k) const { return c_bern[k]; }
    __device__ __forceinline__ double cexp(int i) const { return c_exp[i]; }
    __device__ __forceinline__ double exp2(int j) const { return __ldg(&g_exp2_tab[j]); }
    __device__ __forceinline__ double pcen(int j) const { return __ldg(&g_pcen[j]); }
    __device__ __forceinline__ const double *ptab(int j) const { return &g_ptab[j][0][0]; }
};

__device__ __forceinline__ EdgeVals edge_vals(double x) { return edge_vals(x, GlobalTabs()); }

// Test hook kernel: e^{-x} by exp_neg where it applies (0 <= x < 708).
__global__ void exp_neg_kernel(const double *__restrict__ x, double *__restrict__ out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    out[i] = (v >= 0.0 && v < 708.0) ? exp_neg(v, GlobalTabs()) : exp(-v);
}

// Host: the tables as a kernel parameter (for the sweep with fused emission).
bool planck_tabs(PlanckTabs *out) {
    planck_upload_tables();
    if (cudaMemcpyFromSymbol(out->head, c_head, sizeof(out->head)) != cudaSuccess ||
        cudaMemcpyFromSymbol(out->bern, c_bern, sizeof(out->bern)) != cudaSuccess ||
        cudaMemcpyFromSymbol(out->cexp, c_exp, sizeof(out->cexp)) != cudaSuccess)
        return false;
    void *a = nullptr, *b = nullptr, *c = nullptr;
    if (cudaGetSymbolAddress(&a, g_ptab) != cudaSuccess ||
        cudaGetSymbolAddress(&b, g_pcen) != cudaSuccess ||
        cudaGetSymbolAddress(&c, g_exp2_tab) != cudaSuccess)
        return false;
    out->ptab = static_cast<const double *>(a);
    out->pcen = static_cast<const double *>(b);
    out->exp2 = static_cast<const double *>(c);
    return true;
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
    // counts are warp maxima).
    const int n_nodes = ncell * nn;
    const int t_raw = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t_raw < n_nodes;
    const int t = active ? t_raw : n_nodes - 1;
    const int cell = t / nn, node = t - cell * nn;
    emit_node<RT>(cell, node, active, ncell, nn, G, Gp, edges, s_edges, acT4_scale, inv_cdt, T,
                  sigma, src, gray, qcanon, ctrl + CTRL_STATUS, ST_NONPHYSICAL, GlobalTabs());
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
        o[3] = (phi > 0.0 && m[3] > 0.0) ? m[3] / phi : sP;
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
        o[6] = (phi > 0.0 && m[6] > 0.0) ? m[6] / phi : sP;
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
    // an FP32 problem's sweeps: the double-FP32 evaluation (sm_planck_df.cu)
    if (p->prec == 32 && !q_canon && !p->emit_fp64) return launch_emission_df(p, T, sigma, s, active);
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
