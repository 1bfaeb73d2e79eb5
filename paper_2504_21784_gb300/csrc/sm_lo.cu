// Gray low-order solve and the full time step, FP64 on the device:
//  * the independent LDG low-order system of Sec. 4 (fluxes with kappa =
//    alpha/2 and s = sign(w.n), w = (1, 1); Marshak-type boundary; closure
//    source R1_ind), lumped with the 2-point Gauss-Lobatto rule (Sec. 6);
//  * the Newton iteration of Sec. 5 with frozen gray opacities, the
//    pseudo-fission linearisation of the emission (Eq. pseudo_fission) and the
//    pointwise nonlinear temperature elimination (Eq. nonlinear_T_update);
//  * the Schur complement in E (Eq. schur), symmetric positive definite for
//    lumped forms, solved by Jacobi-preconditioned conjugate gradients in
//    the single-reduction form of Chronopoulos and Gear;
//  * Algorithm 1 (outer fixed point between the transport sweep and the
//    low-order solve) with the relative stopping rule Eq. relative_tol.
//
// Unknowns are nodal (cell corners): E_n and F_n = (F_x, F_y).  With the
// interior faces oriented +x / +y, s = +1, so F^.n takes the low-side F and
// P^ n the high-side E.  The lumped A_FF = m sigma~_F is diagonal, which makes
// S = A_EE - A_EF A_FF^-1 A_FE a stencil over a cell and its four face
// neighbours; its coefficients are assembled once per low-order solve (only
// aE on its diagonal changes between Newton iterations).
//
// GB300 runs FP64 at about 1/64 of its FP32 rate (roughly two FP64 FMAs per
// clock per SM), so these kernels are bound by FP64 instruction count, not by
// memory: the whole working set of a 256x256 mesh is a few MB and stays in
// L2.  The design therefore minimises FP64 work: one thread per cell (the
// four nodes of a cell share their stencil loads and partial sums, read as
// double2 vectors), the stencil of S assembled once per solve, 1/A_FF and
// 1/diag(S) precomputed so that conjugate-gradient iterations divide nothing,
// block and grid sums taken by one warp per block,
// and the pointwise temperature Newton step taken with an FP32 reciprocal of
// its derivative (a quasi-Newton step: the root is unchanged).  PCG scalars
// never leave the device: grid-wide sums are deterministic fixed-order sums
// (no floating-point atomics), and the whole Newton iteration of a low-order
// solve -- set-up, conjugate gradients and finish of every Newton step, and
// the stopping tests -- is one cooperative launch whose blocks meet at grid
// barriers with bounded waits, so the host synchronises once per solve.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "sm_internal.cuh"

namespace smk {
namespace lo {

constexpr int BLOCK = 128;
enum { DONE_NO = 0, DONE_CONVERGED = 1, DONE_BREAKDOWN = 2, DONE_CAPPED = 3, DONE_TIMEOUT = 4 };

struct Scalars {
    double d2, n2;       // outer iteration: squared norms of the change of (T, E) and of (T, E)
    int elim_max;        // most temperature-elimination iterations of any node
    unsigned int count;  // arrivals of the running kernel's blocks
    unsigned int bar_count;  // arrivals at the cooperative kernel's grid barriers
    // statistics of the last low-order solve (cooperative Newton kernel)
    int newton_iters, pcg_total, pcg_max, pcg_capped, status;
};
enum { LO_OK = 0, LO_BREAKDOWN = 1, LO_TIMEOUT = 2, LO_NONFINITE = 3 };

struct Geo {
    int dim, nx, ny, ncell, N;
    double m, c;
    double wfx, wfy;        // Gauss-Lobatto weights of x- and y-faces
    double kx, ky, fx, fy;  // A_FE: volume (c/3) m / h, faces (c/3) wf
    double lx, ly;          // A_EF volume: m / h
    double px, py, bx, by;  // interior penalty (c alpha / 2) wf, boundary c alpha wf
    double c3;              // c / 3
    double alpha;           // Eq. alpha of the S_N set
};

struct Cell {
    int k, ix, iy;
    bool L, R, B, T;  // face neighbours present (left, right, bottom, top)
};

__device__ __forceinline__ Cell cell_of(const Geo &G, int k) {
    Cell C;
    C.k = k;
    C.iy = k / G.nx;
    C.ix = k - C.iy * G.nx;
    C.L = C.ix > 0;
    C.R = C.ix + 1 < G.nx;
    C.B = C.iy > 0;
    C.T = C.iy + 1 < G.ny;
    return C;
}

// the NN nodal values of cell k ([cell][node] arrays, 16-byte aligned)
template <int NN>
__device__ __forceinline__ void ldc(const double *__restrict__ a, int k, double (&v)[NN]) {
    const double2 *p = reinterpret_cast<const double2 *>(a + (size_t)k * NN);
#pragma unroll
    for (int i = 0; i < NN / 2; ++i) {
        const double2 t = p[i];
        v[2 * i] = t.x;
        v[2 * i + 1] = t.y;
    }
}
template <int NN>
__device__ __forceinline__ void stc(double *__restrict__ a, int k, const double (&v)[NN]) {
    double2 *p = reinterpret_cast<double2 *>(a + (size_t)k * NN);
#pragma unroll
    for (int i = 0; i < NN / 2; ++i) p[i] = make_double2(v[2 * i], v[2 * i + 1]);
}

// Accessors of the nodal values of cell k, with loads that bypass L1
// (ld.global.cg): the cooperative low-order kernel reads values that other
// blocks of the same launch wrote (E, x, diag(S) and the PCG's r, w, s).
template <int NN>
__device__ __forceinline__ void ldc_cg(const double *a, int k, double (&v)[NN]) {
    const double2 *p = reinterpret_cast<const double2 *>(a + (size_t)k * NN);
#pragma unroll
    for (int i = 0; i < NN / 2; ++i) {
        const double2 t = __ldcg(p + i);
        v[2 * i] = t.x;
        v[2 * i + 1] = t.y;
    }
}
template <int NN>
struct VecCG {
    const double *v;
    __device__ __forceinline__ void get(int k, double (&o)[NN]) const { ldc_cg<NN>(v, k, o); }
    __device__ __forceinline__ double get1(int k, int n) const {
        return __ldcg(v + (size_t)k * NN + n);
    }
};

// Node numbering inside a cell: n = a + 2b (2D), n = a (1D); a, b = 0 on the
// low x / y side.  x-rows are the node pairs (2b, 2b+1), y-columns (a, a+2).
//
// q = S e = A_EE e - A_EF A_FF^-1 A_FE e on the nodes of cell C; e receives
// the cell's own values.  Per x-row, with s = e_0 + e_1 and ia = 1/A_FF:
//   u_0 = ((c/3) m/h s - (c/3) wf e_0) ia_0        (first-moment rows, A_FE:
//   u_1 = ((c/3) wf e^ - (c/3) m/h s) ia_1          volume -(c/3) div v E, face
//                                                   (c/3)[v.n] E^, E^ the high
//                                                   side / own value on the
//                                                   boundary)
//   (A_EF u)_0 = m/h (u_0 + u_1) - wf u_1^left      (volume -grad u . F, face
//   (A_EF u)_1 = -m/h (u_0 + u_1) + wf u_1          [u] F^.n, F^ the low side)
// and A_EE adds aE e, the penalty (c alpha/2) wf (e - e_nb) on interior
// faces and c alpha wf e on the boundary.  The left neighbour's u_1 needs
// only its own row and this cell's e_0, so it is recomputed here.
// T: the arithmetic (FP64, or FP32 for the inner solves of the mixed-precision
// conjugate gradients), GT its geometry coefficients, IA the 1/A_FF array's
// accessor (ia(k, n)).
template <typename T, int NN, class Acc, class GT, class IA>
__device__ __forceinline__ void schur_cell_t(const GT &G, const Cell &C, const Acc &acc,
                                             const T (&aE)[NN], const IA &iaF, T (&q)[NN],
                                             T (&e)[NN]) {
    T eL[NN], eR[NN], ia[NN];
    acc.get(C.k, e);
    if (C.L) acc.get(C.k - 1, eL);
    if (C.R) acc.get(C.k + 1, eR);
#pragma unroll
    for (int n = 0; n < NN; ++n) ia[n] = iaF(C.k, n);
#pragma unroll
    for (int n = 0; n < NN; ++n) q[n] = aE[n] * e[n];
#pragma unroll
    for (int b = 0; b < NN / 2; ++b) {
        const int n0 = 2 * b, n1 = 2 * b + 1;
        const T s = e[n0] + e[n1];
        const T u0 = (G.kx * s - G.fx * e[n0]) * ia[n0];
        const T u1 = (G.fx * (C.R ? eR[n0] : e[n1]) - G.kx * s) * ia[n1];
        const T sv = G.lx * (u0 + u1);
        T v0 = sv, v1 = -sv;
        if (C.L) {
            const T uL = (G.fx * e[n0] - G.kx * (eL[n0] + eL[n1])) * iaF(C.k - 1, n1);
            v0 -= G.wfx * uL;
            q[n0] += G.px * (e[n0] - eL[n1]);
        } else {
            q[n0] += G.bx * e[n0];
        }
        if (C.R) {
            v1 += G.wfx * u1;
            q[n1] += G.px * (e[n1] - eR[n0]);
        } else {
            q[n1] += G.bx * e[n1];
        }
        q[n0] -= v0;
        q[n1] -= v1;
    }
    if constexpr (NN == 4) {
        T eB[NN], eT[NN];
        if (C.B) acc.get(C.k - G.nx, eB);
        if (C.T) acc.get(C.k + G.nx, eT);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int n0 = a, n1 = a + 2;
            const T s = e[n0] + e[n1];
            const T u0 = (G.ky * s - G.fy * e[n0]) * ia[n0];
            const T u1 = (G.fy * (C.T ? eT[n0] : e[n1]) - G.ky * s) * ia[n1];
            const T sv = G.ly * (u0 + u1);
            T v0 = sv, v1 = -sv;
            if (C.B) {
                const T uB = (G.fy * e[n0] - G.ky * (eB[n0] + eB[n1])) * iaF(C.k - G.nx, n1);
                v0 -= G.wfy * uB;
                q[n0] += G.py * (e[n0] - eB[n1]);
            } else {
                q[n0] += G.by * e[n0];
            }
            if (C.T) {
                v1 += G.wfy * u1;
                q[n1] += G.py * (e[n1] - eT[n0]);
            } else {
                q[n1] += G.by * e[n1];
            }
            q[n0] -= v0;
            q[n1] -= v1;
        }
    }
}

// the FP32 copy of the 1/A_FF array (mixed-precision inner solves)
template <int NN> struct IaF {
    const float *a;
    __device__ __forceinline__ float operator()(int k, int n) const {
        return __ldcg(a + (size_t)k * NN + n);
    }
};

// The stencil of S assembled once per low-order solve: S = A_EE - A_EF
// A_FF^-1 A_FE depends on the Newton iterate only through aE on its diagonal
// (A_FF holds the closures' sigma~_F, fixed for the solve), so every other
// coefficient is formed once from 1/A_FF and the geometry, by differentiating
// the cell formula of schur_cell_t term by term, and a conjugate-gradient
// matrix-vector product costs one FMA per coefficient instead of the formula's
// FP64 work.  Coefficients of cell k at Sc + k * Stencil<NN>::n:
//   2D: [0..3] geometric diagonal g_n (diag(S) = aE_n + g_n); own-cell
//       couplings (0,1) 4, (0,2) 5, (1,0) 6, (1,3) 7, (2,0) 8, (2,3) 9,
//       (3,1) 10, (3,2) 11; neighbour couplings, (row <- cell node):
//       0 <- L0 12, L1 13, B0 14, B2 15, R0 16, T0 17;
//       1 <- R0 18, B1 19, B3 20, T1 21;  2 <- L2 22, L3 23, R2 24, T0 25;
//       3 <- R2 26, T1 27  (L, R, B, T: the left, right, bottom, top cell;
//       zero where that face is a boundary).
//   1D: [0..1] g_n; (0,1) 2, (1,0) 3; 0 <- L0 4, L1 5, R0 6; 1 <- R0 7.
template <int NN> struct Stencil;
template <> struct Stencil<4> { static constexpr int n = 28; };
template <> struct Stencil<2> { static constexpr int n = 8; };

// The coefficients one row pair (x) or node column (y) adds, with k_, f_,
// l_, wf, pen, bnd its kx, fx, lx, wfx, px, bx (or the y ones), ia0 / ia1
// the 1/A_FF of its low / high node, lo / hi whether its low / high face is
// interior and iaLo the low neighbour's 1/A_FF at that neighbour's high node.
// oa = (n0, n1), ob = (n1, n0), hA = (n0 <- hi n0), hB = (n1 <- hi n0),
// lA = (n0 <- lo n0), lB = (n0 <- lo n1).
__device__ __forceinline__ void axis_coefs(double k_, double f_, double l_, double wf, double pen,
                                           double bnd, double ia0, double ia1, bool lo, bool hi,
                                           double iaLo, double *c, int n0, int n1, int oa, int ob,
                                           int hA, int hB, int lA, int lB) {
    // u0 = ia0 (k s - f e_n0), u1 = ia1 (f e^ - k s), s = e_n0 + e_n1,
    // e^ = the high neighbour's e_n0 (interior face) or e_n1 (boundary)
    const double a0 = ia0 * (k_ - f_), a1 = ia0 * k_;
    const double b0 = -ia1 * k_;
    const double b1 = hi ? -ia1 * k_ : ia1 * (f_ - k_);
    const double bH = hi ? ia1 * f_ : 0.0;
    // sv = l (u0 + u1): q_n0 -= sv, q_n1 += sv
    const double s0 = l_ * (a0 + b0), s1 = l_ * (a1 + b1), sH = l_ * bH;
    c[n0] -= s0;
    c[oa] -= s1;
    c[n1] += s1;
    c[ob] += s0;
    if (lo) {
        // q_n0 += wf uL + pen (e_n0 - eL_n1), uL = iaLo (f e_n0 - k (eL_n0 + eL_n1))
        c[n0] += wf * iaLo * f_ + pen;
        c[lA] -= wf * iaLo * k_;
        c[lB] -= wf * iaLo * k_ + pen;
    } else {
        c[n0] += bnd;
    }
    if (hi) {
        // q_n0 -= sv's high part; q_n1 += sv's high part - wf u1 + pen (e_n1 - eH_n0)
        c[hA] -= sH;
        c[n1] += pen - wf * b1;
        c[ob] -= wf * b0;
        c[hB] += sH - wf * bH - pen;
    } else {
        c[n1] += bnd;
    }
}

// One thread per cell: the cell's stencil coefficients from 1/A_FF (its own
// and its low neighbours') and the geometry.
template <int NN>
__global__ void __launch_bounds__(BLOCK)
stencil_kernel(Geo G, const double *__restrict__ iaF, double *__restrict__ Sc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.ncell) return;
    const Cell C = cell_of(G, k);
    constexpr int NS = Stencil<NN>::n;
    double c[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) c[i] = 0.0;
    double ia[NN];
    ldc<NN>(iaF, k, ia);
    if constexpr (NN == 4) {
        const double iaL0 = C.L ? iaF[(size_t)(k - 1) * NN + 1] : 0.0;
        const double iaL1 = C.L ? iaF[(size_t)(k - 1) * NN + 3] : 0.0;
        const double iaB0 = C.B ? iaF[(size_t)(k - G.nx) * NN + 2] : 0.0;
        const double iaB1 = C.B ? iaF[(size_t)(k - G.nx) * NN + 3] : 0.0;
        axis_coefs(G.kx, G.fx, G.lx, G.wfx, G.px, G.bx, ia[0], ia[1], C.L, C.R, iaL0, c, 0, 1,
                   4, 6, 16, 18, 12, 13);
        axis_coefs(G.kx, G.fx, G.lx, G.wfx, G.px, G.bx, ia[2], ia[3], C.L, C.R, iaL1, c, 2, 3,
                   9, 11, 24, 26, 22, 23);
        axis_coefs(G.ky, G.fy, G.ly, G.wfy, G.py, G.by, ia[0], ia[2], C.B, C.T, iaB0, c, 0, 2,
                   5, 8, 17, 25, 14, 15);
        axis_coefs(G.ky, G.fy, G.ly, G.wfy, G.py, G.by, ia[1], ia[3], C.B, C.T, iaB1, c, 1, 3,
                   7, 10, 21, 27, 19, 20);
    } else {
        const double iaL = C.L ? iaF[(size_t)(k - 1) * NN + 1] : 0.0;
        axis_coefs(G.kx, G.fx, G.lx, G.wfx, G.px, G.bx, ia[0], ia[1], C.L, C.R, iaL, c, 0, 1, 2,
                   3, 6, 7, 4, 5);
    }
    double2 *o = reinterpret_cast<double2 *>(Sc + (size_t)k * NS);
#pragma unroll
    for (int i = 0; i < NS / 2; ++i) o[i] = make_double2(c[2 * i], c[2 * i + 1]);
}

// q = S e on the nodes of cell C from the assembled stencil (the operator of
// schur_cell_t up to rounding); e receives the cell's own values.
template <int NN, class Acc>
__device__ __forceinline__ void schur_cell(const Geo &G, const Cell &C, const Acc &acc,
                                           const double (&aE)[NN], const double *__restrict__ Sc,
                                           double (&q)[NN], double (&e)[NN]) {
    constexpr int NS = Stencil<NN>::n;
    double c[NS];
    const double2 *cp = reinterpret_cast<const double2 *>(Sc + (size_t)C.k * NS);
#pragma unroll
    for (int i = 0; i < NS / 2; ++i) {
        const double2 t = __ldg(cp + i);
        c[2 * i] = t.x;
        c[2 * i + 1] = t.y;
    }
    acc.get(C.k, e);
    if constexpr (NN == 4) {
        double eL[4] = {0.0, 0.0, 0.0, 0.0}, eB[4] = {0.0, 0.0, 0.0, 0.0};
        double eR0 = 0.0, eR2 = 0.0, eT0 = 0.0, eT1 = 0.0;
        if (C.L) acc.get(C.k - 1, eL);
        if (C.B) acc.get(C.k - G.nx, eB);
        if (C.R) {
            eR0 = acc.get1(C.k + 1, 0);
            eR2 = acc.get1(C.k + 1, 2);
        }
        if (C.T) {
            eT0 = acc.get1(C.k + G.nx, 0);
            eT1 = acc.get1(C.k + G.nx, 1);
        }
        q[0] = fma(aE[0] + c[0], e[0],
                   fma(c[4], e[1],
                       fma(c[5], e[2],
                           fma(c[12], eL[0],
                               fma(c[13], eL[1],
                                   fma(c[14], eB[0],
                                       fma(c[15], eB[2], fma(c[16], eR0, c[17] * eT0))))))));
        q[1] = fma(aE[1] + c[1], e[1],
                   fma(c[6], e[0],
                       fma(c[7], e[3],
                           fma(c[18], eR0, fma(c[19], eB[1], fma(c[20], eB[3], c[21] * eT1))))));
        q[2] = fma(aE[2] + c[2], e[2],
                   fma(c[8], e[0],
                       fma(c[9], e[3],
                           fma(c[22], eL[2], fma(c[23], eL[3], fma(c[24], eR2, c[25] * eT0))))));
        q[3] = fma(aE[3] + c[3], e[3],
                   fma(c[10], e[1], fma(c[11], e[2], fma(c[26], eR2, c[27] * eT1))));
    } else {
        double eL[2] = {0.0, 0.0}, eR0 = 0.0;
        if (C.L) acc.get(C.k - 1, eL);
        if (C.R) eR0 = acc.get1(C.k + 1, 0);
        q[0] = fma(aE[0] + c[0], e[0],
                   fma(c[2], e[1], fma(c[4], eL[0], fma(c[5], eL[1], c[6] * eR0))));
        q[1] = fma(aE[1] + c[1], e[1], fma(c[3], e[0], c[7] * eR0));
    }
}

// The geometry coefficients in FP32 (the inner solves of the mixed-precision
// conjugate gradients).
struct GeoF {
    int nx;
    float kx, ky, fx, fy, lx, ly, px, py, bx, by, wfx, wfy;
};
__device__ __forceinline__ GeoF geo_f(const Geo &G) {
    GeoF g;
    g.nx = G.nx;
    g.kx = (float)G.kx; g.ky = (float)G.ky; g.fx = (float)G.fx; g.fy = (float)G.fy;
    g.lx = (float)G.lx; g.ly = (float)G.ly; g.px = (float)G.px; g.py = (float)G.py;
    g.bx = (float)G.bx; g.by = (float)G.by; g.wfx = (float)G.wfx; g.wfy = (float)G.wfy;
    return g;
}

// FP32 nodal values of cell k (read past L1: written by other blocks)
template <int NN>
__device__ __forceinline__ void ldf(const float *a, int k, float (&v)[NN]) {
    if constexpr (NN == 4) {
        const float4 t = __ldcg(reinterpret_cast<const float4 *>(a) + k);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        const float2 t = __ldcg(reinterpret_cast<const float2 *>(a) + k);
        v[0] = t.x; v[1] = t.y;
    }
}
template <int NN>
__device__ __forceinline__ void stf(float *a, int k, const float (&v)[NN]) {
    if constexpr (NN == 4)
        reinterpret_cast<float4 *>(a)[k] = make_float4(v[0], v[1], v[2], v[3]);
    else
        reinterpret_cast<float2 *>(a)[k] = make_float2(v[0], v[1]);
}
template <int NN> struct VecF {
    const float *v;
    __device__ __forceinline__ void get(int k, float (&o)[NN]) const { ldf<NN>(v, k, o); }
};
// an FP32 vector read as FP64 (the refinement's residual update r -= S e)
template <int NN> struct VecFD {
    const float *v;
    __device__ __forceinline__ void get(int k, double (&o)[NN]) const {
        float t[NN];
        ldf<NN>(v, k, t);
#pragma unroll
        for (int i = 0; i < NN; ++i) o[i] = (double)t[i];
    }
    __device__ __forceinline__ double get1(int k, int n) const {
        return (double)__ldcg(v + (size_t)k * NN + n);
    }
};
// the inner solve's search direction p = u + beta p_old of cell k, on the fly
template <int NN> struct DirF {
    const float *u, *p;
    float beta;
    __device__ __forceinline__ void get(int k, float (&o)[NN]) const {
        float a[NN], b[NN];
        ldf<NN>(u, k, a);
        ldf<NN>(p, k, b);
#pragma unroll
        for (int i = 0; i < NN; ++i) o[i] = __fmaf_rn(beta, b[i], a[i]);
    }
};

// A_EF u on the nodes of cell C for a materialised u[node][dim].
template <int NN>
__device__ __forceinline__ void ef_cell(const Geo &G, const Cell &C, const double *__restrict__ u,
                                        double (&out)[NN]) {
    constexpr int D = NN == 4 ? 2 : 1;
    const double *uk = u + (size_t)C.k * NN * D;
#pragma unroll
    for (int b = 0; b < NN / 2; ++b) {
        const int n0 = 2 * b, n1 = 2 * b + 1;
        const double sv = G.lx * (uk[n0 * D] + uk[n1 * D]);
        out[n0] = sv - (C.L ? G.wfx * u[((size_t)(C.k - 1) * NN + n1) * D] : 0.0);
        out[n1] = -sv + (C.R ? G.wfx * uk[n1 * D] : 0.0);
    }
    if constexpr (NN == 4) {
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int n0 = a, n1 = a + 2;
            const double sv = G.ly * (uk[n0 * D + 1] + uk[n1 * D + 1]);
            out[n0] += sv - (C.B ? G.wfy * u[((size_t)(C.k - G.nx) * NN + n1) * D + 1] : 0.0);
            out[n1] += -sv + (C.T ? G.wfy * uk[n1 * D + 1] : 0.0);
        }
    }
}

// (A_FE e) components on the nodes of cell C (not divided by A_FF).
template <int NN, class Acc>
__device__ __forceinline__ void fe_cell(const Geo &G, const Cell &C, const Acc &acc,
                                        double (&e)[NN], double (&ax)[NN], double (&ay)[NN]) {
    double eR[NN];
    acc.get(C.k, e);
    if (C.R) acc.get(C.k + 1, eR);
#pragma unroll
    for (int b = 0; b < NN / 2; ++b) {
        const int n0 = 2 * b, n1 = 2 * b + 1;
        const double s = e[n0] + e[n1];
        ax[n0] = G.kx * s - G.fx * e[n0];
        ax[n1] = G.fx * (C.R ? eR[n0] : e[n1]) - G.kx * s;
    }
    if constexpr (NN == 4) {
        double eT[NN];
        if (C.T) acc.get(C.k + G.nx, eT);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int n0 = a, n1 = a + 2;
            const double s = e[n0] + e[n1];
            ay[n0] = G.ky * s - G.fy * e[n0];
            ay[n1] = G.fy * (C.T ? eT[n0] : e[n1]) - G.ky * s;
        }
    }
}

// ---------------------------------------------------------------------------
// Grid-wide sums finished by the last block to arrive: every block writes its
// partial sums, the last one adds all partials in block order (deterministic)
// and resets the arrival counter.  Returns true in thread 0 of the last block,
// with the totals in v.  Every thread of every block must call it.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <int K>
__device__ bool grid_sums(double (&v)[K], double *part, unsigned int *count) {
    __shared__ double sh[BLOCK / 32][K];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
        for (int k = 0; k < K; ++k) sh[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[w][k];
            part[(size_t)blockIdx.x * K + k] = s;
        }
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            s += __ldcg(part + (size_t)b * K + k);
        v[k] = warp_sum(s);
    }
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < K; ++k) sh[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x != 0) return false;
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sh[w][k];
        v[k] = s;
    }
    *count = 0u;
    return true;
}

// ---------------------------------------------------------------------------
// Consistent-method sources (Sec. 4, consistent; the discrete residual
// approach applied to the lumped upwind DG transport): for each node, the
// difference between the LDG face terms evaluated with the high-order moments
// and the moments of the upwind face terms of the transport discretization.
// With F^pm_n = sum_{Omega.n >< 0} w (Omega.n) I and Pi^pm_n = sum_{Omega.n >< 0}
// w Omega (Omega.n) I from the per-quadrant moments qm[node][q][phi, F_x, F_y,
// Pi_xx, Pi_xy, Pi_yy], and K1 / K2 the low / high side of an interior face:
//   R0(K1 node) = w_f [F.n(K1) + (c alpha/2)(E_K1 - E_K2) - F^+_n(K1) - F^-_n(K2)],
//   R0(K2 node) = -R0(K1 node),
//   R1(K1 node) = w_f [(c/3) n E_K2 - Pi^+_n(K1) - Pi^-_n(K2)],  R1(K2 node) = -R1(K1 node),
// and on the boundary (outward n, inflow moments J_in, Pi_in of the side):
//   R0 = w_f [J_in + alpha phi - F^+_n],  R1 = w_f [(c/3) n E - Pi^+_n - Pi_in].
struct Half {
    double Fp, Fm, Pp[2], Pm[2];
};

// half-range moments of node j for the normal +x (axis 0) or +y (axis 1):
// F^pm = sum_{Omega_axis >< 0} w Omega_axis I and the x, y components of
// Pi^pm = sum_{Omega_axis >< 0} w Omega Omega_axis I; quadrants in the
// canonical order (+,+), (-,+), (-,-), (+,-)
__device__ __forceinline__ Half half_pos_axis(const double *__restrict__ qm, int j, int axis) {
    const double *q = qm + (size_t)j * 24;
    const int p0 = 0, p1 = axis == 0 ? 3 : 1;  // quadrants with Omega along +axis
    const int m0 = axis == 0 ? 1 : 2, m1 = axis == 0 ? 2 : 3;
    const int kF = 1 + axis;                    // F_x or F_y
    const int kP0 = axis == 0 ? 3 : 4, kP1 = axis == 0 ? 4 : 5;  // (Pi_xx, Pi_xy) or (Pi_xy, Pi_yy)
    Half h;
    h.Fp = q[p0 * 6 + kF] + q[p1 * 6 + kF];
    h.Fm = q[m0 * 6 + kF] + q[m1 * 6 + kF];
    h.Pp[0] = q[p0 * 6 + kP0] + q[p1 * 6 + kP0];
    h.Pp[1] = q[p0 * 6 + kP1] + q[p1 * 6 + kP1];
    h.Pm[0] = q[m0 * 6 + kP0] + q[m1 * 6 + kP0];
    h.Pm[1] = q[m0 * 6 + kP1] + q[m1 * 6 + kP1];
    return h;
}

__device__ __forceinline__ double qm_tot(const double *__restrict__ qm, int j, int k) {
    const double *q = qm + (size_t)j * 24;
    return q[k] + q[6 + k] + q[12 + k] + q[18 + k];
}

__global__ void __launch_bounds__(BLOCK)
consistent_kernel(Geo G, const double *__restrict__ qm, const double *__restrict__ jin,
                  const double *__restrict__ pin, double *__restrict__ R0,
                  double *__restrict__ R1f) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.ncell) return;
    const Cell C = cell_of(G, k);
    const double ca2 = 0.5 * G.c * G.alpha, c3 = G.c3, ic = 1.0 / G.c;
    for (int nloc = 0; nloc < 4; ++nloc) {
        const int a = nloc & 1, b = nloc >> 1;
        const int j = k * 4 + nloc;
        const double phi = qm_tot(qm, j, 0), Ej = phi * ic;
        double r0 = 0.0, r1[2] = {0.0, 0.0};
        for (int axis = 0; axis < 2; ++axis) {
            const bool high = axis == 0 ? a == 1 : b == 1;  // node on the +axis face of its cell
            const bool has_nb = axis == 0 ? (high ? C.R : C.L) : (high ? C.T : C.B);
            const double wf = axis == 0 ? G.wfx : G.wfy;
            const int side = axis == 0 ? (high ? 1 : 0) : (high ? 3 : 2);
            const Half hj = half_pos_axis(qm, j, axis);
            if (has_nb) {
                const int nbcell = axis == 0 ? (high ? k + 1 : k - 1) : (high ? k + G.nx : k - G.nx);
                const int nbloc = axis == 0 ? ((1 - a) + 2 * b) : (a + 2 * (1 - b));
                const int jn = nbcell * 4 + nbloc;
                const Half hn = half_pos_axis(qm, jn, axis);
                const double En = qm_tot(qm, jn, 0) * ic;
                // K1 = low side, K2 = high side of the face; n = +axis
                const Half &h1 = high ? hj : hn, &h2 = high ? hn : hj;
                const double E1 = high ? Ej : En, E2 = high ? En : Ej;
                const double F1n = qm_tot(qm, high ? j : jn, 1 + axis);
                const double q0 = wf * (F1n + ca2 * (E1 - E2) - h1.Fp - h2.Fm);
                const double qx = wf * ((axis == 0 ? c3 * E2 : 0.0) - h1.Pp[0] - h2.Pm[0]);
                const double qy = wf * ((axis == 1 ? c3 * E2 : 0.0) - h1.Pp[1] - h2.Pm[1]);
                const double sgn = high ? 1.0 : -1.0;  // the K1 node takes +, the K2 node -
                r0 += sgn * q0;
                r1[0] += sgn * qx;
                r1[1] += sgn * qy;
            } else {
                // boundary, outward normal s * e_axis; the half ranges of
                // -e_axis are minus the opposite half ranges of +e_axis
                const double sn = high ? 1.0 : -1.0;
                const double Fp = high ? hj.Fp : -hj.Fm;
                const double Px = high ? hj.Pp[0] : -hj.Pm[0];
                const double Py = high ? hj.Pp[1] : -hj.Pm[1];
                r0 += wf * (jin[side] + G.alpha * phi - Fp);
                r1[0] += wf * ((axis == 0 ? c3 * sn * Ej : 0.0) - Px - pin[side * 2]);
                r1[1] += wf * ((axis == 1 ? c3 * sn * Ej : 0.0) - Py - pin[side * 2 + 1]);
            }
        }
        R0[j] = r0;
        R1f[(size_t)j * 2] = r1[0];
        R1f[(size_t)j * 2 + 1] = r1[1];
    }
}

// The same corrections on the 1D slab (point faces, w_f = 1, n = +-1): the
// half ranges of mu > 0 and mu < 0 are quadrants 0 and 1 of the moment
// layout, so half_pos_axis(., ., 0) applies unchanged.  One thread per cell.
__global__ void __launch_bounds__(BLOCK)
consistent1d_kernel(Geo G, const double *__restrict__ qm, const double *__restrict__ jin,
                    const double *__restrict__ pin, double *__restrict__ R0,
                    double *__restrict__ R1f) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.ncell) return;
    const double ca2 = 0.5 * G.c * G.alpha, c3 = G.c3, ic = 1.0 / G.c;
    for (int a = 0; a < 2; ++a) {
        const int j = k * 2 + a;
        const double phi = qm_tot(qm, j, 0), Ej = phi * ic;
        const bool high = a == 1;  // node on the +x face of its cell
        const bool has_nb = high ? k + 1 < G.nx : k > 0;
        const Half hj = half_pos_axis(qm, j, 0);
        double r0, r1;
        if (has_nb) {
            const int jn = high ? j + 1 : j - 1;  // the neighbour cell's node on this face
            const Half hn = half_pos_axis(qm, jn, 0);
            const double En = qm_tot(qm, jn, 0) * ic;
            const Half &h1 = high ? hj : hn, &h2 = high ? hn : hj;
            const double E1 = high ? Ej : En, E2 = high ? En : Ej;
            const double F1n = qm_tot(qm, high ? j : jn, 1);
            const double sgn = high ? 1.0 : -1.0;
            r0 = sgn * (F1n + ca2 * (E1 - E2) - h1.Fp - h2.Fm);
            r1 = sgn * (c3 * E2 - h1.Pp[0] - h2.Pm[0]);
        } else {
            const double sn = high ? 1.0 : -1.0;
            const int side = high ? 1 : 0;
            const double Fp = high ? hj.Fp : -hj.Fm;
            const double Px = high ? hj.Pp[0] : -hj.Pm[0];
            r0 = jin[side] + G.alpha * phi - Fp;
            r1 = c3 * sn * Ej - Px - pin[side * 2];
        }
        R0[j] = r0;
        R1f[j] = r1;
    }
}

// ---------------------------------------------------------------------------
// E* = phi / c and F* = F from the moments of the previous step's intensity
// (the high-order time-edge sources of Sec. 6.1).  One thread per node.
__global__ void timeedge_kernel(int N, int D, int nm, double inv_c, const double *__restrict__ mom,
                                double *__restrict__ Estar, double *__restrict__ Fstar) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    Estar[t] = mom[(size_t)t * nm] * inv_c;
    for (int d = 0; d < D; ++d) Fstar[(size_t)t * D + d] = mom[(size_t)t * nm + 1 + d];
}

// Per low-order solve (closures fixed), one thread per node: 1/A_FF with
// A_FF = m sigma~_F, the first-moment right-hand side b_F = m F*/(c dt) +
// R1_ind and u_b = A_FF^-1 b_F, where
// R1_ind(v) = int v . sum_g (sigma_F - sigma_g) F_g + int grad_h v : T
//             - int_Gamma0 [v] . {T n}   (Sec. 4, independent closures).
__global__ void __launch_bounds__(BLOCK)
prepare_kernel(Geo G, const double *__restrict__ clo, int nc, double inv_cdt,
               const double *__restrict__ Fstar, const double *__restrict__ R1f,
               double *__restrict__ iaF, double *__restrict__ bF, double *__restrict__ ub,
               Scalars *sc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        sc->elim_max = 0;
        sc->bar_count = 0u;  // the cooperative kernel's barrier starts empty
        sc->status = LO_OK;
    }
    if (t >= G.N) return;
    const int D = G.dim, NN = D == 2 ? 4 : 2;
    const int k = t / NN, n = t - k * NN;
    const int iy = k / G.nx, ix = k - iy * G.nx;
    const int a = n & 1, b = n >> 1;
    auto node = [&](int kk, int aa, int bb) { return kk * NN + aa + 2 * bb; };
    auto Tt = [&](int nd, int i, int j) -> double {  // closure tensor component (i, j)
        const double *cl = clo + (size_t)nd * nc;
        if (D == 1) return cl[2];
        return i != j ? cl[4] : (i == 0 ? cl[3] : cl[5]);
    };
    const double *cl = clo + (size_t)t * nc;
    const double sF = D == 1 ? cl[4] : cl[7];
    const double ia = 1.0 / (G.m * (sF + inv_cdt));
    iaF[t] = ia;
    for (int d = 0; d < D; ++d) {
        double r = G.m * (D == 1 ? cl[6] : cl[9 + d]);
        r += (2 * a - 1) * G.lx * (Tt(node(k, 0, b), d, 0) + Tt(node(k, 1, b), d, 0));
        if (D == 2) r += (2 * b - 1) * G.ly * (Tt(node(k, a, 0), d, 1) + Tt(node(k, a, 1), d, 1));
        if (R1f) {
            r += R1f[(size_t)t * D + d];  // consistent method: face and boundary corrections
        } else {
            // independent method: - int_Gamma0 [v] . {T n}
            if (a == 1 && ix + 1 < G.nx)
                r -= G.wfx * 0.5 * (Tt(t, d, 0) + Tt(node(k + 1, 0, b), d, 0));
            else if (a == 0 && ix > 0)
                r += G.wfx * 0.5 * (Tt(t, d, 0) + Tt(node(k - 1, 1, b), d, 0));
            if (D == 2) {
                if (b == 1 && iy + 1 < G.ny)
                    r -= G.wfy * 0.5 * (Tt(t, d, 1) + Tt(node(k + G.nx, a, 0), d, 1));
                else if (b == 0 && iy > 0)
                    r += G.wfy * 0.5 * (Tt(t, d, 1) + Tt(node(k - G.nx, a, 1), d, 1));
            }
        }
        const double bv = G.m * inv_cdt * Fstar[(size_t)t * D + d] + r;
        bF[(size_t)t * D + d] = bv;
        ub[(size_t)t * D + d] = bv * ia;
    }
}

// ---------------------------------------------------------------------------
// Grid-wide synchronisation for the cooperative low-order kernel (all blocks
// co-resident): a barrier of our own whose wait is bounded in time (a block
// that gives up records a timeout and leaves, and the others then give up at
// their next barrier), and reductions whose per-block partials every block
// sums in the same fixed order after the barrier, so that all blocks take the
// same decisions.  The barrier counts arrivals on one counter that is never
// reset inside a launch (the solve's set-up kernel zeroes it): barrier number
// j is complete once the counter reaches j * nblocks, so a block arrives with
// one release-ordered atomic and waits with acquire loads, and the last
// arrival has nothing more to publish.
struct GridBar {
    unsigned int *count;
    unsigned int nblocks;
    long long limit_ns;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned int *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void atom_add_release_u32(unsigned int *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ long long lo_global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// false: the wait ran out of time (every thread of the block gets the same
// answer).  `target` is the block's running arrival target (thread 0's copy
// is the one used), starting at 0 in every launch.
__device__ bool grid_barrier(const GridBar &b, unsigned &target) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        target += b.nblocks;
        // release: the block's writes (ordered before this thread's by the
        // __syncthreads above) become visible with the arrival
        atom_add_release_u32(b.count, 1u);
        const long long t0 = lo_global_ns();
        while ((int)(ld_acquire_u32(b.count) - target) < 0) {
            if (lo_global_ns() - t0 > b.limit_ns) {
                ok = 0;
                break;
            }
        }
    }
    return __syncthreads_and(ok) != 0;
}

// Block totals of K values into part[bid]; after a barrier, grid_totals
// sums the nb per-block partials in a fixed order (every thread gets them).
// bid / nb: the block's index among the blocks that solve its problem and
// their number (the whole grid for one problem; a share of it in the batched
// launch).  FP64 instructions issue at a small fraction of the FP32 rate on
// this GPU and the conjugate-gradient phases are bound by them, so both sums
// run in one warp (after a shared-memory transpose) rather than in every warp
// of the block: the block's threads only store and load.
template <int K>
__device__ void block_partials(double (&v)[K], double *part, int bid) {
    __shared__ double sh[K][BLOCK];
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = sh[k][lane];
#pragma unroll
            for (int w = 1; w < BLOCK / 32; ++w) t += sh[k][w * 32 + lane];
            t = warp_sum(t);
            if (lane == 0) part[(size_t)bid * K + k] = t;
        }
    }
}

// The grid totals of K values, then M scalars derived from them by
// f(totals, out) in one thread (divisions and square roots taken once per
// block instead of once per thread); every thread gets totals and scalars.
template <int K, int M, class F>
__device__ void grid_totals_f(double (&v)[K], const double *part, int nb, double (&o)[M], F f) {
    __shared__ double tot[K + M];
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double t[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double a = 0.0;
            for (int b = lane; b < nb; b += 32) a += __ldcg(part + (size_t)b * K + k);
            t[k] = warp_sum(a);
        }
        if (lane == 0) {
            double ov[M];
            f(t, ov);
#pragma unroll
            for (int k = 0; k < K; ++k) tot[k] = t[k];
#pragma unroll
            for (int m = 0; m < M; ++m) tot[K + m] = ov[m];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = tot[k];
#pragma unroll
    for (int m = 0; m < M; ++m) o[m] = tot[K + m];
    __syncthreads();
}
struct NoScalars {
    template <int K>
    __device__ void operator()(const double (&)[K], double (&o)[1]) const { o[0] = 0.0; }
};
template <int K>
__device__ void grid_totals(double (&v)[K], const double *part, int nb) {
    double none[1];
    grid_totals_f<K, 1>(v, part, nb, none, NoScalars{});
}

// ---------------------------------------------------------------------------
// The whole Newton iteration of a low-order solve in one cooperative launch:
// per Newton iteration a set-up phase (linearisation, Schur right-hand side,
// residual of the start x = E), the conjugate-gradient phases and the finish
// phase (back-substitution and pointwise temperature elimination), each
// closed by a grid barrier, and the stopping test of Eq. relative_tol taken by
// every block on the same grid totals.  The preconditioner is Jacobi,
// u = r / diag(S).  Two forms of the conjugate gradients (mathematically the
// same iterates):
//  * textbook (SINGLE = false): a matrix-vector phase (p = u + beta p_old
//    formed on the fly for the neighbours, q = S p, p.q) and an update phase
//    (x, r, u; r.r, r.u), two grid reductions per iteration;
//  * single-reduction (SINGLE = true), the form of Chronopoulos and Gear
//    (J. Comput. Appl. Math. 25, 1989): with w = S u, gamma = r.u, delta = w.u,
//      beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old),
//      p = u + beta p, s = w + beta s (= S p), x += alpha p, r -= alpha s,
//    and the next u, w = S u, gamma, delta and r.r in the same phase, one grid
//    reduction per iteration (plus one set-up phase for the first w).  The
//    product needs the new u of the neighbour cells: each cell forms them on
//    the fly from the neighbours' r, w and s of the previous phase, which are
//    double-buffered.  That costs about 40 FP64 operations per cell and saves
//    a barrier, which pays only while the FP64 pipes are lightly loaded; the
//    host picks the form from the cells per SM sub-partition.
// Partial sums of consecutive reductions go to different buffers (A: set-up,
// B / C: the conjugate-gradient phases, D: finish), so one barrier per
// reduction suffices.  Values other blocks wrote in the same launch (E, x and
// the search vectors of neighbour cells) are read past L1.
struct NewtonArgs {
    Geo G;
    const double *clo;
    int nc;
    double a_rad, dt;
    double *T, *E, *F;
    const double *Tstar, *cv, *Estar, *jin2, *R0, *iaF, *ub, *bF;
    const double *Sc;  // the assembled stencil of S (stencil_kernel)
    double inv_dt, inv_cdt;  // 1/dt, 1/(c dt): FP64 division is slow on this GPU
    double *aE, *idiag, *x, *p;
    double *r[2], *w[2], *s[2];  // double-buffered by iteration parity
    double *partA, *partB, *partC, *partD;
    double pcg_rtol, eps_inner, elim_rtol, T_floor;
    int max_pcg, max_inner, max_elim;
    Scalars *sc;
    GridBar bar;
    int withhold;  // test hook: the last block leaves before its first barrier
    // mixed-precision conjugate gradients: FP32 copies of aE, 1/A_FF and
    // 1/diag(S), and the inner solve's r, u, p (double-buffered), q, e
    // (double-buffered by refinement cycle)
    float *fa, *fi, *fd, *fr, *fu, *fp[2], *fq, *fe[2];
};

// The preconditioned residual u of cell k for the next matrix-vector product,
// from values of the previous phase: before the first iteration (START)
// u = r / diag(S), else u = (r - alpha s) / diag(S) with s = w + beta s_old
// (s_old = 0 and beta = 0 in the first iteration).  The owner of the cell
// forms its own r and s with the same operations, so both agree bit for bit.
template <int NN, bool START>
struct NextU {
    const double *r, *w, *s, *idg;
    double alpha, beta;
    __device__ __forceinline__ void get(int k, double (&o)[NN]) const {
        double rv[NN], dv[NN];
        ldc_cg<NN>(r, k, rv);
        ldc_cg<NN>(idg, k, dv);
        if constexpr (START) {
#pragma unroll
            for (int i = 0; i < NN; ++i) o[i] = rv[i] * dv[i];
        } else {
            double wv[NN], sv[NN];
            ldc_cg<NN>(w, k, wv);
            ldc_cg<NN>(s, k, sv);
#pragma unroll
            for (int i = 0; i < NN; ++i) o[i] = fma(-alpha, fma(beta, sv[i], wv[i]), rv[i]) * dv[i];
        }
    }
    __device__ __forceinline__ double get1(int k, int n) const {
        const size_t i = (size_t)k * NN + n;
        const double rv = __ldcg(r + i), dv = __ldcg(idg + i);
        if constexpr (START) {
            return rv * dv;
        } else {
            return fma(-alpha, fma(beta, __ldcg(s + i), __ldcg(w + i)), rv) * dv;
        }
    }
};

// Per Newton iteration, for cell k: linearise the emission about
// the current T (Sec. 5), form aE = m c (sigma~_E - nu sigma_E), the Schur
// right-hand side b_E - A_EF u_b with b_E = m (sigma_P B(T0) + nu q_T0 +
// E*/dt) + the Marshak inflow, 1/diag(S), and the residual of the start
// x = E: r = rhs - S x.  Sums ||rhs||^2 (the PCG stopping test's scale); the
// textbook form also starts u = r / diag(S), p = u and sums r.r and r.u.
template <int NN, bool SINGLE>
__device__ __forceinline__ void newton_setup_cell(const NewtonArgs &A, int k, double (&v)[3]) {
    const Geo &G = A.G;
    const Cell C = cell_of(G, k);
    double T0[NN], Ts[NN], cvv[NN], Es[NN], aE[NN], bE[NN];
    ldc<NN>(A.T, k, T0);
    ldc<NN>(A.Tstar, k, Ts);
    ldc<NN>(A.cv, k, cvv);
    ldc<NN>(A.Estar, k, Es);
    const double inv_cdt = A.inv_cdt;
#pragma unroll
    for (int n = 0; n < NN; ++n) {
        const double *cl = A.clo + ((size_t)k * NN + n) * A.nc;
        const double sE = cl[NN == 4 ? 6 : 3], sP = cl[NN == 4 ? 8 : 5];
        const double Tn = T0[n];
        const double B0 = A.a_rad * G.c * (Tn * Tn * Tn * Tn);
        const double dB = 4.0 * A.a_rad * G.c * (Tn * Tn * Tn);
        const double cv_dt = cvv[n] * A.inv_dt;
        const double den = cv_dt + sP * dB;
        const double rden = den > 0.0 ? 1.0 / den : 0.0;
        const double nu = sP * dB * rden;                     // pseudo-fission coefficient
        const double omnu = den > 0.0 ? cv_dt * rden : 1.0;  // 1 - nu, formed without the difference
        // sigma~_E - nu sigma_E = sigma_E (1 - nu) + 1/(c dt) and sigma_P B + nu q_T0 =
        // sigma_P B (1 - nu) + nu C_v/dt (T* - T): where sigma_P dB >> C_v/dt
        // (optically thick, nu -> 1) the printed differences cancel catastrophically
        // and the Newton iterates would inherit their rounding
        aE[n] = G.m * G.c * (sE * omnu + inv_cdt);
        bE[n] = G.m * (sP * B0 * omnu + nu * cv_dt * (Ts[n] - Tn) + Es[n] * A.inv_dt);
    }
    if (A.R0) {
        // consistent method: face and boundary corrections (the inflow included)
        double r0[NN];
        ldc<NN>(A.R0, k, r0);
#pragma unroll
        for (int n = 0; n < NN; ++n) bE[n] += r0[n];
    } else {
        // Marshak boundary: -2 int_Gamma_b u F_in, F_in the incoming partial current
#pragma unroll
        for (int b = 0; b < NN / 2; ++b) {
            if (!C.L) bE[2 * b] += G.wfx * A.jin2[0];
            if (!C.R) bE[2 * b + 1] += G.wfx * A.jin2[1];
        }
        if constexpr (NN == 4) {
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (!C.B) bE[a] += G.wfy * A.jin2[2];
                if (!C.T) bE[a + 2] += G.wfy * A.jin2[3];
            }
        }
    }
    double efu[NN], q[NN], e[NN], rv[NN], idg[NN], zv[NN];
    ef_cell<NN>(G, C, A.ub, efu);
    schur_cell<NN>(G, C, VecCG<NN>{A.E}, aE, A.Sc, q, e);
#pragma unroll
    for (int n = 0; n < NN; ++n) {
        const double rhs = bE[n] - efu[n];
        rv[n] = rhs - q[n];
        idg[n] = 1.0 / (aE[n] + __ldg(A.Sc + (size_t)k * Stencil<NN>::n + n));  // 1 / diag(S)
        v[0] += rhs * rhs;
        if constexpr (!SINGLE) {
            zv[n] = rv[n] * idg[n];
            v[1] += rv[n] * rv[n];
            v[2] += rv[n] * zv[n];
        }
    }
    stc<NN>(A.aE, k, aE);
    stc<NN>(A.idiag, k, idg);
    stc<NN>(A.x, k, e);
    stc<NN>(A.r[0], k, rv);
    if constexpr (!SINGLE) {
        stc<NN>(A.r[1], k, zv);  // u
        stc<NN>(A.w[0], k, zv);  // p
    }
}

// Textbook form: the search direction of cell k formed on the fly,
// p = u + beta p_old (values of the previous phase, read past L1)
template <int NN>
struct DirCG {
    const double *u, *p;
    double beta;
    __device__ __forceinline__ void get(int k, double (&o)[NN]) const {
        double a[NN], b[NN];
        ldc_cg<NN>(u, k, a);
        ldc_cg<NN>(p, k, b);
#pragma unroll
        for (int i = 0; i < NN; ++i) o[i] = fma(beta, b[i], a[i]);
    }
    __device__ __forceinline__ double get1(int k, int n) const {
        const size_t i = (size_t)k * NN + n;
        return fma(beta, __ldcg(p + i), __ldcg(u + i));
    }
};

// After the linear solve, for cell k: E = x, back-substitution
// F = A_FF^-1 (b_F - A_FE E), then the pointwise nonlinear elimination of T
// (Eq. nonlinear_T_update, lumped): (C_v/dt) T + sigma_P a c T^4 =
// c sigma_E E + (C_v/dt) T*, iterated from the current T and floored at
// T_floor.  The step divides f by an FP32 reciprocal of f' (a quasi-Newton
// step with relative slope error below 1e-7: the root and the stopping test
// are those of Newton's method; FP64 division is expensive on this GPU).
// Sums ||u_new - u_old||^2 and ||u_new||^2 over u = (T, E) for
// Eq. relative_tol.
template <int NN>
__device__ __forceinline__ void newton_finish_cell(const NewtonArgs &A, int k, double (&v)[2],
                                                   int &its_max) {
    constexpr int D = NN == 4 ? 2 : 1;
    const Geo &G = A.G;
    const Cell C = cell_of(G, k);
    double e[NN], ax[NN], ay[NN], ia[NN], Told[NN], Ts[NN], cvv[NN], Eold[NN], Tn[NN];
    fe_cell<NN>(G, C, VecCG<NN>{A.x}, e, ax, ay);
    ldc<NN>(A.iaF, k, ia);
    ldc<NN>(A.T, k, Told);
    ldc<NN>(A.Tstar, k, Ts);
    ldc<NN>(A.cv, k, cvv);
    ldc<NN>(A.E, k, Eold);
#pragma unroll
    for (int n = 0; n < NN; ++n) {
        const size_t nd = (size_t)k * NN + n;
        A.F[nd * D] = (A.bF[nd * D] - ax[n]) * ia[n];
        if constexpr (D == 2) A.F[nd * D + 1] = (A.bF[nd * D + 1] - ay[n]) * ia[n];
        const double *cl = A.clo + nd * A.nc;
        const double sE = cl[NN == 4 ? 6 : 3], sP = cl[NN == 4 ? 8 : 5];
        const double cv_dt = cvv[n] * A.inv_dt;
        const double k4 = sP * A.a_rad * G.c;
        const double rhs = G.c * sE * e[n] + cv_dt * Ts[n];
        double y = Told[n];
        int its;
        for (its = 1; its <= A.max_elim; ++its) {
            const double y3 = y * y * y;
            const double f = cv_dt * y + k4 * y3 * y - rhs;
            const double df = cv_dt + 4.0 * k4 * y3;
            const double adf = fabs(df);
            const double rdf = (adf > 1e-30 && adf < 1e30) ? (double)__frcp_rn((float)df)
                                                           : 1.0 / df;
            const double yn = fmax(y - f * rdf, A.T_floor);
            const bool conv = fabs(yn - y) <= A.elim_rtol * fabs(yn);
            y = yn;
            if (conv) break;
        }
        its_max = max(its_max, min(its, A.max_elim));
        Tn[n] = y;
        const double dT = y - Told[n], dE = e[n] - Eold[n];
        v[0] += dT * dT + dE * dE;
        v[1] += y * y + e[n] * e[n];
    }
    stc<NN>(A.T, k, Tn);
    stc<NN>(A.E, k, e);
}

// The textbook conjugate gradients on S x = b from the state in the FP64
// buffers: x, r = r[0], u = r[1] = r / diag(S), p = u (rz = r.u); buffers p =
// w[0] / w[1] by iteration parity, q = s[0].  Returns the DONE_ code; iters
// counts on from its value.
template <int NN>
__device__ __forceinline__ int cg_textbook(const NewtonArgs &A, const int bid, const int nb,
                                           const int k0, const int stride, unsigned &bar_target,
                                           const double stop, double rz, int &iters) {
    const Geo &G = A.G;
    double *const rb = A.r[0], *const ub = A.r[1], *const qb = A.s[0];
    double beta = 0.0;
    for (;;) {
        const double *po = (iters & 1) ? A.w[1] : A.w[0];
        double *pn = (iters & 1) ? A.w[0] : A.w[1];
        double v1[1] = {0.0};
        for (int k = k0; k < G.ncell; k += stride) {
            const Cell C = cell_of(G, k);
            double aEv[NN], qv[NN], pv[NN];
            ldc<NN>(A.aE, k, aEv);
            schur_cell<NN>(G, C, DirCG<NN>{ub, po, beta}, aEv, A.Sc, qv, pv);
            stc<NN>(pn, k, pv);
            stc<NN>(qb, k, qv);
#pragma unroll
            for (int n = 0; n < NN; ++n) v1[0] += pv[n] * qv[n];
        }
        block_partials<1>(v1, A.partB, bid);
        if (!grid_barrier(A.bar, bar_target)) return DONE_TIMEOUT;
        double o1[2];  // (curvature positive and finite, alpha)
        grid_totals_f<1, 2>(v1, A.partB, nb, o1, [rz](const double (&t)[1], double (&o)[2]) {
            const bool ok = t[0] > 0.0 && isfinite(t[0]) && isfinite(rz);
            o[0] = ok ? 1.0 : 0.0;
            o[1] = ok ? rz / t[0] : 0.0;
        });
        if (o1[0] == 0.0) return DONE_BREAKDOWN;
        const double alpha = o1[1];
        double v2[2] = {0.0, 0.0};
        for (int k = k0; k < G.ncell; k += stride) {
            double pv[NN], qv[NN], dv[NN], xv[NN], rv[NN], zv[NN];
            ldc<NN>(pn, k, pv);
            ldc<NN>(qb, k, qv);
            ldc<NN>(A.idiag, k, dv);
            ldc<NN>(A.x, k, xv);
            ldc<NN>(rb, k, rv);
#pragma unroll
            for (int n = 0; n < NN; ++n) {
                xv[n] = fma(alpha, pv[n], xv[n]);
                rv[n] = fma(-alpha, qv[n], rv[n]);
                zv[n] = rv[n] * dv[n];
                v2[0] += rv[n] * rv[n];
                v2[1] += rv[n] * zv[n];
            }
            stc<NN>(A.x, k, xv);
            stc<NN>(rb, k, rv);
            stc<NN>(ub, k, zv);
        }
        block_partials<2>(v2, A.partC, bid);
        if (!grid_barrier(A.bar, bar_target)) return DONE_TIMEOUT;
        double o2[2];  // (converged, beta)
        grid_totals_f<2, 2>(v2, A.partC, nb, o2,
                            [rz, stop](const double (&t)[2], double (&o)[2]) {
                                o[0] = sqrt(t[0]) <= stop ? 1.0 : 0.0;
                                o[1] = t[1] / rz;
                            });
        ++iters;
        if (o2[0] != 0.0) return DONE_CONVERGED;
        if (iters >= A.max_pcg) return DONE_CAPPED;
        beta = o2[1];
        rz = v2[1];
    }
}

// DONE_ code of a mixed-precision solve whose refinement stopped helping
constexpr int DONE_FALLBACK = 5;

// Mixed-precision conjugate gradients (iterative refinement) on S x = b from
// x = E with the FP64 residual r = r[0] of the set-up: each cycle solves
// S e = r approximately by Jacobi-preconditioned conjugate gradients in FP32
// on FP32 copies of the operator's coefficients (on this GPU FP32 issues at 64
// times the FP64 rate; the operator application is the solve's arithmetic),
// to 1e-5 of the cycle's starting residual, then updates x += e and
// r -= S e in FP64, so the FP64 residual -- the one the stopping test reads --
// falls by about that factor per cycle, down to the same pcg_rtol as the FP64
// solve.  A cycle that does not at least halve the FP64 norm of r returns
// DONE_FALLBACK (the caller continues with the FP64 conjugate gradients from
// x and r).  iters counts the inner iterations and the refinement updates.
template <int NN>
__device__ __forceinline__ int mixed_cg(const NewtonArgs &A, const int bid, const int nb,
                                        const int k0, const int stride, unsigned &bar_target,
                                        const double stop, int &iters) {
    const Geo &G = A.G;
    const GeoF Gf = geo_f(G);
    constexpr float INNER = 1e-5f;
    // cycle start: FP32 copies of the coefficients, r32 = r, u = r / diag(S),
    // e = 0; sums r.r (FP64), r32.u, r32.r32
    double v[3] = {0.0, 0.0, 0.0};
    for (int k = k0; k < G.ncell; k += stride) {
        double aEv[NN], iav[NN], dv[NN], rv[NN];
        ldc<NN>(A.aE, k, aEv);
        ldc<NN>(A.iaF, k, iav);
        ldc<NN>(A.idiag, k, dv);
        ldc<NN>(A.r[0], k, rv);
        float fa[NN], fi[NN], fd[NN], fr[NN], fu[NN], z[NN];
#pragma unroll
        for (int n = 0; n < NN; ++n) {
            fa[n] = (float)aEv[n];
            fi[n] = (float)iav[n];
            fd[n] = (float)dv[n];
            fr[n] = (float)rv[n];
            fu[n] = fr[n] * fd[n];
            z[n] = 0.f;
            v[0] += rv[n] * rv[n];
            v[1] += (double)fr[n] * (double)fu[n];
            v[2] += (double)fr[n] * (double)fr[n];
        }
        stf<NN>(A.fa, k, fa);
        stf<NN>(A.fi, k, fi);
        stf<NN>(A.fd, k, fd);
        stf<NN>(A.fr, k, fr);
        stf<NN>(A.fu, k, fu);
        stf<NN>(A.fp[0], k, fu);  // p = u + 0 p_old reads p_old: keep it finite
        stf<NN>(A.fe[0], k, z);
    }
    block_partials<3>(v, A.partB, bid);
    if (!grid_barrier(A.bar, bar_target)) return DONE_TIMEOUT;
    grid_totals<3>(v, A.partB, nb);
    double rr64 = v[0], rz = v[1], rr32 = v[2];
    if (sqrt(rr64) <= stop) return DONE_CONVERGED;
    for (int cyc = 0;; ++cyc) {
        float *const e = A.fe[cyc & 1];
        // inner FP32 conjugate gradients on S e = r32 from e = 0
        const double inner_stop = (double)INNER * sqrt(rr32);
        double beta = 0.0;
        for (int it = 0;; ++it) {
            const float *po = A.fp[it & 1];
            float *pn = A.fp[(it + 1) & 1];
            double v1[1] = {0.0};
            for (int k = k0; k < G.ncell; k += stride) {
                const Cell C = cell_of(G, k);
                float aEv[NN], qv[NN], pv[NN];
                ldf<NN>(A.fa, k, aEv);
                schur_cell_t<float, NN>(Gf, C, DirF<NN>{A.fu, po, (float)beta}, aEv,
                                        IaF<NN>{A.fi}, qv, pv);
                stf<NN>(pn, k, pv);
                stf<NN>(A.fq, k, qv);
#pragma unroll
                for (int n = 0; n < NN; ++n) v1[0] += (double)pv[n] * (double)qv[n];
            }
            block_partials<1>(v1, A.partC, bid);
            if (!grid_barrier(A.bar, bar_target)) return DONE_TIMEOUT;
            grid_totals<1>(v1, A.partC, nb);
            if (!(v1[0] > 0.0) || !isfinite(v1[0]) || !isfinite(rz)) break;  // refine from here
            const float alpha = (float)(rz / v1[0]);
            double v2[2] = {0.0, 0.0};
            for (int k = k0; k < G.ncell; k += stride) {
                float pv[NN], qv[NN], dv[NN], ev[NN], rv[NN], uv[NN];
                ldf<NN>(pn, k, pv);
                ldf<NN>(A.fq, k, qv);
                ldf<NN>(A.fd, k, dv);
                ldf<NN>(e, k, ev);
                ldf<NN>(A.fr, k, rv);
#pragma unroll
                for (int n = 0; n < NN; ++n) {
                    ev[n] = __fmaf_rn(alpha, pv[n], ev[n]);
                    rv[n] = __fmaf_rn(-alpha, qv[n], rv[n]);
                    uv[n] = rv[n] * dv[n];
                    v2[0] += (double)rv[n] * (double)rv[n];
                    v2[1] += (double)rv[n] * (double)uv[n];
                }
                stf<NN>(e, k, ev);
                stf<NN>(A.fr, k, rv);
                stf<NN>(A.fu, k, uv);
            }
            block_partials<2>(v2, A.partD, bid);
            if (!grid_barrier(A.bar, bar_target)) return DONE_TIMEOUT;
            grid_totals<2>(v2, A.partD, nb);
            ++iters;
            if (sqrt(v2[0]) <= inner_stop || iters >= A.max_pcg || !isfinite(v2[1])) break;
            beta = v2[1] / rz;
            rz = v2[1];
        }
        // refinement: x += e, r -= S e in FP64; the next cycle's r32, u, e = 0
        double v3[3] = {0.0, 0.0, 0.0};
        float *const e_next = A.fe[(cyc + 1) & 1];
        for (int k = k0; k < G.ncell; k += stride) {
            const Cell C = cell_of(G, k);
            double aEv[NN], se[NN], ed[NN], xv[NN], rv[NN];
            ldc<NN>(A.aE, k, aEv);
            schur_cell<NN>(G, C, VecFD<NN>{e}, aEv, A.Sc, se, ed);
            ldc<NN>(A.x, k, xv);
            ldc<NN>(A.r[0], k, rv);
            float fd[NN], fr[NN], fu[NN], z[NN];
            ldf<NN>(A.fd, k, fd);
#pragma unroll
            for (int n = 0; n < NN; ++n) {
                xv[n] += ed[n];
                rv[n] -= se[n];
                fr[n] = (float)rv[n];
                fu[n] = fr[n] * fd[n];
                z[n] = 0.f;
                v3[0] += rv[n] * rv[n];
                v3[1] += (double)fr[n] * (double)fu[n];
                v3[2] += (double)fr[n] * (double)fr[n];
            }
            stc<NN>(A.x, k, xv);
            stc<NN>(A.r[0], k, rv);
            stf<NN>(A.fr, k, fr);
            stf<NN>(A.fu, k, fu);
            stf<NN>(A.fp[0], k, fu);
            stf<NN>(e_next, k, z);
        }
        block_partials<3>(v3, A.partA, bid);
        if (!grid_barrier(A.bar, bar_target)) return DONE_TIMEOUT;
        grid_totals<3>(v3, A.partA, nb);
        ++iters;
        if (!isfinite(v3[0])) return DONE_BREAKDOWN;
        if (sqrt(v3[0]) <= stop) return DONE_CONVERGED;
        if (iters >= A.max_pcg) return DONE_CAPPED;
        if (v3[0] > 0.25 * rr64) return DONE_FALLBACK;  // the cycle did not halve ||r||
        rr64 = v3[0];
        rz = v3[1];
        rr32 = v3[2];
    }
}

// The scalars of an iteration of the single-reduction conjugate gradients
// from the sums t = (gamma = r.u, delta = w.u, r.r) of the last reduction and
// the previous iteration's gamma and alpha: (converged, step defined, alpha,
// beta), taken in one thread.
struct SingleScalars {
    double stop, gam_old, alpha_old;
    bool first;
    __device__ void operator()(const double (&t)[3], double (&o)[4]) const {
        const double gam = t[0], del = t[1];
        const double beta = first ? 0.0 : gam / gam_old;
        const double den = first ? del : del - beta * gam / alpha_old;
        const bool ok = den > 0.0 && isfinite(den) && isfinite(gam);
        o[0] = sqrt(t[2]) <= stop ? 1.0 : 0.0;
        o[1] = ok ? 1.0 : 0.0;
        o[2] = ok ? gam / den : 0.0;
        o[3] = beta;
    }
};

// The Newton iteration of one problem on its nb blocks (bid: this block's
// index among them).  MIXED: the linear solves by mixed-precision conjugate
// gradients (mixed_cg), SINGLE then unused.
template <int NN, bool SINGLE, bool MIXED = false>
__device__ __forceinline__ void lo_newton_body(const NewtonArgs &A, const int bid, const int nb) {
    if (A.withhold && bid == nb - 1) return;
    const Geo &G = A.G;
    const int stride = nb * BLOCK;
    const int k0 = bid * BLOCK + threadIdx.x;
    int status = LO_OK, newton = 0, pcg_total = 0, pcg_max = 0, capped = 0;
    unsigned bar_target = 0;  // arrivals that complete the next grid barrier
    double d1 = -1.0;
    for (int it = 1; it <= A.max_inner; ++it) {
        // set-up: linearisation, r = rhs - S E, ||rhs||^2 (textbook form:
        // also u, p = u, r.r, r.u)
        double v0[3] = {0.0, 0.0, 0.0};
        for (int k = k0; k < G.ncell; k += stride)
            newton_setup_cell<NN, SINGLE || MIXED>(A, k, v0);
        block_partials<3>(v0, A.partA, bid);
        if (!grid_barrier(A.bar, bar_target)) { status = LO_TIMEOUT; break; }
        grid_totals<3>(v0, A.partA, nb);
        const double stop = A.pcg_rtol * sqrt(v0[0]);
        int done = DONE_NO, iters = 0;
        if constexpr (MIXED) {
            done = mixed_cg<NN>(A, bid, nb, k0, stride, bar_target, stop, iters);
            if (done == DONE_FALLBACK) {
                // the FP64 conjugate gradients from the current x and r: u =
                // r / diag(S), p = u; r.r, r.u (partial sums D: the last
                // reduction used A, the first of the loop uses B)
                double vf[2] = {0.0, 0.0};
                double *const pst = (iters & 1) ? A.w[1] : A.w[0];
                for (int k = k0; k < G.ncell; k += stride) {
                    double rv[NN], dv[NN], zv[NN];
                    ldc<NN>(A.r[0], k, rv);
                    ldc<NN>(A.idiag, k, dv);
#pragma unroll
                    for (int n = 0; n < NN; ++n) {
                        zv[n] = rv[n] * dv[n];
                        vf[0] += rv[n] * rv[n];
                        vf[1] += rv[n] * zv[n];
                    }
                    stc<NN>(A.r[1], k, zv);
                    stc<NN>(pst, k, zv);
                }
                block_partials<2>(vf, A.partD, bid);
                if (!grid_barrier(A.bar, bar_target)) {
                    done = DONE_TIMEOUT;
                } else {
                    grid_totals<2>(vf, A.partD, nb);
                    done = sqrt(vf[0]) <= stop
                               ? DONE_CONVERGED
                               : cg_textbook<NN>(A, bid, nb, k0, stride, bar_target, stop, vf[1],
                                                 iters);
                }
            }
        } else if constexpr (SINGLE) {
            // second set-up phase: u = r / diag(S), w = S u; r.u, w.u, r.r;
            // p = s = 0 before the first iteration
            double v3[3] = {0.0, 0.0, 0.0};
            {
                const NextU<NN, true> nu{A.r[0], nullptr, nullptr, A.idiag, 0.0, 0.0};
                double zero[NN];
#pragma unroll
                for (int n = 0; n < NN; ++n) zero[n] = 0.0;
                for (int k = k0; k < G.ncell; k += stride) {
                    const Cell C = cell_of(G, k);
                    double aEv[NN], wv[NN], uv[NN], rv[NN];
                    ldc<NN>(A.aE, k, aEv);
                    schur_cell<NN>(G, C, nu, aEv, A.Sc, wv, uv);
                    ldc<NN>(A.r[0], k, rv);
                    stc<NN>(A.w[0], k, wv);
                    stc<NN>(A.s[1], k, zero);
                    stc<NN>(A.p, k, zero);
#pragma unroll
                    for (int n = 0; n < NN; ++n) {
                        v3[0] += rv[n] * uv[n];
                        v3[1] += wv[n] * uv[n];
                        v3[2] += rv[n] * rv[n];
                    }
                }
            }
            block_partials<3>(v3, A.partB, bid);
            if (!grid_barrier(A.bar, bar_target)) { status = LO_TIMEOUT; break; }
            // sc: the next iteration's (converged, den ok, alpha, beta)
            double sc[4];
            grid_totals_f<3, 4>(v3, A.partB, nb, sc, SingleScalars{stop, 0.0, 0.0, true});
            // conjugate gradients on S E = b from x = E, one reduction per
            // iteration; iteration i reads r_i, w_i (buffers i % 2) and s_{i-1}
            // (buffer (i + 1) % 2) and writes s_i, r_{i+1}, w_{i+1}
            double gam = v3[0];
            while (true) {
                if (sc[0] != 0.0) { done = DONE_CONVERGED; break; }
                if (iters >= A.max_pcg) { done = DONE_CAPPED; break; }
                if (sc[1] == 0.0) { done = DONE_BREAKDOWN; break; }
                const double alpha = sc[2], beta = sc[3];
                const int cur = iters & 1, nxt = cur ^ 1;
                const NextU<NN, false> nu{A.r[cur], A.w[cur], A.s[nxt], A.idiag, alpha, beta};
                double v[3] = {0.0, 0.0, 0.0};
                for (int k = k0; k < G.ncell; k += stride) {
                    const Cell C = cell_of(G, k);
                    double rv[NN], wv[NN], sv[NN], pv[NN], xv[NN], dv[NN];
                    ldc<NN>(A.r[cur], k, rv);
                    ldc<NN>(A.w[cur], k, wv);
                    ldc<NN>(A.s[nxt], k, sv);
                    ldc<NN>(A.p, k, pv);
                    ldc<NN>(A.idiag, k, dv);
                    ldc<NN>(A.x, k, xv);
#pragma unroll
                    for (int n = 0; n < NN; ++n) {
                        pv[n] = fma(beta, pv[n], rv[n] * dv[n]);
                        sv[n] = fma(beta, sv[n], wv[n]);
                        xv[n] = fma(alpha, pv[n], xv[n]);
                        rv[n] = fma(-alpha, sv[n], rv[n]);
                        // r.u and r.r of the new residual (u = r / diag(S), as
                        // the matrix-vector product below forms it)
                        v[0] += rv[n] * (rv[n] * dv[n]);
                        v[2] += rv[n] * rv[n];
                    }
                    stc<NN>(A.p, k, pv);
                    stc<NN>(A.x, k, xv);
                    stc<NN>(A.s[cur], k, sv);
                    stc<NN>(A.r[nxt], k, rv);
                    double aEv[NN], wn[NN], un[NN];
                    ldc<NN>(A.aE, k, aEv);
                    schur_cell<NN>(G, C, nu, aEv, A.Sc, wn, un);
                    stc<NN>(A.w[nxt], k, wn);
#pragma unroll
                    for (int n = 0; n < NN; ++n) v[1] += wn[n] * un[n];
                }
                double *part = cur ? A.partB : A.partC;
                block_partials<3>(v, part, bid);
                if (!grid_barrier(A.bar, bar_target)) { done = DONE_TIMEOUT; break; }
                grid_totals_f<3, 4>(v, part, nb, sc, SingleScalars{stop, gam, alpha, false});
                ++iters;
                gam = v[0];
            }
        } else {
            // textbook form (start x = E, p = u)
            if (sqrt(v0[1]) <= stop)
                done = DONE_CONVERGED;
            else
                done = cg_textbook<NN>(A, bid, nb, k0, stride, bar_target, stop, v0[2], iters);
        }
        if (done == DONE_TIMEOUT) { status = LO_TIMEOUT; break; }
        if (done == DONE_BREAKDOWN) { status = LO_BREAKDOWN; break; }
        pcg_total += iters;
        pcg_max = max(pcg_max, iters);
        if (done != DONE_CONVERGED) ++capped;
        ++newton;
        // finish: back-substitution and pointwise elimination
        double v2[2] = {0.0, 0.0};
        int its_max = 0;
        for (int k = k0; k < G.ncell; k += stride) newton_finish_cell<NN>(A, k, v2, its_max);
        const int wmax = __reduce_max_sync(0xffffffffu, its_max);
        if ((threadIdx.x & 31) == 0 && wmax > 0) atomicMax(&A.sc->elim_max, wmax);
        block_partials<2>(v2, A.partD, bid);
        if (!grid_barrier(A.bar, bar_target)) { status = LO_TIMEOUT; break; }
        grid_totals<2>(v2, A.partD, nb);
        const double dn = sqrt(v2[0]), un = sqrt(v2[1]);
        if (!isfinite(dn)) { status = LO_NONFINITE; break; }
        if (d1 < 0.0) d1 = dn;
        // Eq. relative_tol, plus a round-off guard for an update that is
        // already at round-off level
        if (dn == 0.0 || dn < A.eps_inner * d1 || dn <= 1e-14 * un) break;
    }
    if (bid == 0 && threadIdx.x == 0) {
        Scalars *sc = A.sc;
        sc->newton_iters = newton;
        sc->pcg_total = pcg_total;
        sc->pcg_max = pcg_max;
        sc->pcg_capped = capped;
        if (status != LO_OK) sc->status = status;
    } else if (status == LO_TIMEOUT && threadIdx.x == 0) {
        A.sc->status = LO_TIMEOUT;
    }
}

// at least 4 blocks per SM (128 registers per thread): a 256x256 mesh (512
// blocks of cells) then runs without grid-stride repeats
template <int NN, bool SINGLE, bool MIXED>
__global__ void __launch_bounds__(BLOCK, 4) lo_newton_kernel(const NewtonArgs A) {
    lo_newton_body<NN, SINGLE, MIXED>(A, blockIdx.x, gridDim.x);
}

// The low-order solves of many problems in one cooperative launch: blocks
// first[m] .. first[m + 1] - 1 solve problem m (its own arguments, partial
// sums, barrier counter and scalars), each problem with its own FP64 PCG form
// (form[m]: 0 textbook, 1 single-reduction).
// The problems share nothing, so each runs its own Newton and PCG
// iterations and stopping tests; every block of the launch is co-resident,
// so a problem's barriers wait only on blocks that are running.
template <int NN>
__global__ void __launch_bounds__(BLOCK, 4)
lo_newton_batch_kernel(const NewtonArgs *__restrict__ args, const int *__restrict__ form,
                       const int *__restrict__ first, int n) {
    __shared__ NewtonArgs sA;
    __shared__ int s_m;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n - 1;  // the last m with first[m] <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_m = lo;
    }
    __syncthreads();
    const int m = s_m;
    {
        const unsigned *src = reinterpret_cast<const unsigned *>(args + m);
        unsigned *dst = reinterpret_cast<unsigned *>(&sA);
        static_assert(sizeof(NewtonArgs) % 4 == 0, "word copy");
        for (int i = threadIdx.x; i < (int)(sizeof(NewtonArgs) / 4); i += BLOCK) dst[i] = src[i];
    }
    __syncthreads();
    const int bid = (int)blockIdx.x - first[m], nb = first[m + 1] - first[m];
    if (form[m] == 1)
        lo_newton_body<NN, true>(sA, bid, nb);
    else
        lo_newton_body<NN, false>(sA, bid, nb);
}

// Outer iteration, one thread per node: ||u - u_in||^2 and ||u||^2 for
// u = (T, E), then u_in <- u.
__global__ void __launch_bounds__(BLOCK)
outer_change_kernel(int N, const double *__restrict__ T, const double *__restrict__ E,
                    double *__restrict__ Tin, double *__restrict__ Ein, double *part, Scalars *sc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (t < N) {
        const double dT = T[t] - Tin[t], dE = E[t] - Ein[t];
        v[0] = dT * dT + dE * dE;
        v[1] = T[t] * T[t] + E[t] * E[t];
        Tin[t] = T[t];
        Ein[t] = E[t];
    }
    if (grid_sums<2>(v, part, &sc->count)) {
        sc->d2 = v[0];
        sc->n2 = v[1];
    }
}

}  // namespace lo
}  // namespace smk

// ===========================================================================
// host side
struct sm_lo_state {
    int N = 0, D = 0, NN = 0, nblk_cell = 0, nblk_node = 0;
    double *buf = nullptr;  // every node array in one allocation
    double *aE, *iaF, *bF, *ub, *idiag, *x, *p, *r[2], *wv[2], *s[2], *Estar, *Fstar, *Tstar, *Tin,
        *Ein;
    double *part = nullptr;
    double *jin2 = nullptr;     // [4] 2 |F_in| per side
    double *R0 = nullptr, *R1f = nullptr;  // consistent-method sources [node], [node][2]
    double *qmom_int = nullptr;            // per-quadrant moments used by sm_step
    double *jinc = nullptr, *pinc = nullptr;  // inflow moments J_in [4], Pi_in [4][2]
    double *sigma = nullptr;    // sigma_g(T^k) of the running step
    double *clo = nullptr;      // closures when the caller passes none
    smk::lo::Scalars *sc = nullptr;
    smk::lo::Scalars *h_sc = nullptr;  // pinned mirror
    int coop_grid[3] = {0, 0, 0};  // blocks of the cooperative launch per PCG form (0: not sized)
    float *fbuf = nullptr;         // the mixed-precision solves' FP32 vectors (10 per node)
    double *Sc = nullptr;          // the assembled stencil of S, Stencil<NN>::n per cell
    int nsm = 0;                // SMs of the device (0: not queried yet)
};

namespace {

using smk::lo::BLOCK;
using smk::lo::Geo;

// doubles of the per-block partial-sum buffer: the cooperative kernel's four
// reduction buffers (3 + 3 + 3 + 2 values per block); the outer iteration's
// change norms use the first 2
constexpr size_t PART_PER_BLOCK = 11;

#define SM_LO_CUDA_LAUNCH(call)                                                      \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return lo_fail(SM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        p->launches++;                                                             \
    } while (0)

sm_status lo_fail(sm_status s, const std::string &m) {
    smk::set_last_error(m.c_str());
    return s;
}

#define LO_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return lo_fail(e_ == cudaErrorMemoryAllocation ? SM_ERR_OOM : SM_ERR_CUDA,   \
                           std::string(#call) + ": " + cudaGetErrorString(e_));         \
    } while (0)
#define LO_TRY(expr)                \
    do {                            \
        sm_status s_ = (expr);      \
        if (s_ != SM_OK) return s_; \
    } while (0)

Geo make_geo(const sm_problem *p) {
    Geo G;
    G.dim = p->dim;
    G.nx = p->nx;
    G.ny = p->dim == 2 ? p->ny : 1;
    G.ncell = p->ncell;
    G.N = p->ncell * p->nn;
    const double hx = p->hx, hy = p->dim == 2 ? p->hy : 1.0;
    G.m = p->dim == 1 ? 0.5 * hx : 0.25 * hx * hy;
    G.c = p->desc.c;
    G.wfx = p->dim == 1 ? 1.0 : 0.5 * hy;
    G.wfy = 0.5 * hx;
    G.c3 = G.c / 3.0;
    G.lx = G.m / hx;
    G.ly = G.m / hy;
    G.kx = G.c3 * G.lx;
    G.ky = G.c3 * G.ly;
    G.fx = G.c3 * G.wfx;
    G.fy = G.c3 * G.wfy;
    G.alpha = p->alpha;
    const double ca = G.c * p->alpha;
    G.px = 0.5 * ca * G.wfx;
    G.py = 0.5 * ca * G.wfy;
    G.bx = ca * G.wfx;
    G.by = ca * G.wfy;
    return G;
}

inline bool aligned16(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

sm_status lo_ensure(sm_problem *p) {
    if (p->lo) return SM_OK;
    if ((long long)p->ncell * p->nn > (1LL << 30))
        return lo_fail(SM_ERR_UNSUPPORTED, "the low-order solve supports up to 2^30 nodes");
    p->lo = new sm_lo_state();
    sm_lo_state &w = *p->lo;
    const int N = p->ncell * p->nn, D = p->dim;
    w.N = N;
    w.D = D;
    w.NN = p->nn;
    w.nblk_cell = (p->ncell + BLOCK - 1) / BLOCK;
    w.nblk_node = (N + BLOCK - 1) / BLOCK;
    const size_t nS = 15, nV = 3;  // node arrays and [node][dim] arrays
    const size_t buf_elems = (size_t)N * nS + (size_t)N * D * nV;
    LO_CUDA(cudaMalloc(&w.buf, sizeof(double) * buf_elems));
    double *b = w.buf;
    auto take = [&](size_t n) {
        double *r = b;
        b += n;
        return r;
    };
    w.bF = take((size_t)N * D);
    w.ub = take((size_t)N * D);
    w.Fstar = take((size_t)N * D);
    w.aE = take(N);
    w.iaF = take(N);
    w.idiag = take(N);
    w.x = take(N);
    w.p = take(N);
    for (int i = 0; i < 2; ++i) {
        w.r[i] = take(N);
        w.wv[i] = take(N);
        w.s[i] = take(N);
    }
    w.Estar = take(N);
    w.Tstar = take(N);
    w.Tin = take(N);
    w.Ein = take(N);
    const size_t nblk = (size_t)std::max(w.nblk_cell, w.nblk_node);
    LO_CUDA(cudaMalloc(&w.part, sizeof(double) * PART_PER_BLOCK * nblk));
    LO_CUDA(cudaMalloc(&w.fbuf, sizeof(float) * (size_t)N * 10));
    const size_t nsc = (size_t)p->ncell * (p->nn == 4 ? smk::lo::Stencil<4>::n
                                                      : smk::lo::Stencil<2>::n);
    LO_CUDA(cudaMalloc(&w.Sc, sizeof(double) * nsc));
    p->workspace_bytes += sizeof(double) * nsc;
    p->workspace_bytes += sizeof(float) * (size_t)N * 10;
    LO_CUDA(cudaMalloc(&w.jin2, sizeof(double) * 4));
    {  // consistent method: R0 [N], R1f [N][dim], quadrant moments, inflow moments
        LO_CUDA(cudaMalloc(&w.R0, sizeof(double) * (size_t)N * 3));
        w.R1f = w.R0 + N;
        LO_CUDA(cudaMalloc(&w.qmom_int, sizeof(double) * (size_t)N * 24));
        LO_CUDA(cudaMalloc(&w.jinc, sizeof(double) * 12));
        w.pinc = w.jinc + 4;
        p->workspace_bytes += sizeof(double) * ((size_t)N * 27 + 12);
    }
    LO_CUDA(cudaMalloc(&w.sigma, sizeof(double) * (size_t)p->G * p->ncell));
    LO_CUDA(cudaMalloc(&w.clo, sizeof(double) * (size_t)N * p->nc));
    LO_CUDA(cudaMalloc(&w.sc, sizeof(smk::lo::Scalars)));
    LO_CUDA(cudaMemset(w.sc, 0, sizeof(smk::lo::Scalars)));
    LO_CUDA(cudaMallocHost(&w.h_sc, sizeof(smk::lo::Scalars)));
    p->workspace_bytes += sizeof(double) * (buf_elems + PART_PER_BLOCK * nblk + 4 +
                                            (size_t)p->G * p->ncell +
                                            (size_t)N * p->nc) +
                          sizeof(smk::lo::Scalars);
    // 2 |F_in| per side: 2 sum_{Omega.n<0} w |Omega.n| I_in with the gray
    // isotropic inflow I_in = a c T_bdr^4 / 4 pi (vacuum where T_bdr <= 0)
    const double PI = 3.14159265358979323846;
    const double nrm[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    double jin2[4];
    for (int s = 0; s < 4; ++s) {
        const double Tb = p->desc.T_bdr[s];
        const double Iin = Tb > 0 ? p->desc.a * p->desc.c * Tb * Tb * Tb * Tb / (4.0 * PI) : 0.0;
        double acc = 0.0;
        for (int d = 0; d < p->nd; ++d) {
            const double on = p->omx[d] * nrm[s][0] + (p->dim == 2 ? p->omy[d] * nrm[s][1] : 0.0);
            if (on < 0) acc += p->w[d] * -on;
        }
        jin2[s] = 2.0 * acc * Iin;
    }
    LO_CUDA(cudaMemcpy(w.jin2, jin2, sizeof(jin2), cudaMemcpyHostToDevice));
    {
        // consistent method: J_in = sum_{Omega.n<0} w |Omega.n| I_in and
        // Pi_in = sum_{Omega.n<0} w Omega (Omega.n) I_in per side
        double jp[12] = {0};
        for (int s = 0; s < 4; ++s) {
            const double Tb = p->desc.T_bdr[s];
            const double Iin = Tb > 0 ? p->desc.a * p->desc.c * Tb * Tb * Tb * Tb / (4.0 * PI) : 0.0;
            for (int d = 0; d < p->nd; ++d) {
                const double oy = p->dim == 2 ? p->omy[d] : 0.0;
                const double on = p->omx[d] * nrm[s][0] + oy * nrm[s][1];
                if (on < 0) {
                    jp[s] += p->w[d] * -on * Iin;
                    jp[4 + 2 * s] += p->w[d] * p->omx[d] * on * Iin;
                    jp[4 + 2 * s + 1] += p->w[d] * oy * on * Iin;
                }
            }
        }
        LO_CUDA(cudaMemcpy(w.jinc, jp, sizeof(jp), cudaMemcpyHostToDevice));
    }
    return SM_OK;
}

sm_status read_scalars(sm_problem *p) {
    sm_lo_state &w = *p->lo;
    LO_CUDA(cudaMemcpyAsync(w.h_sc, w.sc, sizeof(smk::lo::Scalars), cudaMemcpyDeviceToHost,
                            p->stream));
    LO_CUDA(cudaStreamSynchronize(p->stream));
    return SM_OK;
}

sm_status check_params(const sm_step_params &prm) {
    if (prm.max_outer < 1 || prm.max_inner < 1 || prm.max_pcg < 1 || prm.max_elim < 1)
        return lo_fail(SM_ERR_INVALID_ARG, "iteration limits must be >= 1");
    if (prm.method != SM_METHOD_INDEPENDENT && prm.method != SM_METHOD_CONSISTENT)
        return lo_fail(SM_ERR_INVALID_ARG, "method must be SM_METHOD_INDEPENDENT or CONSISTENT");
    if (!(prm.eps_outer >= 0) || !(prm.eps_inner >= 0) || !(prm.pcg_rtol > 0) ||
        !(prm.elim_rtol > 0) || !(prm.T_floor > 0))
        return lo_fail(SM_ERR_INVALID_ARG,
                       "tolerances must be >= 0 (eps) or > 0 (pcg_rtol, elim_rtol, T_floor)");
    return SM_OK;
}

sm_status sm_count(sm_lo_state &w) {
    if (w.nsm == 0) {
        int dev = 0;
        LO_CUDA(cudaGetDevice(&dev));
        LO_CUDA(cudaDeviceGetAttribute(&w.nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    return SM_OK;
}

// The PCG form of problem p (0 textbook, 1 single-reduction, 2 mixed
// precision).  The library's choice: the single-reduction form below
// SINGLE_CELLS cells, the textbook form from there on.  Measured on GB300
// (seconds per converged step, the same iterates): the single-reduction form
// saves 9 % on the 64-cell slab, but costs 7 % on the 128^2 gray channel
// (5.32 against 4.97 ms) and 5 % on the 256^2 multigroup mesh, where the extra
// FP64 work of forming the neighbours' u outweighs the saved barrier.  The
// mixed-precision form is not chosen: it needs 1.6x the iterations (each
// refinement cycle restarts the Krylov space) and an iteration, bound by the
// grid barriers' latency rather than by FP64 arithmetic, gets only about a
// quarter cheaper (gray channel 5.81 ms, multigroup 33.7 against 32.3 ms).
constexpr long long SINGLE_CELLS = 4096;
int pcg_form(const sm_problem *p, int nsm) {
    (void)nsm;
    switch (p->lo_pcg_form) {
        case SM_DEBUG_PCG_TEXTBOOK: return 0;
        case SM_DEBUG_PCG_SINGLE: return 1;
        case SM_DEBUG_PCG_MIXED: return 2;
        default: break;
    }
    return p->ncell < SINGLE_CELLS ? 1 : 0;
}
int form_used(int f) {
    return f == 2 ? SM_DEBUG_PCG_MIXED : f == 1 ? SM_DEBUG_PCG_SINGLE : SM_DEBUG_PCG_TEXTBOOK;
}

// The arguments of problem p's Newton kernel on nblocks blocks.
smk::lo::NewtonArgs newton_args(sm_problem *p, sm_lo_state &w, const Geo &G, const double *clo,
                                double *T, double *E, double *F, const double *Tstar,
                                const double *cv, const double *R0, const sm_step_params &prm,
                                int nblocks) {
    const size_t nblk = (size_t)std::max(w.nblk_cell, w.nblk_node);
    smk::lo::NewtonArgs A;
    A.G = G;
    A.clo = clo;
    A.nc = p->nc;
    A.a_rad = p->desc.a;
    A.dt = p->desc.dt;
    A.inv_dt = 1.0 / p->desc.dt;
    A.inv_cdt = 1.0 / (G.c * p->desc.dt);
    A.T = T;
    A.E = E;
    A.F = F;
    A.Tstar = Tstar;
    A.cv = cv;
    A.Estar = w.Estar;
    A.jin2 = w.jin2;
    A.R0 = R0;
    A.iaF = w.iaF;
    A.Sc = w.Sc;
    A.ub = w.ub;
    A.bF = w.bF;
    A.aE = w.aE;
    A.idiag = w.idiag;
    A.x = w.x;
    A.p = w.p;
    for (int i = 0; i < 2; ++i) {
        A.r[i] = w.r[i];
        A.w[i] = w.wv[i];
        A.s[i] = w.s[i];
    }
    // per-block partial sums of the kernel's reductions: A, B, C (up to 3
    // values each), D (2), disjoint
    A.partA = w.part;
    A.partB = w.part + 3 * nblk;
    A.partC = w.part + 6 * nblk;
    A.partD = w.part + 9 * nblk;
    static_assert(PART_PER_BLOCK >= 11, "room for the partial sums A, B, C, D");
    A.pcg_rtol = prm.pcg_rtol;
    A.eps_inner = prm.eps_inner;
    A.elim_rtol = prm.elim_rtol;
    A.T_floor = prm.T_floor;
    A.max_pcg = prm.max_pcg;
    A.max_inner = prm.max_inner;
    A.max_elim = prm.max_elim;
    A.sc = w.sc;
    A.bar.count = &w.sc->bar_count;
    A.bar.nblocks = (unsigned)nblocks;
    A.bar.limit_ns = p->timeout_ns;
    A.withhold = p->fault_withhold_block;
    {
        float *f = w.fbuf;
        float **slots[] = {&A.fa, &A.fi, &A.fd, &A.fr, &A.fu, &A.fp[0], &A.fp[1], &A.fq, &A.fe[0],
                           &A.fe[1]};
        for (int i = 0; i < 10; ++i) *slots[i] = f + (size_t)i * w.N;
    }
    return A;
}

// One cooperative launch runs the whole Newton iteration (all blocks
// co-resident: the grid is at most the blocks that fit on the GPU at once).
template <int NN>
sm_status launch_newton(sm_problem *p, sm_lo_state &w, const Geo &G, const double *clo,
                        double *T, double *E, double *F, const double *Tstar, const double *cv,
                        const double *R0, const sm_step_params &prm) {
    LO_TRY(sm_count(w));
    const int form = pcg_form(p, w.nsm);
    const void *k = form == 2   ? (const void *)smk::lo::lo_newton_kernel<NN, false, true>
                    : form == 1 ? (const void *)smk::lo::lo_newton_kernel<NN, true, false>
                                : (const void *)smk::lo::lo_newton_kernel<NN, false, false>;
    int &grid = w.coop_grid[form];
    if (grid == 0) {
        int per_sm = 0;
        LO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BLOCK, 0));
        if (per_sm < 1) return lo_fail(SM_ERR_CUDA, "the low-order kernel does not fit on an SM");
        grid = std::min(w.nblk_cell, per_sm * w.nsm);
    }
    smk::lo::NewtonArgs A = newton_args(p, w, G, clo, T, E, F, Tstar, cv, R0, prm, grid);
    void *args[] = {&A};
    LO_CUDA(cudaLaunchCooperativeKernel(k, dim3(grid), dim3(BLOCK), args, 0, p->stream));
    p->lo_pcg_form_used = form_used(form);
    return SM_OK;
}

// The Newton iteration of Sec. 5 on the gray system with fixed closures.
// Time-edge sources in w.Estar / w.Fstar; T, E hold the initial guesses and
// receive the result, F receives the flux of the last linear solve.  One
// cooperative launch and one host synchronisation per solve.
template <int NN>
sm_status lo_launch(sm_problem *p, const double *clo, const double *Tstar, const double *cv,
                    double *T, double *E, double *F, const sm_step_params &prm,
                    const double *qmom) {
    sm_lo_state &w = *p->lo;
    const Geo G = make_geo(p);
    cudaStream_t s = p->stream;
    const double dt = p->desc.dt;
    const double *R0 = nullptr, *R1f = nullptr;
    if (qmom) {  // consistent method
        if (NN == 4)
            smk::lo::consistent_kernel<<<w.nblk_cell, BLOCK, 0, s>>>(G, qmom, w.jinc, w.pinc,
                                                                     w.R0, w.R1f);
        else
            smk::lo::consistent1d_kernel<<<w.nblk_cell, BLOCK, 0, s>>>(G, qmom, w.jinc, w.pinc,
                                                                       w.R0, w.R1f);
        LO_CUDA(cudaGetLastError());
        p->launches++;
        R0 = w.R0;
        R1f = w.R1f;
    }
    smk::lo::prepare_kernel<<<w.nblk_node, BLOCK, 0, s>>>(G, clo, p->nc, 1.0 / (G.c * dt),
                                                          w.Fstar, R1f, w.iaF, w.bF, w.ub, w.sc);
    LO_CUDA(cudaGetLastError());
    smk::lo::stencil_kernel<NN><<<w.nblk_cell, BLOCK, 0, s>>>(G, w.iaF, w.Sc);
    LO_CUDA(cudaGetLastError());
    p->launches += 2;
    LO_TRY(launch_newton<NN>(p, w, G, clo, T, E, F, Tstar, cv, R0, prm));
    p->launches++;
    return SM_OK;
}

// Status and statistics of the last low-order solve from the pinned mirror
// of its scalars (the caller has copied and synchronized them).
sm_status lo_collect(sm_problem *p, sm_step_stats *st) {
    sm_lo_state &w = *p->lo;
    const smk::lo::Scalars &h = *w.h_sc;
    if (h.status == smk::lo::LO_TIMEOUT)
        return lo_fail(SM_ERR_TIMEOUT, "a grid barrier of the low-order kernel ran out of time");
    if (h.status == smk::lo::LO_BREAKDOWN)
        return lo_fail(SM_ERR_NO_CONVERGENCE,
                       "conjugate gradients broke down: the Schur complement is not positive "
                       "definite on the search direction, or the data is not finite");
    if (h.status == smk::lo::LO_NONFINITE)
        return lo_fail(SM_ERR_NONPHYSICAL, "the low-order Newton iterate is not finite");
    st->pcg_iters_total += h.pcg_total;
    st->pcg_iters_max = std::max(st->pcg_iters_max, h.pcg_max);
    st->pcg_capped += h.pcg_capped;
    st->newton_iters_total += h.newton_iters;
    st->newton_iters_max = std::max(st->newton_iters_max, h.newton_iters);
    st->elim_iters_max = std::max(st->elim_iters_max, w.h_sc->elim_max);
    return SM_OK;
}

// Launches a low-order solve without waiting for it.
sm_status launch_lo(sm_problem *p, const double *clo, const double *Tstar, const double *cv,
                    double *T, double *E, double *F, const sm_step_params &prm,
                    const double *qmom) {
    return p->dim == 2 ? lo_launch<4>(p, clo, Tstar, cv, T, E, F, prm, qmom)
                       : lo_launch<2>(p, clo, Tstar, cv, T, E, F, prm, qmom);
}

sm_status run_lo(sm_problem *p, const double *clo, const double *Tstar, const double *cv,
                 double *T, double *E, double *F, const sm_step_params &prm, sm_step_stats *st,
                 const double *qmom) {
    LO_TRY(launch_lo(p, clo, Tstar, cv, T, E, F, prm, qmom));
    LO_TRY(read_scalars(p));
    return lo_collect(p, st);
}

// Start of a time step (Algorithm 1) for problem p, on its stream: sigma_g at
// the step's start temperature (frozen for the step, Sec. 3 Rem. opacity),
// the time-edge sources E* = phi/c, F* = F of the previous step's moments
// (Sec. 6.1), T* = T^k, and the start of the outer iteration E = E*, T = T^k.
sm_status step_begin(sm_problem *p, const double *scale, double *T, double *E,
                     const double *moments) {
    sm_lo_state &w = *p->lo;
    cudaStream_t s = p->stream;
    const int N = w.N;
    LO_TRY(sm_opacity(p, T, scale, w.sigma));
    smk::lo::timeedge_kernel<<<w.nblk_node, BLOCK, 0, s>>>(N, w.D, p->nm, 1.0 / p->desc.c,
                                                          moments, w.Estar, w.Fstar);
    LO_CUDA(cudaGetLastError());
    p->launches++;
    LO_CUDA(cudaMemcpyAsync(w.Tstar, T, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    LO_CUDA(cudaMemcpyAsync(w.Tin, T, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    LO_CUDA(cudaMemcpyAsync(w.Ein, w.Estar, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    LO_CUDA(cudaMemcpyAsync(E, w.Estar, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    return SM_OK;
}

// ||u - u_in|| and ||u|| of the outer iteration (u = (T, E)) into the
// scalars, then u_in <- u.
sm_status launch_outer_change(sm_problem *p, const double *T, const double *E) {
    sm_lo_state &w = *p->lo;
    smk::lo::outer_change_kernel<<<w.nblk_node, BLOCK, 0, p->stream>>>(w.N, T, E, w.Tin, w.Ein,
                                                                      w.part, w.sc);
    LO_CUDA(cudaGetLastError());
    p->launches++;
    return SM_OK;
}

sm_status check_lo_problem(sm_problem *p) {
    if (!(p->desc.dt > 0.0))
        return lo_fail(SM_ERR_INVALID_ARG, "the low-order solve needs a time step dt > 0");
    return lo_ensure(p);
}

// Arguments of the batched low-order launch: per problem its Newton kernel
// arguments, its PCG form and its first block (pinned host copies and their
// device mirrors; rewritten before every launch, after the previous one has
// been waited for).
struct BatchLO {
    smk::lo::NewtonArgs *h_args = nullptr, *d_args = nullptr;
    int *h_int = nullptr, *d_int = nullptr;  // single[cap], first[cap + 1]
    int cap = 0;
    int per_sm = 0;  // co-resident blocks of the batched kernel per SM
};

// The low-order solves (independent method) of the problems `members` in one
// cooperative launch on stream s, after each one's preparation kernel.
// Every problem gets blocks in proportion to its cells (at least one, at
// most one per BLOCK cells) out of all the blocks that fit on the GPU at
// once; with fewer blocks than its single-problem launch a problem runs more
// cells per thread (grid-stride loops) and sums its block partials in
// another order.
sm_status batch_lo_launch(sm_batch *b, const std::vector<int> &members,
                          const std::vector<sm_problem *> &probs, const double *const *clo,
                          const double *const *cv, double *const *T, double *const *E,
                          double *const *F, const sm_step_params &prm, cudaStream_t s) {
    const int n = (int)members.size();
    if (n == 0) return SM_OK;
    void *&slot = smk::batch_lo_scratch(b);
    if (!slot) slot = new BatchLO();
    BatchLO &L = *static_cast<BatchLO *>(slot);
    if (L.cap < n) {
        if (L.h_args) cudaFreeHost(L.h_args);
        if (L.d_args) cudaFree(L.d_args);
        if (L.h_int) cudaFreeHost(L.h_int);
        if (L.d_int) cudaFree(L.d_int);
        L.h_args = L.d_args = nullptr;
        L.h_int = L.d_int = nullptr;
        L.cap = 0;
        LO_CUDA(cudaMallocHost(&L.h_args, sizeof(smk::lo::NewtonArgs) * n));
        LO_CUDA(cudaMalloc(&L.d_args, sizeof(smk::lo::NewtonArgs) * n));
        LO_CUDA(cudaMallocHost(&L.h_int, sizeof(int) * (2 * n + 1)));
        LO_CUDA(cudaMalloc(&L.d_int, sizeof(int) * (2 * n + 1)));
        L.cap = n;
    }
    sm_lo_state &w0 = *probs[members[0]]->lo;
    LO_TRY(sm_count(w0));
    const int nsm = w0.nsm;
    const void *k = (const void *)smk::lo::lo_newton_batch_kernel<4>;
    if (L.per_sm == 0) {
        LO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.per_sm, k, BLOCK, 0));
        if (L.per_sm < 1) return lo_fail(SM_ERR_CUDA, "the batched low-order kernel does not fit on an SM");
    }
    const long long cap_blocks = (long long)L.per_sm * nsm;
    if (n > cap_blocks)
        return lo_fail(SM_ERR_UNSUPPORTED, "more batch members than co-resident low-order blocks");
    // blocks per problem: one each, the rest in proportion to the cells
    std::vector<long long> need(n), nb(n, 1);
    long long extra_need = 0;
    for (int i = 0; i < n; ++i) {
        need[i] = probs[members[i]]->lo->nblk_cell;
        extra_need += need[i] - 1;
    }
    const long long rest = cap_blocks - n;
    for (int i = 0; i < n; ++i) {
        const long long e = extra_need <= rest ? need[i] - 1
                                               : (long long)((double)(need[i] - 1) * rest / extra_need);
        nb[i] += std::min(e, need[i] - 1);
    }
    int *form = L.h_int, *first = L.h_int + n;
    first[0] = 0;
    for (int i = 0; i < n; ++i) {
        sm_problem *p = probs[members[i]];
        sm_lo_state &w = *p->lo;
        const int m = members[i];
        const Geo G = make_geo(p);
        smk::lo::prepare_kernel<<<w.nblk_node, BLOCK, 0, s>>>(
            G, clo[m], p->nc, 1.0 / (G.c * p->desc.dt), w.Fstar, nullptr, w.iaF, w.bF, w.ub, w.sc);
        LO_CUDA(cudaGetLastError());
        if (p->nn == 4)
            smk::lo::stencil_kernel<4><<<w.nblk_cell, BLOCK, 0, s>>>(G, w.iaF, w.Sc);
        else
            smk::lo::stencil_kernel<2><<<w.nblk_cell, BLOCK, 0, s>>>(G, w.iaF, w.Sc);
        LO_CUDA(cudaGetLastError());
        p->launches += 2;
        L.h_args[i] = newton_args(p, w, G, clo[m], T[m], E[m], F[m], w.Tstar, cv[m], nullptr, prm,
                                  (int)nb[i]);
        form[i] = pcg_form(p, nsm) == 1 ? 1 : 0;  // the batched launch runs the FP64 forms
        first[i + 1] = first[i] + (int)nb[i];
        p->lo_pcg_form_used = form_used(form[i]);
    }
    LO_CUDA(cudaMemcpyAsync(L.d_args, L.h_args, sizeof(smk::lo::NewtonArgs) * n,
                            cudaMemcpyHostToDevice, s));
    LO_CUDA(cudaMemcpyAsync(L.d_int, L.h_int, sizeof(int) * (2 * n + 1), cudaMemcpyHostToDevice, s));
    const smk::lo::NewtonArgs *da = L.d_args;
    const int *ds = L.d_int, *df = L.d_int + n;
    int nn = n;
    void *args[] = {&da, &ds, &df, &nn};
    LO_CUDA(cudaLaunchCooperativeKernel(k, dim3(first[n]), dim3(BLOCK), args, 0, s));
    probs[members[0]]->launches++;
    return SM_OK;
}

}  // namespace

namespace smk {
void batch_lo_free(void *scratch) {
    if (!scratch) return;
    BatchLO *L = static_cast<BatchLO *>(scratch);
    if (L->h_args) cudaFreeHost(L->h_args);
    if (L->d_args) cudaFree(L->d_args);
    if (L->h_int) cudaFreeHost(L->h_int);
    if (L->d_int) cudaFree(L->d_int);
    delete L;
}
void lo_free(sm_problem *p) {
    if (!p->lo) return;
    sm_lo_state &w = *p->lo;
    void *bufs[] = {w.buf, w.part, w.jin2, w.sigma, w.clo, w.sc, w.R0, w.qmom_int, w.jinc, w.fbuf,
                    w.Sc};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (w.h_sc) cudaFreeHost(w.h_sc);
    delete p->lo;
    p->lo = nullptr;
}
}  // namespace smk

extern "C" {

void sm_default_step_params(sm_step_params *prm) {
    if (!prm) return;
    prm->eps_outer = 1e-3;
    prm->eps_inner = 1e-3;
    prm->pcg_rtol = 1e-10;
    prm->elim_rtol = 1e-10;
    prm->T_floor = 1e-8;
    prm->max_outer = 100;
    prm->max_inner = 30;
    prm->max_pcg = 5000;
    prm->max_elim = 40;
    prm->method = SM_METHOD_INDEPENDENT;
    prm->refine = 0;
}

sm_status sm_loworder_newton(sm_problem *p, const double *closures_dev, const double *T_star_dev,
                             const double *cv_dev, const double *moments_star_dev, double *T_dev,
                             double *E_dev, double *F_dev, const sm_step_params *params,
                             sm_step_stats *stats) {
    if (!p || !closures_dev || !T_star_dev || !cv_dev || !moments_star_dev || !T_dev || !E_dev ||
        !F_dev)
        return lo_fail(SM_ERR_INVALID_ARG, "NULL argument to sm_loworder_newton");
    if (!aligned16(T_star_dev) || !aligned16(cv_dev) || !aligned16(T_dev) || !aligned16(E_dev))
        return lo_fail(SM_ERR_INVALID_ARG, "T, T_star, cv and E must be 16-byte aligned");
    sm_step_params prm;
    if (params)
        prm = *params;
    else
        sm_default_step_params(&prm);
    LO_TRY(check_params(prm));
    LO_TRY(check_lo_problem(p));
    sm_lo_state &w = *p->lo;
    smk::lo::timeedge_kernel<<<w.nblk_node, BLOCK, 0, p->stream>>>(
        w.N, w.D, p->nm, 1.0 / p->desc.c, moments_star_dev, w.Estar, w.Fstar);
    LO_CUDA(cudaGetLastError());
    p->launches++;
    const double *qmom = nullptr;
    if (prm.method == SM_METHOD_CONSISTENT) {
        if (!p->qmom_dev)
            return lo_fail(SM_ERR_INVALID_ARG,
                           "the consistent method needs the per-quadrant moments of the last "
                           "sweep: register a buffer with sm_set_quadrant_moments and sweep");
        qmom = p->qmom_dev;
    }
    sm_step_stats st{};
    LO_TRY(run_lo(p, closures_dev, T_star_dev, cv_dev, T_dev, E_dev, F_dev, prm, &st, qmom));
    st.converged = 1;
    if (stats) *stats = st;
    return SM_OK;
}

sm_status sm_step(sm_problem *p, const double *scale_dev, const double *cv_dev, double *T_dev,
                  double *E_dev, double *F_dev, double *moments_dev, const void *I_prev_dev,
                  void *I_next_dev, double *closures_dev, const sm_step_params *params,
                  sm_step_stats *stats) {
    if (!p || !scale_dev || !cv_dev || !T_dev || !E_dev || !F_dev || !moments_dev || !I_prev_dev ||
        !I_next_dev)
        return lo_fail(SM_ERR_INVALID_ARG, "NULL argument to sm_step");
    if (!aligned16(cv_dev) || !aligned16(T_dev) || !aligned16(E_dev))
        return lo_fail(SM_ERR_INVALID_ARG, "T, cv and E must be 16-byte aligned");
    sm_step_params prm;
    if (params)
        prm = *params;
    else
        sm_default_step_params(&prm);
    LO_TRY(check_params(prm));
    LO_TRY(check_lo_problem(p));
    sm_lo_state &w = *p->lo;
    cudaStream_t s = p->stream;
    double *clo = closures_dev ? closures_dev : w.clo;
    const bool consistent = prm.method == SM_METHOD_CONSISTENT;
    const bool refine = prm.refine != 0;
    if (refine) {
        if (consistent)
            return lo_fail(SM_ERR_UNSUPPORTED, "the FP64 defect correction runs the independent method");
        if (I_prev_dev == I_next_dev)
            return lo_fail(SM_ERR_INVALID_ARG, "I_prev_dev and I_next_dev must not alias");
        LO_TRY(smk::refine_ensure(p));
        smk::refine_take_corrections(p);  // count this step's corrections only
    }
    double *qmom_saved = p->qmom_dev;
    const double *qmom = nullptr;
    if (consistent) {
        // the sweeps of this step also leave their per-quadrant moments
        qmom = qmom_saved ? qmom_saved : w.qmom_int;
        LO_TRY(sm_set_quadrant_moments(p, const_cast<double *>(qmom)));
    }
    LO_TRY(step_begin(p, scale_dev, T_dev, E_dev, moments_dev));
    if (refine) {
        // I^k as pairs of FP32 numbers; the iterate (held as pairs in the
        // caller's I_next buffer until the end of the step) starts there
        LO_TRY(smk::refine_begin(p, static_cast<const double *>(I_prev_dev), I_next_dev));
    }
    sm_step_stats st{};
    double d1 = -1.0;
    for (int it = 1; it <= prm.max_outer; ++it) {
        // high-order solve with the current T: emission, sweep, moments, closures
        if (refine) {
            // residuals of the iterate and FP32 correction sweeps
            SM_LO_CUDA_LAUNCH(smk::launch_emission(p, T_dev, w.sigma, nullptr, s));
            LO_TRY(smk::refine_solve(p, I_next_dev, moments_dev));
            SM_LO_CUDA_LAUNCH(smk::launch_closures_from_T(p, moments_dev, T_dev, w.sigma, clo, s));
        } else {
            LO_TRY(sm_sweep(p, T_dev, w.sigma, I_prev_dev, I_next_dev, moments_dev, clo));
        }
        LO_TRY(sm_synchronize(p));
        LO_TRY(run_lo(p, clo, w.Tstar, cv_dev, T_dev, E_dev, F_dev, prm, &st, qmom));
        LO_TRY(launch_outer_change(p, T_dev, E_dev));
        LO_TRY(read_scalars(p));
        st.outer_iters = it;
        const double dn = std::sqrt(w.h_sc->d2), un = std::sqrt(w.h_sc->n2);
        st.last_change = dn;
        if (d1 < 0) d1 = dn;
        if (dn == 0.0 || dn < prm.eps_outer * d1 || dn <= 1e-14 * un) {
            st.converged = 1;
            break;
        }
    }
    if (refine) {
        LO_TRY(smk::refine_end(p, I_next_dev));  // the iterate back into FP64
        LO_TRY(sm_synchronize(p));
        st.refine_corrections = smk::refine_take_corrections(p);
    }
    if (consistent && !qmom_saved) LO_TRY(sm_set_quadrant_moments(p, nullptr));
    if (stats) *stats = st;
    return SM_OK;
}

sm_status sm_batch_step(sm_batch *b, const double *const *scale_dev,
                        const double *const *cv_dev, double *const *T_dev, double *const *E_dev,
                        double *const *F_dev, double *const *moments_dev,
                        const void *const *I_prev_dev, void *const *I_next_dev,
                        double *const *closures_dev, const sm_step_params *params,
                        sm_step_stats *stats_host) {
    if (!b || !scale_dev || !cv_dev || !T_dev || !E_dev || !F_dev || !moments_dev ||
        !I_prev_dev || !I_next_dev)
        return lo_fail(SM_ERR_INVALID_ARG, "NULL argument to sm_batch_step");
    sm_step_params prm;
    if (params)
        prm = *params;
    else
        sm_default_step_params(&prm);
    LO_TRY(check_params(prm));
    if (prm.method != SM_METHOD_INDEPENDENT)
        return lo_fail(SM_ERR_UNSUPPORTED, "sm_batch_step runs the independent method");
    if (prm.refine)
        return lo_fail(SM_ERR_UNSUPPORTED, "sm_batch_step has no FP64 defect correction");
    const std::vector<sm_problem *> &probs = smk::batch_members(b);
    const int n = (int)probs.size();
    for (int i = 0; i < n; ++i) {
        if (!scale_dev[i] || !cv_dev[i] || !T_dev[i] || !E_dev[i] || !F_dev[i] ||
            !moments_dev[i] || !I_prev_dev[i] || !I_next_dev[i])
            return lo_fail(SM_ERR_INVALID_ARG,
                           "member " + std::to_string(i) + ": NULL argument to sm_batch_step");
        if (!aligned16(cv_dev[i]) || !aligned16(T_dev[i]) || !aligned16(E_dev[i]))
            return lo_fail(SM_ERR_INVALID_ARG, "T, cv and E must be 16-byte aligned");
        LO_TRY(check_lo_problem(probs[i]));
    }
    std::vector<const double *> sig(n);
    std::vector<double *> clo(n);
    for (int i = 0; i < n; ++i) {
        sm_problem *p = probs[i];
        sig[i] = p->lo->sigma;
        clo[i] = closures_dev && closures_dev[i] ? closures_dev[i] : p->lo->clo;
        LO_TRY(step_begin(p, scale_dev[i], T_dev[i], E_dev[i], moments_dev[i]));
    }
    std::vector<sm_step_stats> st(n);
    std::vector<double> d1(n, -1.0);
    std::vector<unsigned char> active(n, 1);
    int n_active = n;
    const cudaStream_t s = smk::batch_stream(b);
    // the batched low-order launch for 2D members (every member of a batch is
    // 2D) unless a test forces one launch per member
    const bool lo_batched = probs[0]->dim == 2 && smk::batch_lo_mode(b) != 0;
    for (int it = 1; it <= prm.max_outer && n_active > 0; ++it) {
        // high-order solve of every unconverged member in one batched pass
        // (emission, one persistent sweep launch, moments, closures)
        LO_TRY(smk::batch_pass(b, T_dev, sig.data(), I_prev_dev, I_next_dev, moments_dev,
                               clo.data(), active.data()));
        // their low-order solves in one cooperative launch (2D members), or
        // one launch each, queued on the batch's stream without waiting in
        // between
        std::vector<int> act;
        for (int i = 0; i < n; ++i)
            if (active[i]) act.push_back(i);
        if (lo_batched)
            LO_TRY(batch_lo_launch(b, act, probs, clo.data(), cv_dev, T_dev, E_dev, F_dev, prm, s));
        for (int i : act) {
            sm_problem *p = probs[i];
            sm_lo_state &w = *p->lo;
            if (!lo_batched)
                LO_TRY(launch_lo(p, clo[i], w.Tstar, cv_dev[i], T_dev[i], E_dev[i], F_dev[i], prm,
                                 nullptr));
            LO_TRY(launch_outer_change(p, T_dev[i], E_dev[i]));
            LO_CUDA(cudaMemcpyAsync(w.h_sc, w.sc, sizeof(smk::lo::Scalars),
                                    cudaMemcpyDeviceToHost, s));
        }
        LO_TRY(smk::batch_status(b));  // synchronizes the stream
        for (int i = 0; i < n; ++i) {
            if (!active[i]) continue;
            sm_problem *p = probs[i];
            const sm_status lr = lo_collect(p, &st[i]);
            if (lr != SM_OK)
                return lo_fail(lr, "member " + std::to_string(i) + ", outer iteration " +
                                       std::to_string(it) + ": " + sm_last_error());
            const double dn = std::sqrt(p->lo->h_sc->d2), un = std::sqrt(p->lo->h_sc->n2);
            st[i].outer_iters = it;
            st[i].last_change = dn;
            if (d1[i] < 0) d1[i] = dn;
            // Eq. relative_tol per member, with the round-off guard of sm_step
            if (dn == 0.0 || dn < prm.eps_outer * d1[i] || dn <= 1e-14 * un) {
                st[i].converged = 1;
                active[i] = 0;
                --n_active;
            }
        }
    }
    if (stats_host)
        for (int i = 0; i < n; ++i) stats_host[i] = st[i];
    return SM_OK;
}

}  // extern "C"
