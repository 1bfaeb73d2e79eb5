// Gray low-order solve and the full time step, FP64 on the device:
//  * the independent LDG low-order system of Sec. 4 (fluxes with kappa =
//    alpha/2 and s = sign(w.n), w = (1, 1); Marshak-type boundary; closure
//    source R1_ind), lumped with the 2-point Gauss-Lobatto rule (Sec. 6);
//  * the Newton iteration of Sec. 5 with frozen gray opacities, the
//    pseudo-fission linearisation of the emission (Eq. pseudo_fission) and the
//    pointwise nonlinear temperature elimination (Eq. nonlinear_T_update);
//  * the Schur complement in E (Eq. schur), symmetric positive definite for
//    lumped forms, solved by preconditioned conjugate gradients;
//  * Algorithm 1 (outer fixed point between the transport sweep and the
//    low-order solve) with the relative stopping rule Eq. relative_tol.
//
// Unknowns are nodal (cell corners): E_n and F_n = (F_x, F_y).  With the
// interior faces oriented +x / +y, s = +1, so F^.n takes the low-side F and
// P^ n the high-side E.  The lumped A_FF = m sigma~_F is diagonal, which lets
// S = A_EE - A_EF A_FF^-1 A_FE be applied matrix-free as a two-hop stencil on
// the structured mesh; the whole working set of a 256x256 mesh (a few MB)
// stays in L2, so these kernels are launch- and latency-bound rather than
// bandwidth-bound.  PCG scalars never leave the device: each kernel's
// reductions are finished by the last block to arrive (deterministic fixed-
// order sums, no atomics on floating point), and chunks of iterations are
// replayed from a CUDA graph; the host only polls a done flag per chunk.
#include <algorithm>
#include <cmath>
#include <string>

#include "sm_internal.cuh"

namespace smk {
namespace lo {

constexpr int BLOCK = 256;
constexpr int PCG_CHUNK = 16;  // PCG iterations per graph replay (even: p buffers alternate)
enum { DONE_NO = 0, DONE_CONVERGED = 1, DONE_BREAKDOWN = 2, DONE_CAPPED = 3 };

struct Scalars {
    double alpha, beta, rz, bnorm, rr, d2, n2, rtol;
    int done, iters, max_iters, elim_max;
    unsigned int count;  // arrivals of the running kernel's blocks
    int pad[3];
};

struct Geo {
    int dim, nx, ny, nn, N;
    double m;         // lumped nodal mass |K| / 2^dim
    double wfx, wfy;  // Gauss-Lobatto face weights of x- and y-faces
    double hx, hy;
    double c, alpha;
};

struct NodeGeo {
    int cell, ix, iy, a, b;
};

__device__ __forceinline__ NodeGeo node_geo(const Geo &G, int t) {
    NodeGeo g;
    g.cell = t / G.nn;
    const int loc = t - g.cell * G.nn;
    g.iy = g.cell / G.nx;
    g.ix = g.cell - g.iy * G.nx;
    g.a = loc & 1;
    g.b = G.nn == 4 ? (loc >> 1) : 0;
    return g;
}
__device__ __forceinline__ int nid(const Geo &G, int cell, int a, int b) {
    return cell * G.nn + (G.nn == 4 ? a + 2 * b : a);
}

// value accessors for the stencil helpers
struct Vec {
    const double *v;
    __device__ double operator()(int j) const { return v[j]; }
};
// PCG search direction formed on the fly: p = z + beta p_old
struct Dir {
    const double *z, *p_old;
    double beta;
    __device__ double operator()(int j) const { return z[j] + beta * p_old[j]; }
};

// Component d of (A_FE e) at node j: first-moment rows, E columns.
//   volume  -(c/3) int div v E  at the Lobatto points,
//   faces   (c/3) int [v.n] E^ with E^ the high-side value on interior faces
//           and the node's own value on the boundary.
template <class X>
__device__ __forceinline__ double fe_comp(const Geo &G, const X &e, int j, int d) {
    const NodeGeo g = node_geo(G, j);
    const double c3 = G.c / 3.0;
    if (d == 0) {
        const double e0 = e(nid(G, g.cell, 0, g.b)), e1 = e(nid(G, g.cell, 1, g.b));
        double v = -c3 * G.m * (2 * g.a - 1) / G.hx * (e0 + e1);
        if (g.a == 1)
            v += c3 * G.wfx * (g.ix + 1 < G.nx ? e(nid(G, g.cell + 1, 0, g.b)) : e1);
        else
            v -= c3 * G.wfx * e0;
        return v;
    }
    const double e0 = e(nid(G, g.cell, g.a, 0)), e1 = e(nid(G, g.cell, g.a, 1));
    double v = -c3 * G.m * (2 * g.b - 1) / G.hy * (e0 + e1);
    if (g.b == 1)
        v += c3 * G.wfy * (g.iy + 1 < G.ny ? e(nid(G, g.cell + G.nx, g.a, 0)) : e1);
    else
        v -= c3 * G.wfy * e0;
    return v;
}

// nodal F values, [node][dim]
struct FVec {
    const double *f;
    int D;
    __device__ double operator()(int j, int d) const { return f[(size_t)j * D + d]; }
};
// F = A_FF^-1 A_FE e formed on the fly (the inner factor of S)
template <class X>
struct FOfE {
    Geo G;
    X e;
    const double *aF;
    __device__ double operator()(int j, int d) const { return fe_comp(G, e, j, d) / aF[j]; }
};

// (A_EF f) at node t: zeroth-moment rows, F columns.
//   volume  -int grad u . F,   faces  int [u] F^.n with F^ the low-side F.
template <class FX>
__device__ __forceinline__ double ef_at(const Geo &G, const FX &f, int t) {
    const NodeGeo g = node_geo(G, t);
    double v = -G.m * (2 * g.a - 1) / G.hx *
               (f(nid(G, g.cell, 0, g.b), 0) + f(nid(G, g.cell, 1, g.b), 0));
    if (g.a == 1) {
        if (g.ix + 1 < G.nx) v += G.wfx * f(t, 0);
    } else if (g.ix > 0) {
        v -= G.wfx * f(nid(G, g.cell - 1, 1, g.b), 0);
    }
    if (G.dim == 2) {
        v += -G.m * (2 * g.b - 1) / G.hy *
             (f(nid(G, g.cell, g.a, 0), 1) + f(nid(G, g.cell, g.a, 1), 1));
        if (g.b == 1) {
            if (g.iy + 1 < G.ny) v += G.wfy * f(t, 1);
        } else if (g.iy > 0) {
            v -= G.wfy * f(nid(G, g.cell - G.nx, g.a, 1), 1);
        }
    }
    return v;
}

// (A_EE e) at node t: nodal absorption aE_t e_t, interior penalty
// (c alpha / 2) int [u][E], boundary c alpha int u E.
template <class X>
__device__ __forceinline__ double ee_at(const Geo &G, double aEt, const X &e, int t) {
    const NodeGeo g = node_geo(G, t);
    const double pen = 0.5 * G.c * G.alpha, bnd = G.c * G.alpha;
    const double et = e(t);
    double v = aEt * et;
    if (g.a == 1)
        v += g.ix + 1 < G.nx ? pen * G.wfx * (et - e(nid(G, g.cell + 1, 0, g.b))) : bnd * G.wfx * et;
    else
        v += g.ix > 0 ? pen * G.wfx * (et - e(nid(G, g.cell - 1, 1, g.b))) : bnd * G.wfx * et;
    if (G.dim == 2) {
        if (g.b == 1)
            v += g.iy + 1 < G.ny ? pen * G.wfy * (et - e(nid(G, g.cell + G.nx, g.a, 0)))
                                 : bnd * G.wfy * et;
        else
            v += g.iy > 0 ? pen * G.wfy * (et - e(nid(G, g.cell - G.nx, g.a, 1))) : bnd * G.wfy * et;
    }
    return v;
}

// S e at node t
template <class X>
__device__ __forceinline__ double schur_at(const Geo &G, double aEt, const double *aF, const X &e,
                                           int t) {
    return ee_at(G, aEt, e, t) - ef_at(G, FOfE<X>{G, e, aF}, t);
}

// Diagonal of S = A_EE + (c/3) A_EF A_FF^-1 A_EF^T (A_FE = -(c/3) A_EF^T):
// S_tt = (A_EE)_tt + (c/3) sum_j (A_EF)_tj^2 / (A_FF)_jj over the F columns
// that row t touches.
__device__ double schur_diag(const Geo &G, double aEt, const double *aF, int t) {
    const NodeGeo g = node_geo(G, t);
    const double pen = 0.5 * G.c * G.alpha, bnd = G.c * G.alpha;
    double dEE = aEt, sum = 0.0;
    {
        const double vol = -G.m * (2 * g.a - 1) / G.hx;
        double c0 = vol, c1 = vol;
        if (g.a == 1) {
            if (g.ix + 1 < G.nx) {
                c1 += G.wfx;
                dEE += pen * G.wfx;
            } else {
                dEE += bnd * G.wfx;
            }
        } else if (g.ix > 0) {
            sum += G.wfx * G.wfx / aF[nid(G, g.cell - 1, 1, g.b)];
            dEE += pen * G.wfx;
        } else {
            dEE += bnd * G.wfx;
        }
        sum += c0 * c0 / aF[nid(G, g.cell, 0, g.b)] + c1 * c1 / aF[nid(G, g.cell, 1, g.b)];
    }
    if (G.dim == 2) {
        const double vol = -G.m * (2 * g.b - 1) / G.hy;
        double c0 = vol, c1 = vol;
        if (g.b == 1) {
            if (g.iy + 1 < G.ny) {
                c1 += G.wfy;
                dEE += pen * G.wfy;
            } else {
                dEE += bnd * G.wfy;
            }
        } else if (g.iy > 0) {
            sum += G.wfy * G.wfy / aF[nid(G, g.cell - G.nx, g.a, 1)];
            dEE += pen * G.wfy;
        } else {
            dEE += bnd * G.wfy;
        }
        sum += c0 * c0 / aF[nid(G, g.cell, g.a, 0)] + c1 * c1 / aF[nid(G, g.cell, g.a, 1)];
    }
    return dEE + (G.c / 3.0) * sum;
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
// E* = phi / c and F* = F from the moments of the previous step's intensity
// (the high-order time-edge sources of Sec. 6.1).
__global__ void timeedge_kernel(int N, int D, int nm, double inv_c, const double *__restrict__ mom,
                                double *__restrict__ Estar, double *__restrict__ Fstar) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    Estar[t] = mom[(size_t)t * nm] * inv_c;
    for (int d = 0; d < D; ++d) Fstar[(size_t)t * D + d] = mom[(size_t)t * nm + 1 + d];
}

// Per low-order solve (closures fixed): aF = m sigma~_F, the first-moment
// right-hand side b_F = m F*/(c dt) + R1_ind and u_b = A_FF^-1 b_F.
// R1_ind(v) = int v . sum_g (sigma_F - sigma_g) F_g + int grad_h v : T
//             - int_Gamma0 [v] . {T n}   (Sec. 4, independent closures).
__global__ void prepare_kernel(Geo G, const double *__restrict__ clo, int nc, double inv_cdt,
                               const double *__restrict__ Fstar, double *__restrict__ aF,
                               double *__restrict__ bF, double *__restrict__ ub, Scalars *sc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) sc->elim_max = 0;
    if (t >= G.N) return;
    const NodeGeo g = node_geo(G, t);
    const int D = G.dim;
    auto Tt = [&](int node, int i, int j) -> double {  // closure tensor component (i, j)
        const double *cl = clo + (size_t)node * nc;
        if (D == 1) return cl[2];
        return i != j ? cl[4] : (i == 0 ? cl[3] : cl[5]);
    };
    const double *cl = clo + (size_t)t * nc;
    const double sF = D == 1 ? cl[4] : cl[7];
    const double aFt = G.m * (sF + inv_cdt);
    aF[t] = aFt;
    for (int d = 0; d < D; ++d) {
        double r = G.m * (D == 1 ? cl[6] : cl[9 + d]);
        r += G.m * (2 * g.a - 1) / G.hx *
             (Tt(nid(G, g.cell, 0, g.b), d, 0) + Tt(nid(G, g.cell, 1, g.b), d, 0));
        if (D == 2)
            r += G.m * (2 * g.b - 1) / G.hy *
                 (Tt(nid(G, g.cell, g.a, 0), d, 1) + Tt(nid(G, g.cell, g.a, 1), d, 1));
        if (g.a == 1 && g.ix + 1 < G.nx)
            r -= G.wfx * 0.5 * (Tt(t, d, 0) + Tt(nid(G, g.cell + 1, 0, g.b), d, 0));
        else if (g.a == 0 && g.ix > 0)
            r += G.wfx * 0.5 * (Tt(t, d, 0) + Tt(nid(G, g.cell - 1, 1, g.b), d, 0));
        if (D == 2) {
            if (g.b == 1 && g.iy + 1 < G.ny)
                r -= G.wfy * 0.5 * (Tt(t, d, 1) + Tt(nid(G, g.cell + G.nx, g.a, 0), d, 1));
            else if (g.b == 0 && g.iy > 0)
                r += G.wfy * 0.5 * (Tt(t, d, 1) + Tt(nid(G, g.cell - G.nx, g.a, 1), d, 1));
        }
        const double b = G.m * inv_cdt * Fstar[(size_t)t * D + d] + r;
        bF[(size_t)t * D + d] = b;
        ub[(size_t)t * D + d] = b / aFt;
    }
}

// Per Newton iteration: linearise about the current T (Sec. 5), form the
// Schur right-hand side b_E - A_EF u_b, the Jacobi diagonal, and start PCG
// from x = E: r = rhs - S x, z = r / diag, p = z.
__global__ void __launch_bounds__(BLOCK)
newton_setup_kernel(Geo G, const double *__restrict__ clo, int nc, double a_rad, double dt,
                    const double *__restrict__ T, const double *__restrict__ Tstar,
                    const double *__restrict__ cv, const double *__restrict__ Estar,
                    const double *__restrict__ jin2, const double *__restrict__ aF,
                    const double *__restrict__ ub, const double *__restrict__ E,
                    double *__restrict__ aE, double *__restrict__ diag, double *__restrict__ x,
                    double *__restrict__ r, double *__restrict__ z, double *__restrict__ p0,
                    double rtol, int max_iters, double *part, Scalars *sc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (t < G.N) {
        const NodeGeo g = node_geo(G, t);
        const int D = G.dim;
        const double *cl = clo + (size_t)t * nc;
        const double sE = D == 1 ? cl[3] : cl[6], sP = D == 1 ? cl[5] : cl[8];
        const double inv_cdt = 1.0 / (G.c * dt);
        const double T0 = T[t];
        const double B0 = a_rad * G.c * T0 * T0 * T0 * T0;
        const double dB = 4.0 * a_rad * G.c * T0 * T0 * T0;
        const double cv_dt = cv[t] / dt;
        const double den = cv_dt + sP * dB;
        const double nu = den > 0.0 ? sP * dB / den : 0.0;  // pseudo-fission coefficient
        const double qT0 = cv_dt * (Tstar[t] - T0) - sP * B0;
        const double aEt = G.m * G.c * (sE + inv_cdt - nu * sE);
        double bE = G.m * (sP * B0 + nu * qT0 + Estar[t] / dt);
        // Marshak boundary: -2 int_Gamma_b u F_in with the incoming partial currents
        if (g.a == 0 && g.ix == 0) bE += G.wfx * jin2[0];
        if (g.a == 1 && g.ix == G.nx - 1) bE += G.wfx * jin2[1];
        if (D == 2) {
            if (g.b == 0 && g.iy == 0) bE += G.wfy * jin2[2];
            if (g.b == 1 && g.iy == G.ny - 1) bE += G.wfy * jin2[3];
        }
        const double rhs = bE - ef_at(G, FVec{ub, D}, t);
        const double dg = schur_diag(G, aEt, aF, t);
        const double rv = rhs - schur_at(G, aEt, aF, Vec{E}, t);
        const double zv = rv / dg;
        aE[t] = aEt;
        diag[t] = dg;
        x[t] = E[t];
        r[t] = rv;
        z[t] = zv;
        p0[t] = zv;
        v[0] = rv * rv;
        v[1] = rv * zv;
        v[2] = rhs * rhs;
    }
    if (grid_sums<3>(v, part, &sc->count)) {
        sc->rr = v[0];
        sc->rz = v[1];
        sc->bnorm = sqrt(v[2]);
        sc->beta = 0.0;
        sc->iters = 0;
        sc->rtol = rtol;
        sc->max_iters = max_iters;
        sc->done = sqrt(v[0]) <= rtol * sc->bnorm ? DONE_CONVERGED : DONE_NO;
    }
}

// PCG, first half of an iteration: p = z + beta p_old (written for this
// node, formed on the fly for its neighbours), q = S p, alpha = rz / (p.q).
__global__ void __launch_bounds__(BLOCK)
pcg_matvec_kernel(Geo G, const double *__restrict__ aE, const double *__restrict__ aF,
                  const double *__restrict__ z, const double *__restrict__ p_old,
                  double *__restrict__ p_new, double *__restrict__ q, double *part, Scalars *sc) {
    if (sc->done) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const Dir p{z, p_old, sc->beta};
    double v[1] = {0.0};
    if (t < G.N) {
        const double pt = p(t);
        const double qt = schur_at(G, aE[t], aF, p, t);
        p_new[t] = pt;
        q[t] = qt;
        v[0] = pt * qt;
    }
    if (grid_sums<1>(v, part, &sc->count)) {
        if (v[0] > 0.0 && isfinite(v[0]) && isfinite(sc->rz))
            sc->alpha = sc->rz / v[0];
        else
            sc->done = DONE_BREAKDOWN;  // S not positive definite on p, or non-finite data
    }
}

// PCG, second half: x += alpha p, r -= alpha q, z = r / diag, stopping test
// ||r|| <= rtol ||b|| and beta = (r.z)_new / (r.z)_old.
__global__ void __launch_bounds__(BLOCK)
pcg_update_kernel(int N, const double *__restrict__ p, const double *__restrict__ q,
                  const double *__restrict__ diag, double *__restrict__ x, double *__restrict__ r,
                  double *__restrict__ z, double *part, Scalars *sc) {
    if (sc->done) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const double alpha = sc->alpha;
    double v[2] = {0.0, 0.0};
    if (t < N) {
        x[t] += alpha * p[t];
        const double rv = r[t] - alpha * q[t];
        const double zv = rv / diag[t];
        r[t] = rv;
        z[t] = zv;
        v[0] = rv * rv;
        v[1] = rv * zv;
    }
    if (grid_sums<2>(v, part, &sc->count)) {
        sc->iters += 1;
        sc->rr = v[0];
        if (sqrt(v[0]) <= sc->rtol * sc->bnorm) {
            sc->done = DONE_CONVERGED;
        } else if (sc->iters >= sc->max_iters) {
            sc->done = DONE_CAPPED;
        } else {
            sc->beta = v[1] / sc->rz;
            sc->rz = v[1];
        }
    }
}

// After the linear solve: E = x, back-substitution F = A_FF^-1 (b_F - A_FE E),
// then the pointwise nonlinear elimination of T (Eq. nonlinear_T_update,
// lumped): (C_v/dt) T + sigma_P a c T^4 = c sigma_E E + (C_v/dt) T*, Newton
// from the current T, floored at T_floor.  Sums ||u_new - u_old||^2 and
// ||u_new||^2 over u = (T, E) for Eq. relative_tol.
__global__ void __launch_bounds__(BLOCK)
newton_finish_kernel(Geo G, const double *__restrict__ clo, int nc, double a_rad, double dt,
                     const double *__restrict__ x, const double *__restrict__ aF,
                     const double *__restrict__ bF, const double *__restrict__ Tstar,
                     const double *__restrict__ cv, double *__restrict__ T, double *__restrict__ E,
                     double *__restrict__ F, double rtol, int maxit, double T_floor, double *part,
                     Scalars *sc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0.0, 0.0};
    int its = 0;
    if (t < G.N) {
        const int D = G.dim;
        const double En = x[t];
        const double inv_aF = 1.0 / aF[t];
        for (int d = 0; d < D; ++d)
            F[(size_t)t * D + d] = (bF[(size_t)t * D + d] - fe_comp(G, Vec{x}, t, d)) * inv_aF;
        const double *cl = clo + (size_t)t * nc;
        const double sE = D == 1 ? cl[3] : cl[6], sP = D == 1 ? cl[5] : cl[8];
        const double cv_dt = cv[t] / dt;
        const double k4 = sP * a_rad * G.c;
        const double rhs = G.c * sE * En + cv_dt * Tstar[t];
        const double Told = T[t];
        double y = Told;
        for (its = 1; its <= maxit; ++its) {
            const double y3 = y * y * y;
            const double f = cv_dt * y + k4 * y3 * y - rhs;
            const double df = cv_dt + 4.0 * k4 * y3;
            const double yn = fmax(y - f / df, T_floor);
            const bool conv = fabs(yn - y) <= rtol * fabs(yn);
            y = yn;
            if (conv) break;
        }
        its = min(its, maxit);
        const double dT = y - Told, dE = En - E[t];
        T[t] = y;
        E[t] = En;
        v[0] = dT * dT + dE * dE;
        v[1] = y * y + En * En;
    }
    const int wmax = __reduce_max_sync(0xffffffffu, its);
    if ((threadIdx.x & 31) == 0 && wmax > 0) atomicMax(&sc->elim_max, wmax);
    if (grid_sums<2>(v, part, &sc->count)) {
        sc->d2 = v[0];
        sc->n2 = v[1];
    }
}

// Outer iteration: ||u - u_in||^2 and ||u||^2 for u = (T, E), then u_in <- u.
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
    int N = 0, D = 0, nblk = 0;
    double *buf = nullptr;  // every node array in one allocation
    double *aE, *aF, *bF, *ub, *diag, *x, *r, *z, *pb[2], *q, *Estar, *Fstar, *Tstar, *Tin, *Ein;
    double *part = nullptr;
    double *jin2 = nullptr;     // [4] 2 |F_in| per side
    double *sigma = nullptr;    // sigma_g(T^k) of the running step
    double *clo = nullptr;      // closures when the caller passes none
    smk::lo::Scalars *sc = nullptr;
    smk::lo::Scalars *h_sc = nullptr;  // pinned mirror
    cudaStream_t cap = nullptr;        // private stream for graph capture
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

using smk::lo::BLOCK;
using smk::lo::Geo;
using smk::lo::PCG_CHUNK;

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
    G.nn = p->nn;
    G.N = p->ncell * p->nn;
    G.hx = p->hx;
    G.hy = p->dim == 2 ? p->hy : 1.0;
    G.m = p->dim == 1 ? 0.5 * p->hx : 0.25 * p->hx * p->hy;
    G.wfx = p->dim == 1 ? 1.0 : 0.5 * p->hy;
    G.wfy = 0.5 * p->hx;
    G.c = p->desc.c;
    G.alpha = p->alpha;
    return G;
}

// Capture PCG_CHUNK iterations (two kernels each) into a graph replayed on
// the problem's stream; the device buffers it names never move.
sm_status build_graph(sm_problem *p, sm_lo_state &w) {
    const Geo G = make_geo(p);
    LO_CUDA(cudaStreamCreateWithFlags(&w.cap, cudaStreamNonBlocking));
    LO_CUDA(cudaStreamBeginCapture(w.cap, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < PCG_CHUNK; ++i) {
        double *po = w.pb[i & 1], *pn = w.pb[(i + 1) & 1];
        smk::lo::pcg_matvec_kernel<<<w.nblk, BLOCK, 0, w.cap>>>(G, w.aE, w.aF, w.z, po, pn, w.q,
                                                                w.part, w.sc);
        smk::lo::pcg_update_kernel<<<w.nblk, BLOCK, 0, w.cap>>>(G.N, pn, w.q, w.diag, w.x, w.r,
                                                                w.z, w.part, w.sc);
    }
    cudaGraph_t g = nullptr;
    LO_CUDA(cudaStreamEndCapture(w.cap, &g));
    w.graph = g;
    LO_CUDA(cudaGraphInstantiate(&w.exec, w.graph, 0));
    return SM_OK;
}

sm_status lo_ensure(sm_problem *p) {
    if (p->lo) return SM_OK;
    if ((long long)p->ncell * p->nn > (1LL << 30))
        return lo_fail(SM_ERR_UNSUPPORTED, "the low-order solve supports up to 2^30 nodes");
    p->lo = new sm_lo_state();
    sm_lo_state &w = *p->lo;
    const int N = p->ncell * p->nn, D = p->dim;
    w.N = N;
    w.D = D;
    w.nblk = (N + BLOCK - 1) / BLOCK;
    const size_t nS = 13, nV = 3;  // node arrays and [node][dim] arrays
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
    w.aF = take(N);
    w.diag = take(N);
    w.x = take(N);
    w.r = take(N);
    w.z = take(N);
    w.pb[0] = take(N);
    w.pb[1] = take(N);
    w.q = take(N);
    w.Estar = take(N);
    w.Tstar = take(N);
    w.Tin = take(N);
    w.Ein = take(N);
    LO_CUDA(cudaMalloc(&w.part, sizeof(double) * 3 * (size_t)w.nblk));
    LO_CUDA(cudaMalloc(&w.jin2, sizeof(double) * 4));
    LO_CUDA(cudaMalloc(&w.sigma, sizeof(double) * (size_t)p->G * p->ncell));
    LO_CUDA(cudaMalloc(&w.clo, sizeof(double) * (size_t)N * p->nc));
    LO_CUDA(cudaMalloc(&w.sc, sizeof(smk::lo::Scalars)));
    LO_CUDA(cudaMemset(w.sc, 0, sizeof(smk::lo::Scalars)));
    LO_CUDA(cudaMallocHost(&w.h_sc, sizeof(smk::lo::Scalars)));
    p->workspace_bytes += sizeof(double) * (buf_elems + 3 * (size_t)w.nblk + 4 +
                                            (size_t)p->G * p->ncell + (size_t)N * p->nc) +
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
    return build_graph(p, w);
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
    if (!(prm.eps_outer >= 0) || !(prm.eps_inner >= 0) || !(prm.pcg_rtol > 0) ||
        !(prm.elim_rtol > 0) || !(prm.T_floor > 0))
        return lo_fail(SM_ERR_INVALID_ARG,
                       "tolerances must be >= 0 (eps) or > 0 (pcg_rtol, elim_rtol, T_floor)");
    return SM_OK;
}

// The Newton iteration of Sec. 5 on the gray system with fixed closures.
// Time-edge sources in w.Estar / w.Fstar; T, E hold the initial guesses and
// receive the result, F receives the flux of the last linear solve.
sm_status lo_solve(sm_problem *p, const double *clo, const double *Tstar, const double *cv,
                   double *T, double *E, double *F, const sm_step_params &prm,
                   sm_step_stats *st) {
    sm_lo_state &w = *p->lo;
    const Geo G = make_geo(p);
    cudaStream_t s = p->stream;
    const double dt = p->desc.dt, a = p->desc.a;
    smk::lo::prepare_kernel<<<w.nblk, BLOCK, 0, s>>>(G, clo, p->nc, 1.0 / (G.c * dt), w.Fstar,
                                                     w.aF, w.bF, w.ub, w.sc);
    LO_CUDA(cudaGetLastError());
    p->launches++;
    double d1 = -1.0;
    const int max_chunks = prm.max_pcg / PCG_CHUNK + 2;
    for (int it = 1; it <= prm.max_inner; ++it) {
        smk::lo::newton_setup_kernel<<<w.nblk, BLOCK, 0, s>>>(
            G, clo, p->nc, a, dt, T, Tstar, cv, w.Estar, w.jin2, w.aF, w.ub, E, w.aE, w.diag, w.x,
            w.r, w.z, w.pb[0], prm.pcg_rtol, prm.max_pcg, w.part, w.sc);
        LO_CUDA(cudaGetLastError());
        p->launches++;
        LO_TRY(read_scalars(p));
        int chunks = 0;
        while (!w.h_sc->done && chunks < max_chunks) {
            LO_CUDA(cudaGraphLaunch(w.exec, s));
            p->launches += 2 * PCG_CHUNK;
            ++chunks;
            LO_TRY(read_scalars(p));
        }
        const int done = w.h_sc->done;
        if (done == smk::lo::DONE_BREAKDOWN)
            return lo_fail(SM_ERR_NO_CONVERGENCE,
                           "conjugate gradients broke down: the Schur complement is not positive "
                           "definite on the search direction, or the data is not finite");
        if (done == smk::lo::DONE_NO)
            return lo_fail(SM_ERR_NO_CONVERGENCE, "conjugate gradients did not stop");
        st->pcg_iters_total += w.h_sc->iters;
        st->pcg_iters_max = std::max(st->pcg_iters_max, w.h_sc->iters);
        if (done == smk::lo::DONE_CAPPED) st->pcg_capped++;
        smk::lo::newton_finish_kernel<<<w.nblk, BLOCK, 0, s>>>(
            G, clo, p->nc, a, dt, w.x, w.aF, w.bF, Tstar, cv, T, E, F, prm.elim_rtol, prm.max_elim,
            prm.T_floor, w.part, w.sc);
        LO_CUDA(cudaGetLastError());
        p->launches++;
        LO_TRY(read_scalars(p));
        st->newton_iters_total++;
        const double dn = std::sqrt(w.h_sc->d2), un = std::sqrt(w.h_sc->n2);
        if (!std::isfinite(dn))
            return lo_fail(SM_ERR_NONPHYSICAL, "the low-order Newton iterate is not finite");
        if (d1 < 0) d1 = dn;
        st->newton_iters_max = std::max(st->newton_iters_max, it);
        // Eq. relative_tol, plus a round-off guard for an update that is
        // already at round-off level
        if (dn == 0.0 || dn < prm.eps_inner * d1 || dn <= 1e-14 * un) break;
    }
    st->elim_iters_max = std::max(st->elim_iters_max, w.h_sc->elim_max);
    return SM_OK;
}

sm_status check_lo_problem(sm_problem *p) {
    if (!(p->desc.dt > 0.0))
        return lo_fail(SM_ERR_INVALID_ARG, "the low-order solve needs a time step dt > 0");
    return lo_ensure(p);
}

}  // namespace

namespace smk {
void lo_free(sm_problem *p) {
    if (!p->lo) return;
    sm_lo_state &w = *p->lo;
    if (w.exec) cudaGraphExecDestroy(w.exec);
    if (w.graph) cudaGraphDestroy(w.graph);
    if (w.cap) cudaStreamDestroy(w.cap);
    void *bufs[] = {w.buf, w.part, w.jin2, w.sigma, w.clo, w.sc};
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
}

sm_status sm_loworder_newton(sm_problem *p, const double *closures_dev, const double *T_star_dev,
                             const double *cv_dev, const double *moments_star_dev, double *T_dev,
                             double *E_dev, double *F_dev, const sm_step_params *params,
                             sm_step_stats *stats) {
    if (!p || !closures_dev || !T_star_dev || !cv_dev || !moments_star_dev || !T_dev || !E_dev ||
        !F_dev)
        return lo_fail(SM_ERR_INVALID_ARG, "NULL argument to sm_loworder_newton");
    sm_step_params prm;
    if (params)
        prm = *params;
    else
        sm_default_step_params(&prm);
    LO_TRY(check_params(prm));
    LO_TRY(check_lo_problem(p));
    sm_lo_state &w = *p->lo;
    smk::lo::timeedge_kernel<<<w.nblk, BLOCK, 0, p->stream>>>(w.N, w.D, p->nm, 1.0 / p->desc.c,
                                                             moments_star_dev, w.Estar, w.Fstar);
    LO_CUDA(cudaGetLastError());
    p->launches++;
    sm_step_stats st{};
    LO_TRY(lo_solve(p, closures_dev, T_star_dev, cv_dev, T_dev, E_dev, F_dev, prm, &st));
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
    sm_step_params prm;
    if (params)
        prm = *params;
    else
        sm_default_step_params(&prm);
    LO_TRY(check_params(prm));
    LO_TRY(check_lo_problem(p));
    sm_lo_state &w = *p->lo;
    cudaStream_t s = p->stream;
    const int N = w.N;
    double *clo = closures_dev ? closures_dev : w.clo;
    // opacities frozen at T^k for the whole step (Sec. 3, Rem. opacity)
    LO_TRY(sm_opacity(p, T_dev, scale_dev, w.sigma));
    smk::lo::timeedge_kernel<<<w.nblk, BLOCK, 0, s>>>(N, w.D, p->nm, 1.0 / p->desc.c, moments_dev,
                                                     w.Estar, w.Fstar);
    LO_CUDA(cudaGetLastError());
    p->launches++;
    LO_CUDA(cudaMemcpyAsync(w.Tstar, T_dev, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    LO_CUDA(cudaMemcpyAsync(w.Tin, T_dev, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    LO_CUDA(cudaMemcpyAsync(w.Ein, w.Estar, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    LO_CUDA(cudaMemcpyAsync(E_dev, w.Estar, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    sm_step_stats st{};
    double d1 = -1.0;
    for (int it = 1; it <= prm.max_outer; ++it) {
        // high-order solve with the current T: emission, sweep, moments, closures
        LO_TRY(sm_sweep(p, T_dev, w.sigma, I_prev_dev, I_next_dev, moments_dev, clo));
        LO_TRY(sm_synchronize(p));
        LO_TRY(lo_solve(p, clo, w.Tstar, cv_dev, T_dev, E_dev, F_dev, prm, &st));
        smk::lo::outer_change_kernel<<<w.nblk, BLOCK, 0, s>>>(N, T_dev, E_dev, w.Tin, w.Ein,
                                                             w.part, w.sc);
        LO_CUDA(cudaGetLastError());
        p->launches++;
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
    if (stats) *stats = st;
    return SM_OK;
}

}  // extern "C"
