// Time-dependent high-order problem, right-edge leakage objective and its
// discrete adjoint (gradient with respect to per-cell opacity scales s_K).
//
// Forward step (Eq. transport with Eq. energy_balance, backward Euler, the
// opacities frozen at the start of the step, sigma^n_{g,K} = s_K f_g(Tbar^n_K)):
//   A_{d,g}(sigma~^n) I^{n+1} = sigma^n_g B_g(T^{n+1})/4pi + I^n/(c dt) + inflow
//   C_v (T^{n+1} - T^n)/dt = sum_g sigma^n_g (phi_g - B_g(T^{n+1}))   (per node)
// converged by the unaccelerated iteration: a full pass (emission at the
// current T, sweep with fused moments) then one Newton step of the nodal
// energy balance with the pass's sum_g sigma_g phi_g, until the relative
// change of T is below tol.
//
// Adjoint step n (the transposed linearisation, run backwards in time), with
// psi = lambda / w_d the transport multiplier and theta the energy multiplier:
//   A(sigma~^n)^T psi^n = sigma^n_g theta^n + psi^{n+1}/(c dt) + right-edge inflow dt m
//   (C_v/dt + sum_g sigma_g B'_g) theta^n = sum_g sigma_g B'_g phipsi_g / 4pi + X^{n+1}
// A(Omega)^T is the upwind operator of -Omega: the same sweep kernel with the
// directions reversed (memory quadrant q^2 for geometric quadrant q), i.e. the
// reversed wavefront.  The opacity sensitivity of the step,
//   G^n_{g,K} = -sum_{nodes of K} [sum_d w_d (psi I - psi B_g/4pi - theta I)] - sum theta B_g,
// gives dJ/ds_K += sum_g G^n_{g,K} f_g(Tbar^n_K) and the chain into the
// previous step X^n = theta C_v/dt + sum_g G^n_{g,K} s_K f'_g(Tbar^n_K)/n_nodes.
// The moments of the adjoint step are taken on the canonical FP64 layout
// (the adjoint is off the hot path; this keeps its reductions plain).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sm_internal.cuh"

namespace smk {
namespace adj {

constexpr int BLOCK = 256;

// Fixed-order sums, so that a forward or adjoint step gives the same bits on
// every run: each block folds its threads' pairs by warp shuffles and then
// across its warps in a fixed order and writes one partial pair; finish_kernel
// (one block) sums the partials in a fixed order into acc.
__device__ __forceinline__ void block_sum2(double a, double b, double *__restrict__ part) {
    __shared__ double sa[BLOCK / 32], sb[BLOCK / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sa[wid] = a;
        sb[wid] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int i = 0; i < BLOCK / 32; ++i) {
            ta += sa[i];
            tb += sb[i];
        }
        part[2 * blockIdx.x] = ta;
        part[2 * blockIdx.x + 1] = tb;
    }
}

__global__ void __launch_bounds__(BLOCK) finish_kernel(int nb, const double *__restrict__ part,
                                                       double *__restrict__ acc) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += BLOCK) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    __shared__ double out[2 * BLOCK];
    out[threadIdx.x] = a;
    out[BLOCK + threadIdx.x] = b;
    __syncthreads();
    for (int h = BLOCK / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            out[threadIdx.x] += out[threadIdx.x + h];
            out[BLOCK + threadIdx.x] += out[BLOCK + threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        acc[0] = out[0];
        acc[1] = out[BLOCK];
    }
}

// One Newton step of the nodal energy balance with sum_g sigma_g phi_g (SE)
// fixed; sum_g sigma_g B_g(T) = a c T^4 sigma_P and sum_g sigma_g B'_g =
// 4 a c T^3 sigma_F from the emission pass at T.  Block partials of
// (|dT|^2, |T|^2) in part.
__global__ void __launch_bounds__(BLOCK)
    energy_kernel(int N, double ac, double dt, const double *__restrict__ Tn,
                  const double *__restrict__ cv, const double *__restrict__ gray,
                  const double *__restrict__ mom, int nm, int ise, double *__restrict__ T,
                  double *__restrict__ part) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double dd = 0.0, tt = 0.0;
    if (t < N) {
        const double T0 = T[t];
        const double cv_dt = cv[t] / dt;
        const double T3 = T0 * T0 * T0;
        const double f =
            cv_dt * (T0 - Tn[t]) + ac * T3 * T0 * gray[2 * t] - mom[(size_t)t * nm + ise];
        const double fp = cv_dt + 4.0 * ac * T3 * gray[2 * t + 1];
        const double Tnew = fmax(T0 - f / fp, 0.1 * T0);  // the safeguard never binds near the root
        T[t] = Tnew;
        dd = (Tnew - T0) * (Tnew - T0);
        tt = Tnew * Tnew;
    }
    block_sum2(dd, tt, part);
}

// Adjoint source records: q = sigma_g theta at the nodes, sigma~, sigma
// (the sweep's record layout); padding groups get no source and sigma~ = 1.
template <typename RT>
__global__ void source_kernel(int ncell, int nn, int G, int Gp, double inv_cdt,
                              const double *__restrict__ sigma, const double *__restrict__ theta,
                              RT *__restrict__ src) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell * Gp) return;
    const int cell = i / Gp, g = i - cell * Gp;
    RT *rec = src + (size_t)i * 8;
    if (g < G) {
        const double sg = sigma[(size_t)g * ncell + cell];
        for (int n = 0; n < nn; ++n) rec[n] = (RT)(sg * theta[(size_t)cell * nn + n]);
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

// theta = (sum_g cB_g sum_d w_d psi_{d,g} + X) / (C_v/dt + sdB) per node;
// Block partials of (|dtheta|^2, |theta|^2) in part.  psi canonical [d][g][node].
__global__ void __launch_bounds__(BLOCK)
    theta_kernel(int N, int nd, int G, const double *__restrict__ w,
                 const double *__restrict__ psi, const double *__restrict__ cB,
                 const double *__restrict__ sdB, const double *__restrict__ cv, double dt,
                 const double *__restrict__ X, double *__restrict__ theta,
                 double *__restrict__ part) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double dd = 0.0, tt = 0.0;
    if (t < N) {
        double s = 0.0;
        for (int g = 0; g < G; ++g) {
            double ph = 0.0;
            for (int d = 0; d < nd; ++d) ph += w[d] * psi[((size_t)d * G + g) * N + t];
            s += cB[(size_t)g * N + t] * ph;
        }
        const double th = (s + (X ? X[t] : 0.0)) / (cv[t] / dt + sdB[t]);
        const double d0 = th - theta[t];
        theta[t] = th;
        dd = d0 * d0;
        tt = th * th;
    }
    block_sum2(dd, tt, part);
}

// G_{g,K} = -sum_{n in K} [sum_d w_d (psi I - psi B4 - theta I) + 4 pi theta B4],
// one thread per (g, cell).
__global__ void sens_kernel(int ncell, int nn, int nd, int G, const double *__restrict__ w,
                            const double *__restrict__ psi, const double *__restrict__ I,
                            const double *__restrict__ B4, const double *__restrict__ theta,
                            double *__restrict__ Gs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G * ncell) return;
    const int g = i / ncell, cell = i - g * ncell;
    const size_t N = (size_t)ncell * nn;
    const double FOUR_PI = 4.0 * 3.14159265358979323846;
    double acc = 0.0;
    for (int n = 0; n < nn; ++n) {
        const size_t t = (size_t)cell * nn + n;
        const double b = B4[(size_t)g * N + t], th = theta[t];
        double s = 0.0;
        for (int d = 0; d < nd; ++d) {
            const size_t o = ((size_t)d * G + g) * N + t;
            const double ps = psi[o], iv = I[o];
            s += w[d] * (ps * iv - ps * b - th * iv);
        }
        acc += s + FOUR_PI * th * b;
    }
    Gs[i] = -acc;
}

// grad_K += sum_g G_{g,K} f_g; X = theta C_v/dt + sum_g G_{g,K} s_K f'_g / nn.
__global__ void chain_kernel(int ncell, int nn, int G, const double *__restrict__ Gs,
                             const double *__restrict__ f, const double *__restrict__ df,
                             const double *__restrict__ scale, const double *__restrict__ theta,
                             const double *__restrict__ cv, double dt, double *__restrict__ X,
                             double *__restrict__ grad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncell) return;
    double gk = 0.0, xk = 0.0;
    for (int g = 0; g < G; ++g) {
        const double Gv = Gs[(size_t)g * ncell + k];
        gk += Gv * f[(size_t)g * ncell + k];
        xk += Gv * df[(size_t)g * ncell + k];
    }
    grad[k] += gk;
    xk *= scale[k] / nn;
    for (int n = 0; n < nn; ++n) {
        const size_t t = (size_t)k * nn + n;
        X[t] = theta[t] * cv[t] / dt + xk;
    }
}

// Outgoing partial current through the right edge, lumped at the face's
// Gauss-Lobatto points: sum_{d: Omega_x > 0} w_d Omega_x sum_g sum (h_y/2) I
// over the right-edge nodes (a = 1 of the last column).  One thread per
// (d, g, row), block partials in part; I canonical.
__global__ void __launch_bounds__(BLOCK)
    leakage_kernel(int nx, int ny, int nn, int nd, int G, double half_hy,
                   const double *__restrict__ omx, const double *__restrict__ w,
                   const double *__restrict__ I, double *__restrict__ part) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < nd * G * ny) {
        const int d = i / (G * ny), r = i - d * G * ny;
        const int g = r / ny, iy = r - g * ny;
        if (omx[d] > 0.0) {
            const size_t N = (size_t)nx * ny * nn;
            const size_t cell = (size_t)iy * nx + nx - 1;
            const size_t o = ((size_t)d * G + g) * N + cell * nn;
            double s = I[o + 1];
            if (nn == 4) s += I[o + 3];
            v = w[d] * omx[d] * half_hy * s;
        }
    }
    block_sum2(v, 0.0, part);
}

}  // namespace adj
}  // namespace smk

struct sm_adj_state {
    double *buf = nullptr;
    double *sigma, *f, *df, *B4, *cB, *sdB, *theta, *Tn, *mom, *Gs, *psi_c, *I_c, *omx, *w, *acc;
    double *part;  // per-block partial pairs of the fixed-order sums
    double *h_acc = nullptr;
    void *inflow_adj = nullptr;  // [4][Gp] in the sweep precision
};

namespace {

using smk::adj::BLOCK;

sm_status a_fail(sm_status s, const std::string &m) {
    smk::set_last_error(m.c_str());
    return s;
}

#define A_CUDA(call)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return a_fail(e_ == cudaErrorMemoryAllocation ? SM_ERR_OOM : SM_ERR_CUDA,  \
                          std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)
#define A_TRY(expr)                 \
    do {                            \
        sm_status s_ = (expr);      \
        if (s_ != SM_OK) return s_; \
    } while (0)

inline int nblk(size_t n) { return (int)((n + BLOCK - 1) / BLOCK); }

sm_status adj_ensure(sm_problem *p) {
    if (p->adj) return SM_OK;
    p->adj = new sm_adj_state();
    sm_adj_state &a = *p->adj;
    const size_t N = (size_t)p->ncell * p->nn, GC = (size_t)p->G * p->ncell, GN = (size_t)p->G * N;
    const size_t canon = (size_t)p->nd * GN;
    const size_t nparts = 2 * (size_t)std::max(nblk(N), nblk((size_t)p->nd * p->G * p->ny));
    const size_t total =
        3 * GC + 2 * GN + 3 * N + N * p->nm + GC + 2 * canon + 2 * p->nd + 4 + nparts;
    A_CUDA(cudaMalloc(&a.buf, sizeof(double) * total));
    double *b = a.buf;
    auto take = [&](size_t n) {
        double *r = b;
        b += n;
        return r;
    };
    a.sigma = take(GC);
    a.f = take(GC);
    a.df = take(GC);
    a.B4 = take(GN);
    a.cB = take(GN);
    a.sdB = take(N);
    a.theta = take(N);
    a.Tn = take(N);
    a.mom = take(N * p->nm);
    a.Gs = take(GC);
    a.psi_c = take(canon);
    a.I_c = take(canon);
    a.omx = take(p->nd);
    a.w = take(p->nd);
    a.acc = take(4);
    a.part = take(nparts);
    A_CUDA(cudaMemcpy(a.omx, p->omx.data(), sizeof(double) * p->nd, cudaMemcpyHostToDevice));
    A_CUDA(cudaMemcpy(a.w, p->w.data(), sizeof(double) * p->nd, cudaMemcpyHostToDevice));
    A_CUDA(cudaMallocHost(&a.h_acc, sizeof(double) * 4));
    // the adjoint of the leakage objective enters as an isotropic inflow
    // dt m through the right edge (m = h_x h_y / 4, the lumped nodal mass)
    const size_t nin = 4 * (size_t)p->Gp;
    A_CUDA(cudaMalloc(&a.inflow_adj, nin * p->rsize));
    const double val = p->desc.dt * 0.25 * p->hx * p->hy;
    std::vector<double> in(nin, 0.0);
    for (int g = 0; g < p->G; ++g) in[1 * p->Gp + g] = val;
    if (p->prec == 32) {
        std::vector<float> f(nin);
        for (size_t i = 0; i < nin; ++i) f[i] = (float)in[i];
        A_CUDA(cudaMemcpy(a.inflow_adj, f.data(), nin * 4, cudaMemcpyHostToDevice));
    } else {
        A_CUDA(cudaMemcpy(a.inflow_adj, in.data(), nin * 8, cudaMemcpyHostToDevice));
    }
    p->workspace_bytes += sizeof(double) * total + nin * p->rsize;
    return SM_OK;
}

// Sums the nb block partials in a fixed order and reads the pair back.
sm_status read_acc(sm_problem *p, int nb, double *out2) {
    sm_adj_state &a = *p->adj;
    smk::adj::finish_kernel<<<1, BLOCK, 0, p->stream>>>(nb, a.part, a.acc);
    A_CUDA(cudaGetLastError());
    p->launches++;
    A_CUDA(cudaMemcpyAsync(a.h_acc, a.acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    A_CUDA(cudaStreamSynchronize(p->stream));
    out2[0] = a.h_acc[0];
    out2[1] = a.h_acc[1];
    return SM_OK;
}

sm_status adjoint_sweep(sm_problem *p, const void *psi_next, void *psi_out) {
    sm_adj_state &a = *p->adj;
    cudaStream_t s = p->stream;
    const int n = p->ncell * p->Gp;
    if (p->prec == 32)
        smk::adj::source_kernel<float><<<nblk(n), BLOCK, 0, s>>>(
            p->ncell, p->nn, p->G, p->Gp, p->inv_cdt, a.sigma, a.theta, (float *)p->d_src);
    else
        smk::adj::source_kernel<double><<<nblk(n), BLOCK, 0, s>>>(
            p->ncell, p->nn, p->G, p->Gp, p->inv_cdt, a.sigma, a.theta, (double *)p->d_src);
    A_CUDA(cudaGetLastError());
    p->launches++;
    A_TRY(smk::sweep_only(p, psi_next, psi_out, nullptr, nullptr, 1));
    A_CUDA(smk::launch_pack(p, a.psi_c, psi_out, 1, s));
    p->launches++;
    return SM_OK;
}

sm_status check_aligned(const void *a, const void *b) {
    if ((reinterpret_cast<uintptr_t>(a) & 15u) || (reinterpret_cast<uintptr_t>(b) & 15u))
        return a_fail(SM_ERR_INVALID_ARG, "packed intensity buffers must be 16-byte aligned");
    return SM_OK;
}

}  // namespace

namespace smk {
void adjoint_free(sm_problem *p) {
    if (!p->adj) return;
    if (p->adj->buf) cudaFree(p->adj->buf);
    if (p->adj->inflow_adj) cudaFree(p->adj->inflow_adj);
    if (p->adj->h_acc) cudaFreeHost(p->adj->h_acc);
    delete p->adj;
    p->adj = nullptr;
}
}  // namespace smk

extern "C" {

sm_status sm_ho_step(sm_problem *p, const double *scale_dev, const double *cv_dev, double *T_dev,
                     const void *I_prev_dev, void *I_next_dev, double tol, int max_iter,
                     int *iters_host) {
    if (!p || !scale_dev || !cv_dev || !T_dev || !I_next_dev)
        return a_fail(SM_ERR_INVALID_ARG, "NULL argument to sm_ho_step");
    if (!(p->desc.dt > 0.0)) return a_fail(SM_ERR_INVALID_ARG, "sm_ho_step needs dt > 0");
    if (!(tol > 0.0) || max_iter < 1)
        return a_fail(SM_ERR_INVALID_ARG, "tol must be > 0 and max_iter >= 1");
    A_TRY(check_aligned(I_prev_dev, I_next_dev));
    A_TRY(adj_ensure(p));
    sm_adj_state &a = *p->adj;
    cudaStream_t s = p->stream;
    const int N = p->ncell * p->nn;
    A_TRY(sm_opacity(p, T_dev, scale_dev, a.sigma));  // frozen for the step
    A_CUDA(cudaMemcpyAsync(a.Tn, T_dev, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    const int ise = p->dim == 2 ? 6 : 3;
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
        A_TRY(sm_sweep(p, T_dev, a.sigma, I_prev_dev, I_next_dev, a.mom, nullptr));
        smk::adj::energy_kernel<<<nblk(N), BLOCK, 0, s>>>(N, p->desc.a * p->desc.c, p->desc.dt,
                                                          a.Tn, cv_dev, p->d_gray, a.mom, p->nm,
                                                          ise, T_dev, a.part);
        A_CUDA(cudaGetLastError());
        p->launches++;
        double h[2];
        A_TRY(read_acc(p, nblk(N), h));
        if (!std::isfinite(h[0]) || !std::isfinite(h[1]))
            return a_fail(SM_ERR_NONPHYSICAL, "the temperature iterate is not finite");
        if (std::sqrt(h[0]) <= tol * std::sqrt(h[1])) break;
    }
    // the intensity of the converged temperature
    A_TRY(sm_sweep(p, T_dev, a.sigma, I_prev_dev, I_next_dev, a.mom, nullptr));
    A_TRY(sm_synchronize(p));
    if (iters_host) *iters_host = std::min(it, max_iter);
    return SM_OK;
}

sm_status sm_leakage(sm_problem *p, const void *I_dev, double *out_host) {
    if (!p || !I_dev || !out_host) return a_fail(SM_ERR_INVALID_ARG, "NULL argument to sm_leakage");
    if (p->dim != 2) return a_fail(SM_ERR_UNSUPPORTED, "sm_leakage is 2D only");
    A_TRY(adj_ensure(p));
    sm_adj_state &a = *p->adj;
    cudaStream_t s = p->stream;
    A_CUDA(smk::launch_pack(p, a.I_c, const_cast<void *>(I_dev), 1, s));
    const int n = p->nd * p->G * p->ny;
    smk::adj::leakage_kernel<<<nblk(n), BLOCK, 0, s>>>(p->nx, p->ny, p->nn, p->nd, p->G,
                                                       0.5 * p->hy, a.omx, a.w, a.I_c, a.part);
    A_CUDA(cudaGetLastError());
    p->launches += 2;
    double h[2];
    A_TRY(read_acc(p, nblk(n), h));
    *out_host = h[0];
    return SM_OK;
}

sm_status sm_adjoint_step(sm_problem *p, const double *scale_dev, const double *cv_dev,
                          const double *T_n_dev, const double *T_np1_dev, const void *I_np1_dev,
                          const void *psi_next_dev, const double *X_next_dev, void *psi_out_dev,
                          double *X_out_dev, double *grad_dev, double tol, int max_iter,
                          int *iters_host) {
    if (!p || !scale_dev || !cv_dev || !T_n_dev || !T_np1_dev || !I_np1_dev || !psi_out_dev ||
        !X_out_dev || !grad_dev)
        return a_fail(SM_ERR_INVALID_ARG, "NULL argument to sm_adjoint_step");
    if (p->dim != 2) return a_fail(SM_ERR_UNSUPPORTED, "the adjoint is 2D only");
    if (!(p->desc.dt > 0.0)) return a_fail(SM_ERR_INVALID_ARG, "the adjoint needs dt > 0");
    if (!(tol > 0.0) || max_iter < 1)
        return a_fail(SM_ERR_INVALID_ARG, "tol must be > 0 and max_iter >= 1");
    if (psi_next_dev == psi_out_dev)
        return a_fail(SM_ERR_INVALID_ARG, "psi_next and psi_out must not alias");
    A_TRY(check_aligned(psi_next_dev, psi_out_dev));
    A_TRY(check_aligned(I_np1_dev, nullptr));
    A_TRY(adj_ensure(p));
    sm_adj_state &a = *p->adj;
    cudaStream_t s = p->stream;
    const int N = p->ncell * p->nn;
    const double dt = p->desc.dt;
    A_TRY(sm_opacity(p, T_n_dev, scale_dev, a.sigma));
    A_CUDA(smk::launch_opacity_shape(p, T_n_dev, a.f, a.df, s));
    A_CUDA(smk::launch_planck_parts(p, T_np1_dev, a.sigma, a.B4, a.cB, a.sdB, s));
    A_CUDA(smk::launch_pack(p, a.I_c, const_cast<void *>(I_np1_dev), 1, s));
    A_CUDA(cudaMemsetAsync(a.theta, 0, sizeof(double) * N, s));
    p->launches += 3;
    // the sweep reads the adjoint inflow for the duration of the step
    const size_t nin = 4 * (size_t)p->Gp * p->rsize;
    A_CUDA(cudaMemcpyAsync(p->d_inflow, a.inflow_adj, nin, cudaMemcpyDeviceToDevice, s));
    sm_status st = SM_OK;
    int it = 0;
    for (it = 1; it <= max_iter && st == SM_OK; ++it) {
        if ((st = adjoint_sweep(p, psi_next_dev, psi_out_dev)) != SM_OK) break;
        smk::adj::theta_kernel<<<nblk(N), BLOCK, 0, s>>>(N, p->nd, p->G, a.w, a.psi_c, a.cB,
                                                         a.sdB, cv_dev, dt, X_next_dev, a.theta,
                                                         a.part);
        p->launches++;
        double h[2];
        if ((st = read_acc(p, nblk(N), h)) != SM_OK) break;
        if (!std::isfinite(h[0])) {
            st = a_fail(SM_ERR_NONPHYSICAL, "the adjoint iterate is not finite");
            break;
        }
        if (std::sqrt(h[0]) <= tol * std::sqrt(h[1])) break;
    }
    if (st == SM_OK) st = adjoint_sweep(p, psi_next_dev, psi_out_dev);  // psi of the final theta
    if (st == SM_OK) {
        const int ng = p->G * p->ncell;
        smk::adj::sens_kernel<<<nblk(ng), BLOCK, 0, s>>>(p->ncell, p->nn, p->nd, p->G, a.w,
                                                         a.psi_c, a.I_c, a.B4, a.theta, a.Gs);
        smk::adj::chain_kernel<<<nblk(p->ncell), BLOCK, 0, s>>>(p->ncell, p->nn, p->G, a.Gs, a.f,
                                                                a.df, scale_dev, a.theta, cv_dev,
                                                                dt, X_out_dev, grad_dev);
        p->launches += 2;
    }
    // restore the problem's own boundary inflow
    const cudaError_t e = smk::launch_inflow(p, s);
    if (st == SM_OK && e != cudaSuccess)
        st = a_fail(SM_ERR_CUDA, std::string("inflow: ") + cudaGetErrorString(e));
    if (st == SM_OK) st = sm_synchronize(p);
    if (iters_host) *iters_host = std::min(it, max_iter);
    return st;
}

}  // extern "C"
