// FP64 defect correction of the transport solve with FP32 sweeps (the FP32
// sweep path refined to FP64 accuracy inside the outer SM iteration).
//
// The state -- the intensity iterate, the previous step's intensity, the
// emission records -- is FP64 (a precision-64 problem).  Each outer iteration
// of Algorithm 1 replaces the FP64 sweep by corrections of the iterate I
// (which starts at I^k), each
//   1. the FP64 residual of the lumped upwind-DG equations (Eq. dgsn_transport
//      with the time term of Eq. smm_be_transport) at I:
//      r = S + (upwind face terms of I) - M I per node, S = q + I^k/(c dt),
//      stored in FP32;
//   2. an FP32 sweep of the correction, M d = r + (upwind face terms of d)
//      with zero inflow (the sweep kernel with q = 0 and r in place of I^k,
//      1/(c dt) -> 1);
//   3. I += d in FP64,
// until a correction is below 1e-8 of the iterate (at most MAX_CORR per outer
// iteration): a correction leaves the FP32 solve's relative error of d, so
// the next one is that much smaller and the iterate reaches the FP64 solution
// of the transport equations for the outer iteration's temperature -- the same
// intensity the FP64 sweep computes, up to rounding.  One correction per outer
// iteration would not do: its FP32 error would enter the closures and, through
// the low-order solve, the next temperature, and the outer iteration carries
// such errors along.  Then the FP64 moments of the iterate, read from it
// directly (the sweep's fused FP32 moments of d would carry FP32 rounding of
// the large first corrections into every later moment).
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
//
// Cost on this GPU: the residual takes about 30 FP64 operations per
// (cell, direction, group), the update 8 and the moments 9, against some 90 of
// the FP64 sweep, and FP64 issues at 1/64 of the FP32 rate; with two
// corrections per outer iteration the refined path costs about what the FP64
// sweep does.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sm_internal.cuh"

namespace smk {

constexpr int MAX_CORR = 4;         // corrections per outer iteration, at most
constexpr double CORR_TOL = 1e-8;   // stop once max |d| <= CORR_TOL max |I|

struct RefineArgs {
    int nx, ny, ncell, NQ, NWT, NGB, DB, LG, GW, Gp;
    double inv_cdt;
    const LaneConst *lanes;
    const double *src;     // [cell][Gp][8] FP64 records: q at the nodes, sigma~, sigma
    const double *inflow;  // [4][Gp] FP64
    const double *I_k;     // packed FP64 I^k (NULL: zero)
    const double *I;       // packed FP64 iterate
    float *r;              // packed FP32 residual (out)
    size_t n_elems;        // packed elements / 4 (one thread each)
};

// One thread per (warp task, cell, slot, lane): the residual of its four
// nodes.  Padding lanes (no direction) get r = 0, so their correction is 0.
__global__ void __launch_bounds__(256) residual_kernel(const RefineArgs R) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= R.n_elems) return;
    const int lane = (int)(e & 31);
    size_t rest = e >> 5;
    const int slot = (int)(rest % R.GW);
    rest /= R.GW;
    const int cell = (int)(rest % R.ncell);
    const int wg = (int)(rest / R.ncell);
    const int q = wg / R.NWT, wt = wg - q * R.NWT;
    const int db = wt / R.NGB, gb = wt - db * R.NGB;
    const LaneConst &L = R.lanes[(q * R.DB + db) * 32 + lane];
    float *ro = R.r + e * 4;
    const int g = gb * R.GW * R.LG + slot * R.LG + L.g_lo;
    if (!L.valid) {
        for (int n = 0; n < 4; ++n) ro[n] = 0.0f;
        return;
    }
    const int sx = (q == 0 || q == 3) ? 1 : -1, sy = q < 2 ? 1 : -1;
    const int au = sx > 0 ? 0 : 1, bu = sy > 0 ? 0 : 1;
    const int nuu = au + 2 * bu, ndu = (1 - au) + 2 * bu;
    const int nud = au + 2 * (1 - bu), ndd = (1 - au) + 2 * (1 - bu);
    const int ix = cell % R.nx, iy = cell / R.nx;
    // the packed elements of the same (warp task, slot, lane) at another cell
    const size_t cell_stride = (size_t)R.GW * 32;
    const double *Ic = R.I + e * 4;
    double I[4], S[4];
    for (int n = 0; n < 4; ++n) I[n] = Ic[n];
    const double *rec = R.src + ((size_t)cell * R.Gp + g) * 8;
    for (int n = 0; n < 4; ++n) S[n] = rec[n];
    if (R.I_k) {
        const double *ik = R.I_k + e * 4;
        for (int n = 0; n < 4; ++n) S[n] = fma(R.inv_cdt, ik[n], S[n]);
    }
    double Xu, Xd, Yu, Yd;
    if (ix - sx >= 0 && ix - sx < R.nx) {
        const double *nb = Ic - (ptrdiff_t)(sx * (ptrdiff_t)cell_stride) * 4;
        Xu = nb[ndu];
        Xd = nb[ndd];
    } else {
        Xu = Xd = R.inflow[(sx > 0 ? 0 : 1) * R.Gp + g];
    }
    if (iy - sy >= 0 && iy - sy < R.ny) {
        const double *nb = Ic - (ptrdiff_t)(sy * (ptrdiff_t)R.nx * (ptrdiff_t)cell_stride) * 4;
        Yu = nb[nud];
        Yd = nb[ndd];
    } else {
        Yu = Yd = R.inflow[(sy > 0 ? 2 : 3) * R.Gp + g];
    }
    const double mu = L.mu, eta = L.eta;
    const double A = rec[4] + mu + eta;
    double r[4];
    r[nuu] = S[nuu] + 2.0 * (mu * Xu + eta * Yu) - (A * I[nuu] + mu * I[ndu] + eta * I[nud]);
    r[ndu] = S[ndu] + 2.0 * eta * Yd - (A * I[ndu] - mu * I[nuu] + eta * I[ndd]);
    r[nud] = S[nud] + 2.0 * mu * Xd - (A * I[nud] - eta * I[nuu] + mu * I[ndd]);
    r[ndd] = S[ndd] - (A * I[ndd] - eta * I[ndu] - mu * I[nud]);
    for (int n = 0; n < 4; ++n) ro[n] = (float)r[n];
}

// I += d (FP64 iterate, FP32 correction, the same packed layout, one
// element of four nodes per thread), with max |d| and max |I| after the
// update: non-negative IEEE numbers order like their bit patterns, so the
// maxima are integer atomics on the bits (no FP64 compare).
__global__ void __launch_bounds__(256) update_kernel(double *__restrict__ I,
                                                     const float *__restrict__ d, size_t n_elems,
                                                     unsigned long long *__restrict__ maxes) {
    unsigned long long md = 0, mi = 0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_elems;
         e += (size_t)gridDim.x * blockDim.x) {
        const float4 dv = reinterpret_cast<const float4 *>(d)[e];
        double2 *ip = reinterpret_cast<double2 *>(I) + e * 2;
        double2 a = ip[0], b = ip[1];
        a.x += (double)dv.x;
        a.y += (double)dv.y;
        b.x += (double)dv.z;
        b.y += (double)dv.w;
        ip[0] = a;
        ip[1] = b;
        const unsigned dm = max(max(__float_as_uint(fabsf(dv.x)), __float_as_uint(fabsf(dv.y))),
                                max(__float_as_uint(fabsf(dv.z)), __float_as_uint(fabsf(dv.w))));
        const unsigned long long abs_mask = 0x7fffffffffffffffull;
        const unsigned long long im =
            max(max((unsigned long long)__double_as_longlong(a.x) & abs_mask,
                    (unsigned long long)__double_as_longlong(a.y) & abs_mask),
                max((unsigned long long)__double_as_longlong(b.x) & abs_mask,
                    (unsigned long long)__double_as_longlong(b.y) & abs_mask));
        md = max(md, (unsigned long long)dm);
        mi = max(mi, im);
    }
    for (int off = 16; off >= 1; off >>= 1) {
        md = max(md, __shfl_xor_sync(0xffffffffu, md, off));
        mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(maxes + 0, md);
        atomicMax(maxes + 1, mi);
    }
}

// FP64 moments of the packed FP64 iterate, per node: one warp per (quadrant,
// direction block, cell); each lane sums its direction's intensities over all
// groups of the direction block, plain and sigma-weighted (sigma_g from the
// records), the sums pass through shared memory, and each lane forms one of
// the 36 moments (4 nodes x {phi, F, P} and sigma-weighted {phi, F}) as the
// dot product of the 32 lanes' sums with their weights; partial moments per
// (quadrant, direction block) go to part[qd][cell][36] for the fixed-order
// reduction.  Padding lanes have zero weights and padding groups zero
// intensity.
constexpr int MOM_WARPS = 4;
__global__ void __launch_bounds__(MOM_WARPS * 32)
moments64_kernel(const double *__restrict__ I, const LaneConst *__restrict__ lanes,
                 const double *__restrict__ src, int ncell, int NQ, int DB, int NGB, int NWT,
                 int GW, int LG, int Gp, double *__restrict__ part) {
    __shared__ double sh[MOM_WARPS][8][33];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const long long wglob = (long long)blockIdx.x * MOM_WARPS + wi;
    if (wglob >= (long long)NQ * DB * ncell) return;
    const int qd = (int)(wglob / ncell), cell = (int)(wglob - (long long)qd * ncell);
    const int q = qd / DB, db = qd - q * DB;
    const LaneConst &L = lanes[qd * 32 + lane];
    double s[4] = {0.0, 0.0, 0.0, 0.0}, ss[4] = {0.0, 0.0, 0.0, 0.0};
    for (int gb = 0; gb < NGB; ++gb) {
        const int wt = db * NGB + gb;
        const size_t e0 = (((size_t)q * NWT + wt) * ncell + cell) * GW;
        for (int gw = 0; gw < GW; ++gw) {
            const int g = gb * GW * LG + gw * LG + L.g_lo;
            const double sg = src[((size_t)cell * Gp + g) * 8 + 5];
            const double2 *ip = reinterpret_cast<const double2 *>(I) + ((e0 + gw) * 32 + lane) * 2;
            const double2 a = ip[0], b = ip[1];
            const double v[4] = {a.x, a.y, b.x, b.y};
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                s[n] += v[n];
                ss[n] = fma(sg, v[n], ss[n]);
            }
        }
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        sh[wi][n][lane] = s[n];
        sh[wi][4 + n][lane] = ss[n];
    }
    __syncwarp();
    for (int m = lane; m < 36; m += 32) {
        const int n = m / 9, k = m - 9 * n;
        const int row = k < 6 ? n : 4 + n, wrow = k < 6 ? k : k - 6;
        double acc = 0.0;
        for (int j = 0; j < 32; ++j) acc = fma(lanes[qd * 32 + j].wm[wrow], sh[wi][row][j], acc);
        part[((size_t)qd * ncell + cell) * 36 + m] = acc;
    }
}

// FP32 records of the correction sweep: no emission (q = 0), the problem's
// sigma~ and sigma rounded to FP32.
__global__ void records32_kernel(const double *__restrict__ rec, float *__restrict__ out,
                                 size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *a = rec + i * 8;
    float *o = out + i * 8;
    for (int k = 0; k < 4; ++k) o[k] = 0.0f;
    o[4] = (float)a[4];
    o[5] = (float)a[5];
    o[6] = 0.0f;
    o[7] = 0.0f;
}

}  // namespace smk

struct sm_refine_state {
    float *r = nullptr, *d = nullptr;  // packed FP32 residual and correction
    float *rec32 = nullptr;            // [cell][Gp][8] FP32 records of the correction sweep
    float *inflow0 = nullptr;          // [4][Gp] zero inflow
    double *part = nullptr;            // [NQ*DB][cell][36] partial moments of the iterate
    unsigned long long *maxes = nullptr;    // max |d|, max |I| of the last update (bits)
    unsigned long long *h_maxes = nullptr;  // pinned mirror
    int W = 0, S = 0, NS = 0;          // tiling of the FP32 correction sweep
    int resident = 0;                  // its CTAs that fit
    int corrections = 0;               // corrections of the running step
};

namespace smk {

void refine_free(sm_problem *p) {
    if (!p->refine) return;
    sm_refine_state &R = *p->refine;
    for (void *b : {(void *)R.r, (void *)R.d, (void *)R.rec32, (void *)R.inflow0, (void *)R.part,
                    (void *)R.maxes})
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
    if (cudaMalloc(&R.r, ie * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&R.d, ie * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&R.rec32, nrec * 8 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&R.inflow0, (size_t)4 * p->Gp * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&R.part, npart * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&R.maxes, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&R.h_maxes, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(R.inflow0, 0, (size_t)4 * p->Gp * sizeof(float)) != cudaSuccess) {
        refine_free(p);
        set_last_error("FP64 defect correction: device allocation failed");
        return SM_ERR_OOM;
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
    p->workspace_bytes += ie * 8 + nrec * 32 + (size_t)16 * p->Gp + npart * 8 + 16;
    return SM_OK;
}

// The transport solve of one outer iteration by defect correction of the
// packed FP64 iterate I (the records hold the emission of the current
// temperature), then the FP64 moments of I into mom.  I_k: the previous
// step's intensity.  Synchronizes the stream after each correction (the
// stopping test reads the maxima).
sm_status refine_solve(sm_problem *p, const double *I_k, double *I, double *mom) {
    sm_refine_state &R = *p->refine;
    cudaStream_t s = p->stream;
    const size_t ie = (size_t)p->NQ * p->NWT * p->ncell * p->GW * 32 * 4;
    const size_t nrec = (size_t)p->ncell * p->Gp;
    auto cuda_fail = [](const char *what) {
        set_last_error(what);
        return SM_ERR_CUDA;
    };
    records32_kernel<<<(unsigned)((nrec + 255) / 256), 256, 0, s>>>(
        static_cast<const double *>(p->d_src), R.rec32, nrec);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail("FP64 defect correction: records launch failed");
    p->launches++;
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
    A.inv_cdt = p->inv_cdt;
    A.lanes = p->d_lanes;
    A.src = static_cast<const double *>(p->d_src);
    A.inflow = static_cast<const double *>(p->d_inflow);
    A.I_k = I_k;
    A.I = I;
    A.r = R.r;
    A.n_elems = ie / 4;
    for (int c = 0; c < MAX_CORR; ++c) {
        residual_kernel<<<(unsigned)((A.n_elems + 255) / 256), 256, 0, s>>>(A);
        if (cudaGetLastError() != cudaSuccess) return cuda_fail("FP64 defect correction: residual launch failed");
        // the FP32 correction sweep: source r, no emission, zero inflow, its
        // own tiling (moments not reduced)
        ++p->epoch;
        SweepArgs a = make_sweep_args(p, R.r, R.d);
        a.src = R.rec32;
        a.inflow = R.inflow0;
        a.inv_cdt = 1.0;
        a.W = R.W;
        a.S = R.S;
        a.NS = R.NS;
        a.n_tasks = R.NS * p->NQ * p->NWT;
        a.publish = publish_rows(a.n_tasks, R.resident);
        if (cudaMemsetAsync(p->d_ctrl, 0, 2 * sizeof(unsigned int), s) != cudaSuccess ||
            launch_sweep2d_prec(32, p, a, std::min(a.n_tasks, R.resident), s) != cudaSuccess ||
            cudaMemsetAsync(R.maxes, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess)
            return cuda_fail("FP64 defect correction: correction sweep launch failed");
        update_kernel<<<std::max<size_t>(1, std::min<size_t>((ie / 4 + 255) / 256, 152 * 8)), 256, 0,
                        s>>>(I, R.d, ie / 4, R.maxes);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(R.h_maxes, R.maxes, 2 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return cuda_fail("FP64 defect correction: update launch failed");
        p->launches += 3;
        ++R.corrections;
        const sm_status st = sm_synchronize(p);  // also reports a wavefront timeout
        if (st != SM_OK) return st;
        unsigned dbits = (unsigned)R.h_maxes[0];
        float dmax;
        std::memcpy(&dmax, &dbits, sizeof(dmax));
        double imax;
        std::memcpy(&imax, &R.h_maxes[1], sizeof(imax));
        if (!std::isfinite(dmax) || !std::isfinite(imax)) {
            set_last_error("FP64 defect correction: the correction is not finite");
            return SM_ERR_NONPHYSICAL;
        }
        if ((double)dmax <= CORR_TOL * imax) break;
    }
    const long long warps = (long long)p->NQ * p->DB * p->ncell;
    moments64_kernel<<<(unsigned)((warps + MOM_WARPS - 1) / MOM_WARPS), MOM_WARPS * 32, 0, s>>>(
        I, p->d_lanes, static_cast<const double *>(p->d_src), p->ncell, p->NQ, p->DB, p->NGB,
        p->NWT, p->GW, p->LG, p->Gp, R.part);
    if (cudaGetLastError() != cudaSuccess ||
        launch_reduce_prec(64, p, R.part, p->NQ * p->DB, mom, nullptr, s) != cudaSuccess)
        return cuda_fail("FP64 defect correction: moments launch failed");
    p->launches += 2;
    return SM_OK;
}

int refine_take_corrections(sm_problem *p) {
    if (!p->refine) return 0;
    const int c = p->refine->corrections;
    p->refine->corrections = 0;
    return c;
}

}  // namespace smk
