// Rows a2 + a3: the lumped upwind-DG transport sweep (Sec. 3, Eqs. upwind and
// dgsn_transport; all forms lumped with the tensor 2-point Gauss-Lobatto rule,
// Sec. 6) fused with the per-node angular-moment reductions (Sec. 2).
//
// Lumped cell system.  With the corner quadrature every mass, reaction and
// face term is nodal.  Dividing the equation of node (x-side, y-side) by its
// mass hx*hy/4 and naming the sides u (upwind) / d (downwind) of the sweep,
// mu = |Omega_x|/hx, eta = |Omega_y|/hy, A = sigma~ + mu + eta:
//   [ A   mu  eta  0  ] [I_uu]   [S_uu + 2 mu X_u + 2 eta Y_u]
//   [-mu  A   0   eta ] [I_du] = [S_du + 2 eta Y_d          ]
//   [-eta 0   A   mu  ] [I_ud]   [S_ud + 2 mu X_d           ]
//   [ 0  -eta -mu  A  ] [I_dd]   [S_dd                      ]
// where X_u, X_d are the upwind x-face inflows of the two node rows, Y_u, Y_d
// the upwind y-face inflows of the two node columns and S = q + I^k/(c dt).
// The matrix is A*I + mu*Jx + eta*Jy with commuting skew parts Jx, Jy
// (Jx^2 = Jy^2 = -I), so with P = A^2 + mu^2 + eta^2 and Z = Jx*Jy:
//   M^{-1} = (A - mu Jx - eta Jy) (P + 2 mu eta Z) / (P^2 - 4 mu^2 eta^2).
// The kernel evaluates this after scaling by 1/A (no overflow in FP32 for
// optical depths up to ~1e9).  1D: [[A, mu], [-mu, A]] with A = sigma~ + mu.
//
// Parallel layout.  A warp task owns 32 lanes x GW slots of (direction, group)
// pairs of one quadrant (lane = direction inside the quadrant, or direction x
// group when a quadrant has fewer than 32 directions).  W warp tasks of the
// same quadrant form a chain; a chain's mesh is cut into column strips of
// TX cells, one CTA per (chain, strip).  A CTA sweeps its strip row by row in
// upwind order; the x-inflow of each row comes from the upwind strip through
// an L2-resident face buffer and a per-(chain, strip) row counter (release /
// acquire), the y-inflow is carried in shared memory.  Tasks are handed out
// by an atomic queue in upwind-strip order, so every awaited producer is
// already running (no deadlock for any grid size), and every wait is bounded
// in time (status word + abort flag, never a trap).  Per cell, each lane sums
// its GW intensities, forms the 36 (2D) weighted moments, and the warp
// reduces them by a transpose-butterfly; the W warps are summed in shared
// memory and written as one partial per (chain, cell).
#include "sm_internal.cuh"

namespace smk {

template <typename RT> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

__device__ __forceinline__ void ld4_stream(const float *p, float (&v)[4]) {
    const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4_stream(const double *p, double (&v)[4]) {
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(p + 2));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4_stream(float *p, const float (&v)[4]) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void st4_stream(double *p, const double (&v)[4]) {
    __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
    __stcs(reinterpret_cast<double2 *>(p + 2), make_double2(v[2], v[3]));
}
__device__ __forceinline__ void ld4_ro(const float *p, float (&v)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4_ro(const double *p, double (&v)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p + 2));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for a producer row counter.  Returns 0 when the counter reached
// target, 1 when the wait gave up (time limit: records ST_TIMEOUT and raises
// the abort flag) or another CTA aborted.
__device__ int wait_flag(const unsigned long long *f, unsigned long long target,
                         unsigned int *ctrl, long long timeout_ns) {
    if (ld_acquire(f) >= target) return 0;
    const long long t0 = global_ns();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
        if (ld_acquire(f) >= target) return 0;
        if (ld_relaxed(ctrl + CTRL_ABORT)) return 1;
        if (global_ns() - t0 > timeout_ns) {
            atomicOr(ctrl + CTRL_STATUS, (unsigned)ST_TIMEOUT);
            atomicExch(ctrl + CTRL_ABORT, 1u);
            return 1;
        }
    }
}

// Transpose-butterfly warp reduction of CNT values per lane: afterwards v[0]
// of lane L holds the warp sum of value index L >> (5 - log2 CNT).
template <int OFF, int CNT, typename RT> struct TRed {
    static __device__ __forceinline__ void run(RT *v, int lane) {
        if constexpr (CNT > 1) {
            constexpr int H = CNT / 2;
            const bool up = (lane & OFF) != 0;
#pragma unroll
            for (int i = 0; i < H; ++i) {
                const RT send = up ? v[i] : v[i + H];
                const RT keep = up ? v[i + H] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
            }
            if constexpr (OFF > 1) TRed<OFF / 2, H, RT>::run(v, lane);
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], OFF);
            if constexpr (OFF > 1) TRed<OFF / 2, 1, RT>::run(v, lane);
        }
    }
};

size_t sweep2d_smem_bytes(int prec, int W, int GW, int TX) {
    const size_t rs = (prec == 32) ? 4 : 8;
    return (size_t)W * GW * TX * 32 * 2 * rs + (size_t)2 * W * TX * 36 * rs;
}

// ---------------------------------------------------------------------------
template <typename RT, int GW>
__global__ void __launch_bounds__(512) sweep2d_kernel(const SweepArgs A) {
    using R2 = typename V2<RT>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_task;
    __shared__ int s_abort;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int W = A.W, TX = A.TX;
    const int nx = A.nx, ny = A.ny, ncell = A.ncell;
    R2 *ycar = reinterpret_cast<R2 *>(smem_raw);                     // [W][GW][TX][32]
    RT *msm = reinterpret_cast<RT *>(ycar + (size_t)W * GW * TX * 32);  // [2][W][TX][36]
    const RT *Qp = static_cast<const RT *>(A.Q);
    const R2 *SGp = static_cast<const R2 *>(A.SG);
    const RT *inflow = static_cast<const RT *>(A.inflow);
    const RT *Ip = static_cast<const RT *>(A.I_prev);
    RT *Io = static_cast<RT *>(A.I_out);
    RT *part = static_cast<RT *>(A.part);
    R2 *face = static_cast<R2 *>(A.face);
    const RT inv_cdt = (RT)A.inv_cdt;
    const RT two = (RT)2;

    for (;;) {
        if (threadIdx.x == 0) s_task = (int)atomicAdd(A.ctrl + CTRL_QUEUE, 1u);
        __syncthreads();
        const int task = s_task;
        if (task >= A.n_tasks) return;
        const int sr = task / A.NCH, ch = task - sr * A.NCH;
        const int q = ch / A.CPQ, cq = ch - q * A.CPQ;
        const int sx = (q == 0 || q == 3) ? 1 : -1;
        const int sy = (q < 2) ? 1 : -1;
        const int strip = sx > 0 ? sr : A.NS - 1 - sr;
        const int x0 = strip * TX;
        const int ws = min(TX, nx - x0);
        const int wt = cq * W + w;
        const bool wvalid = wt < A.NWT;
        const int nvalid = min(W, A.NWT - cq * W);
        const int wtc = wvalid ? wt : 0;
        const int db = wtc / A.NGB, gb = wtc - db * A.NGB;
        const LaneConst &L = A.lanes[(q * A.DB + db) * 32 + lane];
        const RT mu = (RT)L.mu, eta = (RT)L.eta;
        RT wm[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) wm[k] = (RT)L.wm[k];
        const int side_x = sx > 0 ? 0 : 1, side_y = sy > 0 ? 2 : 3;
        int gidx[GW];
        RT bx[GW], by[GW];
#pragma unroll
        for (int gw = 0; gw < GW; ++gw) {
            gidx[gw] = gb * (GW * A.LG) + gw * A.LG + L.g_lo;
            bx[gw] = inflow[side_x * A.Gp + gidx[gw]];
            by[gw] = inflow[side_y * A.Gp + gidx[gw]];
        }
        const int au = sx > 0 ? 0 : 1, bu = sy > 0 ? 0 : 1;
        const int nuu = au + 2 * bu, ndu = (1 - au) + 2 * bu;
        const int nud = au + 2 * (1 - bu), ndd = (1 - au) + 2 * (1 - bu);
        const size_t wtbase = (size_t)(q * A.NWT + wtc) * ncell;
        const bool publish = sr < A.NS - 1;
        unsigned long long *myflag = A.flags + (size_t)ch * A.NS + strip;
        const unsigned long long *upflag = A.flags + (size_t)ch * A.NS + (sr > 0 ? strip - sx : strip);
        // face buffer [chain][strip][row][warp][slot][lane]
        R2 *face_out = face + ((size_t)ch * A.NS + strip) * ny * W * GW * 32;
        const R2 *face_in =
            face + ((size_t)ch * A.NS + (sr > 0 ? strip - sx : strip)) * ny * W * GW * 32;
        const unsigned long long ep = A.epoch << 32;

        for (int jj = 0; jj < ny; ++jj) {
            const int y = sy > 0 ? jj : ny - 1 - jj;
            const int buf = jj & 1;
            if (sr > 0) {
                if (threadIdx.x == 0)
                    s_abort = wait_flag(upflag, ep | (unsigned long long)(jj + 1), A.ctrl,
                                        A.timeout_ns);
                __syncthreads();
                if (s_abort) return;
            }
            if (wvalid) {
                RT Xu[GW], Xd[GW];
#pragma unroll
                for (int gw = 0; gw < GW; ++gw) {
                    if (sr == 0) {
                        Xu[gw] = bx[gw];
                        Xd[gw] = bx[gw];
                    } else {
                        const R2 f = __ldcg(face_in + (((size_t)y * W + w) * GW + gw) * 32 + lane);
                        Xu[gw] = f.x;
                        Xd[gw] = f.y;
                    }
                }
                for (int i = 0; i < ws; ++i) {
                    const int xo = sx > 0 ? i : ws - 1 - i;
                    const int cell = y * nx + x0 + xo;
                    RT s[4] = {0, 0, 0, 0}, ss[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int gw = 0; gw < GW; ++gw) {
                        const int g = gidx[gw];
                        RT S[4];
                        ld4_ro(Qp + ((size_t)g * ncell + cell) * 4, S);
                        const R2 sg = __ldg(SGp + (size_t)g * ncell + cell);
                        const size_t ioff = (((wtbase + cell) * GW + gw) * 32 + lane) * 4;
                        if (Ip) {
                            RT Ik[4];
                            ld4_stream(Ip + ioff, Ik);
#pragma unroll
                            for (int n = 0; n < 4; ++n) S[n] = fma(inv_cdt, Ik[n], S[n]);
                        }
                        R2 *yc = ycar + (((size_t)w * GW + gw) * TX + xo) * 32 + lane;
                        RT Yu, Yd;
                        if (jj == 0) {
                            Yu = by[gw];
                            Yd = by[gw];
                        } else {
                            const R2 t = *yc;
                            Yu = t.x;
                            Yd = t.y;
                        }
                        const RT iA = rcp(sg.x + mu + eta);
                        const RT m = mu * iA, e = eta * iA;
                        const RT ruu = (S[nuu] + two * (mu * Xu[gw] + eta * Yu)) * iA;
                        const RT rdu = fma(two * eta, Yd, S[ndu]) * iA;
                        const RT rud = fma(two * mu, Xd[gw], S[nud]) * iA;
                        const RT rdd = S[ndd] * iA;
                        const RT P = fma(m, m, fma(e, e, (RT)1));
                        const RT z = two * m * e;
                        const RT iD = rcp(fma(P, P, -z * z));
                        const RT wuu = fma(P, ruu, z * rdd);
                        const RT wdu = fma(P, rdu, -z * rud);
                        const RT wud = fma(P, rud, -z * rdu);
                        const RT wdd = fma(P, rdd, z * ruu);
                        RT I4[4];
                        I4[nuu] = (wuu - m * wdu - e * wud) * iD;
                        I4[ndu] = (wdu + m * wuu - e * wdd) * iD;
                        I4[nud] = (wud - m * wdd + e * wuu) * iD;
                        I4[ndd] = (wdd + m * wud + e * wdu) * iD;
                        st4_stream(Io + ioff, I4);
                        R2 yo;
                        yo.x = I4[nud];
                        yo.y = I4[ndd];
                        *yc = yo;
                        Xu[gw] = I4[ndu];
                        Xd[gw] = I4[ndd];
#pragma unroll
                        for (int n = 0; n < 4; ++n) {
                            s[n] += I4[n];
                            ss[n] = fma(sg.y, I4[n], ss[n]);
                        }
                    }
                    RT v[36];
#pragma unroll
                    for (int n = 0; n < 4; ++n) {
#pragma unroll
                        for (int k = 0; k < 6; ++k) v[n * 9 + k] = wm[k] * s[n];
#pragma unroll
                        for (int k = 0; k < 3; ++k) v[n * 9 + 6 + k] = wm[k] * ss[n];
                    }
                    TRed<16, 32, RT>::run(v, lane);
                    TRed<16, 4, RT>::run(v + 32, lane);
                    RT *ms = msm + (((size_t)buf * W + w) * TX + xo) * 36;
                    ms[lane] = v[0];
                    if ((lane & 7) == 0) ms[32 + (lane >> 3)] = v[32];
                }
                if (publish) {
#pragma unroll
                    for (int gw = 0; gw < GW; ++gw) {
                        R2 f;
                        f.x = Xu[gw];
                        f.y = Xd[gw];
                        __stcg(face_out + (((size_t)y * W + w) * GW + gw) * 32 + lane, f);
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0 && publish && !(A.fault_skip_publish && sr == 0)) {
                __threadfence();
                st_release(myflag, ep | (unsigned long long)(jj + 1));
            }
            RT *pdst = part + ((size_t)ch * ncell + (size_t)y * nx + x0) * 36;
            for (int e = threadIdx.x; e < ws * 36; e += blockDim.x) {
                const int xo = e / 36, k = e - xo * 36;
                RT acc = 0;
                for (int w2 = 0; w2 < nvalid; ++w2)
                    acc += msm[(((size_t)buf * W + w2) * TX + xo) * 36 + k];
                pdst[e] = acc;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 1D: one warp per warp task sweeps the whole line (the paper's 1D problems
// have at most a few thousand cells); per-warp partial moments.
template <typename RT, int GW>
__global__ void __launch_bounds__(256) sweep1d_kernel(const SweepArgs A) {
    using R2 = typename V2<RT>::t;
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (gwarp >= A.NQ * A.NWT) return;
    const int q = gwarp / A.NWT, wt = gwarp - q * A.NWT;
    const int sx = q == 0 ? 1 : -1;
    const int nx = A.nx, ncell = A.ncell;
    const int db = wt / A.NGB, gb = wt - db * A.NGB;
    const LaneConst &L = A.lanes[(q * A.DB + db) * 32 + lane];
    const RT mu = (RT)L.mu;
    const RT w0 = (RT)L.wm[0], w1 = (RT)L.wm[1], w2 = (RT)L.wm[2];
    const RT *Qp = static_cast<const RT *>(A.Q);
    const R2 *Qv = reinterpret_cast<const R2 *>(Qp);
    const R2 *SGp = static_cast<const R2 *>(A.SG);
    const RT *inflow = static_cast<const RT *>(A.inflow);
    const R2 *Ip = static_cast<const R2 *>(A.I_prev);
    R2 *Io = static_cast<R2 *>(A.I_out);
    RT *part = static_cast<RT *>(A.part);
    const RT inv_cdt = (RT)A.inv_cdt;
    const RT two = (RT)2;
    int gidx[GW];
    RT X[GW];
    const int side = sx > 0 ? 0 : 1;
#pragma unroll
    for (int gw = 0; gw < GW; ++gw) {
        gidx[gw] = gb * (GW * A.LG) + gw * A.LG + L.g_lo;
        X[gw] = inflow[side * A.Gp + gidx[gw]];
    }
    const int au = sx > 0 ? 0 : 1;
    const size_t wtbase = (size_t)(q * A.NWT + wt) * ncell;
    for (int i = 0; i < nx; ++i) {
        const int cell = sx > 0 ? i : nx - 1 - i;
        RT s[2] = {0, 0}, ss[2] = {0, 0};
#pragma unroll
        for (int gw = 0; gw < GW; ++gw) {
            const int g = gidx[gw];
            const R2 qv = __ldg(Qv + (size_t)g * ncell + cell);
            const R2 sg = __ldg(SGp + (size_t)g * ncell + cell);
            RT S[2] = {qv.x, qv.y};
            const size_t ioff = ((wtbase + cell) * GW + gw) * 32 + lane;
            if (Ip) {
                const R2 ik = __ldcs(Ip + ioff);
                S[0] = fma(inv_cdt, ik.x, S[0]);
                S[1] = fma(inv_cdt, ik.y, S[1]);
            }
            const RT iA = rcp(sg.x + mu);
            const RT m = mu * iA;
            const RT r1 = fma(two * mu, X[gw], S[au]) * iA;
            const RT r2 = S[1 - au] * iA;
            const RT iD = rcp(fma(m, m, (RT)1));
            RT I2[2];
            I2[au] = (r1 - m * r2) * iD;
            I2[1 - au] = (r2 + m * r1) * iD;
            R2 o;
            o.x = I2[0];
            o.y = I2[1];
            __stcs(Io + ioff, o);
            X[gw] = I2[1 - au];
#pragma unroll
            for (int n = 0; n < 2; ++n) {
                s[n] += I2[n];
                ss[n] = fma(sg.y, I2[n], ss[n]);
            }
        }
        RT v[10];
#pragma unroll
        for (int n = 0; n < 2; ++n) {
            v[n * 5 + 0] = w0 * s[n];
            v[n * 5 + 1] = w1 * s[n];
            v[n * 5 + 2] = w2 * s[n];
            v[n * 5 + 3] = w0 * ss[n];
            v[n * 5 + 4] = w1 * ss[n];
        }
        TRed<16, 8, RT>::run(v, lane);
        TRed<16, 2, RT>::run(v + 8, lane);
        RT *pd = part + ((size_t)gwarp * ncell + cell) * 10;
        if ((lane & 3) == 0) pd[lane >> 2] = v[0];
        if ((lane & 15) == 0) pd[8 + (lane >> 4)] = v[8];
    }
}

// ---------------------------------------------------------------------------
template <typename RT, int GW>
static cudaError_t launch2d_t(const SweepArgs &a, int grid, size_t smem, cudaStream_t s) {
    sweep2d_kernel<RT, GW><<<grid, a.W * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename RT>
static const void *kernel2d_ptr(int GW) {
    switch (GW) {
        case 1: return (const void *)sweep2d_kernel<RT, 1>;
        case 2: return (const void *)sweep2d_kernel<RT, 2>;
        default: return (const void *)sweep2d_kernel<RT, 4>;
    }
}

cudaError_t launch_sweep2d(const sm_problem *p, const SweepArgs &a, int grid, cudaStream_t s) {
    const size_t smem = sweep2d_smem_bytes(p->prec, a.W, a.GW, a.TX);
    if (p->prec == 32) {
        switch (a.GW) {
            case 1: return launch2d_t<float, 1>(a, grid, smem, s);
            case 2: return launch2d_t<float, 2>(a, grid, smem, s);
            default: return launch2d_t<float, 4>(a, grid, smem, s);
        }
    }
    switch (a.GW) {
        case 1: return launch2d_t<double, 1>(a, grid, smem, s);
        case 2: return launch2d_t<double, 2>(a, grid, smem, s);
        default: return launch2d_t<double, 4>(a, grid, smem, s);
    }
}

// Configures the shared-memory limit of the 2D kernel for (W, current GW,
// TX) and returns how many CTAs fit on the whole GPU (0 if none).
int sweep2d_max_resident(const sm_problem *p, int W, size_t *smem_out) {
    const size_t smem = sweep2d_smem_bytes(p->prec, W, p->GW, p->TX);
    if (smem_out) *smem_out = smem;
    const void *k = (p->prec == 32) ? kernel2d_ptr<float>(p->GW) : kernel2d_ptr<double>(p->GW);
    int dev = 0, nsm = 0, maxopt = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem + 64 > (size_t)maxopt) return 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, W * 32, smem) != cudaSuccess)
        return 0;
    return per_sm * nsm;
}

cudaError_t launch_sweep1d(const sm_problem *p, const SweepArgs &a, cudaStream_t s) {
    const int warps = a.NQ * a.NWT;
    const int threads = 128;
    const int blocks = (warps * 32 + threads - 1) / threads;
    if (p->prec == 32) {
        switch (a.GW) {
            case 1: sweep1d_kernel<float, 1><<<blocks, threads, 0, s>>>(a); break;
            case 2: sweep1d_kernel<float, 2><<<blocks, threads, 0, s>>>(a); break;
            default: sweep1d_kernel<float, 4><<<blocks, threads, 0, s>>>(a); break;
        }
    } else {
        switch (a.GW) {
            case 1: sweep1d_kernel<double, 1><<<blocks, threads, 0, s>>>(a); break;
            case 2: sweep1d_kernel<double, 2><<<blocks, threads, 0, s>>>(a); break;
            default: sweep1d_kernel<double, 4><<<blocks, threads, 0, s>>>(a); break;
        }
    }
    return cudaGetLastError();
}

}  // namespace smk
