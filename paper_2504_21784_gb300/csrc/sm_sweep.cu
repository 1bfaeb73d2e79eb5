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
// 2D parallel layout (diagonal wavefront).  A warp task owns 32 lanes x GW
// slots of (direction, group) pairs of one quadrant (lane = direction inside
// the quadrant, or direction x group when a quadrant has fewer than 32
// directions).  A CTA takes one warp task over a strip of W cell columns,
// one warp per column; each warp walks its column in upwind row order with
// the y-inflow carried in registers.  The x-inflow of a row comes from the
// warp of the upwind column through a shared-memory ring of RING rows, each
// slot guarded by a "full" and an "empty" mbarrier (the waiting warp is
// suspended by the hardware instead of polling), and across strips from the upwind CTA
// through an L2-resident face buffer and a per-(warp task, strip) row counter
// (release / acquire).  So the W warps of a CTA run one row apart, a staircase
// wavefront with no CTA-wide barrier inside a task.  Each warp prefetches
// the I^k and source records of its next S rows with TMA bulk copies
// (cp.async.bulk, mbarrier completion) into shared memory.  Tasks come from an
// atomic queue in upwind-strip order, so every awaited producer is already
// running (no deadlock for any grid size), and every wait is bounded in time
// (status word + abort flag, never a trap).  Per cell, each lane sums its GW
// intensities (plain and sigma-weighted, per node), the warp transposes the
// sums through shared memory, each lane forms one of the 36 weighted moments
// as a dot product over the 32 lanes (the last four split over octets of
// lanes and finished by shuffles), and the warp task stores them in its own
// slot of the per-(warp task, cell) partial moments; the reduction sums the
// warp tasks in a fixed order, so the moments are reproducible bit for bit.
#include <stdint.h>
#include <string.h>

#include "sm_internal.cuh"

namespace smk {

template <typename RT> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

__device__ __forceinline__ void st4_stream(float *p, const float (&v)[4]) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void st4_stream(double *p, const double (&v)[4]) {
    __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
    __stcs(reinterpret_cast<double2 *>(p + 2), make_double2(v[2], v[3]));
}
__device__ __forceinline__ void lds4(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void lds4(const double *p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    const double2 b = *reinterpret_cast<const double2 *>(p + 2);
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
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// orders this thread's generic-proxy view of global memory before its later
// async-proxy (TMA) reads of it
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- mbarrier / TMA bulk-copy helpers (inline PTX) ----------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// arrive (release, CTA scope) of the executing thread
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// global -> shared bulk copy; bytes and both addresses multiples of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Records a timeout in the status word, raises the global and CTA abort flags.
__device__ __forceinline__ void raise_timeout(unsigned int *ctrl, volatile int *s_abort) {
    atomicOr(ctrl + CTRL_STATUS, (unsigned)ST_TIMEOUT);
    atomicExch(ctrl + CTRL_ABORT, 1u);
    *s_abort = 1;
}

// Bounded wait (every lane) for a TMA stage.  false: timed out or aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned int *ctrl,
                                          long long timeout_ns, volatile int *s_abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31) == 0) {
            if (*s_abort) return false;
            if (global_ns() - t0 > timeout_ns) {
                raise_timeout(ctrl, s_abort);
                return false;
            }
        }
    }
}

// Bounded wait (every lane) for a producer row counter in global memory.
__device__ __forceinline__ bool flag_wait_geq(const unsigned long long *f,
                                              unsigned long long target, unsigned long long &seen,
                                              unsigned int *ctrl, long long timeout_ns,
                                              volatile int *s_abort) {
    if (seen >= target) return true;
    seen = ld_acquire(f);
    if (seen >= target) return true;
    const long long t0 = global_ns();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        seen = ld_acquire(f);
        if (seen >= target) return true;
        if (*s_abort || ld_relaxed(ctrl + CTRL_ABORT)) {
            *s_abort = 1;
            return false;
        }
        if (global_ns() - t0 > timeout_ns) {
            raise_timeout(ctrl, s_abort);
            return false;
        }
    }
}

// Transpose-butterfly warp reduction of CNT values per lane: afterwards v[0]
// of lane L holds the warp sum of value index L >> (5 - log2 CNT).  Steps stop
// at offset STOP (exclusive of smaller offsets) when STOP > 0.
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

constexpr int RING = 2;   // rows of x-face buffering between neighbouring warps
constexpr int SREC = 8;   // source record: q at 4 nodes, sigma~, sigma, 2 pad
constexpr int MROW = 36;  // padded row length of the moment transpose buffers

// Reciprocal: the FP32 path uses the hardware approximation (relative error
// below 2^-22, far inside the FP32 sweep's tolerance); FP64 stays IEEE.
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_fast(double x) { return __drcp_rn(x); }

// Correctly rounded product and sum that the compiler never contracts into an
// FMA: every rounding of the cell solve is fixed by the source, so the same
// problem gives bit-identical intensities from every kernel it is compiled
// into (single-problem and batched launches).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

__host__ __device__ inline size_t stage_bytes(int rsize, int GW, int GSLOT) {
    return (size_t)GW * 32 * 4 * rsize + (size_t)GSLOT * SREC * rsize;
}
// ---------------------------------------------------------------------------
// Shared-memory layout of one 2D sweep CTA: W warps, each owning S stages of
// stg bytes (prefetched I^k and source records), an x-face ring for ring_gw
// slots and the per-lane moment weights; after them W*S stage mbarriers and
// the ring mbarriers (W*RING "full", W*RING "empty").  A row's stage, once
// its cell solves have read it,
// doubles as that row's moment transpose buffer ([8][MROW]) before the
// prefetch of a later row overwrites it, so a stage is at least that large.
struct Layout2D {
    size_t stg, wsz, ring_off, wt_off;
};

__host__ __device__ inline Layout2D layout2d(int rsize, int S, size_t stg, int ring_gw) {
    Layout2D L;
    const size_t mb = ((size_t)8 * MROW * rsize + 15) & ~(size_t)15;
    L.stg = stg > mb ? stg : mb;
    L.ring_off = (size_t)S * L.stg;
    L.wt_off = L.ring_off + (size_t)RING * ring_gw * 32 * 2 * rsize;
    L.wsz = L.wt_off + (size_t)6 * MROW * rsize;
    return L;
}

__host__ __device__ inline size_t layout2d_total(const Layout2D &L, int W, int S) {
    return (size_t)W * L.wsz + (size_t)W * S * 8 + (size_t)2 * W * RING * 8 + 64;
}

size_t sweep2d_smem_bytes(int prec, int W, int GW, int S, int GSLOT) {
    const int rs = prec == 32 ? 4 : 8;
    return layout2d_total(layout2d(rs, S, stage_bytes(rs, GW, GSLOT), GW), W, S);
}

size_t sweep2d_batch_smem_bytes(int prec, int W, int S, size_t stg, int ring_gw) {
    return layout2d_total(layout2d(prec == 32 ? 4 : 8, S, stg, ring_gw), W, S);
}

size_t sweep2d_stage_bytes(int prec, int GW, int GSLOT) {
    return stage_bytes(prec == 32 ? 4 : 8, GW, GSLOT);
}

// ---------------------------------------------------------------------------
// Fused emission (EmitArgs): the Planck tables reached through the kernel
// parameter.
struct ParamTabs {
    const PlanckTabs *t;
    __device__ __forceinline__ double head(int k) const { return t->head[k]; }
    __device__ __forceinline__ double bern(int k) const { return t->bern[k]; }
    __device__ __forceinline__ double cexp(int i) const { return t->cexp[i]; }
    __device__ __forceinline__ double exp2(int j) const { return __ldg(t->exp2 + j); }
    __device__ __forceinline__ double pcen(int j) const { return __ldg(t->pcen + j); }
    __device__ __forceinline__ const double *ptab(int j) const { return t->ptab + (size_t)j * 2 * NTAY; }
};

// Strip of the r-th place in the order the strips are first needed: the
// quadrants with Omega_x > 0 start at strip 0, the others at strip NS - 1.
__device__ __forceinline__ int emit_strip_of_rank(int r, int NS) {
    return (r & 1) ? NS - 1 - (r >> 1) : (r >> 1);
}

// One emission item (8 cells of strip s, one node per lane) by the calling
// warp, then its completion released to strip s's counter.  Kept out of line
// so that the sweep's register allocation does not grow with it.
template <typename RT>
__device__ __noinline__ void emit_item(const EmitArgs &E, RT *src, unsigned int *ctrl, int item,
                                       const float *s_edges) {
    const int lane = threadIdx.x & 31;
    const int s = emit_strip_of_rank(item / E.per_strip, E.NS);
    const int k = item % E.per_strip;
    const int x0 = s * E.W, ws = min(E.W, E.nx - x0);
    const int ncells = ws * E.ny;
    if (8 * k < ncells) {  // (warp-uniform) the ragged strip's surplus items are empty
        int ci = 8 * k + (lane >> 2);
        const bool active = ci < ncells;
        if (!active) ci = ncells - 1;  // a copy of a real node, nothing stored
        const int cell = (ci / ws) * E.nx + x0 + (ci % ws);
        emit_node<RT>(cell, lane & 3, active, E.ncell, 4, E.G, E.Gp, E.edges, s_edges,
                      E.acT4_scale, E.inv_cdt, E.T, E.sigma, src, E.gray, nullptr,
                      ctrl + CTRL_STATUS, ST_NONPHYSICAL, ParamTabs{&E.tabs});
    }
    __threadfence();  // every lane's records, before the release below
    __syncwarp();
    if (lane == 0) red_release_add_u32(E.ctr + 1 + s, 1u);
}

// Claims the next emission item for the calling warp (-1: none left).
__device__ __forceinline__ int emit_claim(const EmitArgs &E) {
    int it = 0;
    if ((threadIdx.x & 31) == 0) it = (int)atomicAdd(E.ctr, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    return it < E.items ? it : -1;
}

// Before a task of strip s issues its first copy of the source records: wait
// until the strip's emission is complete, processing emission items while
// any is left (every item is claimed by a running warp and never waits, so
// the wait ends); then order the strip's records before this warp's TMA
// reads.  false: the wait ran out of time or the sweep was aborted.
template <typename RT>
__device__ bool emit_wait_strip(const EmitArgs &E, RT *src, unsigned int *ctrl, int s,
                                const float *s_edges, volatile int *s_abort) {
    const int lane = threadIdx.x & 31;
    const unsigned need = (unsigned)E.per_strip;
    long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        unsigned done = 0;
        if (lane == 0) done = ld_acquire_u32(E.ctr + 1 + s);
        done = __shfl_sync(0xffffffffu, done, 0);
        if (done >= need) break;
        const int item = emit_claim(E);
        if (item >= 0) {
            emit_item<RT>(E, src, ctrl, item, s_edges);
            continue;
        }
        // every item is taken: the strip's last ones are being finished
        if (t0 == 0) t0 = global_ns();
        __nanosleep(128);
        if ((it & 15) == 0) {
            const bool stop = *s_abort || ld_relaxed(ctrl + CTRL_ABORT) ||
                              global_ns() - t0 > E.timeout_ns;
            if (__any_sync(0xffffffffu, stop)) {
                if (global_ns() - t0 > E.timeout_ns) raise_timeout(ctrl, s_abort);
                *s_abort = 1;
                return false;
            }
        }
    }
    if (lane == 0) fence_proxy_async_global();
    __syncwarp();
    return true;
}

// One task of the 2D sweep: strip sr of warp task wg (quadrant Q, direction
// block, group block) of the problem A, every warp of the CTA sweeping one
// cell column of the strip from the upwind to the downwind edge.  The
// quadrant is a template parameter so that the upwind/downwind roles of the
// four nodes are compile-time register indices.
template <typename RT, int GW, int Q, bool MOM, class Args>
__device__ __forceinline__ void sweep2d_task_q(const Args &A, const Layout2D &Lay, const int task,
                                             unsigned char *smem_raw, uint64_t *bars,
                                             uint64_t *ring_bars, uint32_t &ring_p,
                                             uint32_t &ring_c, volatile int *s_abort,
                                             uint32_t &phase, const unsigned long long epoch,
                                             const EmitArgs *E, const float *s_edges) {
    using R2 = typename V2<RT>::t;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int W = A.W, S = A.S;
    const int nx = A.nx, ny = A.ny;
    const int GSLOT = GW * A.LG;
    const size_t stg = Lay.stg, wsz = Lay.wsz, ring_off = Lay.ring_off;
    unsigned char *wbase = smem_raw + (size_t)w * wsz;
    uint64_t *mybars = bars + (size_t)w * S;
    RT *Wt = reinterpret_cast<RT *>(wbase + Lay.wt_off);  // [6][MROW]: weights per lane
    const RT *src = static_cast<const RT *>(A.src);
    const RT *inflow = static_cast<const RT *>(A.inflow);
    const RT *Ip = static_cast<const RT *>(A.I_prev);
    RT *Io = static_cast<RT *>(A.I_out);
    RT *acc = static_cast<RT *>(A.mom_acc);
    R2 *face = static_cast<R2 *>(A.face);
    const RT inv_cdt = (RT)A.inv_cdt;
    const RT two = (RT)2;
    const uint32_t bytes_I = Ip ? (uint32_t)(GW * 32 * 4 * sizeof(RT)) : 0u;
    const uint32_t bytes_S = (uint32_t)(GSLOT * SREC * sizeof(RT));
    // moment this lane assembles whole, m = n*9 + k, and the eighth of moment
    // 32 + lane/8 (source lanes 4 (lane % 8) .. +3) it adds to its octet's sum
    const int m1 = lane, n1 = m1 / 9, k1 = m1 % 9;
    const int vrow1 = k1 < 6 ? n1 : 4 + n1, wrow1 = k1 < 6 ? k1 : k1 - 6;
    const int m2 = 32 + (lane >> 3), k2 = m2 % 9;
    const int vrow2 = k2 < 6 ? 3 : 7, wrow2 = k2 < 6 ? k2 : k2 - 6;
    const int c2 = 4 * (lane & 7);
    const int NWG = A.NQ * A.NWT;
    const int sr = task / NWG, wg = task - sr * NWG;
    constexpr int q = Q;
    const int wt = wg - q * A.NWT;
    constexpr int sx = (Q == 0 || Q == 3) ? 1 : -1;
    constexpr int sy = (Q < 2) ? 1 : -1;
    const int strip = sx > 0 ? sr : A.NS - 1 - sr;
    const int x0 = A.strip_x0 ? __ldg(A.strip_x0 + strip) : strip * W;
    const int ws = A.strip_x0 ? __ldg(A.strip_x0 + strip + 1) - x0 : min(W, nx - x0);
    if (w >= ws) return;  // idle column of a ragged strip
    const int xw = sx > 0 ? x0 + w : x0 + ws - 1 - w;
    const int db = wt / A.NGB, gb = wt - db * A.NGB;
    const LaneConst &L = A.lanes[(q * A.DB + db) * 32 + lane];
    const RT mu = (RT)L.mu, eta = (RT)L.eta;
    const RT two_mu = mul_rn((RT)2, mu), two_eta = mul_rn((RT)2, eta);
#pragma unroll
    for (int k = 0; k < 6; ++k) Wt[k * MROW + lane] = (RT)L.wm[k];
    const int g_lo = L.g_lo;
    const int side_x = sx > 0 ? 0 : 1, side_y = sy > 0 ? 2 : 3;
    RT X0[GW], X1[GW], Y0[GW], Y1[GW];  // x-inflow (rows u,d), y-inflow (columns u,d)
    // boundary x-inflow of this lane's slots (first column of strip 0), slot
    // gw at bxin[gw * A.LG]; re-read per row rather than held in registers
    const RT *bxin = inflow + side_x * A.Gp + gb * GSLOT + g_lo;
#pragma unroll
    for (int gw = 0; gw < GW; ++gw) {
        const int g = gb * GSLOT + gw * A.LG + g_lo;
        const RT by = inflow[side_y * A.Gp + g];
        Y0[gw] = by;
        Y1[gw] = by;
    }
    constexpr int au = sx > 0 ? 0 : 1, bu = sy > 0 ? 0 : 1;
    constexpr int nuu = au + 2 * bu, ndu = (1 - au) + 2 * bu;
    constexpr int nud = au + 2 * (1 - bu), ndd = (1 - au) + 2 * (1 - bu);
    // memory quadrant of the intensities: the geometric one, or its reverse
    // for adjoint sweeps (the transposed operator of Omega is that of -Omega)
    const size_t wtbase = ((size_t)(A.reverse ? (q ^ 2) : q) * A.NWT + wt) * A.ncell;
    const bool global_in = (w == 0) && sr > 0;
    const bool global_out = (w == ws - 1) && sr < A.NS - 1;
    const size_t fidx_out = ((size_t)wg * A.NS + strip) * ny;
    const size_t fidx_in = ((size_t)wg * A.NS + (sr > 0 ? strip - sx : strip)) * ny;
    unsigned long long *myflag = A.flags + (size_t)wg * A.NS + strip;
    const unsigned long long *upflag =
        A.flags + (size_t)wg * A.NS + (sr > 0 ? strip - sx : strip);
    const unsigned long long ep = epoch << 32;
    unsigned long long seen = 0;
    const R2 *ring_in =
        w > 0 ? reinterpret_cast<const R2 *>(smem_raw + (size_t)(w - 1) * wsz + ring_off)
              : nullptr;
    R2 *ring_out = reinterpret_cast<R2 *>(wbase + ring_off);
    __syncwarp();  // weights visible to the whole warp

    auto row_y = [&](int jj) { return sy > 0 ? jj : ny - 1 - jj; };
    auto issue = [&](int jj) {  // lane 0: TMA for row jj into stage jj % S
        const int st = jj % S;
        unsigned char *dst = wbase + (size_t)st * stg;
        const int cell = row_y(jj) * nx + xw;
        mbar_arrive_expect_tx(mybars + st, bytes_I + bytes_S);
        if (Ip) bulk_g2s(dst, Ip + ((wtbase + cell) * GW) * 32 * 4, bytes_I, mybars + st);
        bulk_g2s(dst + bytes_I, src + ((size_t)cell * A.Gp + (size_t)gb * GSLOT) * SREC,
                 bytes_S, mybars + st);
    };
    int issued = -1;    // highest row whose copy was issued
    int consumed = 0;   // rows whose stage has been waited for
    // fused emission: this strip's source records must be complete first
    if (E && !emit_wait_strip<RT>(*E, const_cast<RT *>(src), A.ctrl, strip, s_edges, s_abort))
        return;
    if (lane == 0) {
        fence_proxy_async_smem();
        for (int jj = 0; jj < min(S, ny); ++jj) issue(jj);
    }
    issued = min(S, ny) - 1;
    bool ok = true;
    int jj = 0;
    for (; jj < ny && ok; ++jj) {
        const int y = row_y(jj);
        const int st = jj % S;
        // (a) x-inflow
        if (w == 0 && sr == 0) {
#pragma unroll
            for (int gw = 0; gw < GW; ++gw) {
                const RT b = __ldg(bxin + gw * A.LG);
                X0[gw] = b;
                X1[gw] = b;
            }
        } else if (global_in) {
            ok = flag_wait_geq(upflag, ep | (unsigned long long)(jj + 1), seen, A.ctrl,
                               A.timeout_ns, s_abort);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
#pragma unroll
            for (int gw = 0; gw < GW; ++gw) {
                const R2 f = __ldcg(face + ((fidx_in + y) * GW + gw) * 32 + lane);
                X0[gw] = f.x;
                X1[gw] = f.y;
            }
        } else {
            // the upwind column's ring: wait until its row is in ("full"),
            // read it, hand the slot back ("empty"); every lane waits and
            // arrives (acquire / release of its own accesses)
            const uint32_t c = ring_c;
            const int slot = (int)(c % RING);
            ok = mbar_wait(ring_bars + (w - 1) * RING + slot, (c / RING) & 1u, A.ctrl,
                           A.timeout_ns, s_abort);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
#pragma unroll
            for (int gw = 0; gw < GW; ++gw) {
                const R2 f = ring_in[(slot * GW + gw) * 32 + lane];
                X0[gw] = f.x;
                X1[gw] = f.y;
            }
            mbar_arrive(ring_bars + (W + w - 1) * RING + slot);
            ring_c = c + 1;
        }
        // (b) this row's prefetched I^k and sources
        ok = mbar_wait(mybars + st, (phase >> st) & 1u, A.ctrl, A.timeout_ns, s_abort);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        phase ^= 1u << st;
        consumed = jj + 1;
        const RT *sbI = reinterpret_cast<const RT *>(wbase + (size_t)st * stg) + lane * 4;
        const RT *sbS = reinterpret_cast<const RT *>(wbase + (size_t)st * stg + bytes_I) +
                        (size_t)g_lo * SREC;
        // (c) cell solves, reading the stage slot by slot
        RT s4[4] = {0, 0, 0, 0}, ss4[4] = {0, 0, 0, 0};
        const int cell = y * nx + xw;
        RT *io = Io + (((wtbase + cell) * GW) * 32 + lane) * 4;
#pragma unroll
        for (int gw = 0; gw < GW; ++gw) {
            RT Sn[4], Ik[4];
            lds4(sbS + (size_t)gw * A.LG * SREC, Sn);
            const RT sgt = sbS[(size_t)gw * A.LG * SREC + 4];
            const RT sgm = sbS[(size_t)gw * A.LG * SREC + 5];
            if (Ip) {
                lds4(sbI + (size_t)gw * 128, Ik);
#pragma unroll
                for (int n = 0; n < 4; ++n) Sn[n] = fma(inv_cdt, Ik[n], Sn[n]);
            }
            const RT iA = rcp_fast(add_rn(add_rn(sgt, mu), eta));
            const RT m = mul_rn(mu, iA), e = mul_rn(eta, iA);
            const RT ruu = mul_rn(fma(two, fma(mu, X0[gw], mul_rn(eta, Y0[gw])), Sn[nuu]), iA);
            const RT rdu = mul_rn(fma(two_eta, Y1[gw], Sn[ndu]), iA);
            const RT rud = mul_rn(fma(two_mu, X1[gw], Sn[nud]), iA);
            const RT rdd = mul_rn(Sn[ndd], iA);
            const RT P = fma(m, m, fma(e, e, (RT)1));
            const RT z = mul_rn(mul_rn(two, m), e);
            const RT iD = rcp_fast(fma(P, P, -mul_rn(z, z)));
            const RT wuu = fma(P, ruu, mul_rn(z, rdd));
            const RT wdu = fma(P, rdu, -mul_rn(z, rud));
            const RT wud = fma(P, rud, -mul_rn(z, rdu));
            const RT wdd = fma(P, rdd, mul_rn(z, ruu));
            RT I4[4];
            I4[nuu] = mul_rn(fma(-e, wud, fma(-m, wdu, wuu)), iD);
            I4[ndu] = mul_rn(fma(-e, wdd, fma(m, wuu, wdu)), iD);
            I4[nud] = mul_rn(fma(e, wuu, fma(-m, wdd, wud)), iD);
            I4[ndd] = mul_rn(fma(e, wdu, fma(m, wud, wdd)), iD);
            st4_stream(io + (size_t)gw * 128, I4);
            X0[gw] = I4[ndu];  // x-outflow -> next column
            X1[gw] = I4[ndd];
            Y0[gw] = I4[nud];  // y-outflow -> next row
            Y1[gw] = I4[ndd];
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                s4[n] = add_rn(s4[n], I4[n]);
                ss4[n] = fma(sgm, I4[n], ss4[n]);
            }
        }
        // (d) hand the x-outflow downwind
        if (w < ws - 1) {
            // this column's ring: once the slot's previous row has been read
            // ("empty"), write the row and mark it "full"
            const uint32_t r = ring_p;
            const int slot = (int)(r % RING);
            if (r >= RING) {
                ok = mbar_wait(ring_bars + (W + w) * RING + slot, ((r / RING) + 1) & 1u, A.ctrl,
                               A.timeout_ns, s_abort);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
            }
#pragma unroll
            for (int gw = 0; gw < GW; ++gw) {
                R2 f;
                f.x = X0[gw];
                f.y = X1[gw];
                ring_out[(slot * GW + gw) * 32 + lane] = f;
            }
            mbar_arrive(ring_bars + w * RING + slot);
            ring_p = r + 1;
        } else if (global_out) {
#pragma unroll
            for (int gw = 0; gw < GW; ++gw) {
                R2 f;
                f.x = X0[gw];
                f.y = X1[gw];
                __stcg(face + ((fidx_out + y) * GW + gw) * 32 + lane, f);
            }
            __syncwarp();
            // release the rows to the downwind strip in batches of A.publish:
            // the gpu-scope fence is paid once per batch
            if (lane == 0 && !(A.fault_skip_publish && sr == 0) &&
                ((jj + 1) % max(A.publish, 1) == 0 || jj + 1 == ny)) {
                __threadfence();
                st_release(myflag, ep | (unsigned long long)(jj + 1));
            }
        }
        // (e) moments of this cell (MOM; the defect correction's sweeps take
        // the moments of the iterate instead): transpose through shared
        // memory (this row's stage, read by every lane by now), then lane m
        // forms moment m = n*9 + k as a dot product over the 32 lanes
        if constexpr (MOM) {
            RT *Mb = reinterpret_cast<RT *>(wbase + (size_t)st * stg);  // [8][MROW]
            __syncwarp();
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                Mb[n * MROW + lane] = s4[n];
                Mb[(4 + n) * MROW + lane] = ss4[n];
            }
            __syncwarp();
            // four partial sums per dot product: dependent chains of 8, not 32
            RT d1p[4] = {0, 0, 0, 0};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                RT a[4], b[4];
                lds4(Mb + vrow1 * MROW + 4 * i, a);
                lds4(Wt + wrow1 * MROW + 4 * i, b);
#pragma unroll
                for (int t = 0; t < 4; ++t) d1p[t] = fma(a[t], b[t], d1p[t]);
            }
            const RT d1 = (d1p[0] + d1p[1]) + (d1p[2] + d1p[3]);
            RT d2;
            {
                RT c[4], e4[4];
                lds4(Mb + vrow2 * MROW + c2, c);
                lds4(Wt + wrow2 * MROW + c2, e4);
                d2 = fma(c[3], e4[3], fma(c[2], e4[2], fma(c[1], e4[1], c[0] * e4[0])));
                d2 += __shfl_xor_sync(0xffffffffu, d2, 1);
                d2 += __shfl_xor_sync(0xffffffffu, d2, 2);
                d2 += __shfl_xor_sync(0xffffffffu, d2, 4);
            }
            // this warp task's share of the cell's moments: a slot of its own
            // (no atomics), summed over the warp tasks in a fixed order by the
            // reduction, so that the moments do not depend on the schedule
            RT *ac = acc + ((size_t)wg * A.ncell + cell) * 36;
            ac[m1] = d1;
            if ((lane & 7) == 0) ac[m2] = d2;
        }
        // the stage is free: prefetch row jj + S into it (the proxy fence
        // orders this warp's reads and writes of it before the copy)
        __syncwarp();
        if (lane == 0 && jj + S < ny) {
            fence_proxy_async_smem();
            issue(jj + S);
        }
        if (jj + S < ny) issued = jj + S;
    }
    if (!ok) {
        // wait (bounded) for this warp's copies still in flight, then leave
        const long long t0 = global_ns();
        for (int r = consumed; r <= issued; ++r) {
            const int st = r % S;
            while (!mbar_try_wait(mybars + st, (phase >> st) & 1u)) {
                if (global_ns() - t0 > A.timeout_ns) break;
            }
            phase ^= 1u << st;
        }
        *s_abort = 1;
    }
}

template <typename RT, int GW, bool MOM = true, class Args>
__device__ __forceinline__ void sweep2d_task(const Args &A, const Layout2D &Lay, const int task,
                                             unsigned char *smem_raw, uint64_t *bars,
                                             uint64_t *ring_bars, uint32_t &ring_p,
                                             uint32_t &ring_c, volatile int *s_abort,
                                             uint32_t &phase, const unsigned long long epoch,
                                             const EmitArgs *E = nullptr,
                                             const float *s_edges = nullptr) {
    const int NWG = A.NQ * A.NWT;
    const int q = (task % NWG) / A.NWT;
    switch (q) {
        case 0:
            sweep2d_task_q<RT, GW, 0, MOM>(A, Lay, task, smem_raw, bars, ring_bars, ring_p, ring_c,
                                      s_abort, phase, epoch, E, s_edges);
            break;
        case 1:
            sweep2d_task_q<RT, GW, 1, MOM>(A, Lay, task, smem_raw, bars, ring_bars, ring_p, ring_c,
                                      s_abort, phase, epoch, E, s_edges);
            break;
        case 2:
            sweep2d_task_q<RT, GW, 2, MOM>(A, Lay, task, smem_raw, bars, ring_bars, ring_p, ring_c,
                                      s_abort, phase, epoch, E, s_edges);
            break;
        default:
            sweep2d_task_q<RT, GW, 3, MOM>(A, Lay, task, smem_raw, bars, ring_bars, ring_p, ring_c,
                                      s_abort, phase, epoch, E, s_edges);
            break;
    }
}

// barrier of the W sweep warps only (the fused emission warps never join it)
__device__ __forceinline__ void sweep_warps_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// W sweep warps (one per cell column of the strip), plus E.warps fused
// emission warps when E.warps > 0 (EmitArgs).
template <typename RT, int GW, bool MOM = true>
__global__ void __launch_bounds__(512) sweep2d_kernel(const __grid_constant__ SweepArgs A,
                                                      const __grid_constant__ EmitArgs E) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_task;
    __shared__ volatile int s_abort;
    const int W = A.W, S = A.S;
    const Layout2D Lay = layout2d((int)sizeof(RT), S, stage_bytes((int)sizeof(RT), GW, GW * A.LG), GW);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)W * Lay.wsz);
    uint64_t *ring_bars = bars + (size_t)W * S;
    float *s_edges = reinterpret_cast<float *>(
        smem_raw + ((layout2d_total(Lay, W, S) + 15) & ~(size_t)15));
    if (threadIdx.x < W * S) mbar_init(bars + threadIdx.x, 1);
    if (threadIdx.x < 2 * W * RING) mbar_init(ring_bars + threadIdx.x, 32);
    if (threadIdx.x == 0) s_abort = 0;
    if (E.warps)
        for (int i = threadIdx.x; i <= E.G; i += blockDim.x) s_edges[i] = (float)E.edges[i];
    fence_mbar_init();
    __syncthreads();
    if ((int)(threadIdx.x >> 5) >= W) {
        // fused emission warps: emission items until none is left (they never
        // wait on anything, so every strip's emission completes)
        RT *src = static_cast<RT *>(const_cast<void *>(A.src));
        while (!s_abort && !ld_relaxed(A.ctrl + CTRL_ABORT)) {
            const int item = emit_claim(E);
            if (item < 0) break;
            emit_item<RT>(E, src, A.ctrl, item, s_edges);
        }
        return;
    }
    const EmitArgs *Ep = E.warps ? &E : nullptr;
    uint32_t phase = 0;   // parity bit per stage of this warp
    uint32_t ring_p = 0;  // rows this warp has put in its ring, all tasks
    uint32_t ring_c = 0;  // rows this warp has taken from the upwind ring
    for (;;) {
        sweep_warps_sync(W * 32);
        if (threadIdx.x == 0) s_task = (int)atomicAdd(A.ctrl + CTRL_QUEUE, 1u);
        sweep_warps_sync(W * 32);
        const int task = s_task;
        if (task >= A.n_tasks || s_abort) return;
        sweep2d_task<RT, GW, MOM>(A, Lay, task, smem_raw, bars, ring_bars, ring_p, ring_c,
                                  &s_abort, phase, A.epoch, Ep, s_edges);
    }
}

// Many problems in one persistent launch: the tasks of all problems are taken
// from one queue, in an order that keeps each problem's own upwind task order
// (a task waits only on earlier tasks of its problem, which are claimed by
// running CTAs, so the launch cannot deadlock for any grid size).  Each task's
// problem arguments are copied to shared memory and the task body is chosen
// by the problem's slots per lane (GW); the shared-memory layout is sized for
// the largest stage and ring of the batch.

template <typename RT>
__global__ void __launch_bounds__(512) sweep2d_batch_kernel(const __grid_constant__ BatchSweepArgs B) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int2 s_task;
    __shared__ volatile int s_abort;
    __shared__ __align__(16) SweepArgs s_args;
    const int W = B.W, S = B.S;
    const Layout2D Lay = layout2d((int)sizeof(RT), S, B.stg, B.ring_gw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)W * Lay.wsz);
    uint64_t *ring_bars = bars + (size_t)W * S;
    if (threadIdx.x < W * S) mbar_init(bars + threadIdx.x, 1);
    if (threadIdx.x < 2 * W * RING) mbar_init(ring_bars + threadIdx.x, 32);
    if (threadIdx.x == 0) s_abort = 0;
    fence_mbar_init();
    const unsigned long long epoch = *B.epoch;
    uint32_t phase = 0, ring_p = 0, ring_c = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int t = (int)atomicAdd(B.ctrl + CTRL_QUEUE, 1u);
            s_task = t < B.n_tasks ? B.tasks[t] : make_int2(-1, -1);
        }
        __syncthreads();
        const int2 pt = s_task;
        if (pt.x < 0 || s_abort) return;
        {
            const int *from = reinterpret_cast<const int *>(B.args + pt.x);
            int *to = reinterpret_cast<int *>(&s_args);
            for (int i = threadIdx.x; i < (int)(sizeof(SweepArgs) / sizeof(int)); i += blockDim.x)
                to[i] = from[i];
        }
        __syncthreads();
        // a member not swept this pass: none of its tasks runs, so none waits
        if (s_args.active && *s_args.active == 0) continue;
        switch (s_args.GW) {
            case 1:
                sweep2d_task<RT, 1>(s_args, Lay, pt.y, smem_raw, bars, ring_bars, ring_p, ring_c,
                                    &s_abort, phase, epoch);
                break;
            case 2:
                sweep2d_task<RT, 2>(s_args, Lay, pt.y, smem_raw, bars, ring_bars, ring_p, ring_c,
                                    &s_abort, phase, epoch);
                break;
            case 4:
                sweep2d_task<RT, 4>(s_args, Lay, pt.y, smem_raw, bars, ring_bars, ring_p, ring_c,
                                    &s_abort, phase, epoch);
                break;
            default:
                sweep2d_task<RT, 8>(s_args, Lay, pt.y, smem_raw, bars, ring_bars, ring_p, ring_c,
                                    &s_abort, phase, epoch);
                break;
        }
    }
}

// ---------------------------------------------------------------------------
// 1D: one warp per warp task sweeps the whole line (the paper's 1D problems
// have at most a few thousand cells); per-warp partial moments.
// Q: the direction half (0: mu > 0, 1: mu < 0), a template parameter so that
// the upwind/downwind node roles are compile-time register indices.
template <typename RT, int GW, int Q>
__device__ __forceinline__ void sweep1d_warp(const SweepArgs &A, const int gwarp) {
    using R2 = typename V2<RT>::t;
    const int lane = threadIdx.x & 31;
    constexpr int q = Q;
    const int wt = gwarp - q * A.NWT;
    constexpr int sx = q == 0 ? 1 : -1;
    const int nx = A.nx, ncell = A.ncell;
    const int db = wt / A.NGB, gb = wt - db * A.NGB;
    const LaneConst &L = A.lanes[(q * A.DB + db) * 32 + lane];
    const RT mu = (RT)L.mu;
    const RT w0 = (RT)L.wm[0], w1 = (RT)L.wm[1], w2 = (RT)L.wm[2];
    const RT *src = static_cast<const RT *>(A.src);
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
    constexpr int au = sx > 0 ? 0 : 1;
    const size_t wtbase = (size_t)(q * A.NWT + wt) * ncell;
    for (int i = 0; i < nx; ++i) {
        const int cell = sx > 0 ? i : nx - 1 - i;
        RT s[2] = {0, 0}, ss[2] = {0, 0};
#pragma unroll
        for (int gw = 0; gw < GW; ++gw) {
            const RT *rec = src + ((size_t)cell * A.Gp + gidx[gw]) * SREC;
            const R2 qv = __ldg(reinterpret_cast<const R2 *>(rec));
            const RT sgt = __ldg(rec + 4), sgm = __ldg(rec + 5);
            RT S[2] = {qv.x, qv.y};
            const size_t ioff = ((wtbase + cell) * GW + gw) * 32 + lane;
            if (Ip) {
                const R2 ik = __ldcs(Ip + ioff);
                S[0] = fma(inv_cdt, ik.x, S[0]);
                S[1] = fma(inv_cdt, ik.y, S[1]);
            }
            const RT iA = rcp(sgt + mu);
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
                ss[n] = fma(sgm, I2[n], ss[n]);
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

template <typename RT, int GW>
__global__ void __launch_bounds__(256) sweep1d_kernel(const SweepArgs A) {
    const int gwarp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (gwarp >= A.NQ * A.NWT) return;
    if (gwarp < A.NWT)
        sweep1d_warp<RT, GW, 0>(A, gwarp);
    else
        sweep1d_warp<RT, GW, 1>(A, gwarp);
}

// ---------------------------------------------------------------------------
// Lets kernel k use up to the device's opt-in shared memory per block (less
// its static shared memory), so that problems of different sizes sharing one
// kernel instantiation can all launch; false if smem does not fit.
static bool allow_dynamic_smem(const void *k, size_t smem, int *nsm) {
    int dev = 0, maxopt = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return false;
    const size_t limit = (size_t)maxopt - fa.sharedSizeBytes;
    if (smem > limit) return false;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) ==
           cudaSuccess;
}

template <typename RT>
static const void *kernel2d_ptr(int GW) {
    switch (GW) {
        case 1: return (const void *)sweep2d_kernel<RT, 1>;
        case 2: return (const void *)sweep2d_kernel<RT, 2>;
        case 4: return (const void *)sweep2d_kernel<RT, 4>;
        default: return (const void *)sweep2d_kernel<RT, 8>;
    }
}

// The FP32 kernel without the moment stage (the defect correction's sweeps,
// SweepArgs::mom_acc NULL).
static const void *kernel2d_nomom_ptr(int GW) {
    switch (GW) {
        case 1: return (const void *)sweep2d_kernel<float, 1, false>;
        case 2: return (const void *)sweep2d_kernel<float, 2, false>;
        case 4: return (const void *)sweep2d_kernel<float, 4, false>;
        default: return (const void *)sweep2d_kernel<float, 8, false>;
    }
}

// Dynamic shared memory of a 2D sweep CTA: the sweep layout, plus the group
// edges in FP32 for fused emission warps.
static size_t sweep2d_smem_total(int prec, int W, int GW, int S, int GSLOT, int emit_warps,
                                 int G) {
    size_t smem = sweep2d_smem_bytes(prec, W, GW, S, GSLOT);
    if (emit_warps) smem = ((smem + 15) & ~(size_t)15) + (size_t)(G + 1) * sizeof(float);
    return smem;
}

// The 2D sweep kernel of arithmetic precision prec for problem p's layout and
// tiling (the FP32 correction sweeps of an FP64 problem's defect correction).
int sweep2d_max_resident_prec(int prec, const sm_problem *p, int W, int S, size_t *smem_out) {
    const size_t smem = sweep2d_smem_bytes(prec, W, p->GW, S, p->GSLOT);
    if (smem_out) *smem_out = smem;
    const void *k = (prec == 32) ? kernel2d_ptr<float>(p->GW) : kernel2d_ptr<double>(p->GW);
    int nsm = 0;
    if (!allow_dynamic_smem(k, smem, &nsm)) return 0;
    // the FP32 kernel without moments runs with the same tiling: same limit
    if (prec == 32 && !allow_dynamic_smem(kernel2d_nomom_ptr(p->GW), smem, &nsm)) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, W * 32, smem) != cudaSuccess)
        return 0;
    return per_sm * nsm;
}

cudaError_t launch_sweep2d_prec(int prec, const sm_problem *p, const SweepArgs &a, int grid,
                                cudaStream_t s) {
    EmitArgs none;
    memset(&none, 0, sizeof(none));
    const size_t smem = sweep2d_smem_bytes(prec, a.W, a.GW, a.S, a.GW * a.LG);
    const void *k = (prec == 32) ? (a.mom_acc ? kernel2d_ptr<float>(a.GW)
                                              : kernel2d_nomom_ptr(a.GW))
                                 : kernel2d_ptr<double>(a.GW);
    SweepArgs args = a;
    void *params[] = {&args, &none};
    return cudaLaunchKernel(k, dim3(grid), dim3(a.W * 32), params, smem, s);
}

cudaError_t launch_sweep2d(const sm_problem *p, const SweepArgs &a, int grid, cudaStream_t s,
                           const EmitArgs *e) {
    EmitArgs none;
    memset(&none, 0, sizeof(none));
    EmitArgs ea = e ? *e : none;
    const size_t smem = sweep2d_smem_total(p->prec, a.W, a.GW, a.S, a.GW * a.LG, ea.warps, p->G);
    const void *k = (p->prec == 32) ? kernel2d_ptr<float>(a.GW) : kernel2d_ptr<double>(a.GW);
    SweepArgs args = a;
    void *params[] = {&args, &ea};
    return cudaLaunchKernel(k, dim3(grid), dim3((a.W + ea.warps) * 32), params, smem, s);
}

// Configures the shared-memory limit of the 2D kernel for (W, S, emission
// warps) and returns how many CTAs fit on the whole GPU (0 if none).
int sweep2d_max_resident(const sm_problem *p, int W, int S, size_t *smem_out, int emit_warps) {
    const size_t smem = sweep2d_smem_total(p->prec, W, p->GW, S, p->GSLOT, emit_warps, p->G);
    if (smem_out) *smem_out = smem;
    if ((W + emit_warps) * 32 > 512) return 0;
    const void *k = (p->prec == 32) ? kernel2d_ptr<float>(p->GW) : kernel2d_ptr<double>(p->GW);
    int nsm = 0;
    if (!allow_dynamic_smem(k, smem, &nsm)) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (W + emit_warps) * 32, smem) !=
        cudaSuccess)
        return 0;
    return per_sm * nsm;
}

cudaError_t launch_sweep2d_batch(int prec, const BatchSweepArgs &b, int grid, size_t smem,
                                 cudaStream_t s) {
    const void *k = prec == 32 ? (const void *)sweep2d_batch_kernel<float>
                               : (const void *)sweep2d_batch_kernel<double>;
    BatchSweepArgs args = b;
    void *params[] = {&args};
    return cudaLaunchKernel(k, dim3(grid), dim3(b.W * 32), params, smem, s);
}

int sweep2d_batch_max_resident(int prec, int W, size_t smem) {
    const void *k = prec == 32 ? (const void *)sweep2d_batch_kernel<float>
                               : (const void *)sweep2d_batch_kernel<double>;
    int nsm = 0;
    if (!allow_dynamic_smem(k, smem, &nsm)) return 0;
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
            case 4: sweep1d_kernel<float, 4><<<blocks, threads, 0, s>>>(a); break;
            default: sweep1d_kernel<float, 8><<<blocks, threads, 0, s>>>(a); break;
        }
    } else {
        switch (a.GW) {
            case 1: sweep1d_kernel<double, 1><<<blocks, threads, 0, s>>>(a); break;
            case 2: sweep1d_kernel<double, 2><<<blocks, threads, 0, s>>>(a); break;
            case 4: sweep1d_kernel<double, 4><<<blocks, threads, 0, s>>>(a); break;
            default: sweep1d_kernel<double, 8><<<blocks, threads, 0, s>>>(a); break;
        }
    }
    return cudaGetLastError();
}

}  // namespace smk
