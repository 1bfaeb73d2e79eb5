// sm_sweep_static: the hot-path pass of sm_sweep (emission, wavefront sweep
// with fused moments, moment sums and closures) for small 2D problems, for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available -- a host
// thread that must not block on the allocator or synchronize the device
// (cudaMalloc can do both), a process whose device memory is fully reserved
// by another allocator, or a fixed-memory-budget embedding that forbids
// dynamic allocation.  Such a caller cannot use sm_create_problem (which
// allocates the workspace), so this entry point takes the descriptor and
// caller-owned inputs / outputs only, and keeps every intermediate buffer in
// one file-scope device array of SM_STATIC_SCRATCH_BYTES.  It calls no
// cudaMalloc, cudaFree or other allocating routine; its host state lives on
// the stack (only an error message, when there is one, is copied into the
// library's thread-local error string).
//
// The scratch array exists once per GPU that loads the library and is held
// until the process exits.  Host code cannot use the array's name as a
// device address, so the first call on each device (with that device
// current) looks the address up with cudaGetSymbolAddress and caches it; the
// first call in the process also uploads the Planck tables (synchronous
// copies to constant memory).  Two threads making their first call at once both look the
// address up and store the same value (an atomic store).  All calls share
// the array: calls that overlap on the GPU (two streams, two threads, two
// devices' worth of work on one device) race and corrupt each other.  The
// call is synchronous on its stream only: it reads the device status with an
// asynchronous copy on that stream and waits for that stream, not for the
// device.  Host stack use is about 40 KB (the lane tables of at most 16
// quadrant x direction-block rows).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "sm_internal.cuh"

namespace {

constexpr size_t SM_STATIC_SCRATCH_BYTES = 16u << 20;  // 16 MiB per device
constexpr int MAX_DEVICES = 128;
constexpr int MAX_DIRS = 512;       // 4 quadrants x up to 128 directions
constexpr int MAX_LANE_ROWS = 16;   // quadrants x direction blocks: 4 x (128 / 32)
constexpr int MAX_GROUPS = 256;

static __device__ __align__(256) unsigned char g_static_scratch[SM_STATIC_SCRATCH_BYTES];

std::atomic<void *> g_scratch_addr[MAX_DEVICES];  // zero-initialised (static storage)

sm_status static_fail(sm_status s, const char *msg) {
    smk::set_last_error(msg);  // reported by sm_last_error()
    return s;
}

// Gauss-Legendre rule (ascending) into fixed arrays: Newton on P_n with the
// three-term recurrence, starting from cos(pi (4i+3)/(4n+2)).
void gl_fixed(int n, double *x, double *w) {
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        long double z = cosl(pi * (4.0L * i + 3.0L) / (4.0L * n + 2.0L)), dp = 1.0L;
        for (int it = 0; it < 60; ++it) {
            long double p0 = 1.0L, p1 = z;
            for (int k = 2; k <= n; ++k) {
                long double p2 = ((2.0L * k - 1.0L) * z * p1 - (k - 1.0L) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0L; }
            dp = n * (z * p1 - p0) / (z * z - 1.0L);
            const long double dz = p1 / dp;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        long double p0 = 1.0L, p1 = z;
        for (int k = 2; k <= n; ++k) {
            long double p2 = ((2.0L * k - 1.0L) * z * p1 - (k - 1.0L) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0L; }
        dp = n * (z * p1 - p0) / (z * z - 1.0L);
        x[n - 1 - i] = (double)z;
        w[n - 1 - i] = (double)(2.0L / ((1.0L - z * z) * dp * dp));
    }
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

sm_status sm_sweep_static(const sm_problem_desc *d, void *stream, const double *T,
                          const double *sigma, const double *I_prev_canon, double *I_out_canon,
                          double *moments, double *closures) {
    if (!d) return static_fail(SM_ERR_INVALID_ARG, "desc is NULL");
    if (!T || !sigma || !I_out_canon)
        return static_fail(SM_ERR_INVALID_ARG, "T_nodal_dev, sigma_dev and I_out_dev are required");
    if (const char *why = smk::check_desc(d)) return static_fail(SM_ERR_INVALID_ARG, why);
    if (d->dim != 2) return static_fail(SM_ERR_INVALID_ARG, "sm_sweep_static supports dim = 2 only");
    if (d->n_groups > MAX_GROUPS)
        return static_fail(SM_ERR_INVALID_ARG, "sm_sweep_static supports n_groups <= 256");
    // each factor is bounded (by check_desc and here) before the product
    if (d->n_polar > 128 || d->n_azim > 128 || d->n_polar * d->n_azim > 128)
        return static_fail(SM_ERR_INVALID_ARG, "need 1 <= n_polar * n_azim <= 128");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return static_fail(SM_ERR_CUDA, "no current CUDA device");
    void *addr = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!addr) {
        const cudaError_t e = cudaGetSymbolAddress(&addr, g_static_scratch);
        if (e != cudaSuccess || !addr)
            return static_fail(SM_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        g_scratch_addr[dev].store(addr, std::memory_order_release);
    }
    unsigned char *base = static_cast<unsigned char *>(addr);
    smk::planck_upload_tables();

    // A problem description on the stack: scalar fields only (its vectors stay
    // empty and never allocate); device pointers point into the scratch.
    sm_problem p;
    p.desc = *d;
    p.dim = 2;
    p.nx = d->nx;
    p.ny = d->ny;
    p.ncell = p.nx * p.ny;
    p.nn = 4;
    p.nm = 9;
    p.nc = 11;
    p.G = d->n_groups;
    p.NQ = 4;
    p.hx = (d->x1 - d->x0) / p.nx;
    p.hy = (d->y1 - d->y0) / p.ny;
    p.inv_cdt = d->dt > 0.0 ? 1.0 / (d->c * d->dt) : 0.0;
    p.prec = d->precision;
    p.rsize = p.prec == 32 ? 4 : 8;
    p.stream = (cudaStream_t)stream;

    // quadrature (same set and order as sm_create_problem)
    const int np = d->n_polar, na = d->n_azim;
    double gx[256], gw[256];
    gl_fixed(2 * np, gx, gw);
    double omx[MAX_DIRS], omy[MAX_DIRS], wq[MAX_DIRS];
    const double PI = 3.14159265358979323846;
    const int sgx[4] = {1, -1, -1, 1}, sgy[4] = {1, 1, -1, -1};
    int nd = 0;
    for (int q = 0; q < 4; ++q)
        for (int ip = 0; ip < np; ++ip) {
            const double xi = gx[np + ip], st = std::sqrt(1.0 - xi * xi);
            for (int ia = 0; ia < na; ++ia) {
                const double phi = (ia + 0.5) * (0.5 * PI) / na;
                omx[nd] = sgx[q] * st * std::cos(phi);
                omy[nd] = sgy[q] * st * std::sin(phi);
                wq[nd] = 2.0 * gw[np + ip] * (0.5 * PI) / na;
                ++nd;
            }
        }
    p.nd = nd;
    p.DQ = np * na;
    int dqp = 1;
    while (dqp < p.DQ) dqp <<= 1;
    p.DQP = p.DQ <= 32 ? dqp : ((p.DQ + 31) / 32) * 32;
    p.DQL = std::min(p.DQP, 32);
    p.LG = 32 / p.DQL;
    p.DB = p.DQP / p.DQL;
    p.GW = d->groups_per_warp ? d->groups_per_warp : 1;
    p.GSLOT = p.GW * p.LG;
    p.Gp = ((p.G + p.GSLOT - 1) / p.GSLOT) * p.GSLOT;
    p.NGB = p.Gp / p.GSLOT;
    p.NWT = p.DB * p.NGB;
    if (p.NQ * p.DB > MAX_LANE_ROWS) return static_fail(SM_ERR_INVALID_ARG, "too many directions");

    smk::LaneConst lanes[MAX_LANE_ROWS * 32];
    int dir_of[MAX_LANE_ROWS * 32];
    for (int q = 0; q < 4; ++q)
        for (int db = 0; db < p.DB; ++db)
            for (int lane = 0; lane < 32; ++lane) {
                smk::LaneConst &L = lanes[(q * p.DB + db) * 32 + lane];
                std::memset(&L, 0, sizeof(L));
                const int dq = db * p.DQL + (lane % p.DQL);
                L.g_lo = lane / p.DQL;
                const int dc = dq < p.DQ ? q * p.DQ + dq : -1;
                const int ds = dc >= 0 ? dc : q * p.DQ;
                const double ox = omx[ds], oy = omy[ds], wt = dc >= 0 ? wq[ds] : 0.0;
                L.mu = std::fabs(ox) / p.hx;
                L.eta = std::fabs(oy) / p.hy;
                L.wm[0] = wt;
                L.wm[1] = wt * ox;
                L.wm[2] = wt * oy;
                L.wm[3] = wt * (ox * ox - 1.0 / 3.0);
                L.wm[4] = wt * ox * oy;
                L.wm[5] = wt * (oy * oy - 1.0 / 3.0);
                L.valid = dc >= 0;
                dir_of[(q * p.DB + db) * 32 + lane] = dc;
            }
    const int nlanes = p.NQ * p.DB * 32;

    // tiling: the first shape whose shared memory fits
    const int w_try[] = {8, 4, 2, 1};
    const int s_try[] = {3, 2};
    bool tiled = false;
    for (int w : w_try) {
        for (int st : s_try) {
            p.W = w;
            p.S = st;
            size_t smem = 0;
            if (smk::sweep2d_max_resident(&p, p.W, p.S, &smem) > 0) {
                tiled = true;
                break;
            }
        }
        if (tiled) break;
    }
    if (!tiled) return static_fail(SM_ERR_UNSUPPORTED, "no sweep tiling fits");
    p.NS = (p.nx + p.W - 1) / p.W;
    const size_t nwg = (size_t)p.NQ * p.NWT;

    // carve the scratch
    const size_t ielems = (size_t)p.NQ * p.NWT * p.ncell * p.GW * 32 * p.nn;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t o_ctrl = take(smk::CTRL_WORDS * sizeof(unsigned int));
    const size_t o_flags = take(nwg * p.NS * sizeof(unsigned long long));
    const size_t o_edges = take(sizeof(double) * (p.G + 1));
    const size_t o_inflow = take(4 * (size_t)p.Gp * p.rsize);
    const size_t o_lanes = take(sizeof(smk::LaneConst) * nlanes);
    const size_t o_dir = take(sizeof(int) * nlanes);
    const size_t o_src = take((size_t)p.ncell * p.Gp * 8 * p.rsize);
    const size_t o_gray = take((size_t)p.ncell * p.nn * 2 * sizeof(double));
    const size_t o_acc = take(nwg * p.ncell * 36 * p.rsize);
    const size_t o_face = take(nwg * p.NS * p.ny * p.GW * 32 * 2 * p.rsize);
    const size_t o_mom = take((size_t)p.ncell * p.nn * p.nm * sizeof(double));
    const size_t o_Ip = take(ielems * p.rsize);
    const size_t o_Io = take(ielems * p.rsize);
    if (off > SM_STATIC_SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "problem needs %zu bytes of scratch; sm_sweep_static is limited to %zu",
                 off, SM_STATIC_SCRATCH_BYTES);
        return static_fail(SM_ERR_INVALID_ARG, msg);
    }
    p.d_ctrl = reinterpret_cast<unsigned int *>(base + o_ctrl);
    p.d_flags = reinterpret_cast<unsigned long long *>(base + o_flags);
    p.flags_count = nwg * p.NS;
    p.d_edges = reinterpret_cast<double *>(base + o_edges);
    p.d_inflow = base + o_inflow;
    p.d_lanes = reinterpret_cast<smk::LaneConst *>(base + o_lanes);
    p.d_dir_of = reinterpret_cast<int *>(base + o_dir);
    p.d_src = base + o_src;
    p.d_gray = reinterpret_cast<double *>(base + o_gray);
    p.d_mom_acc = base + o_acc;
    p.d_face = base + o_face;
    p.d_mom_tmp = reinterpret_cast<double *>(base + o_mom);
    void *Ip = base + o_Ip;
    void *Io = base + o_Io;

    cudaStream_t s = p.stream;
#define ST_CUDA(x)                                                          \
    do {                                                                    \
        if ((x) != cudaSuccess) return static_fail(SM_ERR_CUDA, #x " failed"); \
    } while (0)
    // what must start at zero: control words (queue, abort, status) and the
    // wavefront row counters (epoch 1 below); every partial moment slot is
    // written by its warp task
    ST_CUDA(cudaMemsetAsync(base + o_ctrl, 0, smk::CTRL_WORDS * sizeof(unsigned int), s));
    ST_CUDA(cudaMemsetAsync(base + o_flags, 0, nwg * p.NS * 8, s));
    ST_CUDA(cudaMemcpyAsync(p.d_edges, d->group_edges, sizeof(double) * (p.G + 1),
                            cudaMemcpyHostToDevice, s));
    ST_CUDA(cudaMemcpyAsync(p.d_lanes, lanes, sizeof(smk::LaneConst) * nlanes,
                            cudaMemcpyHostToDevice, s));
    ST_CUDA(cudaMemcpyAsync(p.d_dir_of, dir_of, sizeof(int) * nlanes, cudaMemcpyHostToDevice, s));
    ST_CUDA(smk::launch_inflow(&p, s));
    if (I_prev_canon) ST_CUDA(smk::launch_pack(&p, I_prev_canon, Ip, 0, s));
    ST_CUDA(smk::launch_emission(&p, T, sigma, nullptr, s));
    smk::SweepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nx = p.nx; a.ny = p.ny; a.ncell = p.ncell; a.NQ = p.NQ; a.NWT = p.NWT; a.NGB = p.NGB;
    a.DB = p.DB; a.LG = p.LG; a.GW = p.GW; a.Gp = p.Gp; a.W = p.W; a.S = p.S; a.NS = p.NS;
    a.n_tasks = p.NS * p.NQ * p.NWT; a.inv_cdt = p.inv_cdt;
    a.lanes = p.d_lanes; a.src = p.d_src; a.inflow = p.d_inflow;
    a.I_prev = I_prev_canon ? Ip : nullptr; a.I_out = Io; a.mom_acc = p.d_mom_acc;
    a.face = p.d_face; a.flags = p.d_flags; a.ctrl = p.d_ctrl; a.epoch = 1;
    a.timeout_ns = 2000000000LL;
    a.fault_skip_publish = 0;
    size_t smem = 0;
    const int resident = smk::sweep2d_max_resident(&p, p.W, p.S, &smem);
    if (resident <= 0) return static_fail(SM_ERR_UNSUPPORTED, "sweep tiling does not fit");
    a.publish = smk::publish_rows(a.n_tasks, resident);
    ST_CUDA(smk::launch_sweep2d(&p, a, std::min(a.n_tasks, resident), s));
    ST_CUDA(smk::launch_reduce(&p, p.d_mom_acc, (int)nwg, moments ? moments : p.d_mom_tmp,
                               closures, s, nullptr, p.NWT));
    ST_CUDA(smk::launch_pack(&p, I_out_canon, Io, 1, s));
    // the status words, read on this stream only (no device-wide synchronization)
    unsigned int ctrl[smk::CTRL_WORDS];
    ST_CUDA(cudaMemcpyAsync(ctrl, base + o_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, s));
    ST_CUDA(cudaStreamSynchronize(s));
#undef ST_CUDA
    if (ctrl[smk::CTRL_STATUS] & smk::ST_TIMEOUT)
        return static_fail(SM_ERR_TIMEOUT, "a wavefront wait exceeded its time limit");
    if (ctrl[smk::CTRL_STATUS] & smk::ST_NONPHYSICAL)
        return static_fail(SM_ERR_NONPHYSICAL, "non-positive or non-finite temperature");
    return SM_OK;
}

}  // extern "C"
