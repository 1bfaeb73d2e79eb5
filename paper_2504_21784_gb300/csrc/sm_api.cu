// Host implementation of the C ABI declared in include/sm.h: problem set-up
// (S_N quadrature, lane mapping, workspace), launch orchestration of the hot
// path (emission -> sweep -> reduction/closures), timing and status.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sm_internal.cuh"

namespace {

thread_local std::string g_err;

sm_status fail(sm_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

#define SM_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? SM_ERR_OOM : SM_ERR_CUDA,        \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
        }                                                                                  \
    } while (0)

// n-point Gauss-Legendre rule on [-1, 1] (ascending nodes): Newton's method on
// P_n from the asymptotic initial guess cos(pi (4i+3)/(4n+2)), with P_n and
// P_n' from the three-term recurrence in long double.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        long double z = cosl(pi * (4.0L * i + 3.0L) / (4.0L * n + 2.0L));
        long double dp = 1.0L;
        for (int it = 0; it < 60; ++it) {
            long double p0 = 1.0L, p1 = z;
            for (int k = 2; k <= n; ++k) {
                long double p2 = ((2.0L * k - 1.0L) * z * p1 - (k - 1.0L) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) {
                p1 = z;
                p0 = 1.0L;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0L);
            long double dz = p1 / dp;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        long double p0 = 1.0L, p1 = z;
        for (int k = 2; k <= n; ++k) {
            long double p2 = ((2.0L * k - 1.0L) * z * p1 - (k - 1.0L) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) {
            p1 = z;
            p0 = 1.0L;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0L);
        x[n - 1 - i] = (double)z;
        w[n - 1 - i] = (double)(2.0L / ((1.0L - z * z) * dp * dp));
    }
}

int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

template <typename T>
sm_status dev_alloc(T **ptr, size_t bytes, size_t *acc) {
    if (*ptr) {
        cudaFree(*ptr);
        *ptr = nullptr;
    }
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void **)ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? SM_ERR_OOM : SM_ERR_CUDA,
                    std::string("cudaMalloc(") + std::to_string(bytes) + "): " +
                        cudaGetErrorString(e));
    }
    if (acc) *acc += bytes;
    return SM_OK;
}

void free_all(sm_problem *p) {
    void *bufs[] = {p->d_edges, p->d_inflow, p->d_lanes, p->d_dir_of, p->d_src,
                    p->d_mom_acc, p->d_gray, p->d_part, p->d_face, p->d_flags,
                    p->ctrl_borrowed ? nullptr : p->d_ctrl, p->d_mom_tmp, p->d_T_tmp,
                    p->d_sig_tmp, p->d_clo_tmp, p->d_emit_ctr, p->d_strip_x0};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete p->tabs;
    p->tabs = nullptr;
    smk::lo_free(p);
    smk::adjoint_free(p);
    smk::refine_free(p);
    for (auto &e : p->ev_pool)
        if (e) cudaEventDestroy(e);
    p->ev_pool.clear();
}

constexpr int MAX_TIMED_SWEEPS = 4096;

// Events of the n-th timed sweep (created on first use).
cudaEvent_t *timing_events(sm_problem *p, int n) {
    if (n >= MAX_TIMED_SWEEPS) return nullptr;
    while ((int)p->ev_pool.size() < 4 * (n + 1)) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        p->ev_pool.push_back(e);
    }
    return &p->ev_pool[4 * n];
}

// First cell column of each strip (and nx) for strips of W columns with
// `tail` strips of W/2 columns at each end of the x range; empty when that
// layout does not exist (tail > 0 needs an even W and at least one strip of
// W columns in between).
std::vector<int> strip_layout(int nx, int W, int tail) {
    std::vector<int> x0;
    if (tail <= 0) return x0;
    const int h = W / 2, mid = nx - 2 * tail * h;
    if (W % 2 || h < 1 || mid < W) return x0;
    int x = 0;
    for (int i = 0; i < tail; ++i, x += h) x0.push_back(x);
    for (; x < tail * h + mid; x += W) x0.push_back(x);
    x = tail * h + mid;
    for (int i = 0; i < tail; ++i, x += h) x0.push_back(x);
    x0.push_back(nx);
    return x0;
}

// (Re)allocate the tiling-dependent workspace: W cell columns (= warps) per
// CTA and S prefetched rows per warp for the 2D sweep, E warps per CTA
// computing the emission inside the sweep kernel (0: its own kernel; E < 0
// keeps the current number), and `tail` half-width strips at each end of the
// x range (shorter tasks for the partial last wave of the persistent grid;
// tail < 0 keeps the current number, which falls to 0 where the layout does
// not exist).  The strips' tasks go through the queue in the same upwind
// order either way.
sm_status apply_tiling(sm_problem *p, int W, int S, int E = -1, int tail = -1) {
    if (p->dim == 1) {
        p->W = 1;
        p->S = 0;
        p->NS = 1;
        const size_t pb = (size_t)p->NQ * p->NWT * p->ncell * p->nn * p->nm * p->rsize;
        if (!p->d_part) {
            sm_status st = dev_alloc(&p->d_part, pb, nullptr);
            if (st) return st;
        }
    } else {
        if (W < 1 || W > 16) return fail(SM_ERR_INVALID_ARG, "strip_width must be in 1..16");
        if (S < 2 || S > 8) return fail(SM_ERR_INVALID_ARG, "prefetch_rows must be in 2..8");
        if (E < 0) E = p->emit_warps;
        if (E > 4 || W + E > 16)
            return fail(SM_ERR_INVALID_ARG, "emission warps: 0..4 and strip_width + warps <= 16");
        if (E > 0 && p->batch_owned)
            return fail(SM_ERR_UNSUPPORTED, "batch members run the emission as its own kernel");
        if (tail < 0) tail = p->tail;
        if (tail > 0 && (E > 0 || p->batch_owned))
            return fail(SM_ERR_UNSUPPORTED,
                        "half-width end strips need the separate emission kernel and a problem "
                        "of its own");
        std::vector<int> x0 = strip_layout(p->nx, W, tail);
        if (x0.empty()) tail = 0;
        const int old_W = p->W, old_S = p->S;
        p->W = W;
        p->S = S;
        size_t smem = 0;
        const int resident = smk::sweep2d_max_resident(p, W, S, &smem, E);
        if (resident <= 0) {
            p->W = old_W;
            p->S = old_S;
            return fail(SM_ERR_UNSUPPORTED, "tiling needs " + std::to_string(smem) +
                                                " B of shared memory per CTA (too much)");
        }
        p->resident = resident;
        p->emit_warps = E;
        p->tail = tail;
        p->NS = tail > 0 ? (int)x0.size() - 1 : (p->nx + W - 1) / W;
        if (tail > 0) {
            sm_status st = dev_alloc(&p->d_strip_x0, sizeof(int) * x0.size(), nullptr);
            if (st) return st;
            SM_CUDA(cudaMemcpy(p->d_strip_x0, x0.data(), sizeof(int) * x0.size(),
                               cudaMemcpyHostToDevice));
        }
        if (E > 0) {
            if (!p->tabs) {
                p->tabs = new smk::PlanckTabs();
                if (!smk::planck_tabs(p->tabs)) return fail(SM_ERR_CUDA, "Planck tables");
            }
            sm_status st = dev_alloc(&p->d_emit_ctr, sizeof(unsigned int) * (1 + p->NS), nullptr);
            if (st) return st;
        }
        const size_t nwg = (size_t)p->NQ * p->NWT;
        const size_t fb = nwg * p->NS * p->ny * p->GW * 32 * 2 * p->rsize;
        if (fb != p->face_bytes || !p->d_face) {
            sm_status st = dev_alloc(&p->d_face, fb, nullptr);
            if (st) return st;
            p->face_bytes = fb;
        }
        const size_t nf = nwg * p->NS;
        if (nf != p->flags_count || !p->d_flags) {
            sm_status st = dev_alloc(&p->d_flags, nf * sizeof(unsigned long long), nullptr);
            if (st) return st;
            SM_CUDA(cudaMemset(p->d_flags, 0, nf * sizeof(unsigned long long)));
            p->flags_count = nf;
        }
    }
    const size_t mom_scratch = p->dim == 2
                                   ? (size_t)p->NQ * p->NWT * p->ncell * 36 * p->rsize
                                   : (size_t)p->NQ * p->NWT * p->ncell * p->nn * p->nm * p->rsize;
    p->workspace_bytes = (size_t)p->Gp * p->ncell * 8 * p->rsize +         // source records
                         (size_t)p->ncell * p->nn * 2 * 8 +                 // gray spectra
                         mom_scratch + p->face_bytes + p->flags_count * 8 +  // sweep scratch
                         (size_t)p->ncell * p->nn * (p->nm + p->nc + 1) * 8 +  // staging
                         (size_t)p->G * p->ncell * 8;
    return SM_OK;
}

smk::SweepArgs make_args(const sm_problem *p, const void *I_prev, void *I_out) {
    smk::SweepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nx = p->nx;
    a.ny = p->ny;
    a.ncell = p->ncell;
    a.NQ = p->NQ;
    a.NWT = p->NWT;
    a.NGB = p->NGB;
    a.DB = p->DB;
    a.LG = p->LG;
    a.GW = p->GW;
    a.Gp = p->Gp;
    a.W = p->W;
    a.S = p->S;
    a.NS = p->NS;
    a.n_tasks = p->NS * p->NQ * p->NWT;
    a.inv_cdt = p->inv_cdt;
    a.lanes = p->d_lanes;
    a.src = p->d_src;
    a.inflow = p->d_inflow;
    a.I_prev = I_prev;
    a.I_out = I_out;
    a.part = p->d_part;
    a.mom_acc = p->d_mom_acc;
    a.face = p->d_face;
    a.flags = p->d_flags;
    a.ctrl = p->d_ctrl;
    a.epoch = p->epoch;
    a.timeout_ns = p->timeout_ns;
    a.fault_skip_publish = p->fault_skip_publish;
    a.publish = smk::publish_rows(a.n_tasks, p->resident);
    a.strip_x0 = p->tail > 0 ? p->d_strip_x0 : nullptr;
    return a;
}

sm_status check_ptr(const void *ptr, const char *name) {
    if (!ptr) return fail(SM_ERR_INVALID_ARG, std::string(name) + " is NULL");
    return SM_OK;
}

// The packed intensity is read by TMA bulk copies and written with 16-byte
// vector stores: both buffers must start on a 16-byte boundary.
sm_status check_intensity_align(const void *I_prev, const void *I_out) {
    if ((reinterpret_cast<uintptr_t>(I_prev) & 15u) || (reinterpret_cast<uintptr_t>(I_out) & 15u))
        return fail(SM_ERR_INVALID_ARG, "packed intensity buffers must be 16-byte aligned");
    return SM_OK;
}

// Sweep kernel and reduction of one pass.  The source records are in place,
// unless T_emit is given: then the sweep kernel's fused emission warps write
// them from T_emit and sigma_emit (2D, p->emit_warps > 0).
sm_status sweep_pass(sm_problem *p, const void *I_prev, void *I_out, double *mom, double *clo,
                     int reverse, cudaEvent_t *ev, const double *T_emit = nullptr,
                     const double *sigma_emit = nullptr) {
    cudaStream_t s = p->stream;
    ++p->epoch;
    smk::SweepArgs a = make_args(p, I_prev, I_out);
    a.reverse = reverse;
    const bool qm = p->qmom_dev != nullptr && !reverse;
    a.qmom = qm && p->dim == 2 ? 1 : 0;  // 1D: the per-warp partials are per half already
    if (p->dim == 2) {
        SM_CUDA(cudaMemsetAsync(p->d_ctrl, 0, 2 * sizeof(unsigned int), s));
        const int grid = std::min(a.n_tasks, p->resident);
        if (T_emit) {
            smk::EmitArgs e;
            std::memset(&e, 0, sizeof(e));
            e.warps = p->emit_warps;
            e.G = p->G;
            e.Gp = p->Gp;
            e.ncell = p->ncell;
            e.nx = p->nx;
            e.ny = p->ny;
            e.W = p->W;
            e.NS = p->NS;
            e.per_strip = (p->W * p->ny + 7) / 8;
            e.items = e.per_strip * p->NS;
            e.acT4_scale = p->desc.a * p->desc.c / (4.0 * 3.14159265358979323846);
            e.inv_cdt = p->inv_cdt;
            e.edges = p->d_edges;
            e.T = T_emit;
            e.sigma = sigma_emit;
            e.gray = p->d_gray;
            e.ctr = p->d_emit_ctr;
            e.timeout_ns = p->timeout_ns;
            e.tabs = *p->tabs;
            SM_CUDA(cudaMemsetAsync(p->d_emit_ctr, 0, sizeof(unsigned int) * (1 + p->NS), s));
            SM_CUDA(smk::launch_sweep2d(p, a, grid, s, &e));
        } else {
            SM_CUDA(smk::launch_sweep2d(p, a, grid, s));
        }
    } else {
        SM_CUDA(smk::launch_sweep1d(p, a, s));
    }
    p->launches++;
    if (ev) SM_CUDA(cudaEventRecord(ev[2], s));
    if (mom || clo) {
        double *m = mom ? mom : p->d_mom_tmp;
        if (p->dim == 2)
            SM_CUDA(smk::launch_reduce(p, p->d_mom_acc, p->NQ * p->NWT, m, clo, s,
                                       qm ? p->qmom_dev : nullptr, p->NWT));
        else
            SM_CUDA(smk::launch_reduce(p, p->d_part, p->NQ * p->NWT, m, clo, s,
                                       qm ? p->qmom_dev : nullptr, p->NWT));
        p->launches++;
    }
    return SM_OK;
}

// The hot path without argument checks: emission, sweep, reduction.
sm_status run_sweep(sm_problem *p, const double *T, const double *sigma, const void *I_prev,
                    void *I_out, double *mom, double *clo) {
    cudaStream_t s = p->stream;
    cudaEvent_t *ev = p->profiling ? timing_events(p, p->n_timed) : nullptr;
    if (ev) SM_CUDA(cudaEventRecord(ev[0], s));
    const bool fused = p->dim == 2 && p->emit_warps > 0;
    if (!fused) {
        SM_CUDA(smk::launch_emission(p, T, sigma, nullptr, s));
        p->launches++;
    }
    if (ev) SM_CUDA(cudaEventRecord(ev[1], s));
    // the moments are always summed in a full pass (into scratch when mom is NULL)
    sm_status st = sweep_pass(p, I_prev, I_out, mom ? mom : p->d_mom_tmp, clo, 0, ev,
                              fused ? T : nullptr, fused ? sigma : nullptr);
    if (st != SM_OK) return st;
    if (ev) {
        SM_CUDA(cudaEventRecord(ev[3], s));
        p->n_timed++;
    }
    return SM_OK;
}

}  // namespace

namespace smk {
void set_last_error(const char *msg) { g_err = msg; }
sm_status apply_tiling_ext(sm_problem *p, int W, int S) { return apply_tiling(p, W, S, 0); }
sm_status sweep_only(sm_problem *p, const void *I_prev, void *I_out, double *mom, double *clo,
                     int reverse) {
    if (reverse && p->dim != 2)
        return fail(SM_ERR_UNSUPPORTED, "reversed (adjoint) sweeps are 2D only");
    return sweep_pass(p, I_prev, I_out, mom, clo, reverse, nullptr);
}
SweepArgs make_sweep_args(const sm_problem *p, const void *I_prev, void *I_out) {
    return make_args(p, I_prev, I_out);
}
}  // namespace smk

namespace smk {
const char *check_desc(const sm_problem_desc *d) {
    if (d->dim != 1 && d->dim != 2) return "dim must be 1 or 2";
    if (d->nx < 1 || (d->dim == 2 && d->ny < 1)) return "empty mesh: nx and ny must be >= 1";
    if ((long long)d->nx * (d->dim == 2 ? d->ny : 1) > (1LL << 30))
        return "mesh too large (more than 2^30 cells)";
    if (!std::isfinite(d->x0) || !std::isfinite(d->x1) || !(d->x1 > d->x0) ||
        (d->dim == 2 && (!std::isfinite(d->y0) || !std::isfinite(d->y1) || !(d->y1 > d->y0))))
        return "domain extent must be finite and positive";
    if (d->n_groups < 1 || !d->group_edges) return "n_groups must be >= 1 with group_edges";
    for (int g = 0; g <= d->n_groups; ++g) {
        if (!(d->group_edges[g] > 0.0) || !std::isfinite(d->group_edges[g]))
            return "group edges must be positive and finite";
        if (g > 0 && !(d->group_edges[g] > d->group_edges[g - 1]))
            return "group edges must be ascending";
    }
    if (d->dim == 1 && (d->n_polar < 2 || d->n_polar % 2 || d->n_polar > 4096))
        return "1D quadrature order must be even, 2..4096";
    // each factor bounded before any product of the two is formed
    if (d->dim == 2 && (d->n_polar < 1 || d->n_azim < 1 || d->n_polar > 4096 || d->n_azim > 4096))
        return "2D quadrature needs 1 <= n_polar, n_azim <= 4096";
    if (!(d->a > 0.0) || !(d->c > 0.0) || !std::isfinite(d->a) || !std::isfinite(d->c))
        return "a and c must be finite and > 0";
    if (!std::isfinite(d->dt)) return "dt must be finite";
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(d->T_bdr[k])) return "boundary temperatures must be finite";
    if (d->precision != 32 && d->precision != 64) return "precision must be 32 or 64";
    if (d->opacity_kind != SM_OPACITY_POWER && d->opacity_kind != SM_OPACITY_LARSEN)
        return "unknown opacity_kind";
    if (!std::isfinite(d->opacity_alpha)) return "opacity_alpha must be finite";
    if (d->groups_per_warp != 0 && d->groups_per_warp != 1 && d->groups_per_warp != 2 &&
        d->groups_per_warp != 4 && d->groups_per_warp != 8)
        return "groups_per_warp must be 0, 1, 2, 4 or 8";
    if (d->strip_width < 0 || d->strip_width > 16) return "strip_width out of range (0..16)";
    if (d->prefetch_rows < 0 || d->prefetch_rows > 8 || d->prefetch_rows == 1)
        return "prefetch_rows must be 0 or 2..8";
    return nullptr;
}
}  // namespace smk

extern "C" {

const char *sm_last_error(void) { return g_err.c_str(); }

const char *sm_status_string(sm_status s) {
    switch (s) {
        case SM_OK: return "SM_OK";
        case SM_ERR_INVALID_ARG: return "SM_ERR_INVALID_ARG";
        case SM_ERR_CUDA: return "SM_ERR_CUDA";
        case SM_ERR_OOM: return "SM_ERR_OOM";
        case SM_ERR_NO_CONVERGENCE: return "SM_ERR_NO_CONVERGENCE";
        case SM_ERR_NONPHYSICAL: return "SM_ERR_NONPHYSICAL";
        case SM_ERR_TIMEOUT: return "SM_ERR_TIMEOUT";
        case SM_ERR_UNSUPPORTED: return "SM_ERR_UNSUPPORTED";
    }
    return "SM_ERR_UNKNOWN";
}

// standalone: the problem is swept on its own (not as a batch member), so the
// automatic slots-per-lane choice also keeps enough independent wavefront
// chains to fill the GPU.
static sm_status create_problem(const sm_problem_desc *d, void *stream, sm_problem **out,
                                int standalone) {
    if (!d || !out) return fail(SM_ERR_INVALID_ARG, "desc and out must be non-NULL");
    *out = nullptr;
    if (const char *why = smk::check_desc(d)) return fail(SM_ERR_INVALID_ARG, why);

    smk::planck_upload_tables();
    smk::planck_df_upload_tables();
    sm_problem *p = new sm_problem();
    p->desc = *d;
    p->edges.assign(d->group_edges, d->group_edges + d->n_groups + 1);
    p->desc.group_edges = p->edges.data();
    p->dim = d->dim;
    p->nx = d->nx;
    p->ny = d->dim == 2 ? d->ny : 1;
    p->ncell = p->nx * p->ny;
    p->nn = d->dim == 2 ? 4 : 2;
    p->nm = d->dim == 2 ? 9 : 5;
    p->nc = d->dim == 2 ? 11 : 7;
    p->G = d->n_groups;
    p->NQ = d->dim == 2 ? 4 : 2;
    p->hx = (d->x1 - d->x0) / p->nx;
    p->hy = d->dim == 2 ? (d->y1 - d->y0) / p->ny : 1.0;
    p->inv_cdt = d->dt > 0.0 ? 1.0 / (d->c * d->dt) : 0.0;
    p->prec = d->precision;
    p->rsize = p->prec == 32 ? 4 : 8;
    p->stream = (cudaStream_t)stream;

    // ---- quadrature in canonical order
    const double PI = 3.14159265358979323846;
    if (p->dim == 1) {
        std::vector<double> x, w;
        gauss_legendre(d->n_polar, x, w);
        p->nd = d->n_polar;
        p->omx = x;
        p->omy.assign(p->nd, 0.0);
        p->w.resize(p->nd);
        for (int i = 0; i < p->nd; ++i) p->w[i] = 2.0 * PI * w[i];
        p->DQ = p->nd / 2;
    } else {
        std::vector<double> x, w;
        gauss_legendre(2 * d->n_polar, x, w);
        const int np = d->n_polar, na = d->n_azim;
        p->nd = 4 * np * na;
        p->DQ = np * na;
        const int sgx[4] = {1, -1, -1, 1}, sgy[4] = {1, 1, -1, -1};
        for (int q = 0; q < 4; ++q)
            for (int ip = 0; ip < np; ++ip) {
                const double xi = x[np + ip], wp = w[np + ip];
                const double st = std::sqrt(1.0 - xi * xi);
                for (int ia = 0; ia < na; ++ia) {
                    const double phi = (ia + 0.5) * (0.5 * PI) / na;
                    p->omx.push_back(sgx[q] * st * std::cos(phi));
                    p->omy.push_back(sgy[q] * st * std::sin(phi));
                    p->w.push_back(2.0 * wp * (0.5 * PI) / na);
                }
            }
    }
    {
        double sa = 0, sw = 0;
        for (int i = 0; i < p->nd; ++i) {
            sa += p->w[i] * std::fabs(p->omx[i]);
            sw += p->w[i];
        }
        p->alpha = sa / sw;
    }

    // ---- lane mapping
    p->DQP = p->DQ <= 32 ? next_pow2(p->DQ) : ((p->DQ + 31) / 32) * 32;
    p->DQL = std::min(p->DQP, 32);
    p->LG = 32 / p->DQL;
    p->DB = p->DQP / p->DQL;
    int GW = d->groups_per_warp;
    if (GW == 0) {
        const int gpl = (p->G + p->LG - 1) / p->LG;  // slots per lane if GW were unlimited
        const int gmax = d->precision == 32 ? 8 : 4;
        GW = 1;
        while (GW < gmax && gpl >= 2 * GW) GW *= 2;
        // chains: quadrants x direction blocks x group blocks, each an
        // independent wavefront pipeline; measured on a 128^2 x 64 x 16 sweep,
        // 16 chains of 2 slots beat 4 chains of 8 by 24 %
        auto chains = [&](int gw) { return p->NQ * p->DB * ((p->G + gw * p->LG - 1) / (gw * p->LG)); };
        if (standalone)
            while (GW > 1 && chains(GW) < 16) GW /= 2;
    }
    p->GW = GW;
    p->GSLOT = GW * p->LG;
    p->Gp = ((p->G + p->GSLOT - 1) / p->GSLOT) * p->GSLOT;
    p->NGB = p->Gp / p->GSLOT;
    p->NWT = p->DB * p->NGB;

    std::vector<smk::LaneConst> lanes((size_t)p->NQ * p->DB * 32);
    std::vector<int> dir_of(lanes.size(), -1);
    for (int q = 0; q < p->NQ; ++q)
        for (int db = 0; db < p->DB; ++db)
            for (int lane = 0; lane < 32; ++lane) {
                smk::LaneConst &L = lanes[(q * p->DB + db) * 32 + lane];
                std::memset(&L, 0, sizeof(L));
                const int dq = db * p->DQL + (lane % p->DQL);  // direction inside the quadrant
                L.g_lo = lane / p->DQL;
                int d_can = -1;
                if (dq < p->DQ) {
                    if (p->dim == 2) {
                        d_can = q * p->DQ + dq;
                    } else {
                        // 1D "quadrants": q = 0 -> mu > 0 (upper half of the GL nodes),
                        // q = 1 -> mu < 0 (lower half)
                        d_can = (q == 0) ? p->DQ + dq : dq;
                    }
                }
                // padding lanes reuse a valid direction with zero weight
                const int ds = d_can >= 0 ? d_can : (p->dim == 2 ? q * p->DQ : (q == 0 ? p->DQ : 0));
                const double ox = p->omx[ds], oy = p->omy[ds];
                const double wt = d_can >= 0 ? p->w[ds] : 0.0;
                L.mu = std::fabs(ox) / p->hx;
                L.eta = p->dim == 2 ? std::fabs(oy) / p->hy : 0.0;
                if (p->dim == 2) {
                    L.wm[0] = wt;
                    L.wm[1] = wt * ox;
                    L.wm[2] = wt * oy;
                    L.wm[3] = wt * (ox * ox - 1.0 / 3.0);
                    L.wm[4] = wt * ox * oy;
                    L.wm[5] = wt * (oy * oy - 1.0 / 3.0);
                } else {
                    L.wm[0] = wt;
                    L.wm[1] = wt * ox;
                    L.wm[2] = wt * (ox * ox - 1.0 / 3.0);
                }
                L.valid = d_can >= 0;
                dir_of[(q * p->DB + db) * 32 + lane] = d_can;
            }

    // ---- allocations
    sm_status st;
    size_t acc = 0;
#define SM_TRY(x)            \
    do {                     \
        st = (x);            \
        if (st) {            \
            free_all(p);     \
            delete p;        \
            return st;       \
        }                    \
    } while (0)
    SM_TRY(dev_alloc(&p->d_edges, sizeof(double) * (p->G + 1), &acc));
    SM_TRY(dev_alloc(&p->d_inflow, 4 * (size_t)p->Gp * p->rsize, &acc));
    SM_TRY(dev_alloc(&p->d_lanes, sizeof(smk::LaneConst) * lanes.size(), &acc));
    SM_TRY(dev_alloc(&p->d_dir_of, sizeof(int) * dir_of.size(), &acc));
    SM_TRY(dev_alloc(&p->d_src, (size_t)p->Gp * p->ncell * 8 * p->rsize, &acc));
    if (p->dim == 2)
        SM_TRY(dev_alloc(&p->d_mom_acc, (size_t)p->NQ * p->NWT * p->ncell * 36 * p->rsize, &acc));
    SM_TRY(dev_alloc(&p->d_gray, (size_t)p->ncell * p->nn * 2 * sizeof(double), &acc));
    SM_TRY(dev_alloc(&p->d_ctrl, smk::CTRL_WORDS * sizeof(unsigned int), &acc));
    SM_TRY(dev_alloc(&p->d_mom_tmp, (size_t)p->ncell * p->nn * p->nm * sizeof(double), &acc));
    SM_TRY(dev_alloc(&p->d_clo_tmp, (size_t)p->ncell * p->nn * p->nc * sizeof(double), &acc));
    SM_TRY(dev_alloc(&p->d_T_tmp, (size_t)p->ncell * p->nn * sizeof(double), &acc));
    SM_TRY(dev_alloc(&p->d_sig_tmp, (size_t)p->G * p->ncell * sizeof(double), &acc));
    auto cuda_try = [&](cudaError_t e, const char *what) -> sm_status {
        if (e == cudaSuccess) return SM_OK;
        return fail(SM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    SM_TRY(cuda_try(cudaMemcpy(p->d_edges, p->edges.data(), sizeof(double) * (p->G + 1),
                               cudaMemcpyHostToDevice), "edges"));
    SM_TRY(cuda_try(cudaMemcpy(p->d_lanes, lanes.data(), sizeof(smk::LaneConst) * lanes.size(),
                               cudaMemcpyHostToDevice), "lanes"));
    SM_TRY(cuda_try(cudaMemcpy(p->d_dir_of, dir_of.data(), sizeof(int) * dir_of.size(),
                               cudaMemcpyHostToDevice), "dir_of"));
    SM_TRY(cuda_try(cudaMemset(p->d_ctrl, 0, smk::CTRL_WORDS * sizeof(unsigned int)), "ctrl"));
    SM_TRY(cuda_try(smk::launch_inflow(p, p->stream), "inflow"));
    p->launches++;

    // ---- tiling
    if (p->dim == 2) {
        // auto: the widest strip (most warps per CTA) whose shared memory
        // fits, with two prefetched rows
        int W = d->strip_width, S = d->prefetch_rows;
        if (S == 0) S = 2;
        if (W == 0) {
            st = SM_ERR_UNSUPPORTED;
            for (int wc : {16, 12, 8, 4, 2})
                if ((st = apply_tiling(p, wc, S)) == SM_OK) break;
        } else {
            st = apply_tiling(p, W, S);
        }
        if (st) {
            free_all(p);
            delete p;
            return st;
        }
    } else {
        SM_TRY(apply_tiling(p, 0, 0));
    }
    SM_TRY(cuda_try(cudaStreamSynchronize(p->stream), "create sync"));
#undef SM_TRY
    *out = p;
    return SM_OK;
}

sm_status sm_create_problem(const sm_problem_desc *d, void *stream, sm_problem **out) {
    return create_problem(d, stream, out, 1);
}

sm_status sm_destroy_problem(sm_problem *p) {
    if (!p) return SM_OK;
    if (p->batch_owned)
        return fail(SM_ERR_INVALID_ARG, "this problem belongs to a batch: destroy the batch");
    cudaStreamSynchronize(p->stream);
    free_all(p);
    delete p;
    return SM_OK;
}

sm_status sm_get_info(const sm_problem *p, sm_problem_info *o) {
    if (!p || !o) return fail(SM_ERR_INVALID_ARG, "NULL argument");
    std::memset(o, 0, sizeof(*o));
    o->dim = p->dim;
    o->nx = p->nx;
    o->ny = p->ny;
    o->n_dir = p->nd;
    o->n_groups = p->G;
    o->n_cells = p->ncell;
    o->n_nodes = p->nn;
    o->n_moments = p->nm;
    o->n_closures = p->nc;
    o->precision = p->prec;
    o->dirs_per_quadrant = p->DQP;
    o->groups_per_lane_row = p->LG;
    o->groups_per_warp = p->GW;
    o->n_groups_padded = p->Gp;
    o->n_warp_tasks = p->NWT;
    o->strip_width = p->W;
    o->prefetch_rows = p->S;
    o->n_tasks = p->dim == 2 ? p->NS * p->NQ * p->NWT : p->NQ * p->NWT;
    o->n_strips = p->NS;
    o->intensity_elems = (size_t)p->NQ * p->NWT * p->ncell * p->GW * 32 * p->nn;
    o->intensity_bytes = o->intensity_elems * p->rsize;
    o->workspace_bytes = p->workspace_bytes;
    o->alpha = p->alpha;
    o->emission_warps = p->emit_warps;
    o->tail_strips = p->tail;
    return SM_OK;
}

sm_status sm_set_stream(sm_problem *p, void *stream) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    p->stream = (cudaStream_t)stream;
    return SM_OK;
}

sm_status sm_set_tiling(sm_problem *p, int strip_width, int prefetch_rows) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    if (p->batch_owned)
        return fail(SM_ERR_INVALID_ARG, "this problem belongs to a batch: sweep it with sm_batch_sweep");
    if (p->dim == 1) return SM_OK;
    SM_CUDA(cudaStreamSynchronize(p->stream));
    return apply_tiling(p, strip_width > 0 ? strip_width : p->W,
                        prefetch_rows > 0 ? prefetch_rows : p->S);
}

sm_status sm_set_tail_strips(sm_problem *p, int n) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    if (p->batch_owned)
        return fail(SM_ERR_INVALID_ARG, "this problem belongs to a batch: sweep it with sm_batch_sweep");
    if (n < 0 || n > 4) return fail(SM_ERR_INVALID_ARG, "tail strips must be in 0..4");
    if (p->dim == 1) return n == 0 ? SM_OK : fail(SM_ERR_UNSUPPORTED, "tail strips are a 2D sweep feature");
    SM_CUDA(cudaStreamSynchronize(p->stream));
    return apply_tiling(p, p->W, p->S, -1, n);
}

sm_status sm_set_emission_warps(sm_problem *p, int warps) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    if (p->batch_owned)
        return fail(SM_ERR_INVALID_ARG, "this problem belongs to a batch: sweep it with sm_batch_sweep");
    if (warps < 0 || warps > 4) return fail(SM_ERR_INVALID_ARG, "emission warps must be in 0..4");
    if (p->dim == 1)
        return warps == 0 ? SM_OK
                          : fail(SM_ERR_UNSUPPORTED, "fused emission is a 2D sweep feature");
    SM_CUDA(cudaStreamSynchronize(p->stream));
    return apply_tiling(p, p->W, p->S, warps);
}

sm_status sm_get_quadrature(const sm_problem *p, double *omx, double *omy, double *w) {
    if (!p || !omx || !omy || !w) return fail(SM_ERR_INVALID_ARG, "NULL argument");
    std::copy(p->omx.begin(), p->omx.end(), omx);
    std::copy(p->omy.begin(), p->omy.end(), omy);
    std::copy(p->w.begin(), p->w.end(), w);
    return SM_OK;
}

sm_status sm_opacity(sm_problem *p, const double *T, const double *scale, double *sigma) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    sm_status st;
    if ((st = check_ptr(T, "T_nodal_dev")) || (st = check_ptr(scale, "scale_dev")) ||
        (st = check_ptr(sigma, "sigma_dev")))
        return st;
    SM_CUDA(smk::launch_opacity(p, T, scale, sigma, p->stream));
    p->launches++;
    return SM_OK;
}

sm_status sm_emission(sm_problem *p, const double *T, const double *sigma, double *q) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    sm_status st;
    if ((st = check_ptr(T, "T_nodal_dev")) || (st = check_ptr(sigma, "sigma_dev"))) return st;
    SM_CUDA(smk::launch_emission(p, T, sigma, q, p->stream));
    p->launches++;
    return SM_OK;
}

sm_status sm_sweep(sm_problem *p, const double *T, const double *sigma, const void *I_prev,
                   void *I_out, double *mom, double *clo) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    if (p->batch_owned)
        return fail(SM_ERR_INVALID_ARG, "this problem belongs to a batch: sweep it with sm_batch_sweep");
    sm_status st;
    if ((st = check_ptr(T, "T_nodal_dev")) || (st = check_ptr(sigma, "sigma_dev")) ||
        (st = check_ptr(I_out, "I_out_dev")))
        return st;
    if (I_prev == I_out) return fail(SM_ERR_INVALID_ARG, "I_prev_dev must not alias I_out_dev");
    if ((st = check_intensity_align(I_prev, I_out))) return st;
    return run_sweep(p, T, sigma, I_prev, I_out, mom, clo);
}

sm_status sm_closures(sm_problem *p, const double *mom, const double *T, const double *sigma,
                      double *clo) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    sm_status st;
    if ((st = check_ptr(mom, "moments_dev")) || (st = check_ptr(T, "T_nodal_dev")) ||
        (st = check_ptr(sigma, "sigma_dev")) || (st = check_ptr(clo, "closures_dev")))
        return st;
    SM_CUDA(smk::launch_closures_from_T(p, mom, T, sigma, clo, p->stream));
    p->launches++;
    return SM_OK;
}

sm_status sm_sweep_host(sm_problem *p, const double *T_host, const double *sigma_host,
                        const void *I_prev, void *I_out, double *mom_host, double *clo_host) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    if (p->batch_owned)
        return fail(SM_ERR_INVALID_ARG, "this problem belongs to a batch: sweep it with sm_batch_sweep");
    sm_status st;
    if ((st = check_ptr(T_host, "T_nodal_host")) || (st = check_ptr(sigma_host, "sigma_host")) ||
        (st = check_ptr(I_out, "I_out_dev")))
        return st;
    if (I_prev == I_out) return fail(SM_ERR_INVALID_ARG, "I_prev_dev must not alias I_out_dev");
    if ((st = check_intensity_align(I_prev, I_out))) return st;
    cudaStream_t s = p->stream;
    const size_t tb = (size_t)p->ncell * p->nn * sizeof(double);
    const size_t sb = (size_t)p->G * p->ncell * sizeof(double);
    SM_CUDA(cudaMemcpyAsync(p->d_T_tmp, T_host, tb, cudaMemcpyHostToDevice, s));
    SM_CUDA(cudaMemcpyAsync(p->d_sig_tmp, sigma_host, sb, cudaMemcpyHostToDevice, s));
    st = run_sweep(p, p->d_T_tmp, p->d_sig_tmp, I_prev, I_out, p->d_mom_tmp,
                   clo_host ? p->d_clo_tmp : nullptr);
    if (st) return st;
    if (mom_host)
        SM_CUDA(cudaMemcpyAsync(mom_host, p->d_mom_tmp,
                                (size_t)p->ncell * p->nn * p->nm * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
    if (clo_host)
        SM_CUDA(cudaMemcpyAsync(clo_host, p->d_clo_tmp,
                                (size_t)p->ncell * p->nn * p->nc * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
    return sm_synchronize(p);
}

sm_status sm_pack_intensity(sm_problem *p, const double *canon, void *packed) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    sm_status st;
    if ((st = check_ptr(canon, "I_canon_dev")) || (st = check_ptr(packed, "I_packed_dev")))
        return st;
    SM_CUDA(smk::launch_pack(p, canon, packed, 0, p->stream));
    p->launches++;
    return SM_OK;
}

sm_status sm_unpack_intensity(sm_problem *p, const void *packed, double *canon) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    sm_status st;
    if ((st = check_ptr(canon, "I_canon_dev")) || (st = check_ptr(packed, "I_packed_dev")))
        return st;
    SM_CUDA(smk::launch_pack(p, canon, const_cast<void *>(packed), 1, p->stream));
    p->launches++;
    return SM_OK;
}

sm_status sm_synchronize(sm_problem *p) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    SM_CUDA(cudaStreamSynchronize(p->stream));
    unsigned int ctrl[smk::CTRL_WORDS];
    SM_CUDA(cudaMemcpy(ctrl, p->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost));
    const unsigned int status = ctrl[smk::CTRL_STATUS];
    if (status) {
        SM_CUDA(cudaMemset(p->d_ctrl + smk::CTRL_STATUS, 0, sizeof(unsigned int)));
        if (status & smk::ST_TIMEOUT)
            return fail(SM_ERR_TIMEOUT, "a wavefront wait exceeded its time limit");
        return fail(SM_ERR_NONPHYSICAL, "non-positive or non-finite temperature");
    }
    return SM_OK;
}

sm_status sm_set_quadrant_moments(sm_problem *p, double *qmom_dev) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    if (p->batch_owned) return fail(SM_ERR_INVALID_ARG, "this problem belongs to a batch");
    SM_CUDA(cudaStreamSynchronize(p->stream));
    // the partial moments are kept per warp task, hence per quadrant: the
    // reduction forms the quadrant sums from them
    p->qmom_dev = qmom_dev;
    return SM_OK;
}

sm_status sm_set_profiling(sm_problem *p, int enable) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    SM_CUDA(cudaStreamSynchronize(p->stream));
    p->profiling = enable != 0;
    p->n_timed = 0;
    return SM_OK;
}

sm_status sm_get_kernel_times(sm_problem *p, double *ms, int *count) {
    if (!p || !ms || !count) return fail(SM_ERR_INVALID_ARG, "NULL argument");
    SM_CUDA(cudaStreamSynchronize(p->stream));
    ms[0] = ms[1] = ms[2] = 0.0;
    for (int n = 0; n < p->n_timed; ++n) {
        cudaEvent_t *ev = &p->ev_pool[4 * n];
        for (int k = 0; k < 3; ++k) {
            float t = 0.f;
            SM_CUDA(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
            ms[k] += t;
        }
    }
    *count = p->n_timed;
    p->n_timed = 0;
    return SM_OK;
}

int64_t sm_launch_count(const sm_problem *p) { return p ? p->launches : 0; }

sm_status sm_autotune(sm_problem *p, const double *T, const double *sigma, const void *I_prev,
                      void *I_out, int reps) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    if (p->batch_owned)
        return fail(SM_ERR_INVALID_ARG, "this problem belongs to a batch: sweep it with sm_batch_sweep");
    sm_status st;
    if ((st = check_ptr(T, "T_nodal_dev")) || (st = check_ptr(sigma, "sigma_dev")) ||
        (st = check_ptr(I_out, "I_out_dev")))
        return st;
    if (p->dim == 1) return SM_OK;
    if (I_prev == I_out) return fail(SM_ERR_INVALID_ARG, "I_prev_dev must not alias I_out_dev");
    if ((st = check_intensity_align(I_prev, I_out))) return st;
    if (reps < 1) reps = 3;
    // strip width x prefetch depth x fused emission warps (0: the emission
    // kernel runs before the sweep) x half-width end strips (with the
    // separate emission kernel only)
    const int w_c[] = {2, 4, 6, 8, 12, 14, 16};
    const int s_c[] = {2, 3, 4};
    const int e_c[] = {0, 2, 4};
    const int t_c[] = {0, 1, 2};
    int best_w = p->W, best_s = p->S, best_e = p->emit_warps, best_t = p->tail;
    float best_ms = 1e30f;
    const bool prof = p->profiling;
    p->profiling = false;
    cudaEvent_t a, b;
    SM_CUDA(cudaEventCreate(&a));
    SM_CUDA(cudaEventCreate(&b));
    for (int wc : w_c) {
        if (wc > p->nx && wc != 2) continue;
        for (int sc : s_c) {
            for (int ec : e_c) {
                if (wc + ec > 16) continue;
                for (int tc : t_c) {
                    if (tc > 0 && ec > 0) continue;
                    if (apply_tiling(p, wc, sc, ec, tc) != SM_OK) continue;
                    if (p->tail != tc) continue;  // that layout does not exist here
                    st = run_sweep(p, T, sigma, I_prev, I_out, nullptr, nullptr);  // warm-up
                    if (st) break;
                    SM_CUDA(cudaEventRecord(a, p->stream));
                    for (int r = 0; r < reps && !st; ++r)
                        st = run_sweep(p, T, sigma, I_prev, I_out, nullptr, nullptr);
                    SM_CUDA(cudaEventRecord(b, p->stream));
                    SM_CUDA(cudaEventSynchronize(b));
                    float ms = 0;
                    SM_CUDA(cudaEventElapsedTime(&ms, a, b));
                    if (st == SM_OK && ms < best_ms) {
                        best_ms = ms;
                        best_w = p->W;
                        best_s = p->S;
                        best_e = p->emit_warps;
                        best_t = p->tail;
                    }
                }
                if (st) break;
            }
            if (st) break;
        }
        if (st) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    p->profiling = prof;
    sm_status sync = sm_synchronize(p);
    sm_status fin = apply_tiling(p, best_w, best_s, best_e, best_t);
    if (st) return st;
    if (sync) return sync;
    return fin;
}

// Test hooks (not part of the public header): shorten the wavefront wait
// limit and make the first strip of every chain withhold its row counters,
// so that a test can exercise the bounded-wait / status path without any
// fault.  Both are host-side settings of this problem only.
sm_status sm_debug_set_wait_limit_ns(sm_problem *p, long long ns) {
    if (!p || ns <= 0) return fail(SM_ERR_INVALID_ARG, "bad argument");
    p->timeout_ns = ns;
    return SM_OK;
}
sm_status sm_debug_skip_publish(sm_problem *p, int enable) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    p->fault_skip_publish = enable != 0;
    return SM_OK;
}
sm_status sm_debug_withhold_lo_block(sm_problem *p, int enable) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    p->fault_withhold_block = enable != 0;
    return SM_OK;
}

sm_status sm_debug_set_pcg_form(sm_problem *p, int form) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    if (form != SM_DEBUG_PCG_AUTO && form != SM_DEBUG_PCG_TEXTBOOK && form != SM_DEBUG_PCG_SINGLE &&
        form != SM_DEBUG_PCG_MIXED)
        return fail(SM_ERR_INVALID_ARG, "form must be SM_DEBUG_PCG_AUTO, _TEXTBOOK, _SINGLE or _MIXED");
    p->lo_pcg_form = form;
    return SM_OK;
}

sm_status sm_debug_set_emission_fp64(sm_problem *p, int fp64) {
    if (!p) return fail(SM_ERR_INVALID_ARG, "NULL problem");
    p->emit_fp64 = fp64 != 0;
    return SM_OK;
}

sm_status sm_debug_get_pcg_form(const sm_problem *p, int *form) {
    if (!p || !form) return fail(SM_ERR_INVALID_ARG, "NULL problem or output");
    *form = p->lo_pcg_form_used;
    return SM_OK;
}

}  // extern "C"

namespace smk {
sm_status create_batch_member(const sm_problem_desc *d, void *stream, sm_problem **out) {
    return create_problem(d, stream, out, 0);
}
}  // namespace smk
