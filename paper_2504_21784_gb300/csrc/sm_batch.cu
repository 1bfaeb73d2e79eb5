// Many independent 2D problems (uneven meshes, group and direction counts)
// swept in one persistent launch.  The batch owns one sm_problem per member
// for its per-problem data (sources, lane constants, inflow, face buffers,
// row counters, moment accumulators); the sweep of every member runs in one
// launch of sweep2d_batch_kernel, whose CTAs take (problem, task) items from
// one queue.  The whole pass -- a one-thread prologue (task queue, abort flag,
// epoch), per-problem emission, the batched sweep, per-problem moment sums
// and closures -- is recorded once as a CUDA graph for a
// given set of caller buffers and replayed afterwards; per-problem kernels sit
// on parallel branches of the graph so that small members run concurrently.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "sm_internal.cuh"

namespace smk {

// Resets the batch's task queue and abort flag and advances its epoch (the
// row counters of every member are tagged with it).
__global__ void batch_prologue_kernel(unsigned int *ctrl, unsigned long long *epoch) {
    ctrl[CTRL_QUEUE] = 0u;
    ctrl[CTRL_ABORT] = 0u;
    *epoch += 1ull;
}

}  // namespace smk

struct sm_batch {
    std::vector<sm_problem *> probs;
    int prec = 32;
    cudaStream_t stream = nullptr;   // the caller's stream
    cudaStream_t cap = nullptr;      // private stream for graph capture
    std::vector<cudaStream_t> side;  // branches of the per-problem work
    std::vector<cudaEvent_t> ev;     // fork / join events
    unsigned int *d_ctrl = nullptr;  // [CTRL_WORDS], shared with every member
    unsigned long long *d_epoch = nullptr;
    int *d_active = nullptr;         // [n] member swept by the next pass (1) or skipped (0)
    bool all_active = true;          // d_active holds all ones
    int2 *d_tasks = nullptr;
    int n_tasks = 0, tasks_cap = 0;
    int W = 8, S = 2, ring_gw = 1, resident = 0;
    size_t stg = 0, smem = 0;
    double updates = 0.0;
    struct Entry {
        std::vector<uintptr_t> key;
        smk::SweepArgs *d_args = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        unsigned long long last_use = 0;
    };
    std::vector<Entry> cache;
    unsigned long long clock = 0;
    long long launches = 0;
    // profiling: passes run live (not from a graph) with 4 events each around
    // the emission, the batched sweep and the reductions
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    int n_timed = 0;
    smk::SweepArgs *d_args_live = nullptr;
    void *lo_scratch = nullptr;  // the batched low-order launch's arguments (sm_lo.cu)
    int lo_batched = 1;          // low-order solves in one launch (1) or one per member (0)
};

namespace {

constexpr int N_SIDE = 8;     // parallel branches for the per-problem kernels
constexpr int CACHE_MAX = 4;  // graphs kept (e.g. the two buffer roles of a time loop)

sm_status b_fail(sm_status s, const std::string &m) {
    smk::set_last_error(m.c_str());
    return s;
}

#define B_CUDA(call)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return b_fail(e_ == cudaErrorMemoryAllocation ? SM_ERR_OOM : SM_ERR_CUDA,  \
                          std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)
#define B_TRY(expr)                 \
    do {                            \
        sm_status s_ = (expr);      \
        if (s_ != SM_OK) return s_; \
    } while (0)

void drop_entry(sm_batch::Entry &e) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.graph) cudaGraphDestroy(e.graph);
    if (e.d_args) cudaFree(e.d_args);
    e = sm_batch::Entry();
}

void clear_cache(sm_batch *b) {
    for (auto &e : b->cache) drop_entry(e);
    b->cache.clear();
}

// Tiling of every member, the shared-memory layout of the batched kernel
// (largest stage and x-face ring of the batch) and the merged task order.
sm_status set_tiling(sm_batch *b, int W, int S) {
    B_CUDA(cudaStreamSynchronize(b->stream));
    clear_cache(b);
    size_t stg = 0;
    int ring_gw = 1;
    for (sm_problem *p : b->probs) {
        B_TRY(smk::apply_tiling_ext(p, W, S));
        stg = std::max(stg, smk::sweep2d_stage_bytes(b->prec, p->GW, p->GSLOT));
        ring_gw = std::max(ring_gw, p->GW);
    }
    const size_t smem = smk::sweep2d_batch_smem_bytes(b->prec, W, S, stg, ring_gw);
    const int resident = smk::sweep2d_batch_max_resident(b->prec, W, smem);
    if (resident <= 0)
        return b_fail(SM_ERR_UNSUPPORTED, "batched tiling needs " + std::to_string(smem) +
                                              " B of shared memory per CTA (too much)");
    // Merge the members' task lists by their relative position (task + 1/2)
    // / n_tasks: each member keeps its own upwind order, which is all the
    // queue needs to be free of deadlock, and the members progress together.
    struct Item {
        double key;
        int p, t;
    };
    std::vector<Item> items;
    for (int i = 0; i < (int)b->probs.size(); ++i) {
        const sm_problem *p = b->probs[i];
        const int n = p->NS * p->NQ * p->NWT;
        for (int t = 0; t < n; ++t) items.push_back({(t + 0.5) / n, i, t});
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const Item &a, const Item &c) { return a.key < c.key; });
    std::vector<int2> tasks(items.size());
    for (size_t k = 0; k < items.size(); ++k) tasks[k] = make_int2(items[k].p, items[k].t);
    if ((int)tasks.size() > b->tasks_cap) {
        if (b->d_tasks) cudaFree(b->d_tasks);
        b->d_tasks = nullptr;
        B_CUDA(cudaMalloc(&b->d_tasks, sizeof(int2) * tasks.size()));
        b->tasks_cap = (int)tasks.size();
    }
    B_CUDA(cudaMemcpy(b->d_tasks, tasks.data(), sizeof(int2) * tasks.size(),
                      cudaMemcpyHostToDevice));
    b->n_tasks = (int)tasks.size();
    b->W = W;
    b->S = S;
    b->stg = stg;
    b->ring_gw = ring_gw;
    b->smem = smem;
    b->resident = resident;
    return SM_OK;
}

struct Ptrs {
    const double *const *T;
    const double *const *sigma;
    const void *const *I_prev;
    void *const *I_out;
    double *const *mom;
    double *const *clo;
};

sm_status check_ptrs(const sm_batch *b, const Ptrs &q) {
    if (!q.T || !q.sigma || !q.I_out)
        return b_fail(SM_ERR_INVALID_ARG, "T, sigma and I_out pointer arrays are required");
    for (size_t i = 0; i < b->probs.size(); ++i) {
        if (!q.T[i] || !q.sigma[i] || !q.I_out[i])
            return b_fail(SM_ERR_INVALID_ARG,
                          "problem " + std::to_string(i) + ": T, sigma and I_out must be non-NULL");
        const void *ip = q.I_prev ? q.I_prev[i] : nullptr;
        if ((reinterpret_cast<uintptr_t>(ip) & 15u) ||
            (reinterpret_cast<uintptr_t>(q.I_out[i]) & 15u))
            return b_fail(SM_ERR_INVALID_ARG, "packed intensity buffers must be 16-byte aligned");
        if (ip && ip == q.I_out[i])
            return b_fail(SM_ERR_INVALID_ARG, "I_prev and I_out must not alias");
    }
    return SM_OK;
}

std::vector<uintptr_t> make_key(const sm_batch *b, const Ptrs &q) {
    std::vector<uintptr_t> k;
    const size_t n = b->probs.size();
    k.reserve(6 * n);
    for (size_t i = 0; i < n; ++i) {
        k.push_back(reinterpret_cast<uintptr_t>(q.T[i]));
        k.push_back(reinterpret_cast<uintptr_t>(q.sigma[i]));
        k.push_back(reinterpret_cast<uintptr_t>(q.I_prev ? q.I_prev[i] : nullptr));
        k.push_back(reinterpret_cast<uintptr_t>(q.I_out[i]));
        k.push_back(reinterpret_cast<uintptr_t>(q.mom ? q.mom[i] : nullptr));
        k.push_back(reinterpret_cast<uintptr_t>(q.clo ? q.clo[i] : nullptr));
    }
    return k;
}

// The members' sweep arguments for the buffers q.
std::vector<smk::SweepArgs> member_args(const sm_batch *b, const Ptrs &q) {
    const size_t n = b->probs.size();
    std::vector<smk::SweepArgs> args(n);
    for (size_t i = 0; i < n; ++i) {
        args[i] = smk::make_sweep_args(b->probs[i], q.I_prev ? q.I_prev[i] : nullptr, q.I_out[i]);
        args[i].ctrl = b->d_ctrl;
        args[i].active = b->d_active + i;
        // the members share one queue: the batch's task count decides
        args[i].publish = smk::publish_rows(b->n_tasks, b->resident);
    }
    return args;
}

// Enqueues one pass on stream c (being captured, or live): prologue,
// per-problem emission on parallel branches, the batched
// sweep, per-problem moment sums and closures.  ev (live profiling only):
// four timing events recorded before the emissions, around the sweep and
// after the reductions.
sm_status enqueue_pass(sm_batch *b, const Ptrs &q, const smk::SweepArgs *d_args,
                       cudaStream_t c, cudaEvent_t *ev) {
    const size_t n = b->probs.size();
    smk::BatchSweepArgs B;
    B.args = d_args;
    B.tasks = b->d_tasks;
    B.n_tasks = b->n_tasks;
    B.W = b->W;
    B.S = b->S;
    B.ring_gw = b->ring_gw;
    B.stg = b->stg;
    B.ctrl = b->d_ctrl;
    B.epoch = b->d_epoch;
    const int grid = std::min(b->n_tasks, b->resident);
    if (ev) B_CUDA(cudaEventRecord(ev[0], c));
    smk::batch_prologue_kernel<<<1, 1, 0, c>>>(b->d_ctrl, b->d_epoch);
    // per-problem emission on parallel branches
    B_CUDA(cudaEventRecord(b->ev[0], c));
    for (int k = 0; k < N_SIDE; ++k) B_CUDA(cudaStreamWaitEvent(b->side[k], b->ev[0], 0));
    for (size_t i = 0; i < n; ++i) {
        sm_problem *p = b->probs[i];
        cudaStream_t s = b->side[i % N_SIDE];
        B_CUDA(smk::launch_emission(p, q.T[i], q.sigma[i], nullptr, s, b->d_active + i));
    }
    for (int k = 0; k < N_SIDE; ++k) {
        B_CUDA(cudaEventRecord(b->ev[1 + k], b->side[k]));
        B_CUDA(cudaStreamWaitEvent(c, b->ev[1 + k], 0));
    }
    if (ev) B_CUDA(cudaEventRecord(ev[1], c));
    B_CUDA(smk::launch_sweep2d_batch(b->prec, B, grid, b->smem, c));
    if (ev) B_CUDA(cudaEventRecord(ev[2], c));
    // per-problem moment sums and closures
    B_CUDA(cudaEventRecord(b->ev[0], c));
    for (int k = 0; k < N_SIDE; ++k) B_CUDA(cudaStreamWaitEvent(b->side[k], b->ev[0], 0));
    for (size_t i = 0; i < n; ++i) {
        sm_problem *p = b->probs[i];
        double *m = (q.mom && q.mom[i]) ? q.mom[i] : p->d_mom_tmp;
        B_CUDA(smk::launch_reduce(p, p->d_mom_acc, p->NQ * p->NWT, m, q.clo ? q.clo[i] : nullptr,
                                  b->side[i % N_SIDE], nullptr, p->NWT, b->d_active + i));
    }
    for (int k = 0; k < N_SIDE; ++k) {
        B_CUDA(cudaEventRecord(b->ev[1 + k], b->side[k]));
        B_CUDA(cudaStreamWaitEvent(c, b->ev[1 + k], 0));
    }
    if (ev) B_CUDA(cudaEventRecord(ev[3], c));
    return SM_OK;
}

// Records the pass for the buffers q into a graph.
sm_status record(sm_batch *b, const Ptrs &q, sm_batch::Entry &e) {
    const size_t n = b->probs.size();
    const std::vector<smk::SweepArgs> args = member_args(b, q);
    B_CUDA(cudaMalloc(&e.d_args, sizeof(smk::SweepArgs) * n));
    B_CUDA(cudaMemcpy(e.d_args, args.data(), sizeof(smk::SweepArgs) * n, cudaMemcpyHostToDevice));
    cudaStream_t c = b->cap;
    B_CUDA(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal));
    const sm_status st = enqueue_pass(b, q, e.d_args, c, nullptr);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c, &g);
    e.graph = g;
    if (st != SM_OK) return st;
    B_CUDA(ce);
    B_CUDA(cudaGraphInstantiate(&e.exec, e.graph, 0));
    return SM_OK;
}

// One pass launched directly on the batch's stream with timing events.
sm_status run_live(sm_batch *b, const Ptrs &q) {
    const size_t n = b->probs.size();
    if (!b->d_args_live) B_CUDA(cudaMalloc(&b->d_args_live, sizeof(smk::SweepArgs) * n));
    const std::vector<smk::SweepArgs> args = member_args(b, q);
    // from pageable memory: staged before the call returns
    B_CUDA(cudaMemcpyAsync(b->d_args_live, args.data(), sizeof(smk::SweepArgs) * n,
                           cudaMemcpyHostToDevice, b->stream));
    cudaEvent_t *ev = nullptr;
    if (b->n_timed < 4096) {
        while ((int)b->ev_pool.size() < 4 * (b->n_timed + 1)) {
            cudaEvent_t e;
            B_CUDA(cudaEventCreate(&e));
            b->ev_pool.push_back(e);
        }
        ev = &b->ev_pool[4 * b->n_timed++];
    }
    B_TRY(enqueue_pass(b, q, b->d_args_live, b->stream, ev));
    b->launches += 2 + 2 * (long long)n;
    return SM_OK;
}

// Which members the next pass sweeps (one flag per member; NULL: all).  The
// flags live on the device, so the recorded graphs stay valid.
sm_status set_active(sm_batch *b, const unsigned char *active) {
    const size_t n = b->probs.size();
    bool all = true;
    if (active)
        for (size_t i = 0; i < n; ++i) all = all && active[i];
    if (all && b->all_active) return SM_OK;
    std::vector<int> v(n, 1);
    if (active)
        for (size_t i = 0; i < n; ++i) v[i] = active[i] ? 1 : 0;
    // from pageable memory: the call returns once v has been staged
    B_CUDA(cudaMemcpyAsync(b->d_active, v.data(), sizeof(int) * n, cudaMemcpyHostToDevice,
                           b->stream));
    b->all_active = all;
    return SM_OK;
}

sm_status run(sm_batch *b, const Ptrs &q) {
    if (b->profiling) return run_live(b, q);
    std::vector<uintptr_t> key = make_key(b, q);
    sm_batch::Entry *hit = nullptr;
    for (auto &e : b->cache)
        if (e.key == key) hit = &e;
    if (!hit) {
        if ((int)b->cache.size() >= CACHE_MAX) {
            auto old = std::min_element(b->cache.begin(), b->cache.end(),
                                        [](const sm_batch::Entry &x, const sm_batch::Entry &y) {
                                            return x.last_use < y.last_use;
                                        });
            B_CUDA(cudaStreamSynchronize(b->stream));
            drop_entry(*old);
            b->cache.erase(old);
        }
        sm_batch::Entry e;
        e.key = key;
        const sm_status st = record(b, q, e);
        if (st != SM_OK) {
            drop_entry(e);
            return st;
        }
        b->cache.push_back(e);
        hit = &b->cache.back();
    }
    hit->last_use = ++b->clock;
    B_CUDA(cudaGraphLaunch(hit->exec, b->stream));
    b->launches += 2 + 2 * (long long)b->probs.size();
    return SM_OK;
}

}  // namespace

namespace smk {
const std::vector<sm_problem *> &batch_members(const sm_batch *b) { return b->probs; }
cudaStream_t batch_stream(const sm_batch *b) { return b->stream; }
void *&batch_lo_scratch(sm_batch *b) { return b->lo_scratch; }
int &batch_lo_mode(sm_batch *b) { return b->lo_batched; }
sm_status batch_pass(sm_batch *b, const double *const *T, const double *const *sigma,
                     const void *const *I_prev, void *const *I_out, double *const *mom,
                     double *const *clo, const unsigned char *active_host) {
    const Ptrs q{T, sigma, I_prev, I_out, mom, clo};
    B_TRY(check_ptrs(b, q));
    B_TRY(set_active(b, active_host));
    return run(b, q);
}
sm_status batch_status(sm_batch *b) {
    unsigned int status = 0;
    B_CUDA(cudaMemcpyAsync(&status, b->d_ctrl + smk::CTRL_STATUS, sizeof(status),
                           cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(cudaStreamSynchronize(b->stream));
    if (!status) return SM_OK;
    B_CUDA(cudaMemsetAsync(b->d_ctrl + smk::CTRL_STATUS, 0, sizeof(unsigned int), b->stream));
    if (status & smk::ST_TIMEOUT)
        return b_fail(SM_ERR_TIMEOUT, "a wavefront wait exceeded its time limit");
    return b_fail(SM_ERR_NONPHYSICAL, "non-positive or non-finite temperature");
}
}  // namespace smk

extern "C" {

sm_status sm_create_batch(const sm_problem_desc *descs, int n, void *stream, sm_batch **out) {
    if (!descs || !out || n < 1)
        return b_fail(SM_ERR_INVALID_ARG, "descs, out and n >= 1 are required");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (descs[i].dim != 2)
            return b_fail(SM_ERR_INVALID_ARG, "batched problems must be 2D");
        if (descs[i].precision != descs[0].precision)
            return b_fail(SM_ERR_INVALID_ARG, "batched problems must share one precision");
    }
    sm_batch *b = new sm_batch();
    b->prec = descs[0].precision;
    b->stream = static_cast<cudaStream_t>(stream);
    auto bail = [&](sm_status s) {
        sm_destroy_batch(b);
        return s;
    };
    const std::vector<int> ones(n, 1);
    if (cudaMalloc(&b->d_ctrl, smk::CTRL_WORDS * sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&b->d_epoch, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&b->d_active, sizeof(int) * n) != cudaSuccess ||
        cudaMemcpy(b->d_active, ones.data(), sizeof(int) * n, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(b->d_ctrl, 0, smk::CTRL_WORDS * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(b->d_epoch, 0, sizeof(unsigned long long)) != cudaSuccess)
        return bail(b_fail(SM_ERR_OOM, "batch control words"));
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(b_fail(SM_ERR_CUDA, "capture stream"));
    b->side.resize(N_SIDE, nullptr);
    for (auto &s : b->side)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return bail(b_fail(SM_ERR_CUDA, "branch stream"));
    b->ev.resize(1 + N_SIDE, nullptr);
    for (auto &e : b->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return bail(b_fail(SM_ERR_CUDA, "fork event"));
    for (int i = 0; i < n; ++i) {
        sm_problem *p = nullptr;
        const sm_status st = smk::create_batch_member(&descs[i], stream, &p);
        if (st != SM_OK) return bail(st);
        // the member reports to the batch's control words
        cudaFree(p->d_ctrl);
        p->d_ctrl = b->d_ctrl;
        p->ctrl_borrowed = true;
        p->batch_owned = true;
        b->probs.push_back(p);
        b->updates += (double)p->ncell * p->nd * p->G;
    }
    const sm_status st = set_tiling(b, 8, 2);
    if (st != SM_OK) {
        const sm_status st2 = set_tiling(b, 4, 2);
        if (st2 != SM_OK) return bail(st2);
    }
    *out = b;
    return SM_OK;
}

sm_status sm_destroy_batch(sm_batch *b) {
    if (!b) return SM_OK;
    cudaStreamSynchronize(b->stream);
    clear_cache(b);
    for (sm_problem *p : b->probs) {
        p->batch_owned = false;
        sm_destroy_problem(p);
    }
    for (auto s : b->side)
        if (s) cudaStreamDestroy(s);
    for (auto e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->d_tasks) cudaFree(b->d_tasks);
    if (b->d_ctrl) cudaFree(b->d_ctrl);
    if (b->d_epoch) cudaFree(b->d_epoch);
    if (b->d_active) cudaFree(b->d_active);
    if (b->d_args_live) cudaFree(b->d_args_live);
    for (auto e : b->ev_pool) cudaEventDestroy(e);
    smk::batch_lo_free(b->lo_scratch);
    delete b;
    return SM_OK;
}

sm_status sm_debug_set_batch_lo(sm_batch *b, int batched) {
    if (!b) return b_fail(SM_ERR_INVALID_ARG, "NULL batch");
    b->lo_batched = batched != 0;
    return SM_OK;
}

sm_status sm_batch_problem(sm_batch *b, int i, sm_problem **out) {
    if (!b || !out || i < 0 || i >= (int)b->probs.size())
        return b_fail(SM_ERR_INVALID_ARG, "batch member index out of range");
    *out = b->probs[i];
    return SM_OK;
}

sm_status sm_batch_get_info(const sm_batch *b, sm_batch_info *o) {
    if (!b || !o) return b_fail(SM_ERR_INVALID_ARG, "NULL argument");
    o->n_problems = (int)b->probs.size();
    o->n_tasks = b->n_tasks;
    o->strip_width = b->W;
    o->prefetch_rows = b->S;
    o->resident_ctas = b->resident;
    o->graphs_cached = (int)b->cache.size();
    o->smem_bytes = b->smem;
    o->updates = b->updates;
    o->launches = b->launches;
    return SM_OK;
}

sm_status sm_batch_set_stream(sm_batch *b, void *stream) {
    if (!b) return b_fail(SM_ERR_INVALID_ARG, "NULL batch");
    b->stream = static_cast<cudaStream_t>(stream);
    for (sm_problem *p : b->probs) p->stream = b->stream;
    return SM_OK;
}

sm_status sm_batch_set_tiling(sm_batch *b, int strip_width, int prefetch_rows) {
    if (!b) return b_fail(SM_ERR_INVALID_ARG, "NULL batch");
    return set_tiling(b, strip_width > 0 ? strip_width : b->W,
                      prefetch_rows > 0 ? prefetch_rows : b->S);
}

sm_status sm_batch_sweep(sm_batch *b, const double *const *T_dev, const double *const *sigma_dev,
                         const void *const *I_prev_dev, void *const *I_out_dev,
                         double *const *moments_dev, double *const *closures_dev) {
    if (!b) return b_fail(SM_ERR_INVALID_ARG, "NULL batch");
    const Ptrs q{T_dev, sigma_dev, I_prev_dev, I_out_dev, moments_dev, closures_dev};
    B_TRY(check_ptrs(b, q));
    B_TRY(set_active(b, nullptr));
    return run(b, q);
}

sm_status sm_batch_synchronize(sm_batch *b) {
    if (!b) return b_fail(SM_ERR_INVALID_ARG, "NULL batch");
    B_CUDA(cudaStreamSynchronize(b->stream));
    unsigned int ctrl[smk::CTRL_WORDS];
    B_CUDA(cudaMemcpy(ctrl, b->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost));
    const unsigned int status = ctrl[smk::CTRL_STATUS];
    if (status) {
        B_CUDA(cudaMemset(b->d_ctrl + smk::CTRL_STATUS, 0, sizeof(unsigned int)));
        if (status & smk::ST_TIMEOUT)
            return b_fail(SM_ERR_TIMEOUT, "a wavefront wait exceeded its time limit");
        return b_fail(SM_ERR_NONPHYSICAL, "non-positive or non-finite temperature");
    }
    return SM_OK;
}

sm_status sm_batch_set_profiling(sm_batch *b, int enable) {
    if (!b) return b_fail(SM_ERR_INVALID_ARG, "NULL batch");
    B_CUDA(cudaStreamSynchronize(b->stream));
    b->profiling = enable != 0;
    b->n_timed = 0;
    return SM_OK;
}

sm_status sm_batch_get_kernel_times(sm_batch *b, double *ms, int *count) {
    if (!b || !ms || !count) return b_fail(SM_ERR_INVALID_ARG, "NULL argument");
    B_CUDA(cudaStreamSynchronize(b->stream));
    ms[0] = ms[1] = ms[2] = 0.0;
    for (int k = 0; k < b->n_timed; ++k) {
        cudaEvent_t *ev = &b->ev_pool[4 * k];
        for (int j = 0; j < 3; ++j) {
            float t = 0.f;
            B_CUDA(cudaEventElapsedTime(&t, ev[j], ev[j + 1]));
            ms[j] += t;
        }
    }
    *count = b->n_timed;
    b->n_timed = 0;
    return SM_OK;
}

sm_status sm_batch_autotune(sm_batch *b, const double *const *T_dev,
                            const double *const *sigma_dev, const void *const *I_prev_dev,
                            void *const *I_out_dev, int reps) {
    if (!b) return b_fail(SM_ERR_INVALID_ARG, "NULL batch");
    const Ptrs q{T_dev, sigma_dev, I_prev_dev, I_out_dev, nullptr, nullptr};
    B_TRY(check_ptrs(b, q));
    B_TRY(set_active(b, nullptr));
    if (reps < 1) reps = 1;
    cudaEvent_t e0, e1;
    B_CUDA(cudaEventCreate(&e0));
    B_CUDA(cudaEventCreate(&e1));
    const int Ws[] = {2, 4, 6, 8, 12, 16};
    const int Ss[] = {2, 3, 4};
    float best = 1e30f;
    int bW = b->W, bS = b->S;
    sm_status result = SM_OK;
    for (int W : Ws) {
        for (int S : Ss) {
            if (set_tiling(b, W, S) != SM_OK) continue;
            if ((result = run(b, q)) != SM_OK) break;  // records the graph, warms up
            cudaEventRecord(e0, b->stream);
            for (int r = 0; r < reps && result == SM_OK; ++r) result = run(b, q);
            cudaEventRecord(e1, b->stream);
            if (result != SM_OK) break;
            if ((result = sm_batch_synchronize(b)) != SM_OK) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bW = W;
                bS = S;
            }
        }
        if (result != SM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const sm_status st = set_tiling(b, bW, bS);
    return result != SM_OK ? result : st;
}

sm_status sm_batch_tune_slots(const sm_problem_desc *descs, int n, void *stream, int reps,
                              int *gw_out) {
    if (!descs || n < 1 || !gw_out) return b_fail(SM_ERR_INVALID_ARG, "descs, n >= 1, gw_out");
    if (reps < 1) reps = 1;
    // every member's automatic choice (the largest that its groups fill)
    std::vector<int> auto_gw(n);
    {
        sm_batch *b = nullptr;
        B_TRY(sm_create_batch(descs, n, stream, &b));
        for (int i = 0; i < n; ++i) auto_gw[i] = b->probs[i]->GW;
        sm_destroy_batch(b);
    }
    const int caps[] = {8, 4, 2, 1};
    float best = 1e30f;
    std::vector<int> best_gw(auto_gw);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    B_CUDA(cudaEventCreate(&e0));
    B_CUDA(cudaEventCreate(&e1));
    sm_status result = SM_OK;
    for (int cap : caps) {
        std::vector<sm_problem_desc> d(descs, descs + n);
        std::vector<int> gw(n);
        bool differs = cap == caps[0];
        for (int i = 0; i < n; ++i) {
            gw[i] = descs[i].groups_per_warp ? descs[i].groups_per_warp : std::min(cap, auto_gw[i]);
            d[i].groups_per_warp = gw[i];
            differs = differs || gw[i] != std::min(cap * 2, auto_gw[i]);
        }
        if (!differs) continue;  // the same layout as the previous cap
        sm_batch *b = nullptr;
        if ((result = sm_create_batch(d.data(), n, stream, &b)) != SM_OK) break;
        // synthetic inputs: T = 1 at every node, unit opacity, zero intensities
        std::vector<void *> owned;
        std::vector<const double *> T(n), sg(n);
        std::vector<const void *> Ip(n);
        std::vector<void *> Io(n);
        for (int i = 0; i < n && result == SM_OK; ++i) {
            const sm_problem *p = b->probs[i];
            const size_t nn = (size_t)p->ncell * p->nn, ng = (size_t)p->G * p->ncell;
            const size_t ib = (size_t)p->NQ * p->NWT * p->ncell * p->GW * 32 * p->nn * p->rsize;
            void *t = nullptr, *s = nullptr, *a = nullptr, *o = nullptr;
            if (cudaMalloc(&t, nn * sizeof(double)) != cudaSuccess ||
                cudaMalloc(&s, ng * sizeof(double)) != cudaSuccess ||
                cudaMalloc(&a, ib) != cudaSuccess || cudaMalloc(&o, ib) != cudaSuccess) {
                for (void *x : {t, s, a, o})
                    if (x) cudaFree(x);
                result = b_fail(SM_ERR_OOM, "slot tuning buffers");
                break;
            }
            owned.insert(owned.end(), {t, s, a, o});
            const std::vector<double> one(std::max(nn, ng), 1.0);
            cudaMemcpy(t, one.data(), nn * sizeof(double), cudaMemcpyHostToDevice);
            cudaMemcpy(s, one.data(), ng * sizeof(double), cudaMemcpyHostToDevice);
            cudaMemset(a, 0, ib);
            T[i] = static_cast<const double *>(t);
            sg[i] = static_cast<const double *>(s);
            Ip[i] = a;
            Io[i] = o;
        }
        float ms = 1e30f;
        if (result == SM_OK)
            result = sm_batch_autotune(b, T.data(), sg.data(), Ip.data(), Io.data(), 1);
        if (result == SM_OK) {
            const Ptrs q{T.data(), sg.data(), Ip.data(), Io.data(), nullptr, nullptr};
            result = run(b, q);  // warm-up (records the graph)
            cudaEventRecord(e0, b->stream);
            for (int r = 0; r < reps && result == SM_OK; ++r) result = run(b, q);
            cudaEventRecord(e1, b->stream);
            if (result == SM_OK) result = sm_batch_synchronize(b);
            if (result == SM_OK) cudaEventElapsedTime(&ms, e0, e1);
        }
        sm_destroy_batch(b);
        for (void *x : owned) cudaFree(x);
        if (result != SM_OK) break;
        if (ms < best) {
            best = ms;
            best_gw = gw;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != SM_OK) return result;
    for (int i = 0; i < n; ++i) gw_out[i] = best_gw[i];
    return SM_OK;
}

}  // extern "C"
