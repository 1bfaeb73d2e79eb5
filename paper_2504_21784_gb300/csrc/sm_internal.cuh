// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sm.h"
#include "../../include/sm_debug.h"
#include "sm_planck.cuh"

namespace smk {

// ---------------------------------------------------------------------------
// Per-lane direction constants of one warp task (quadrant, direction block).
// mu = |Omega_x|/hx, eta = |Omega_y|/hy; wm = w * {1, Ox, Oy, Ox^2-1/3,
// Ox*Oy, Oy^2-1/3} (1D: w * {1, mu, mu^2-1/3}); g_lo = group offset of the
// lane inside a lane row; valid = 0 for padding lanes.
struct LaneConst {
    double mu, eta;
    double wm[6];
    int g_lo;
    int valid;
};

// Device control block: [0] work-queue counter, [1] abort flag (both reset per
// sweep launch), [2] sticky status bits (cleared by sm_synchronize).
enum { CTRL_QUEUE = 0, CTRL_ABORT = 1, CTRL_STATUS = 2, CTRL_WORDS = 4 };
// status bits written by kernels
enum { ST_TIMEOUT = 1u, ST_NONPHYSICAL = 2u };

struct SweepArgs {
    int nx, ny, ncell;
    int NQ, NWT, NGB, DB, LG, GW, Gp;
    int W;            // 2D: cell columns per CTA = warps per CTA (1D: unused)
    int S;            // 2D: rows prefetched per warp (TMA stages)
    int NS;           // 2D: strips
    int n_tasks;      // 2D: NS * NQ * NWT
    double inv_cdt;
    const LaneConst *lanes;  // [NQ][DB][32]
    const void *src;         // [cell][Gp][8] sweep precision: q at 4 nodes, sigma~, sigma, 0, 0
    const void *inflow;      // [4][Gp]
    const void *I_prev;      // packed or null
    void *I_out;             // packed
    void *part;              // 1D: [NQ*NWT][cell][10] per-warp partial moments
    void *mom_acc;           // 2D: [NQ*NWT][cell][36] partial moments per warp task
    void *face;              // 2D: [NQ*NWT][NS][ny][GW][32][2]
    unsigned long long *flags;  // 2D: [NQ*NWT][NS]
    unsigned int *ctrl;
    unsigned long long epoch;
    long long timeout_ns;
    int fault_skip_publish;  // test hook: strip 0 never publishes
    int reverse;             // 2D: sweep -Omega for every direction; I_prev / I_out of
                             // geometric quadrant q live at quadrant q^2 (adjoint sweeps)
    int qmom;                // 2D: per-quadrant moments wanted (the partials keep them apart)
    int publish;             // 2D: rows per release of a strip's x-faces downwind
    const int *active;       // batch member: its tasks are skipped while *active == 0
                             // (NULL: always swept)
    const int *strip_x0;     // 2D: [NS + 1] first cell column of each strip and nx
                             // (NULL: strip s starts at s * W, the last one ragged)
};

// Emission fused into the 2D sweep kernel: `warps` extra warps per CTA
// compute the emission (row a1) of the strips ahead of the sweep while the
// sweep warps stream, and sweep warps whose task's strip is not ready yet help
// with it.  Work items are 8 cells (32 nodes) of one strip, taken in the
// order the strips are first needed (0, NS-1, 1, NS-2, ...: quadrants sweep
// the strips from both sides); every strip has `per_strip` items (the ragged
// last strip's surplus items are empty).  ctr[0] is the item queue and
// ctr[1 + s] the items of strip s done (zeroed before each launch).
struct EmitArgs {
    int warps;                 // 0: the emission runs as its own kernel before the sweep
    int G, Gp, ncell, nx, ny, W, NS, per_strip, items;
    double acT4_scale, inv_cdt;
    const double *edges, *T, *sigma;
    double *gray;
    unsigned int *ctr;
    long long timeout_ns;
    PlanckTabs tabs;
};

// Rows per release of a strip's x-faces to the downwind strip: the release
// costs a gpu-scope fence, so a sweep with several tasks per resident CTA
// (throughput-bound) batches 8 rows; one with fewer tasks than twice the
// resident CTAs (latency-bound: every strip of a chain in flight at once)
// releases every 2 rows to shorten the lag between strips.
inline int publish_rows(int n_tasks, int resident) { return n_tasks >= 2 * resident ? 8 : 2; }

// sm_create_problem for a batch member: the automatic slots-per-lane choice
// maximises the work per warp (the batch supplies the parallelism).
sm_status create_batch_member(const sm_problem_desc *d, void *stream, sm_problem **out);

// Many problems in one persistent 2D sweep launch (sweep2d_batch_kernel).
struct BatchSweepArgs {
    const SweepArgs *args;  // [n_problems] (their ctrl is the batch's)
    const int2 *tasks;      // [n_tasks] (problem, task of that problem)
    int n_tasks;
    int W, S, ring_gw;      // CTA width and stages; x-face ring sized for ring_gw slots
    size_t stg;             // stage bytes: the largest of the batch
    unsigned int *ctrl;
    const unsigned long long *epoch;  // advanced by the batch prologue
};

// launchers (return cudaError_t of the launch)
cudaError_t launch_opacity(const sm_problem *p, const double *T, const double *scale,
                           double *sigma, cudaStream_t s);
cudaError_t launch_emission(const sm_problem *p, const double *T, const double *sigma,
                            double *q_canon, cudaStream_t s, const int *active = nullptr);
cudaError_t launch_inflow(const sm_problem *p, cudaStream_t s);
cudaError_t launch_planck_parts(const sm_problem *p, const double *T, const double *sigma,
                                double *B4, double *cB, double *sdB, cudaStream_t s);
cudaError_t launch_opacity_shape(const sm_problem *p, const double *T, double *f, double *df,
                                 cudaStream_t s);
cudaError_t launch_closures_from_T(const sm_problem *p, const double *mom, const double *T,
                                   const double *sigma, double *out, cudaStream_t s);
cudaError_t launch_sweep2d(const sm_problem *p, const SweepArgs &a, int grid, cudaStream_t s,
                           const EmitArgs *e = nullptr);
cudaError_t launch_sweep1d(const sm_problem *p, const SweepArgs &a, cudaStream_t s);
cudaError_t launch_reduce(const sm_problem *p, const void *part, int n_part, double *mom,
                          double *clo, cudaStream_t s, double *qmom = nullptr,
                          int sets_per_q = 1, const int *active = nullptr);
cudaError_t launch_pack(const sm_problem *p, const double *canon, void *packed, int unpack,
                        cudaStream_t s);
// CTAs of the 2D sweep that fit on the GPU for W sweep warps, S stages and
// emit_warps fused emission warps (0 if none fit); *smem_out: bytes per CTA.
int sweep2d_max_resident(const sm_problem *p, int W, int S, size_t *smem_out, int emit_warps = 0);
// The 2D sweep kernel and the 2D reduction in an explicit arithmetic precision
// for problem p's layout and tiling (FP32 correction sweeps of FP64 problems).
int sweep2d_max_resident_prec(int prec, const sm_problem *p, int W, int S, size_t *smem_out);
cudaError_t launch_sweep2d_prec(int prec, const sm_problem *p, const SweepArgs &a, int grid,
                                cudaStream_t s);
cudaError_t launch_reduce_prec(int prec, const sm_problem *p, const void *part, int n_part,
                               double *mom, double *clo, cudaStream_t s);
// FP64-accurate defect correction with FP32 sweeps (sm_refine.cu): workspace
// on first use (FP64 2D problems only); at the start of a step I^k and the
// iterate (in the caller's packed FP64 buffer I) as pairs of FP32 numbers;
// the transport solve of one outer iteration by corrections of the iterate
// (residual, FP32 correction sweep, I += d, until the corrections are small)
// and the moments of I; at the end of the step I joined back into FP64;
// release.
sm_status refine_ensure(sm_problem *p);
sm_status refine_begin(sm_problem *p, const double *I_k, void *I);
sm_status refine_solve(sm_problem *p, void *I, double *mom);
sm_status refine_end(sm_problem *p, void *I);
int refine_take_corrections(sm_problem *p);  // corrections since the last call
void refine_free(sm_problem *p);
size_t sweep2d_smem_bytes(int prec, int W, int GW, int S, int GSLOT);
size_t sweep2d_stage_bytes(int prec, int GW, int GSLOT);
size_t sweep2d_batch_smem_bytes(int prec, int W, int S, size_t stg, int ring_gw);
cudaError_t launch_sweep2d_batch(int prec, const BatchSweepArgs &b, int grid, size_t smem,
                                 cudaStream_t s);
int sweep2d_batch_max_resident(int prec, int W, size_t smem);
void planck_upload_tables(void);
// double-FP32 emission of an FP32-sweep problem (sm_planck_df.cu); the
// tables' host copies it derives its own tables from (sm_planck.cu)
cudaError_t launch_emission_df(const sm_problem *p, const double *T, const double *sigma,
                               cudaStream_t s, const int *active);
bool planck_df_upload_tables(void);  // once per device (synchronous copies)
// Fills the Planck tables' kernel-parameter form (uploads them first); false
// on a CUDA error.
bool planck_tabs(PlanckTabs *out);
// Descriptor checks shared by sm_create_problem and sm_sweep_static: NULL when
// the descriptor is valid, else a static message (allocates nothing).
const char *check_desc(const sm_problem_desc *d);
// Set the thread-local message returned by sm_last_error() (no allocation
// beyond the message string of at most 255 characters).
void set_last_error(const char *msg);
// Free the low-order workspace (no-op when the low-order solve never ran).
void lo_free(sm_problem *p);
// The sweep of one problem without its emission (the caller has written the
// source records): sweep kernel and, when mom is non-NULL, the moment sums
// and closures.  reverse = 1 sweeps -Omega (adjoint sweeps, 2D only).
sm_status sweep_only(sm_problem *p, const void *I_prev, void *I_out, double *mom, double *clo,
                     int reverse);
// Free the adjoint workspace (no-op when unused).
void adjoint_free(sm_problem *p);
// The batch object as seen by the time step (sm_batch_step): its members, its
// stream, one whole pass (graph replay) for the members whose active flag is
// set (active_host: one flag per member; NULL: all), and the device status
// of the last passes (SM_OK, TIMEOUT or NONPHYSICAL; cleared).
const std::vector<sm_problem *> &batch_members(const sm_batch *b);
cudaStream_t batch_stream(const sm_batch *b);
sm_status batch_pass(sm_batch *b, const double *const *T, const double *const *sigma,
                     const void *const *I_prev, void *const *I_out, double *const *mom,
                     double *const *clo, const unsigned char *active_host);
sm_status batch_status(sm_batch *b);
// Scratch of the batched low-order launch (sm_lo.cu), kept with the batch
// and released with it.
void *&batch_lo_scratch(sm_batch *b);
// 1 (default): the members' low-order solves in one cooperative launch;
// 0: one launch per member (test hook sm_debug_set_batch_lo).
int &batch_lo_mode(sm_batch *b);
void batch_lo_free(void *scratch);
// Tiling and sweep arguments of one problem (used by the batch object).
sm_status apply_tiling_ext(sm_problem *p, int W, int S);
SweepArgs make_sweep_args(const sm_problem *p, const void *I_prev, void *I_out);

}  // namespace smk

struct sm_batch;      // batched problems (sm_batch.cu)
struct sm_lo_state;   // low-order solve workspace, created on first use
struct sm_refine_state;  // defect-correction workspace, created on first use
struct sm_adj_state;  // adjoint workspace, created on first use

struct sm_problem {
    // descriptor copy
    sm_problem_desc desc;
    std::vector<double> edges;
    int dim, nx, ny, ncell, nn, nm, nc, G, nd, NQ;
    double hx, hy, inv_cdt;
    int prec;  // 32 or 64
    size_t rsize;
    // quadrature (canonical order)
    std::vector<double> omx, omy, w;
    double alpha;
    // lane mapping
    int DQ, DQP, DQL, LG, DB, GW, GSLOT, Gp, NGB, NWT;
    // tiling (2D): W cell columns (= warps) per CTA, S prefetched rows per warp
    int W, S, NS;
    int emit_warps = 0;  // 2D: emission warps fused into the sweep kernel (0: separate kernel)
    int tail = 0;        // 2D: half-width strips at each end of the x range (0: uniform strips)
    int emit_fp64 = 0;   // FP32 problem: sweeps take the FP64 emission kernel (test hook)
    int *d_strip_x0 = nullptr;  // [NS + 1] first column of each strip when tail > 0
    int resident = 0;  // 2D sweep CTAs that fit on the GPU for (W, S, emit_warps)
    unsigned int *d_emit_ctr = nullptr;  // [1 + NS] fused-emission queue and strip counters
    smk::PlanckTabs *tabs = nullptr;     // host copy of the tables' parameter form
    // device buffers
    double *d_edges = nullptr;      // [G+1]
    void *d_inflow = nullptr;       // [4][Gp] sweep precision
    smk::LaneConst *d_lanes = nullptr;
    int *d_dir_of = nullptr;        // [NQ][DB][32] canonical direction (or -1)
    void *d_src = nullptr;          // [cell][Gp][8] source records
    void *d_mom_acc = nullptr;      // 2D: [NQ*NWT][cell][36] partial moments per warp task
    double *d_gray = nullptr;       // [cell][node][2] sigma_P, sigma_F
    void *d_part = nullptr;         // 1D: per-warp partial moments
    void *d_face = nullptr;
    size_t face_bytes = 0;
    unsigned long long *d_flags = nullptr;
    size_t flags_count = 0;
    unsigned int *d_ctrl = nullptr;
    double *d_mom_tmp = nullptr;
    double *d_T_tmp = nullptr;      // host-input staging for sm_sweep_host
    double *d_sig_tmp = nullptr;
    double *d_clo_tmp = nullptr;
    unsigned long long epoch = 0;
    long long timeout_ns = 2000000000LL;
    int fault_skip_publish = 0;
    int fault_withhold_block = 0;  // test hook: a low-order block skips its barriers
    int lo_pcg_form = 0;           // test hook: SM_DEBUG_PCG_* (0: the library's choice)
    int lo_pcg_form_used = 0;      // form of the last low-order solve (0: none yet)
    cudaStream_t stream = nullptr;
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;  // 4 events per timed sweep, read back lazily
    int n_timed = 0;
    int64_t launches = 0;
    size_t workspace_bytes = 0;
    sm_lo_state *lo = nullptr;
    sm_refine_state *refine = nullptr;
    sm_adj_state *adj = nullptr;
    double *qmom_dev = nullptr;  // per-quadrant moments [cell][node][4][6] filled by each sweep
    bool qmom_acc4 = false;      // (unused: the partial moments are per warp task)
    bool batch_owned = false;    // member of an sm_batch: swept only by the batch
    bool ctrl_borrowed = false;  // d_ctrl belongs to the batch
};

