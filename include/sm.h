/*
 * sm.h -- C ABI of the GB300 (sm_103a) Second Moment thermal-radiative-transfer
 * hot path: the lumped upwind-DG discrete-ordinates transport sweep over every
 * direction and group, fused with the angular-moment reductions and the gray
 * low-order closures of Olivier, Warsa & Park, "Efficient, Nonlinear Second
 * Moment Methods for Multigroup Thermal Radiative Transfer" (arXiv 2504.21784).
 *
 * Conventions for every entry point
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *    library never frees them.  Pointers named *_host are host pointers.
 *  - Every call is asynchronous on the problem's CUDA stream unless stated.
 *    Device-side conditions (a wavefront wait that ran out of time) are
 *    reported by sm_synchronize().
 *  - No exception crosses the ABI.  A non-zero sm_status is returned and a
 *    thread-local message is available from sm_last_error().
 *  - All arrays are dense and C-ordered:
 *      cell  = iy*nx + ix                      (1D: ny = 1)
 *      node  = a + 2*b  (2D; a = x side, b = y side, 0 = low), node = a (1D);
 *              nodes are the corners (Gauss-Lobatto points) of each cell
 *      T_nodal[cell][node], sigma[g][cell], q[g][cell][node],
 *      canonical intensity I[d][g][cell][node]
 *    Direction order: 1D ascending Gauss-Legendre mu; 2D quadrant-major
 *    (signs of (Omega_x, Omega_y): (+,+), (-,+), (-,-), (+,-)), then polar
 *    cosine ascending, then azimuth.
 *  - The intensity that persists between calls (I^k and the new I) lives in
 *    an opaque packed layout of sm_problem_info.intensity_bytes bytes in the
 *    sweep precision; convert with sm_pack_intensity / sm_unpack_intensity.
 */
#ifndef SM_TRT_H
#define SM_TRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SM_OK = 0,
    SM_ERR_INVALID_ARG = 1,    /* bad descriptor, size or pointer */
    SM_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    SM_ERR_OOM = 3,            /* device allocation failed */
    SM_ERR_NO_CONVERGENCE = 4, /* conjugate gradients broke down in the low-order solve */
    SM_ERR_NONPHYSICAL = 5,    /* non-positive temperature or NaN input */
    SM_ERR_TIMEOUT = 6,        /* a device wavefront wait exceeded its time limit */
    SM_ERR_UNSUPPORTED = 7     /* valid but not implemented (e.g. a tile shape) */
} sm_status;

/* opacity models (Sec. 6.1 power law; Sec. 6.2 form alpha (1 - e^{-nu/T}) / nu^3) */
enum { SM_OPACITY_POWER = 0, SM_OPACITY_LARSEN = 1 };

typedef struct sm_problem sm_problem; /* opaque, owned by the library */

/* Problem descriptor; every field is copied by sm_create_problem. */
typedef struct {
    int dim;                   /* 1 or 2 */
    int nx, ny;                /* cells per axis (ny ignored in 1D) */
    double x0, x1, y0, y1;     /* uniform structured mesh on [x0,x1] x [y0,y1] */
    int n_groups;              /* G >= 1 */
    const double *group_edges; /* host, G+1 ascending positive edges nu_1..nu_{G+1} */
    int n_polar;               /* 1D: Gauss-Legendre order (even); 2D: polar cosines per octant */
    int n_azim;                /* 2D: azimuths per octant (ignored in 1D) */
    double a, c;               /* radiation constant, speed of light */
    double dt;                 /* time step; <= 0 selects the steady operator (no 1/(c dt)) */
    int opacity_kind;          /* SM_OPACITY_POWER or SM_OPACITY_LARSEN */
    double opacity_alpha;      /* alpha of SM_OPACITY_LARSEN */
    double T_bdr[4];           /* boundary temperature per side: left, right, bottom, top;
                                  <= 0 means vacuum (zero inflow) */
    int precision;             /* sweep arithmetic: 32 (FP32) or 64 (FP64) */
    int groups_per_warp;       /* (d,g) slots per lane of a warp task: 1, 2, 4, 8; 0 = auto:
                                  the largest power of two up to 8 (FP32) or 4 (FP64) that
                                  the groups fill, halved while the problem has fewer than
                                  16 independent wavefront chains (quadrant x direction
                                  block x group block); batch members keep the largest */
    int strip_width;           /* 2D: cell columns per CTA, one warp per column, 1..16; 0 = auto:
                                  the widest of 16, 12, 8, 4, 2 whose shared memory fits */
    int prefetch_rows;         /* 2D: rows each warp prefetches by TMA, 2..8; 0 = auto (2) */
} sm_problem_desc;

typedef struct {
    int dim, nx, ny;
    int n_dir, n_groups, n_cells, n_nodes;
    int n_moments;             /* 9 in 2D, 5 in 1D (per node) */
    int n_closures;            /* 11 in 2D, 7 in 1D (per node) */
    int precision;
    int dirs_per_quadrant;     /* padded to the lane mapping */
    int groups_per_lane_row;   /* groups interleaved across the 32 lanes */
    int groups_per_warp;       /* (d,g) slots per lane */
    int n_groups_padded;
    int n_warp_tasks;          /* per quadrant */
    int strip_width, prefetch_rows, n_tasks, n_strips;
    size_t intensity_elems;    /* packed intensity elements (padding included) */
    size_t intensity_bytes;
    size_t workspace_bytes;    /* device scratch the library owns */
    double alpha;              /* Eq. alpha: sum w |Omega.n| / sum w with S_N quadrature */
    int emission_warps;        /* 2D: warps per sweep CTA computing the emission (0: own kernel) */
    int tail_strips;           /* 2D: half-width strips at each end of the x range (0: uniform) */
} sm_problem_info;

/* Create a problem: builds the S_N set (Sec. 2; Gauss-Legendre in 1D,
 * square product set in 2D, weights summing to 4 pi), the group-edge tables
 * and the lane mapping, and allocates the device workspace.  stream is a
 * cudaStream_t (NULL = legacy default stream).  Errors: INVALID_ARG for an
 * empty mesh, G < 1, non-ascending edges, an odd 1D order or an unsupported
 * tile; OOM; CUDA. */
sm_status sm_create_problem(const sm_problem_desc *desc, void *stream, sm_problem **out);

/* Free the workspace and the problem.  NULL is accepted. */
sm_status sm_destroy_problem(sm_problem *p);

sm_status sm_get_info(const sm_problem *p, sm_problem_info *out);

/* Rebind the CUDA stream used by subsequent calls. */
sm_status sm_set_stream(sm_problem *p, void *stream);

/* Change the 2D wavefront strip width (cell columns, one warp each, per CTA)
 * and the TMA prefetch depth in rows (the packed intensity layout does not
 * depend on them).  0 keeps the current value. */
sm_status sm_set_tiling(sm_problem *p, int strip_width, int prefetch_rows);

/* Where the emission (row a1) of a 2D pass runs.  0 (the default): its own
 * kernel, before the sweep kernel.  1..4: fused into the sweep kernel --
 * every sweep CTA gets that many extra warps (strip_width + warps <= 16)
 * that compute the emission of the strips ahead of the sweep, strip by
 * strip in the order the strips are first needed, on the FP64 pipes the
 * streaming sweep leaves idle; a sweep task whose strip is not complete yet
 * computes emission items itself until it is.  The source records are the
 * same either way (the Planck evaluation is shared).  Batch members refuse
 * (UNSUPPORTED), and so does a problem with tail strips (below).  sm_autotune
 * also picks among 0, 2 and 4.  Synchronizes. */
sm_status sm_set_emission_warps(sm_problem *p, int warps);

/* Strip layout of the 2D wavefront: n (0..4) strips of strip_width / 2 cell
 * columns at each end of the x range, full-width strips in between (0, the
 * default: every strip full width, the last one ragged).  The persistent
 * sweep grid takes the strips' tasks in upwind order; the sweeps in both x
 * directions end on half-width strips, so the last, partial wave of tasks is
 * shorter.  The results do not depend on the layout (the packed intensity
 * layout does not change).  Needs an even strip_width, at least one
 * full-width strip in between (else the layout falls back to 0, reported by
 * sm_get_info) and the separate emission kernel (UNSUPPORTED with fused
 * emission warps or for a batch member).  sm_autotune also picks among 0, 1
 * and 2.  Synchronizes. */
sm_status sm_set_tail_strips(sm_problem *p, int n);

/* Copy the discrete ordinates {Omega_d, w_d} (Sec. 2) to host arrays of
 * n_dir entries each in the canonical order (omy is all zero in 1D). */
sm_status sm_get_quadrature(const sm_problem *p, double *omx_host, double *omy_host,
                            double *w_host);

/* Multigroup opacity sigma_{g,K} from the element-average temperature
 * (Sec. 3, Rem. opacity): POWER: s_K Tbar^-3; LARSEN: s_K alpha
 * (1 - e^{-E_g/Tbar}) / E_g^3 with E_g the geometric mean of the group's
 * edges (Sec. 6.2).  T_nodal_dev[cell][node], scale_dev[cell] (s_K),
 * sigma_dev[g][cell] out, all FP64. */
sm_status sm_opacity(sm_problem *p, const double *T_nodal_dev, const double *scale_dev,
                     double *sigma_dev);

/* a1. Emission source q_{g,n} = sigma_g a c T_n^4 b_g(T_n) / 4 pi at every
 * node (Eq. smm_be_transport, Eq. planck, lumped), b_g by the Planck series
 * in FP64 with the lowest edge taken to 0 and the highest to infinity
 * (sum_g b_g = 1).  Fills the internal source buffer used by the next sweep
 * and the nodal Planck- and Rosseland-collapsed opacities sigma_P, sigma_F
 * (Sec. 2) used by the closures.  q_dev[g][cell][node] (FP64) receives a
 * copy when non-NULL.  A non-positive or non-finite temperature is recorded
 * in the device status and reported by sm_synchronize() as NONPHYSICAL. */
sm_status sm_emission(sm_problem *p, const double *T_nodal_dev, const double *sigma_dev,
                      double *q_dev);

/* One pass of the hot path (rows a1-a4):
 *   a1 emission from T_nodal (as sm_emission);
 *   a2 the lumped upwind DG cell solves of Eq. dgsn_transport for every
 *      (direction, group) in wavefront order, sigma~ = sigma + 1/(c dt) and
 *      the time-edge source I^k/(c dt) of Eq. smm_be_transport, isotropic
 *      inflow B_g(T_bdr)/4 pi (Eq. transport BC);
 *   a3 fused per-node moments summed over all (d,g):
 *      2D [phi, Fx, Fy, Txx, Txy, Tyy, SE, SFx, SFy], 1D [phi, F, T, SE, SF]
 *      with phi = sum w I (= c E), F = sum w Omega I, T = sum w (Omega Omega
 *      - I/3) I (in-plane block), SE = sum_g sigma_g sum_d w I,
 *      SF = sum_g sigma_g sum_d w Omega I (Sec. 2, Eqs. sigmaE and
 *      additive_mg_correction numerators);
 *   a4 closures (as sm_closures) when closures_dev is non-NULL.
 * I_prev_dev: packed I^k (NULL: zero, i.e. no time-edge source).
 * I_out_dev: packed new intensity (required; must not alias I_prev_dev).
 * moments_dev[cell][node][n_moments] FP64 (may be NULL).
 * closures_dev[cell][node][n_closures] FP64 (may be NULL). */
sm_status sm_sweep(sm_problem *p, const double *T_nodal_dev, const double *sigma_dev,
                   const void *I_prev_dev, void *I_out_dev, double *moments_dev,
                   double *closures_dev);

/* a4. Closures of the gray low-order system from moments (Sec. 2):
 * sigma_E = SE/phi (Eq. sigmaE; sigma_P where phi <= 0 or SE <= 0: the
 * lumped intensity has no positivity fix-up, and the mean of the positive
 * group opacities is undefined for such weights), sigma_F =
 * sum r_g sigma_g / sum r_g (Eq. sigmaF), sigma_P = sum b_g sigma_g / sum b_g,
 * additive correction sum_g (sigma_F - sigma_g) F_g = sigma_F F - SF
 * (Eq. additive_mg_correction), with nodal spectra at T_nodal.
 * Output per node: 2D [E, Fx, Fy, Txx, Txy, Tyy, sigE, sigF, sigP, Cx, Cy],
 * 1D [E, F, T, sigE, sigF, sigP, C];  E = phi / c. */
sm_status sm_closures(sm_problem *p, const double *moments_dev, const double *T_nodal_dev,
                      const double *sigma_dev, double *closures_dev);

/* ------------------------------------------------------------------------
 * Gray low-order solve and the full time step (Sec. 4 independent LDG
 * system, Sec. 5 Newton iteration, Algorithm 1).  All low-order arithmetic
 * is FP64 on the device: a low-order solve is one cooperative launch (the
 * Newton iteration with its conjugate-gradient solves and stopping tests),
 * after which the host reads its statistics; sm_step also reads the outer
 * iteration's change per iteration.  Both calls therefore synchronize the
 * problem's stream and cannot be captured into a CUDA graph.
 * ---------------------------------------------------------------------- */

/* Iteration controls.  Defaults (sm_default_step_params) are the paper's
 * (Sec. 6): eps = 1e-3 in Eq. relative_tol for the outer and the Newton
 * iterations, 1e-10 relative residual for conjugate gradients and for the
 * pointwise elimination, caps of 100 outer, 30 Newton and 40 elimination
 * iterations.  The paper preconditions conjugate gradients with algebraic
 * multigrid and caps it at 50; this library preconditions with the exact
 * diagonal of the Schur complement (Jacobi), which needs more iterations,
 * so max_pcg defaults to 5000. */
/* low-order closures (Sec. 4): independent (first-moment corrections only)
 * or consistent (face and boundary corrections from the half-range moments
 * of the high-order intensity, so that the converged low-order solution
 * equals the high-order moments; 1D and 2D) */
enum { SM_METHOD_INDEPENDENT = 0, SM_METHOD_CONSISTENT = 1 };

typedef struct {
    double eps_outer;   /* Eq. relative_tol for Algorithm 1's fixed point */
    double eps_inner;   /* Eq. relative_tol for the low-order Newton iteration */
    double pcg_rtol;    /* stop when ||b - S E||_2 <= pcg_rtol ||b||_2 */
    double elim_rtol;   /* pointwise elimination stops when |dT| <= elim_rtol |T| */
    double T_floor;     /* lower bound imposed on T by the elimination */
    int max_outer, max_inner, max_pcg, max_elim;
    int method;         /* SM_METHOD_INDEPENDENT (default) or SM_METHOD_CONSISTENT */
    int refine;         /* 1: FP64 defect correction with FP32 sweeps (see sm_step) */
} sm_step_params;

/* Iteration counts of one call. */
typedef struct {
    int outer_iters;        /* Algorithm 1 iterations (0 for sm_loworder_newton) */
    int newton_iters_total; /* low-order Newton iterations, summed over outer iterations */
    int newton_iters_max;   /* ... largest in one low-order solve */
    int pcg_iters_total;    /* conjugate-gradient iterations, summed */
    int pcg_iters_max;      /* ... largest in one linear solve */
    int pcg_capped;         /* linear solves that stopped at max_pcg */
    int elim_iters_max;     /* largest pointwise elimination count at any node */
    int converged;          /* 1 when the outer iteration met eps_outer within max_outer */
    double last_change;     /* ||u^{l} - u^{l-1}||_2, u = (T, E), of the last outer iteration */
    int refine_corrections; /* FP32 correction sweeps of the step (params->refine = 1), else 0 */
} sm_step_stats;

void sm_default_step_params(sm_step_params *params_host);

/* Solve the gray low-order system with fixed closures by the Newton
 * iteration of Sec. 5: gray opacities frozen, emission linearised about the
 * current T with the pseudo-fission coefficient of Eq. pseudo_fission, the
 * linear system reduced to the Schur complement in E (Eq. schur; symmetric
 * positive definite), solved by Jacobi-preconditioned conjugate gradients,
 * F recovered by back-substitution and T updated by the pointwise
 * nonlinear elimination of Eq. nonlinear_T_update; stops by
 * Eq. relative_tol on u = (T, E).
 *   closures_dev[cell][node][n_closures]: as produced by sm_closures;
 *   T_star_dev[cell][node]: temperature at the previous time step (T*);
 *   cv_dev[cell][node]: heat capacity C_v (> 0);
 *   moments_star_dev[cell][node][n_moments]: moments of the previous step's
 *     intensity; E* = phi / c and F* = F are the time-edge sources (Sec. 6.1);
 *   T_dev, E_dev [cell][node]: initial guesses on entry, solution on exit;
 *   F_dev[cell][node][dim]: flux of the last linear solve (out).
 * Boundary: Marshak-type with the gray isotropic inflow of desc.T_bdr.
 * params->method = SM_METHOD_CONSISTENT uses the consistent sources from
 * the per-quadrant moments of the last sweep (registered with
 * sm_set_quadrant_moments).  Needs desc.dt > 0.  Errors: INVALID_ARG, NO_CONVERGENCE (conjugate
 * gradients broke down), NONPHYSICAL (non-finite iterate), CUDA, OOM (the
 * low-order workspace is allocated on first use).  A capped iteration is
 * not an error: see stats.  stats_host may be NULL. */
/* Register (or, with NULL, drop) a caller buffer qmom_dev[cell][node][4][6]
 * that every following sweep of p fills with the per-quadrant moments of the
 * new intensity (quadrants in the canonical order; per quadrant phi, F_x,
 * F_y, Pi_xx, Pi_xy, Pi_yy with Pi = sum w Omega Omega I, all groups): the
 * input of the consistent method, from which every half-range current and
 * second moment on axis-aligned faces follows.  1D: quadrant 0 holds the
 * directions with mu > 0, quadrant 1 those with mu < 0 (phi, F, 0, Pi_xx,
 * 0, 0; quadrants 2 and 3 zero), the same layout.  In 2D the moment
 * accumulator grows to four quadrants (allocated here).  Synchronizes. */
sm_status sm_set_quadrant_moments(sm_problem *p, double *qmom_dev);

sm_status sm_loworder_newton(sm_problem *p, const double *closures_dev, const double *T_star_dev,
                             const double *cv_dev, const double *moments_star_dev, double *T_dev,
                             double *E_dev, double *F_dev, const sm_step_params *params_host,
                             sm_step_stats *stats_host);

/* One time step of Algorithm 1 (semi-implicit backward Euler, Eq. smm_be):
 * multigroup opacities sigma_g(T^k) from sm_opacity at the step's start
 * temperature, then repeat { sm_sweep with the current T (emission, sweep,
 * moments, closures); sm_loworder_newton } until Eq. relative_tol holds for
 * u = (T, E) or max_outer is reached.  E starts at E* and T at T^k.
 *   scale_dev[cell]: opacity scale s_K (as sm_opacity);
 *   cv_dev[cell][node]: C_v;
 *   T_dev[cell][node]: T^k on entry, T^{k+1} on exit;
 *   E_dev[cell][node], F_dev[cell][node][dim]: low-order solution (out);
 *   moments_dev[cell][node][n_moments]: on entry the moments of I_prev (the
 *     time-edge sources), on exit those of I_next;
 *   I_prev_dev: packed I^k; I_next_dev: packed I^{k+1} (out; no aliasing);
 *   closures_dev[cell][node][n_closures]: last closures (out; may be NULL).
 * With params->refine = 1 (2D, a precision-64 problem: FP64 state and
 * emission, independent method) each outer iteration replaces the FP64 sweep
 * by defect corrections of the intensity iterate (which starts at I^k): the
 * residual of the lumped DG equations at the iterate, an FP32 sweep of the
 * correction with zero inflow and the update, repeated (at most 4 times)
 * until a correction is below 1e-8 of the iterate; then the moments of the
 * iterate.  The residual, the update and the moment sums run in double-FP32
 * arithmetic (each value a pair of FP32 numbers, about 48 significant bits,
 * on the FP32 pipes), so the FP32 sweeps give the FP64 sweep's intensity to
 * about 1e-14 and the step the FP64 step's result; during the step I_next
 * and a library buffer of the same size hold the iterate as such pairs in
 * turn (I_next's contents are unspecified if the step fails), and I_next
 * receives it in FP64 at the step's end.  stats->refine_corrections
 * counts the corrections.  Synchronizes after each correction.  All of
 * the refined path's sweeps are FP32 sweeps with the problem's slots per
 * lane, whose automatic value for precision 64 is capped at 4: a problem
 * made for refined steps runs faster with groups_per_warp set to what the
 * FP32 rule gives (8 where the groups fill it).
 * With params->method = SM_METHOD_CONSISTENT (2D) the sweeps also form
 * per-quadrant moments (in the buffer registered with
 * sm_set_quadrant_moments, else in the library's own) and the low-order
 * solves use the consistent sources; the step then converges to the
 * converged high-order step of sm_ho_step.
 * Errors as sm_sweep and sm_loworder_newton.  Synchronous. */
sm_status sm_step(sm_problem *p, const double *scale_dev, const double *cv_dev, double *T_dev,
                  double *E_dev, double *F_dev, double *moments_dev, const void *I_prev_dev,
                  void *I_next_dev, double *closures_dev, const sm_step_params *params_host,
                  sm_step_stats *stats_host);

/* End-to-end variant of sm_sweep for callers holding host buffers: copies
 * T_nodal_host and sigma_host to the device, runs sm_sweep, copies moments
 * and closures back to the host arrays (either may be NULL) and waits for
 * completion.  Host buffers should be pinned for full copy bandwidth.  The
 * intensity stays device resident (I_prev_dev, I_out_dev as in sm_sweep). */
sm_status sm_sweep_host(sm_problem *p, const double *T_nodal_host, const double *sigma_host,
                        const void *I_prev_dev, void *I_out_dev, double *moments_host,
                        double *closures_host);

/* Convert between the canonical FP64 layout I[d][g][cell][node] and the
 * packed sweep layout (rounded to the sweep precision; padding slots are
 * zeroed by pack and skipped by unpack). */
sm_status sm_pack_intensity(sm_problem *p, const double *I_canon_dev, void *I_packed_dev);
sm_status sm_unpack_intensity(sm_problem *p, const void *I_packed_dev, double *I_canon_dev);

/* Wait for the problem's stream and report device-side status: SM_OK, or
 * SM_ERR_TIMEOUT when a wavefront wait gave up (the sweep output is then
 * invalid).  Clears the device status word. */
sm_status sm_synchronize(sm_problem *p);

/* Pick strip_width, prefetch_rows, the fused emission warps (0, 2 or 4) and
 * the tail strips (0, 1 or 2, with the separate emission kernel only) by
 * timing each candidate whole pass on the given inputs with CUDA events
 * (reps timed passes each after one warm-up); the fastest is kept.
 * Overwrites I_out_dev.  Synchronous. */
sm_status sm_autotune(sm_problem *p, const double *T_nodal_dev, const double *sigma_dev,
                      const void *I_prev_dev, void *I_out_dev, int reps);

/* Kernel timing with CUDA events on the problem's stream.  While enabled,
 * each sweep records (without any synchronization) events around its
 * emission, sweep and reduction kernels, for up to 4096 sweeps;
 * sm_get_kernel_times synchronizes and returns the summed milliseconds and
 * the number of sweeps timed, then resets them.
 * ms_host[0] = emission, [1] = sweep kernel, [2] = moment reduction/closures. */
sm_status sm_set_profiling(sm_problem *p, int enable);
sm_status sm_get_kernel_times(sm_problem *p, double *ms_host, int *count_host);

/* Allocation-free variant of sm_sweep for small 2D problems (the paper has
 * no counterpart: it is a service to callers of this library).
 *
 * For callers that cannot call cudaMalloc -- a thread that must not block on
 * the allocator or synchronize the device, a process whose device memory is
 * fully reserved by another allocator, or an embedding with a fixed memory
 * budget -- and therefore cannot use sm_create_problem, which allocates a
 * workspace.  It runs the same pass as sm_sweep (emission, sweep with fused
 * moments, moment sums and closures) for the problem described by desc
 * (dim must be 2; tile fields are chosen internally), with every
 * intermediate buffer in one static device array of 16 MiB that the library
 * holds on every GPU that loads it, until the process exits.  It allocates
 * nothing: no cudaMalloc, cudaFree or other allocating routine.
 *
 * Inputs and outputs are caller-owned device arrays in the canonical
 * layouts: T_nodal_dev[cell][4], sigma_dev[g][cell], I_prev_canon_dev and
 * I_out_canon_dev [d][g][cell][4] (FP64; I_prev may be NULL),
 * moments_dev[cell][4][9] and closures_dev[cell][4][11] (either may be NULL).
 * A problem whose scratch would exceed 16 MiB is rejected with
 * SM_ERR_INVALID_ARG and a message giving the size it needs (for example,
 * 32x32 cells x 32 directions x 8 groups in FP32 fits).
 *
 * The first call on a device (with that device current) looks up the
 * array's device address with cudaGetSymbolAddress, and the first call in
 * the process uploads the Planck tables (synchronous copies).  The call
 * waits for its own stream only (a
 * cudaStream_t, NULL for the legacy default stream): the device status is
 * read by an asynchronous copy on that stream, then that stream is
 * synchronized; it returns SM_ERR_TIMEOUT or SM_ERR_NONPHYSICAL like
 * sm_synchronize.  It uses about 40 KB of the calling thread's stack.  All
 * calls share the one array, which keeps the previous call's contents (the
 * parts that must start at zero are cleared by each call): calls that
 * overlap on the GPU race.  Descriptor errors are those of
 * sm_create_problem, plus dim != 2, n_groups > 256 and n_polar * n_azim
 * > 128 (each factor is checked before the product). */
sm_status sm_sweep_static(const sm_problem_desc *desc, void *stream, const double *T_nodal_dev,
                          const double *sigma_dev, const double *I_prev_canon_dev,
                          double *I_out_canon_dev, double *moments_dev, double *closures_dev);

/* ------------------------------------------------------------------------
 * Batched problems: many independent 2D problems -- uneven meshes, group and
 * direction counts, material layouts -- swept in ONE persistent launch.  The
 * batch owns one problem per member (created from descs[i]; precision must
 * be the same for all, dim must be 2, tile fields are ignored: the batch's
 * strip width and prefetch depth apply to every member).  Every CTA of the
 * batched sweep takes (member, task) items from one queue, ordered so that
 * each member keeps its own upwind order.  A call to sm_batch_sweep runs
 * the whole pass for every member -- emission (a1), sweep with fused
 * moments (a2, a3), moment sums and closures (a4) -- recorded the first time
 * as a CUDA graph for that set of buffers and replayed on later calls with
 * the same buffers (up to 4 buffer sets are kept, e.g. the two roles of the
 * intensity buffers in a time loop).  The paper runs independent problems
 * one after another; batching them is this library's addition.
 * ---------------------------------------------------------------------- */
typedef struct sm_batch sm_batch; /* opaque, owned by the library */

typedef struct {
    int n_problems;
    int n_tasks;        /* queue items of one batched sweep */
    int strip_width, prefetch_rows;
    int resident_ctas;  /* persistent grid of the batched sweep */
    int graphs_cached;
    size_t smem_bytes;  /* dynamic shared memory per CTA */
    double updates;     /* sum over members of cells x directions x groups */
    int64_t launches;   /* kernels launched by batched sweeps so far */
} sm_batch_info;

/* stream: cudaStream_t (NULL = legacy default stream).  Errors as
 * sm_create_problem, plus INVALID_ARG for n < 1, a 1D member or mixed
 * precisions. */
sm_status sm_create_batch(const sm_problem_desc *descs, int n, void *stream, sm_batch **out);
/* Destroys the batch and its members.  NULL is accepted. */
sm_status sm_destroy_batch(sm_batch *b);
/* Borrowed handle of member i, for sm_get_info, sm_get_quadrature,
 * sm_opacity, sm_emission, sm_closures, sm_pack_intensity and
 * sm_unpack_intensity.  sm_sweep, sm_sweep_host, sm_autotune, sm_set_tiling,
 * sm_step and sm_destroy_problem refuse batch members (INVALID_ARG): their
 * wavefront counters belong to the batch; sm_batch_step advances them. */
sm_status sm_batch_problem(sm_batch *b, int i, sm_problem **out);
sm_status sm_batch_get_info(const sm_batch *b, sm_batch_info *out);
sm_status sm_batch_set_stream(sm_batch *b, void *stream);
/* Strip width 1..16 and prefetch depth 2..8 for every member (0 keeps the
 * current value).  Synchronizes the stream; drops the recorded graphs. */
sm_status sm_batch_set_tiling(sm_batch *b, int strip_width, int prefetch_rows);
/* One pass for every member.  Each argument is a HOST array of n device
 * pointers, laid out as for sm_sweep: T_nodal[i], sigma[i], I_prev[i] (the
 * array or an entry may be NULL: no time-edge source), I_out[i] (required,
 * 16-byte aligned, not aliasing I_prev[i]), moments[i] and closures[i]
 * (arrays or entries may be NULL).  Asynchronous on the batch's stream;
 * sm_batch_synchronize reports device-side status. */
sm_status sm_batch_sweep(sm_batch *b, const double *const *T_nodal_dev,
                         const double *const *sigma_dev, const void *const *I_prev_dev,
                         void *const *I_out_dev, double *const *moments_dev,
                         double *const *closures_dev);
/* Waits for the batch's stream; SM_OK, SM_ERR_TIMEOUT or SM_ERR_NONPHYSICAL
 * (then clears the status). */
sm_status sm_batch_synchronize(sm_batch *b);
/* Picks the strip width and prefetch depth of the batch by timing each
 * candidate (W in 2..16, S in 2..4) on the given buffers with CUDA events,
 * reps timed passes after one warm-up; keeps the fastest.  Overwrites
 * I_out.  Synchronous. */
sm_status sm_batch_autotune(sm_batch *b, const double *const *T_nodal_dev,
                            const double *const *sigma_dev, const void *const *I_prev_dev,
                            void *const *I_out_dev, int reps);

/* Slots per lane -- the (direction, group) pairs each lane of a warp task
 * carries, i.e. the (d,g) work per CTA -- for the members of a batch,
 * picked by timing (this library's autotuner; the packed layout depends on
 * it, so it is chosen before the batch is created): for each cap c = 8, 4,
 * 2, 1 a temporary batch is built from descs whose members take min(c,
 * their automatic choice), its strip width and prefetch depth are autotuned,
 * and reps passes are timed on synthetic inputs (T = 1, unit opacity, zero
 * intensities; the sweep's cost does not depend on the values).  The
 * members' slots of the fastest cap go to gw_out[i] (n entries), for use as
 * descs[i].groups_per_warp; members whose descriptor fixes groups_per_warp
 * keep it.  Allocates and frees its temporary buffers.  Synchronous. */
sm_status sm_batch_tune_slots(const sm_problem_desc *descs, int n, void *stream, int reps,
                              int *gw_out);

/* Kernel timing of batched passes with CUDA events on the batch's stream.
 * While enabled, each pass runs live (launched directly, not replayed from a
 * graph) with events around its three stages, for up to 4096 passes;
 * sm_batch_get_kernel_times synchronizes and returns the summed milliseconds
 * and the number of passes timed, then resets them.  ms_host[0] = prologue,
 * emissions, [1] = the batched sweep kernel, [2] =
 * moment sums and closures. */
sm_status sm_batch_set_profiling(sm_batch *b, int enable);
sm_status sm_batch_get_kernel_times(sm_batch *b, double *ms_host, int *count_host);

/* One time step of Algorithm 1 for every member of the batch (the batched
 * form of sm_step, independent closures): per outer iteration ONE batched
 * pass (emission, the persistent sweep launch over all unconverged members,
 * moments and closures, replayed from a CUDA graph), then the FP64
 * low-order Newton solves of all unconverged members in ONE cooperative
 * launch (each member on its own share of the co-resident blocks, in
 * proportion to its cells, with its own grid barriers, Newton and PCG
 * iterations and stopping tests) and each member's change of u = (T, E);
 * one host synchronisation per outer iteration.  Each member stops by
 * Eq. relative_tol on its own, exactly as sm_step would: a converged member
 * is skipped by later passes (its tasks, emission and reductions are masked
 * on the device, so the recorded graphs stay valid) and keeps the results
 * of its last iteration.  Each argument is a HOST array of n device
 * pointers laid out as sm_step's (I_prev[i], I_next[i] packed in member i's
 * layout; closures may be NULL or hold NULL entries: the library's own
 * buffer).  stats_host (may be NULL) receives n entries.  Errors as sm_step,
 * plus UNSUPPORTED for params->method = SM_METHOD_CONSISTENT.  Synchronous. */
sm_status sm_batch_step(sm_batch *b, const double *const *scale_dev, const double *const *cv_dev,
                        double *const *T_dev, double *const *E_dev, double *const *F_dev,
                        double *const *moments_dev, const void *const *I_prev_dev,
                        void *const *I_next_dev, double *const *closures_dev,
                        const sm_step_params *params_host, sm_step_stats *stats_host);

/* ------------------------------------------------------------------------
 * Time-dependent high-order problem and its discrete adjoint: the gradient
 * of the time-integrated right-edge leakage with respect to per-cell opacity
 * scales s_K (sigma_{g,K} = s_K f_g(Tbar_K), opacities frozen at the start of
 * each step).  The forward being differentiated is the converged high-order
 * system of each backward-Euler step -- the lumped DG transport of
 * Eq. dgsn_transport with the time term of Eq. smm_be_transport and the
 * nodal energy balance C_v (T - T*)/dt = sum_g sigma_g (phi_g - B_g(T))
 * (Eq. energy_balance) -- which the SM iteration with consistent closures
 * and the unaccelerated iteration both converge to.  Adjoint differentiation
 * is this library's addition; the paper does not differentiate.
 * ---------------------------------------------------------------------- */

/* One backward-Euler step converged by the unaccelerated iteration: a full
 * pass (emission at the current T, sweep, moments) then one Newton step of
 * the nodal energy balance, until ||dT|| <= tol ||T||; a final pass makes
 * I_next the intensity of the converged T.  T_dev[cell][node]: T^n on entry,
 * T^{n+1} on exit; scale_dev[cell]: s_K; cv_dev[cell][node]; I_prev_dev:
 * packed I^n (NULL: zero); I_next_dev: packed I^{n+1} (out).  *iters_host
 * (may be NULL) receives the passes taken.  Needs dt > 0.  Synchronous. */
sm_status sm_ho_step(sm_problem *p, const double *scale_dev, const double *cv_dev, double *T_dev,
                     const void *I_prev_dev, void *I_next_dev, double tol, int max_iter,
                     int *iters_host);

/* Outgoing partial current through the right edge (x = x1) of a packed
 * intensity, lumped at the face's Gauss-Lobatto points:
 * sum_{d: Omega_x > 0} w_d Omega_x sum_g sum_{right-edge nodes} (h_y/2) I.
 * 2D only.  Synchronous. */
sm_status sm_leakage(sm_problem *p, const void *I_dev, double *out_host);

/* One adjoint step, run backwards in time after sm_ho_step produced
 * (T_n, T_np1, I_np1): solves the transposed linearised step by source
 * iteration -- reversed-direction sweeps (the transposed upwind operator of
 * Omega is that of -Omega: the reversed wavefront), the leakage entering as
 * the isotropic inflow dt h_x h_y / 4 through the right edge, the energy
 * multiplier theta per node -- until ||dtheta|| <= tol ||theta||.
 *   psi_next_dev: packed transport multiplier of step n+1 (NULL for the last
 *     step); X_next_dev[cell][node]: the later step's dependence on T^{n+1}
 *     (NULL for the last step);
 *   psi_out_dev (packed) and X_out_dev[cell][node]: the same for step n;
 *   grad_dev[cell]: dJ/ds_K of this step is ADDED to it.
 * The packed multiplier is stored at the original directions' positions
 * (sm_unpack_intensity gives it in canonical order).  2D only; needs dt > 0.
 * Synchronous. */
sm_status sm_adjoint_step(sm_problem *p, const double *scale_dev, const double *cv_dev,
                          const double *T_n_dev, const double *T_np1_dev, const void *I_np1_dev,
                          const void *psi_next_dev, const double *X_next_dev, void *psi_out_dev,
                          double *X_out_dev, double *grad_dev, double tol, int max_iter,
                          int *iters_host);

/* Number of kernels this problem has launched since creation. */
int64_t sm_launch_count(const sm_problem *p);

const char *sm_last_error(void);
const char *sm_status_string(sm_status s);

#ifdef __cplusplus
}
#endif
#endif /* SM_TRT_H */
