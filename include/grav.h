/*
 * grav.h -- C ABI of libgrav, the GB300 (sm_103a) implementation of the
 * data-parallel hot path of adaptive force updates (Grudic 2020, "Accelerating
 * self-gravitating hydrodynamics simulations with adaptive force updates",
 * Sections 2 and 3).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Array pointers are CUDA DEVICE pointers owned by the caller.  The library
 *    never allocates device memory: calls that need scratch space take a
 *    caller-provided `workspace` of at least the size the matching
 *    `*_workspace_bytes` query returns (256-byte aligned).
 *  - Every compute call is asynchronous on `stream` (a cudaStream_t passed as
 *    void*; NULL is the legacy default stream) and returns an int status:
 *    GRAV_OK on success, a negative GRAV_E* code otherwise.  Host-side argument
 *    checks happen before anything is launched; a call that returns an error
 *    has launched nothing unless the code is GRAV_ECUDA.
 *  - Conditions that can only be seen on the device (non-finite inputs,
 *    out-of-range indices or bins, a bounded wait that gave up) are OR-ed as
 *    GRAV_FLAG_* bits into the optional device word `flags_dev` (nullable);
 *    the caller reads it when it wants to.  No exception, abort or trap
 *    crosses this boundary and no kernel spins without an iteration bound.
 *  - grav_last_error_string() describes the last failing call of the calling
 *    host thread.
 *  - Layouts: positions, velocities, accelerations and jerks are [n][3]
 *    row-major FP64; the tidal tensor is [n][6] FP64 in the order
 *    xx, yy, zz, xy, xz, yz; masses, potentials and timesteps are [n] FP64;
 *    flags are one byte per element (0 = false, non-zero = true).
 *
 * Notation: element i's position x_i, velocity v_i, mass m_i; d = x_j - x_i,
 * v_ji = v_j - v_i, r = |d|; the softened kernel is the cubic spline of
 * compact support radius h, entering through f(r) = M(<r)/(m r^3) and
 * g(r) = f'(r)/r (f = r^-3 and g = -3 r^-5 for r >= h).
 */
#ifndef GRAV_H
#define GRAV_H

#include <stdint.h>

#if defined(__GNUC__)
#define GRAV_API __attribute__((visibility("default")))
#else
#define GRAV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define GRAV_OK          0
#define GRAV_EINVAL     -1   /* bad argument (null pointer, size, alignment, parameter) */
#define GRAV_ECUDA      -2   /* a CUDA runtime call or kernel launch failed */
#define GRAV_ENONFINITE -3   /* reserved: non-finite input (reported via GRAV_FLAG_NONFINITE) */
#define GRAV_ETIMEOUT   -4   /* reserved: bounded device wait expired (GRAV_FLAG_TIMEOUT) */
#define GRAV_ENOMEM     -5   /* workspace smaller than the matching *_workspace_bytes */

/* Device flag bits OR-ed into *flags_dev. */
#define GRAV_FLAG_NONFINITE 1  /* a position, velocity, mass or a_bar was NaN or Inf */
#define GRAV_FLAG_TIMEOUT   2  /* a bounded wait on a shared-memory copy gave up */
#define GRAV_FLAG_BADINDEX  4  /* a target index outside [0, n_src), or a bin outside [0, k_max] */
#define GRAV_FLAG_NOCONVERGE 8 /* a support iteration of grav_soft_solve ran out of iterations */
#define GRAV_FLAG_OVERFLOW  16 /* a tree build or walk exceeded its node bound (not expected) */

/* Arithmetic of the force sums. */
#define GRAV_F64   0  /* all pair arithmetic and sums in FP64 */
#define GRAV_MIXED 1  /* FP64 positions offset to FP32 per source tile, FP32 pair
                         arithmetic, compensated FP32 tile sums, FP64 final sums */

typedef struct grav_params {
    double G;            /* gravitational constant (> 0) */
    double h;            /* softening support radius (> 0); Newtonian beyond h */
    double eta;          /* tidal-timestep tolerance of Eq. (tidaltimestep) (> 0), e.g. 0.01 */
    int32_t precision;   /* GRAV_F64 or GRAV_MIXED */
    int32_t want_pot;    /* non-zero: also evaluate the potential Phi_i */
    int32_t tile_config; /* -1 = library default (grav_default_tile_config), else an
                            index < grav_tile_config_count(precision) */
    int32_t max_split;   /* upper bound on source splits per target block; 0 = default */
    double box;          /* > 0: periodic cube [0, box)^3, every pair taken to its nearest
                            periodic image (the paper's Zeldovich setting); 0: open */
} grav_params;

/* Describes one tile configuration (for the autotuner). */
typedef struct grav_tile_info {
    int32_t threads;          /* threads per CTA */
    int32_t targets_per_thread;
    int32_t sources_per_tile; /* S: sources staged per shared-memory tile */
    int32_t targets_per_block;/* threads * targets_per_thread */
    int32_t unroll;           /* unroll depth of the Newtonian pair loop (mixed), 0 if fixed */
    int32_t shared_accumulators; /* 1: compensated sums kept in shared memory */
} grav_tile_info;

/* One independent system of a batched launch: elements [offset, offset + n)
 * of the packed arrays, softened with support h (Eq. 4 per system; h = 0:
 * the call's grav_params h).  Systems are given in ascending,
 * non-overlapping order. */
typedef struct grav_system {
    int64_t offset;
    int64_t n;
    double h;
} grav_system;

GRAV_API const char *grav_last_error_string(void);
GRAV_API const char *grav_version(void);
GRAV_API int32_t grav_tile_config_count(int32_t precision);
/* Describes configuration `index` of a precision; index -1 describes the
 * default of a small open-boundary evaluation.  GRAV_EINVAL for a bad
 * precision or index, or a NULL out. */
GRAV_API int grav_tile_config(int32_t precision, int32_t index, grav_tile_info *out);
/* The configuration that tile_config = -1 selects for an evaluation of
 * n_targets targets (the n_idx_max of the call): open boundaries
 * (periodic = soft = 0), a periodic box (periodic != 0) or adaptive softening
 * (soft != 0).  768-thread CTAs from 8192 targets, 256-thread CTAs below
 * (the same in every mode).  Returns
 * the index (>= 0), or GRAV_EINVAL for a bad precision or n_targets < 0.  A
 * property of the library's kernels; the paper has no counterpart. */
GRAV_API int32_t grav_default_tile_config(int32_t precision, int32_t periodic, int32_t soft,
                                          int64_t n_targets);

/* ------------------------------------------------------------------------ */
/* Selection: Eq. (3), Eq. (updatecondition) and Section 3's power-of-two     */
/* block timesteps.  Time is counted in integer ticks of dt_min; an element   */
/* of bin k (0 <= k <= k_max <= 62) takes steps of 2^(k_max-k) ticks and is   */
/* active at ticks that are multiples of its step.                            */
/* ------------------------------------------------------------------------ */

/*
 * grav_select_due -- Eq. (3) and Eq. (updatecondition).
 * For each element i active at `tick` (>= 0): tf_ticks[i] += 2^(k_max-bin[i]);
 * due_out[i] = (tf_ticks[i]*dt_min >= q_f*dt_grav[i]) evaluated as two
 * correctly rounded FP64 products and a compare (bit-identical on any IEEE
 * machine); a due element's counter is reset to 0 because its force is
 * re-evaluated in this substep.  active_out/due_out get 1/0; inactive elements
 * keep their counter and get 0/0.  dt_grav[i] == 0 means "never evaluated"
 * and is always due.  A bin outside [0, k_max] makes the element inactive and
 * sets GRAV_FLAG_BADINDEX.
 *   n         number of elements (>= 0)
 *   bin       int8[n]  (in)
 *   tf_ticks  int64[n] (in/out) ticks since the last force evaluation
 *   dt_grav   f64[n]   (in) tidal timestep from each element's last evaluation
 *   q_f       update tolerance (>= 0); dt_min > 0 the tick length
 *   active_out, due_out  uint8[n] (out)
 *   elapsed_out int64[n] (out, nullable): for due elements, T_f before the
 *             reset (ticks since the previous evaluation); others untouched
 */
GRAV_API int grav_select_due(int64_t n, int64_t tick, int32_t k_max, const int8_t *bin,
                    int64_t *tf_ticks, const double *dt_grav, double q_f, double dt_min,
                    uint8_t *active_out, uint8_t *due_out, int64_t *elapsed_out,
                    int32_t *flags_dev, void *stream);

/*
 * grav_compact_active -- the due set as an index list (follows from
 * Eq. (updatecondition): only due elements are evaluated).
 * idx_out[0..c) = the indices i with flags[i] != 0, ascending; *count_dev = c
 * written on the device (no host synchronisation).  idx_out has room for n
 * entries; entries past c are left unchanged.  n <= INT32_MAX.
 * workspace: >= grav_compact_workspace_bytes(n) bytes.
 */
GRAV_API int64_t grav_compact_workspace_bytes(int64_t n);
GRAV_API int grav_compact_active(int64_t n, const uint8_t *flags, int32_t *idx_out, int32_t *count_dev,
                        void *workspace, int64_t workspace_bytes, void *stream);

/*
 * grav_compact_active_noalloc -- the same compaction as grav_compact_active
 * (identical output) for callers that cannot allocate device memory, so
 * cannot provide a workspace: for example a host code that has reserved the
 * whole device memory pool for itself, or a time-step loop that must not
 * stall on cudaMalloc's implicit device synchronisation.  The paper has no
 * counterpart; this is a property of the library, not of the method.
 *  - Allocates nothing: its scratch (one int32 per block of 4096 flags) is a
 *    fixed array inside the library, present on every device that loads the
 *    library until the process exits (64 KiB per device).
 *  - n is limited to GRAV_COMPACT_NOALLOC_MAX_N (2^26); larger n returns
 *    GRAV_EINVAL before anything is launched.
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any
 *    stream capture.  The address is kept per device ordinal until the
 *    process exits and is not looked up again: after cudaDeviceReset on a
 *    device (which ends its primary context) the kept address may no longer
 *    be valid there, so do not call this entry point on a device after
 *    resetting it.
 *  - All calls share the array.  Each call writes every scratch element it
 *    reads, so nothing needs clearing between calls, but calls whose kernels
 *    overlap on the GPU (other streams, other threads) race on it: serialise
 *    them.
 */
#define GRAV_COMPACT_NOALLOC_MAX_N 67108864
GRAV_API int grav_compact_active_noalloc(int64_t n, const uint8_t *flags, int32_t *idx_out,
                                         int32_t *count_dev, void *stream);

/*
 * grav_predict -- the first-order jerk predictor, Eq. (jerkupdate), in closed
 * form: for active, not-due elements
 *     a_out[i] = a_last[i] + j_last[i] * (tf_ticks[i] * dt_min)
 * (one correctly rounded product for the elapsed time, then a product and a
 * sum per component, no fused multiply-add); for active due elements
 * a_out[i] = a_last[i]; inactive elements are not written.  The paper's
 * incremental update g += j dt_i summed over the steps since the last
 * evaluation equals this closed form in exact arithmetic.
 * a_out may alias neither a_last nor j_last.
 */
GRAV_API int grav_predict(int64_t n, const uint8_t *active, const uint8_t *due, const double *a_last,
                 const double *j_last, const int64_t *tf_ticks, double dt_min, double *a_out,
                 void *stream);

/*
 * grav_push_history -- log past accelerations for the polynomial predictor
 * (Section 2.2: "logging some number of past g_i values").  For every
 * element with due[i] != 0, called after grav_select_due and BEFORE the new
 * evaluation overwrites a_last and dt_grav:
 *     a_prev[i]  = a_last[i]                       ([n][3])
 *     dt_prev[i] = elapsed[i] * dt_min             (gap between its last two
 *                                                  evaluations, one rounding)
 * where elapsed comes from grav_select_due's elapsed_out; an element never
 * evaluated before (dt_grav[i] == 0) gets dt_prev[i] = 0 (no history).
 * Only due elements are written.  a_prev may not alias a_last.  Nothing
 * depends on the absolute tick, so a loop of 2^k_max ticks captured as a
 * CUDA graph replays correctly.
 */
GRAV_API int grav_push_history(int64_t n, const uint8_t *due, const int64_t *elapsed,
                               const double *dt_grav, const double *a_last, double *a_prev,
                               double *dt_prev, double dt_min, void *stream);

/*
 * grav_predict_poly -- the first-order polynomial predictor of Section 2.2,
 * the paper's alternative to the jerk: for active, not-due elements with
 * dt_prev > 0,
 *     a_out = a_last + (a_last - a_prev) * (tau / dt_prev),  tau = T_f dt_min
 * (tau, the ratio, the difference, the product and the sum each correctly
 * rounded, no fused multiply-add); with dt_prev = 0 (a single evaluation so
 * far) and for active due elements a_out = a_last; inactive elements are not
 * written.  a_out may alias neither a_last nor a_prev.
 */
GRAV_API int grav_predict_poly(int64_t n, const uint8_t *active, const uint8_t *due,
                               const double *a_last, const double *a_prev, const double *dt_prev,
                               const int64_t *tf_ticks, double dt_min, double *a_out, void *stream);

/*
 * grav_assign_bins -- Section 2's dt_i = min(dt_grav_i, dt_hydro_i) placed on
 * Section 3's power-of-two bins, for elements active at `tick`.
 * The target bin is the smallest k in [0, k_max] with dt_max * 2^-k <= dt_i
 * (exact comparison of mantissas and exponents; dt_i = +inf -> 0; dt_i <= 0 or
 * NaN -> k_max); a step may only grow at a tick that is a multiple of the new
 * step, so the bin is raised to the smallest k aligned with `tick`.
 * dt_hydro is nullable (no limit).  Inactive elements keep their bin.
 */
GRAV_API int grav_assign_bins(int64_t n, int64_t tick, int32_t k_max, double dt_max, const uint8_t *active,
                     const double *dt_grav, const double *dt_hydro, int8_t *bin, void *stream);

/* ------------------------------------------------------------------------ */
/* Force evaluation: Eq. (4), Section 3's tidal tensor and tidal timestep.    */
/* ------------------------------------------------------------------------ */

/*
 * grav_eval_active -- direct summation over all n_src sources j != i of
 *   a_i   = G sum_j m_j f(r) d                                      (g of the paper)
 *   j_i   = G sum_j m_j [ f(r) v_ji + g(r) (d . v_ji) d ]          (Eq. 4, softened)
 *   T_i   = -G sum_j m_j [ f(r) I + g(r) d d^T ]   = d a_i / d x_i (Section 3)
 *   Phi_i = -G sum_j m_j phi(r)                                     (if want_pot)
 *   dt_grav_i = sqrt(eta) (||T_i||_F^2 / 6)^(-1/4)            (Eq. tidaltimestep)
 * at the targets i = idx[0..c), c = *n_idx_dev (device word, e.g. from
 * grav_compact_active) or n_idx_max when n_idx_dev is NULL; idx NULL means
 * targets 0..n_src-1 (then n_idx_max must equal n_src).  Results are
 * scattered to row i of acc [n_src][3], jerk [n_src][3], tidal [n_src][6],
 * pot [n_src] (nullable unless want_pot) and dt_grav [n_src] (nullable); rows
 * of non-targets are not written.  The self term j == i is excluded by index.
 * c must not exceed n_idx_max (the launch is sized for n_idx_max).
 * workspace: >= grav_eval_workspace_bytes(p, n_src, n_idx_max) bytes.
 */
GRAV_API int64_t grav_eval_workspace_bytes(const grav_params *p, int64_t n_src, int64_t n_idx_max);
GRAV_API int grav_eval_active(const grav_params *p, int64_t n_src, const double *pos, const double *vel,
                     const double *mass, const int32_t *idx, const int32_t *n_idx_dev,
                     int64_t n_idx_max, double *acc, double *jerk, double *tidal, double *pot,
                     double *dt_grav, int32_t *flags_dev, void *workspace,
                     int64_t workspace_bytes, void *stream);

/*
 * grav_eval_backward -- adjoint of grav_eval_active over all n elements as
 * targets (the paper has no adjoint; derived from Eq. 4 and the tidal tensor).
 * For a loss L(a, W) with a_bar = dL/da ([n][3], nullable = 0) and
 * w_bar = dL/dW, W = 1/2 sum_i m_i Phi_i the potential energy:
 *   pos_bar_k  = T_k a_bar_k + G m_k sum_{i!=k} [ f a_bar_i + g d (d . a_bar_i) ]
 *                - w_bar m_k a_k
 *   mass_bar_k = -G sum_{i!=k} f (d . a_bar_i) + w_bar Phi_k,   d = x_i - x_k.
 * acc, tidal and pot are the forward results at all n elements (acc and pot
 * are read only when w_bar != 0, tidal only when a_bar is given).  Pair terms
 * are recomputed, never stored.  pos_bar [n][3] and mass_bar [n] are written.
 * workspace: >= grav_backward_workspace_bytes(p, n) bytes.
 */
GRAV_API int64_t grav_backward_workspace_bytes(const grav_params *p, int64_t n);
GRAV_API int grav_eval_backward(const grav_params *p, int64_t n, const double *pos, const double *mass,
                       const double *a_bar, double w_bar, const double *acc, const double *tidal,
                       const double *pot, double *pos_bar, double *mass_bar, int32_t *flags_dev,
                       void *workspace, int64_t workspace_bytes, void *stream);

/*
 * grav_eval_backward_batched -- grav_eval_backward over many independent
 * systems in one persistent launch (the batched form of the adjoint above,
 * as grav_eval_batched is of the force evaluation).  systems [n_sys] is the
 * DEVICE array of grav_eval_batched ({offset, n, h}, h = 0: p->h); every
 * element of a system is a target, and its sums run over its own system's
 * elements only, with its system's support h.  Work items are (system,
 * target block) pairs taken longest system first through an atomic ticket;
 * each element's sums are formed by one CTA over its system's tiles in a
 * fixed order, so a system's results equal grav_eval_backward on that system
 * alone with max_split = 1, bit for bit.  Elements of no system, and of a
 * system that is skipped (out of range, overlapping, bad h: see
 * grav_eval_batched; GRAV_FLAG_BADINDEX), are not written, except that with
 * a_bar == NULL the elementwise potential-energy terms are written at every
 * element of [0, n_total).  Open boundaries only (p->box = 0).
 * workspace: >= grav_backward_batched_workspace_bytes(p, n_sys, n_total).
 */
GRAV_API int64_t grav_backward_batched_workspace_bytes(const grav_params *p, int32_t n_sys,
                                                       int64_t n_total);
GRAV_API int grav_eval_backward_batched(const grav_params *p, int32_t n_sys, const grav_system *systems,
                                        int64_t n_total, const double *pos, const double *mass,
                                        const double *a_bar, double w_bar, const double *acc,
                                        const double *tidal, const double *pot, double *pos_bar,
                                        double *mass_bar, int32_t *flags_dev, void *workspace,
                                        int64_t workspace_bytes, void *stream);

/*
 * grav_eval_batched -- grav_eval_active over many independent systems in one
 * persistent launch (pattern (2) of the batched workloads; the paper's method
 * per system is unchanged).  systems [n_sys] is a DEVICE array of
 * {offset, n, h} describing systems packed back to back in pos/vel/mass
 * (ascending, non-overlapping, inside [0, n_total)); the sources of a target
 * are the elements of its own system only, and its sums use its system's
 * support h (p->h where h = 0), rounded to FP32 exactly as the host rounds
 * p->h, so a system's results do not depend on how h reached the kernel.  idx[0..c) are GLOBAL target
 * indices in ascending order (for example grav_compact_active over the
 * packed due flags), c = *n_idx_dev or n_idx_max; each system's targets are
 * found on the device by binary search, so counts never visit the host and
 * the call can be captured in a CUDA graph.  Outputs are scattered to the
 * targets' rows as in grav_eval_active.
 * Work is split into (system, target block) items, ordered by decreasing
 * per-item cost (system size) and taken by a fixed grid of CTAs through an
 * atomic ticket; each target's sum is formed by one CTA over its system's
 * tiles in a fixed order, so results do not depend on scheduling and equal
 * grav_eval_active on that system alone with max_split = 1.
 * A system that is out of range, overlaps its predecessor or has an h that
 * is neither 0 nor finite and positive is skipped and sets
 * GRAV_FLAG_BADINDEX; targets that belong to no system are not evaluated.
 * n_sys <= GRAV_BATCH_MAX_SYSTEMS.
 * workspace: >= grav_batched_workspace_bytes(p, n_sys, n_total) bytes.
 */
#define GRAV_BATCH_MAX_SYSTEMS 16384
GRAV_API int64_t grav_batched_workspace_bytes(const grav_params *p, int32_t n_sys, int64_t n_total);
GRAV_API int grav_eval_batched(const grav_params *p, int32_t n_sys, const grav_system *systems,
                               int64_t n_total, const double *pos, const double *vel,
                               const double *mass, const int32_t *idx, const int32_t *n_idx_dev,
                               int64_t n_idx_max, double *acc, double *jerk, double *tidal,
                               double *pot, double *dt_grav, int32_t *flags_dev, void *workspace,
                               int64_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Adaptive softening: Section 3 runs every problem with fully adaptive       */
/* softening and the extra force terms of Price & Monaghan (2007) that keep   */
/* the energy conserved.  Readings (the paper gives no formulas): each        */
/* element i has its own support h_i, fixed by the mass-density constraint    */
/* (4 pi/3) h_i^3 rho_i = n_ngb m_i, rho_i = sum_j m_j W(r_ij, h_i) with the  */
/* self term; a pair uses the mean of the kernels of supports h_i and h_j;    */
/* the correction term makes a_i = -grad_i U / m_i for the potential energy   */
/* U = (1/2) sum_i m_i Phi_i with every h following the constraint.           */
/* ------------------------------------------------------------------------ */

typedef struct grav_soft_params {
    double n_ngb;        /* effective neighbour number of the constraint (> 32/3, e.g. 32) */
    double tol;          /* stop when |(4 pi/3) h^3 rho - n_ngb m| <= tol n_ngb m (>= 1e-15) */
    int32_t max_iter;    /* iterations per element (1..10000); then GRAV_FLAG_NOCONVERGE */
    int32_t pad;
} grav_soft_params;

/*
 * grav_soft_solve -- supports and correction coefficients of n elements.
 * Per element: safeguarded Newton iterations on h (starting from h_inout[i]
 * > 0, each step limited to a factor of 2 and kept in a bracket; a step
 * leaving it doubles h or bisects) until the constraint holds to tol; then
 * from the sums at that h
 *   Omega_i = 1 + h_i / (3 rho_i) sum_j m_j dW(r_ij, h_i)/dh      (j = i included)
 *   zeta_i  = -h_i / (3 rho_i Omega_i) sum_{j != i} m_j dpsi(r_ij, h_i)/dh
 * (psi the potential kernel; dh/drho = -h/(3 rho)).  All FP64.
 *   pos [n][3], mass [n] (> 0): device, in
 *   h_inout [n]: device, in: starting guesses, out: supports
 *   zeta_out, omega_out [n], iters_out [n] (iterations, -1 if the limit ran
 *   out): device, out, each nullable
 * A mass or guess that is not positive and finite sets GRAV_FLAG_NONFINITE
 * and leaves that element's outputs unwritten.
 * workspace: >= grav_soft_workspace_bytes(n) bytes, 256-byte aligned.
 */
GRAV_API int64_t grav_soft_workspace_bytes(int64_t n);
GRAV_API int grav_soft_solve(const grav_soft_params *sp, int64_t n, const double *pos,
                             const double *mass, double *h_inout, double *zeta_out,
                             double *omega_out, int32_t *iters_out, int32_t *flags_dev,
                             void *workspace, int64_t workspace_bytes, void *stream);

/*
 * grav_eval_soft -- grav_eval_active with per-element supports h_elem [n_src]
 * (device, > 0; p->h is only validated) and, when zeta (device [n_src],
 * nullable) is given, the correction term:
 *   a_i   = G sum_j m_j fbar d
 *           - (G/2) sum_j m_j [zeta_i W_r(r,h_i) + zeta_j W_r(r,h_j)] d / r
 *   j_i   = G sum_j m_j [ fbar v_ji + gbar (d . v_ji) d ]
 *   T_i   = -G sum_j m_j [ fbar I + gbar d d^T ]
 *   Phi_i = -G sum_j m_j (phi(r,h_i) + phi(r,h_j)) / 2
 * with fbar = (f(r,h_i) + f(r,h_j))/2, gbar likewise and W_r = dW/dr; jerk and
 * tidal tensor are those of the averaged pair force at fixed supports.  Open
 * boundaries only (p->box must be 0); targets, outputs, precisions and tile
 * configurations as in grav_eval_active.  A support that is not positive and
 * finite sets GRAV_FLAG_NONFINITE.
 * workspace: >= grav_eval_soft_workspace_bytes(p, n_src, n_idx_max) bytes.
 */
GRAV_API int64_t grav_eval_soft_workspace_bytes(const grav_params *p, int64_t n_src,
                                                int64_t n_idx_max);
GRAV_API int grav_eval_soft(const grav_params *p, int64_t n_src, const double *pos,
                            const double *vel, const double *mass, const double *h_elem,
                            const double *zeta, const int32_t *idx, const int32_t *n_idx_dev,
                            int64_t n_idx_max, double *acc, double *jerk, double *tidal,
                            double *pot, double *dt_grav, int32_t *flags_dev, void *workspace,
                            int64_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Approximate solver: Section 3's oct-tree code.  A node of side L is always */
/* split when it subtends L/r > Theta (Theta = 0.5 in the paper), r the       */
/* distance from the target to the node's centre of mass; optionally also the */
/* relative criterion the paper supplements (a node is opened unless          */
/* G M L^2 <= alpha |a_old| r^4).  Nodes are monopoles: mass, centre of mass  */
/* and mean velocity, so accepted nodes contribute to a, j, T and Phi as one  */
/* moving point mass with the same softened pair terms as the direct sum.     */
/* ------------------------------------------------------------------------ */

typedef struct grav_tree_params {
    double theta;        /* opening angle (>= 0; 0 opens every node: the direct sum) */
    double alpha;        /* relative criterion (0 = off; needs a_old) */
    int32_t leaf_size;   /* a node of at most this many elements is a leaf (1..64) */
    int32_t pad;
} grav_tree_params;

/*
 * grav_eval_tree -- builds the oct-tree of all n elements and evaluates a, j,
 * T, Phi (if p->want_pot) and dt_grav at the targets (idx / n_idx_dev /
 * n_idx_max as in grav_eval_active; with idx NULL every element, walked in
 * tree order), FP64 throughout (p->precision is not used; p->box must be 0).
 * The tree (root cube, 63-bit Morton keys of 2^21 cells per axis, elements
 * ordered by (key, index), leaves of at most leaf_size elements or 21 levels
 * deep, monopole moments summed in order) and every opening decision are
 * defined so that an FP64 evaluation on any machine builds the same tree and
 * takes the same branches.
 *   a_old [n][3]: device, nullable; the previous accelerations for alpha > 0
 *   order_out [n]: device int32, nullable; the elements in tree order
 *   stats_dev [2]: device int64, nullable; [0] nodes built, [1] interactions
 *                  (accepted nodes plus leaf pairs) summed over the targets
 * Requires n < 2^29 and a node bound below 2^31 (about 13 n / leaf_size).
 * workspace: >= grav_tree_workspace_bytes(n, leaf_size) bytes, 256-aligned.
 */
GRAV_API int64_t grav_tree_workspace_bytes(int64_t n, int32_t leaf_size);
GRAV_API int grav_eval_tree(const grav_params *p, const grav_tree_params *tp, int64_t n,
                            const double *pos, const double *vel, const double *mass,
                            const double *a_old, const int32_t *idx, const int32_t *n_idx_dev,
                            int64_t n_idx_max, double *acc, double *jerk, double *tidal,
                            double *pot, double *dt_grav, int32_t *order_out,
                            long long *stats_dev, int32_t *flags_dev, void *workspace,
                            int64_t workspace_bytes, void *stream);

/*
 * grav_selftest_wait_timeout -- failure-detection self-test (not part of the
 * method).  Launches one CTA whose shared-memory barrier waits for a transfer
 * that is never issued; the wait gives up after `limit` polls (1..2^20), sets
 * GRAV_FLAG_TIMEOUT in *flags_dev and the kernel returns.  This call then
 * synchronises `stream`, reads the flag word and returns GRAV_ETIMEOUT when
 * the bit is set (the expected outcome) or GRAV_OK.  Nothing faults, traps or
 * hangs, and the CUDA context remains usable.
 */
GRAV_API int grav_selftest_wait_timeout(uint32_t limit, int32_t *flags_dev, void *stream);

/* ------------------------------------------------------------------------ */
/* Measurement helper (not part of the method).                               */
/* ------------------------------------------------------------------------ */

/*
 * grav_measure_fma_peak -- times a register-resident FMA throughput kernel
 * (FP32 when precision == GRAV_MIXED, FP64 when GRAV_F64, packed FP32x2
 * when GRAV_PEAK_F32X2) on the current
 * device with CUDA events and returns the achieved FLOP/s (FMA = 2 flops).
 * Synchronises the stream.  Used to state the CUDA-core peak that the force
 * kernels are measured against.
 */
#define GRAV_PEAK_F32X2 2
GRAV_API int grav_measure_fma_peak(int32_t precision, double seconds_target, double *flops_per_s,
                          void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GRAV_H */
