/*
 * osqp_gb300.h — C ABI of a GB300-native (sm_103a) implementation of the
 * operator-splitting QP method of Stellato et al., "OSQP: An Operator
 * Splitting Solver for Quadratic Programs" (arXiv:1711.08013).
 *
 *   minimize  ½ xᵀPx + qᵀx   subject to  l ≤ Ax ≤ u          (Eq. pb:qp, §1.1)
 *
 * Every step of the solve runs in this library's own CUDA kernels: modified
 * Ruiz equilibration (Alg. 2, §5.1), the per-constraint ρ vector (§5.2), the
 * ADMM iteration of Algorithm 1 (§3.2) with the indirect linear solve of
 * §3.1 — Jacobi-preconditioned conjugate gradients on
 * (P + σI + AᵀRA) x̃ = σx − q + Aᵀ(Rz − y), z̃ = Ax̃ — the unscaled termination
 * and infeasibility tests (§3.4 in the scaled form of §5.1), adaptive ρ̄ with
 * an on-device Jacobi rebuild (§5.2), and unscaling (Eq. pb:scaled_qp).
 *
 * Conventions shared by every entry point
 *  - Matrices are CSC (§7): column pointers (n_cols+1), row indices sorted
 *    and unique within each column, values.  P is given by its upper
 *    triangle (row ≤ column); A is m × n.  Indices are int32, values FP64.
 *  - A bound with |value| ≥ 1e20 (or ±INFINITY) is infinite.  Row i is an
 *    equality row when l_i == u_i exactly (§5.2).
 *  - Host pointers unless the name says _device.  The library copies all
 *    inputs; the caller keeps ownership of its arrays.  The solver owns its
 *    device memory (one allocation, sized at setup) until osqp_cleanup.
 *  - Every call returns OSQP_OK (0) or a negative OSQP_ERR_* code and never
 *    aborts; a failed call leaves the solver usable unless it returned
 *    OSQP_ERR_CUDA or OSQP_ERR_DEVICE.
 *  - A solver is bound to the CUDA device current at setup and to the stream
 *    given there (NULL = the legacy default stream).  One host thread per
 *    solver; different solvers may be used from different threads.
 */
#ifndef OSQP_GB300_H
#define OSQP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define OSQP_OK 0
#define OSQP_ERR_DIMS (-1)      /* n < 1, m < 0, or sizes that disagree */
#define OSQP_ERR_CSC (-2)       /* bad pointers / unsorted / out-of-range indices / P not upper */
#define OSQP_ERR_NONFINITE (-3) /* NaN or Inf in P, A or q; NaN in l or u */
#define OSQP_ERR_LGTU (-4)      /* some l_i > u_i */
#define OSQP_ERR_SETTINGS (-5)  /* α ∉ (0,2), ρ ≤ 0, σ ≤ 0, ε < 0, … */
#define OSQP_ERR_CUDA (-6)      /* a CUDA runtime call failed */
#define OSQP_ERR_OOM (-7)       /* device allocation failed */
#define OSQP_ERR_ARG (-8)       /* NULL solver or required pointer */
#define OSQP_ERR_DEVICE (-9)    /* a device-side wait ran out of time (grid barrier) */
#define OSQP_ERR_LIMIT (-10)    /* size beyond what this entry point supports */

/* ---- solver status (osqp_info.status) ----------------------------------- */
#define OSQP_UNSOLVED 0
#define OSQP_SOLVED 1
#define OSQP_MAX_ITER 2
#define OSQP_PRIMAL_INFEASIBLE 3 /* certificate: osqp_get_certificate(prim_inf_y) */
#define OSQP_DUAL_INFEASIBLE 4   /* certificate: osqp_get_certificate(dual_inf_x) */
#define OSQP_TIME_LIMIT 5
#define OSQP_NUMERICAL_ERROR 6   /* non-finite residuals */

/* ---- precision modes ------------------------------------------------------ */
#define OSQP_PRECISION_FP64 0       /* matrices, PCG and iterates in FP64 */
#define OSQP_PRECISION_FP32_MIXED 1 /* scaled matrices and PCG vectors in FP32,
                                       CG scalars in double-float on FP32
                                       instructions; iterates, residual norms,
                                       termination, ρ ratios and certificates
                                       in FP64.  The tolerances are met on the
                                       problem with its scaled matrices rounded
                                       to FP32 */

typedef struct {
  int32_t n_rows, n_cols, nnz;
  const int32_t* colptr; /* n_cols + 1 */
  const int32_t* rowind; /* nnz */
  const double* val;     /* nnz */
} osqp_csc;

typedef struct {
  double rho;                    /* ρ̄⁰ (§5.2), default 0.1 */
  double sigma;                  /* σ (§5.2), default 1e-6 */
  double alpha;                  /* relaxation α ∈ (0,2) (§5.2), default 1.6 */
  double eps_abs, eps_rel;       /* §3.4, defaults 1e-3 (§7) */
  double eps_pinf, eps_dinf;     /* §3.4, defaults 1e-4 (§7) */
  double adaptive_rho_tolerance; /* update ρ̄ when ≥ this factor away (§5.2), default 5 */
  double eps_equil;              /* Alg. 2 stopping tolerance, default 1e-3 */
  double pcg_tol_fraction;       /* κ: PCG stops at ‖r‖∞ ≤ κ·min(‖r̄_prim‖∞, ‖r̄_dual‖∞)
                                    of the last check, default 0.15 */
  double pcg_tol_floor;          /* τ: and never below τ·‖rhs‖∞, default 1e-10; in the
                                    FP32-mixed mode also never below 1e-5·‖r⁰‖∞ of the
                                    iteration (its residual is recomputed in FP64 at the
                                    next ADMM iteration) */
  double time_limit;             /* seconds of device time for one solve, 0 = none */
  int32_t max_iter;              /* ADMM iterations, default 4000 */
  int32_t check_interval;        /* termination checked every k iterations, default 25 */
  int32_t adaptive_rho;          /* 0/1, default 1 */
  int32_t scaling_iters;         /* Ruiz passes (0 = no scaling), default 10 */
  int32_t max_rho_updates;       /* default 20 */
  int32_t pcg_max_iter;          /* PCG iterations per ADMM iteration, default 100 */
  int32_t precision;             /* OSQP_PRECISION_*, default FP64 */
  int32_t warm_start;            /* 1: osqp_solve starts from the current iterates
                                    (§6); 0: from zero.  Default 1 */
  int32_t launch;                /* 0 auto, 1 one persistent block, 2 whole-GPU
                                    cooperative grid, 3 one thread-block cluster
                                    of 8 CTAs (OSQP_ERR_CUDA at setup if the
                                    device cannot host such a cluster) */
  int32_t polish;                /* 1: solution polishing (§4) after a solved run:
                                    active sets from the sign of y, the
                                    δ-regularised reduced KKT system of Eq.
                                    (kkt_polish_reg) solved by FP64 Jacobi-PCG in
                                    eliminated form, iterative refinement (Eq.
                                    iterative_refinement); the result replaces the
                                    ADMM solution only when y has the signs of Eq.
                                    (compl_slack) on the active rows and both
                                    residuals are no larger.  Default 0 */
  int32_t polish_refine_iter;    /* refinement passes, default 3 */
  double delta;                  /* δ of Eq. (kkt_polish_reg), default 1e-6 */
  int32_t autotune;              /* 1 = time the candidate row partitions (group
                                    widths 1…32) at setup and use the fastest: per
                                    shape class of matrices in osqp_batch_setup, per
                                    matrix in osqp_setup on the whole-GPU grid team;
                                    0 = the row-length rule.  Default 1 */
  int32_t pad2;
} osqp_settings;

typedef struct {
  int32_t status, iter, pcg_iters, rho_updates, ruiz_passes, launch;
  double obj_val;    /* ½xᵀPx + qᵀx of the returned x */
  double prim_res;   /* ‖Ax − z‖∞ at the last check (unscaled, §3.4) */
  double dual_res;   /* ‖Px + q + Aᵀy‖∞ at the last check (unscaled) */
  double rho_estimate;
  double setup_time; /* seconds: scaling, ρ and Jacobi build (device events) */
  double solve_time; /* seconds: the ADMM iterations and unscaling (device events) */
  int32_t polished;  /* 1 polished solution returned, -1 polishing rejected, 0 not run */
  int32_t pad;
} osqp_info;

typedef struct osqp_solver osqp_solver;

/* Fill *s with the defaults of §5.2 and §7 and this library's readings. */
void osqp_set_default_settings(osqp_settings* s);

/* Text for an OSQP_ERR_* code or an OSQP_* status (static storage). */
const char* osqp_error_message(int32_t code);

/* §1.1 problem statement and §7 CSC input.  Validates, builds the sparse
 * structure of [P̄ Āᵀ] and Ā, allocates all device memory, copies the data
 * and runs Ruiz scaling, the ρ vector and the Jacobi diagonal on the device.
 * stream: a cudaStream_t or NULL.  On success *out owns the solver. */
int32_t osqp_setup(osqp_solver** out, const osqp_csc* P_upper, const double* q,
                   const osqp_csc* A, const double* l, const double* u,
                   const osqp_settings* settings, void* stream);

/* Run Algorithm 1 to termination on the solver's stream and wait for it;
 * fills the info returned by osqp_get_solution. */
int32_t osqp_solve(osqp_solver* s);

/* As osqp_solve, but only enqueues the work on the stream (no host wait).
 * Results are valid once the stream reaches this point. */
int32_t osqp_solve_async(osqp_solver* s);

/* §6 "vectors as parameters": new q, l, u (host, NULL = unchanged) are
 * scaled with the stored D, E, c; equality rows and the ρ vector / Jacobi
 * diagonal are rebuilt.  The iterates are kept (warm start). */
int32_t osqp_update_vectors(osqp_solver* s, const double* q, const double* l, const double* u);

/* §6 "matrices as parameters": new values of P (upper) and A in the CSC
 * order given at setup (host, NULL = unchanged).  Ruiz scaling, ρ and the
 * Jacobi diagonal are recomputed; no symbolic work is repeated. */
int32_t osqp_update_matrices(osqp_solver* s, const double* P_val, const double* A_val);

/* Reload every numeric input from HOST memory (same layouts: P_val
 * nnz(P_upper), q n, A_val nnz(A), l m, u m), rescale and reset the
 * iterates; enqueued on the solver's stream (the copies are asynchronous
 * when the host arrays are page-locked).  Inputs are not validated beyond
 * NULL checks. */
int32_t osqp_load_data(osqp_solver* s, const double* P_val, const double* q,
                       const double* A_val, const double* l, const double* u);

/* Reload every numeric input from DEVICE memory (same layouts as above:
 * P_val nnz(P_upper), q n, A_val nnz(A), l m, u m) and rescale, enqueued on
 * the solver's stream without a host wait.  Iterates are reset to zero. */
int32_t osqp_load_data_device(osqp_solver* s, const double* P_val, const double* q,
                              const double* A_val, const double* l, const double* u);

/* Set ρ̄ (> 0): rebuilds the ρ vector and the Jacobi diagonal on the
 * device; no refactorisation exists on this path (§3.1, indirect method). */
int32_t osqp_update_rho(osqp_solver* s, double rho_bar);

/* §6 warm start: x⁰ = D⁻¹x, z⁰ = Āx⁰, y⁰ = cE⁻¹y (host, NULL = zero). */
int32_t osqp_warm_start(osqp_solver* s, const double* x, const double* y);

/* Copy the last solution (unscaled: x = Dx̄, z = E⁻¹z̄, y = c⁻¹Eȳ) to host
 * arrays (any may be NULL) and the info of the last solve (also after
 * osqp_solve_async).  Waits for the stream. */
int32_t osqp_get_solution(osqp_solver* s, double* x, double* y, double* z, osqp_info* info);

/* Enqueue device-to-device copies of the unscaled x (n) and y (m). */
int32_t osqp_get_solution_device(osqp_solver* s, double* x_device, double* y_device);

/* Infeasibility certificates of §5.1: c⁻¹Eδȳ (m) and Dδx̄ (n); zero unless
 * the status is the matching infeasibility. */
int32_t osqp_get_certificate(osqp_solver* s, double* prim_inf_y, double* dual_inf_x);

/* Release device memory and the solver. */
int32_t osqp_cleanup(osqp_solver* s);

/* ---- batched solves -------------------------------------------------------
 * Many independent QPs of the form of Eq. (pb:qp), each with its own sizes
 * and sparsity, resident on the device together and solved by one persistent
 * launch: every CTA takes whole problems from a device work counter (largest
 * first) and runs the complete solve of the single-problem entry points for
 * them (Alg. 2 scaling, Algorithm 1 with PCG, §3.4/§5.1 termination, §5.2 ρ̄
 * adaptation).  Problems share no reduction, so a problem's result does not
 * depend on which other problems are in the batch (it may depend, at the
 * rounding level, on whether one CTA or a cluster solved it; see below).
 *
 * Work order is longest first: by each problem's device time in its previous
 * launch when every problem of the launch has one, else by size.  In a
 * whole-batch launch with more problems than CTAs and known times, the
 * problems whose time exceeds the fair share (total / CTAs) are solved
 * by clusters of 8 CTAs on a second stream beside the one-CTA kernel (they
 * would otherwise set the wall time); osqp_batch_get reports launch = 3 for
 * them.  settings->launch = 1 keeps every problem on one CTA. */
typedef struct osqp_batch osqp_batch;

/* count problems; P_upper[i], A[i] (host CSC as for osqp_setup) and
 * q[i], l[i], u[i] (host arrays).  One device allocation holds everything.
 * The settings apply to every problem; settings->launch other than 1 only
 * allows the heavy-problem clusters described above. */
int32_t osqp_batch_setup(osqp_batch** out, int32_t count, const osqp_csc* P_upper,
                         const double* const* q, const osqp_csc* A, const double* const* l,
                         const double* const* u, const osqp_settings* settings, void* stream);

/* Solve every problem and wait; problems marked by setup, osqp_batch_reset
 * or matrix data are scaled first, problems whose vectors changed are
 * refreshed, all others warm-start from their last iterates (§6) unless
 * settings->warm_start == 0. */
int32_t osqp_batch_solve(osqp_batch* b);

/* As osqp_batch_solve without waiting; results are read after the stream
 * reaches this point (osqp_batch_get waits). */
int32_t osqp_batch_solve_async(osqp_batch* b);

/* Solve only the k problems listed in idx (distinct indices) and wait. */
int32_t osqp_batch_solve_subset(osqp_batch* b, const int32_t* idx, int32_t k);

/* Mark every problem for a cold solve: rescale, ρ̄ = ρ̄⁰, zero iterates. */
int32_t osqp_batch_reset(osqp_batch* b);

/* §6 vectors as parameters for problem i (host arrays, NULL = unchanged);
 * applied at the next solve, which warm-starts problem i. */
int32_t osqp_batch_update_vectors(osqp_batch* b, int32_t i, const double* q, const double* l,
                                  const double* u);

/* §6 vectors as parameters for every problem at once: q_all (Σ n_i values),
 * l_all and u_all (Σ m_i values each), concatenated in problem order (host
 * arrays; q_all may be NULL = unchanged, l_all and u_all are both given or
 * both NULL).  Validated on the host like osqp_batch_update_vectors, copied
 * with one transfer per array into a device staging buffer (allocated by
 * the first whole-batch call) and scattered on the device; every problem
 * warm-starts at the next solve.  Enqueued on the batch's stream (page-locked
 * arrays keep the copies asynchronous).  OSQP_ERR_ARG while a slot launch
 * is in flight. */
int32_t osqp_batch_update_all(osqp_batch* b, const double* q_all, const double* l_all,
                              const double* u_all);

/* Unscaled x (Σ n_i) and y (Σ m_i) of every problem, concatenated in problem
 * order (host arrays, either may be NULL): gathered on the device and copied
 * with one transfer per array.  Waits for in-flight slots and the stream. */
int32_t osqp_batch_get_all(osqp_batch* b, double* x_all, double* y_all);

/* Unscaled x (n_i), y (m_i), z (m_i) of problem i (host arrays, any may be
 * NULL) and its info (solve_time = that problem's device time inside the
 * last launch, setup_time = the whole launch's device time).  Waits for the
 * stream. */
int32_t osqp_batch_get(osqp_batch* b, int32_t i, double* x, double* y, double* z,
                       osqp_info* info);

/* ---- overlapping launches (continuous batching) ----------------------------
 * Up to OSQP_BATCH_MAX_SLOTS subset launches may be in flight at once, each
 * on its own stream, so problems submitted while others run start as soon
 * as CTAs free up and their work overlaps on the device.  A problem may be
 * in at most one launch at a time. */
#define OSQP_BATCH_MAX_SLOTS 32

/* Copy new q/l/u for the k problems idx[0..k) (host arrays, any pointer
 * array or entry may be NULL = unchanged; page-locked memory keeps the
 * copies asynchronous) and launch their warm-started solve on `slot`.
 * Returns at once; OSQP_ERR_ARG if the slot is busy or a problem is in
 * flight. */
int32_t osqp_batch_launch(osqp_batch* b, int32_t slot, const int32_t* idx, int32_t k,
                          const double* const* q, const double* const* l,
                          const double* const* u);

/* 1 if the slot is idle or its launch finished (the slot is then retired
 * and its problems may be read or launched again), 0 if still running. */
int32_t osqp_batch_slot_query(osqp_batch* b, int32_t slot);

/* Wait for the slot's launch and retire it. */
int32_t osqp_batch_slot_wait(osqp_batch* b, int32_t slot);

/* 1 if a slot launch containing problem i solves its problems on clusters
 * of 8 CTAs (problem i has at least 2^17 nonzeros in Kn = [P̄ Āᵀ] and Ā
 * together, the device can host such a cluster and settings->launch ≠ 1),
 * else 0.  A server may launch such problems on their own slots. */
int32_t osqp_batch_uses_cluster(const osqp_batch* b, int32_t i);

/* Device bytes that problem i occupies (its data, iterates and work arrays). */
int64_t osqp_batch_footprint(const osqp_batch* b, int32_t i);

/* Row partition of problem i (a schedule choice; the paper has no
 * counterpart): groups[0] and groups[1] receive the lanes per row (group
 * width G of the sliced layout) of its Kn = [P̄ Āᵀ] and Ā products. */
int32_t osqp_batch_schedule(const osqp_batch* b, int32_t i, int32_t* groups);

/* The autotuner's table (settings->autotune): one entry per shape class of
 * matrices.  Returns the number of classes (0 when the rule was used); for
 * k < min(classes, cap), info[6k .. 6k+5] = {kind (0 Kn, 1 Ā), log2-rows
 * bucket, mean-length bucket, log2-longest-row bucket, representative
 * problem, chosen G} and cycles[6k .. 6k+5] = the measured cycles of G = 1, 2,
 * 4, 8, 16, 32 (host arrays, may be NULL).  OSQP_ERR_ARG for a NULL batch. */
int32_t osqp_batch_tuning(const osqp_batch* b, int32_t cap, int32_t* info, double* cycles);

int32_t osqp_batch_cleanup(osqp_batch* b);

/* Diagnostic read-back of the scaling and the preconditioner (host arrays,
 * any may be NULL; waits for the stream): D (n) and E (m) of Alg. 2 with
 * the cost factor c (§5.1), and the Jacobi diagonal (n) of the reduced
 * system of §3.1 for the current ρ̄,
 *   jacobi_j = P̄_jj + σ + Σ_i ρ_i Ā_ij²,  ρ_i = ρ̄, or 10³ρ̄ on equality rows (§5.2),
 * in the scaled data P̄ = cDPD, Ā = EAD, as the last setup, update or ρ̄
 * change left it (within a solve an adaptive ρ̄ update rebuilds it; the
 * values read after the solve belong to the final ρ̄).  Returns OSQP_ERR_ARG
 * for a NULL solver, OSQP_ERR_CUDA on a failed copy. */
int32_t osqp_diag_scaling(osqp_solver* s, double* D, double* E, double* c, double* jacobi);

/* Row partition of a single problem (a schedule choice; the paper has no
 * counterpart): groups[0], groups[1] = lanes per row (group width G) of the
 * Kn = [P̄ Āᵀ] and Ā products, groups[2] = 1 when the widths were measured
 * (settings->autotune on the whole-GPU grid team: every candidate G = 1, 2,
 * 4, 8, 16, 32 of each matrix timed over 20 products at setup; the fastest
 * is used unless the rule's width is within 3 % of it), 0 when the
 * row-length rule chose them, -1 when a CUDA call of the timing failed (the
 * rule's widths are then in force and the solver works as with autotune = 0).  Widths chosen by timing can differ between
 * two setups of the same problem, and with them the rounding of the
 * products; autotune = 0 gives the same arithmetic on every setup.  ms (12 values, may be NULL) receives the
 * measured milliseconds per timed launch of each candidate, Kn then Ā
 * (zeros without tuning). */
int32_t osqp_diag_schedule(osqp_solver* s, int32_t* groups, double* ms);

/* Diagnostic of the bounded grid barrier that every multi-CTA solve relies
 * on (the paper has no counterpart).  Launches four cooperative CTAs on the
 * current device, one of which never arrives at the barrier; the others must
 * give up after timeout_s seconds (0 < timeout_s ≤ 10), record the timeout
 * and return, leaving the context usable.  Returns OSQP_OK when exactly
 * that happened, OSQP_ERR_DEVICE if the barrier did not report the timeout,
 * OSQP_ERR_ARG for a bad timeout, OSQP_ERR_CUDA on a CUDA error.  Allocates
 * and frees a few bytes of device memory; synchronises the device. */
int32_t osqp_diag_barrier_timeout(double timeout_s);

/* Diagnostic of the sliced sparse layout that osqp_setup builds for every
 * matrix (host only: no device work).  Input: the CSR row pointers of an
 * nrows-row matrix (rowptr[0] = 0, non-decreasing; nnz = rowptr[nrows]) and
 * the number of warps that run its products (16 for one CTA, 16 per CTA of
 * a grid).  Rows of at most max(256, 8·mean) nonzeros are sorted by
 * decreasing length (stable in the row index) into slices of 32/G rows,
 * G = stats[0] lanes per row; step t of a slice holds one nonzero per lane
 * at first + 32t + lane, a row's j-th nonzero on lane G·(its place in the
 * slice) + j mod G at step ⌊j/G⌋.  Longer rows follow the slices in CSR
 * order and are split into chunks of 256 positions.
 * Outputs (host, caller-owned): pos[k] (nnz entries, may be NULL) = the
 * position of CSR entry k; chunks (4 per chunk, may be NULL) = row, first
 * position, end position, and 1 for the first chunk of its row else 0; stats[6] =
 * {G, long-row threshold, slices, positions including padding, long rows,
 * chunks}.  Returns OSQP_ERR_ARG for a negative nrows, NULL rowptr or stats,
 * nwarps < 1; OSQP_ERR_CSC for row pointers that do not start at 0 or
 * decrease. */
int32_t osqp_diag_sliced_layout(int32_t nrows, const int32_t* rowptr, int64_t nwarps,
                                int32_t* pos, int32_t* chunks, int32_t* stats);

#ifdef __cplusplus
}
#endif
#endif /* OSQP_GB300_H */
