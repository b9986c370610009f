/*
 * CPU oracle for the OSQP ADMM method (arXiv:1711.08013) — TEST INFRASTRUCTURE.
 *
 * A plain, slow FP64 implementation of what the GPU path computes, written
 * from the paper and used only by the tests, the package smoke check and the
 * benchmark's CPU-baseline leg.  It shares no code, header or constant with
 * the CUDA library; the status values below are numerically equal to the
 * library's so that results can be compared, and are defined here on their
 * own.
 *
 * Linear solve: the direct method of §3.1 — a fill-reducing minimum-degree
 * ordering of the quasi-definite KKT matrix of Eq. (kkt), then a sparse
 * LDLᵀ factorisation (symbolic + numeric phases) and forward/backward solves.
 */
#ifndef OSQP_ORACLE_H
#define OSQP_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORACLE_UNSOLVED = 0,
  ORACLE_SOLVED = 1,
  ORACLE_MAX_ITER = 2,
  ORACLE_PRIMAL_INFEASIBLE = 3,
  ORACLE_DUAL_INFEASIBLE = 4,
  ORACLE_NUMERICAL_ERROR = 6
};

typedef struct {
  double rho;                     /* ρ̄⁰ (§5.2, default 0.1) */
  double sigma;                   /* σ (§5.2, default 1e-6) */
  double alpha;                   /* α ∈ (0, 2) (§5.2, default 1.6) */
  double eps_abs, eps_rel;        /* §3.4 / §7 (default 1e-3) */
  double eps_pinf, eps_dinf;      /* §3.4 / §7 (default 1e-4) */
  double adaptive_rho_tolerance;  /* §5.2: update when 5× larger or smaller */
  double eps_equil;               /* Alg. 2 stopping tolerance */
  int max_iter;
  int check_interval;             /* termination checked every k iterations */
  int adaptive_rho;               /* 0/1 */
  int scaling_iters;              /* upper bound on Ruiz passes (0 = no scaling) */
  int max_rho_updates;
  int warm_start;                 /* 1: x, y on input are the initial guess (§6) */
  int polish;                     /* 1: solution polishing (§4) after a solved run */
  int polish_refine_iter;         /* iterative-refinement passes of §4 (default 3) */
  double delta;                   /* regularisation δ of Eq. kkt_polish_reg (default 1e-6) */
} oracle_settings;

typedef struct {
  int status, iter, rho_updates, ruiz_passes;
  double obj_val, prim_res, dual_res, rho_bar;
  double setup_time, solve_time;
  long long nnz_L;
  int polished;                   /* 1 accepted, -1 tried and rejected, 0 not tried */
  int pad;
} oracle_info;

/* Solve min ½xᵀPx+qᵀx s.t. l ≤ Ax ≤ u.  P: upper triangle, CSC, n × n;
 * A: CSC, m × n; bounds with |v| ≥ 1e20 are infinite.  Outputs (caller
 * owned): x (n), y (m), z (m), prim_cert (m, c⁻¹Eδȳ), dual_cert (n, Dδx̄).
 * Returns 0, or a negative value for invalid input / factorisation failure. */
int oracle_solve(int n, int m,
                 const int* Pp, const int* Pi, const double* Px, const double* q,
                 const int* Ap, const int* Ai, const double* Ax,
                 const double* l, const double* u, const oracle_settings* s,
                 double* x, double* y, double* z, double* prim_cert, double* dual_cert,
                 oracle_info* info);

/* Alg. 2 alone: returns D (n), E (m), c, and the scaled data in the input
 * patterns (Pbar_x: full symmetric P in CSC of the full pattern given by
 * Pfp/Pfi; Abar_x in A's pattern), q̄, l̄, ū.  Returns the number of passes. */
int oracle_ruiz(int n, int m, const int* Pfp, const int* Pfi, const double* Pfx,
                const double* q, const int* Ap, const int* Ai, const double* Ax,
                const double* l, const double* u, int scaling_iters, double eps_equil,
                double* D, double* E, double* c, double* Pbar_x, double* qbar,
                double* Abar_x, double* lbar, double* ubar);

/* Minimum-degree ordering of a symmetric pattern (full CSC, diagonal optional). */
int oracle_min_degree(int N, const int* Kp, const int* Ki, int* perm);

/* Factor the symmetric quasi-definite K (upper triangle CSC, diagonal
 * present) as PKPᵀ = LDLᵀ and solve K t = g for nrhs right-hand sides stored
 * column by column.  Returns nnz(L) ≥ 0 or a negative error. */
long long oracle_ldl_solve(int N, const int* Kp, const int* Ki, const double* Kx,
                           int nrhs, const double* g, double* t, double* Dout);

#ifdef __cplusplus
}
#endif
#endif
