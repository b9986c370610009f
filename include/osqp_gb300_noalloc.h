/*
 * osqp_gb300_noalloc.h — one solve entry point that allocates nothing.
 *
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory when they solve: code inside a CUDA-graph
 * capture that must not reach the allocator, plugins whose host framework
 * owns every device allocation, and real-time loops that forbid
 * cudaMalloc/cudaFree after start-up.
 */
#ifndef OSQP_GB300_NOALLOC_H
#define OSQP_GB300_NOALLOC_H

#include "osqp_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Size of the statically allocated device work array: 16 MiB on every GPU
 * that loads the library, held until the process exits. */
#define OSQP_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* Solve one small QP (same problem, settings, algorithm and one-CTA solver
 * as osqp_setup + osqp_solve with settings->launch = 1) without any
 * allocation: no cudaMalloc, cudaFree or allocating library call.  Every
 * intermediate array, including the CSR structure that osqp_setup would
 * build on the host, lives in the library's static work array.
 *
 * Inputs (DEVICE pointers, CSC as in osqp_setup, P upper triangle, indices
 * sorted within columns): P_colptr (n+1), P_rowind/P_val (P_nnz), q (n),
 * A_colptr (n+1), A_rowind/A_val (A_nnz), l, u (m).  settings: host.
 * Outputs: x (n) and y (m), DEVICE pointers written with the unscaled
 * solution; info (host, may be NULL).  stream: cudaStream_t or NULL.
 *
 * Returns OSQP_ERR_LIMIT when the problem needs more than
 * OSQP_NOALLOC_SCRATCH_BYTES of work space (about 2·nnz(P) + nnz(A) values
 * and indices plus ~45 vectors of length n or m) or has a row of [P Aᵀ]
 * (the full symmetric P part and the column of A together) or of A longer
 * than 8192 entries; OSQP_ERR_CSC for malformed CSC; OSQP_ERR_NONFINITE for
 * a NaN or infinity in P, A or q or a NaN bound, and OSQP_ERR_LGTU for some
 * l_i > u_i (these input checks of osqp_setup run on the device here, CSC
 * structure first, then values); the usual codes for bad settings.  The
 * call waits for the stream.
 *
 * Inside a stream capture (stream is capturing) nothing may wait, so the
 * call only enqueues the solve and returns OSQP_OK; info must then be NULL
 * (else OSQP_ERR_ARG).  Every replay of the captured graph reads the input
 * buffers and writes x, y when it runs, so one graph solves successive
 * problems of the same n, m and nonzero counts whose values, q, l and u the
 * caller rewrites in place between replays (a control loop).  The status,
 * iteration counts and any device-side rejection of a replay (malformed CSC,
 * too large) are read afterwards with osqp_noalloc_get_info.
 *
 * The first call made with a given device current looks up the work array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  Every call shares the array and overwrites it: calls whose
 * kernels overlap on the GPU (different streams without ordering, or
 * threads) race, so serialise them.  The kernel clears every counter it
 * relies on; the rest of the array keeps the previous call's contents. */
int32_t osqp_solve_noalloc(int32_t n, int32_t m, const int32_t* P_colptr,
                           const int32_t* P_rowind, const double* P_val, int32_t P_nnz,
                           const double* q, const int32_t* A_colptr, const int32_t* A_rowind,
                           const double* A_val, int32_t A_nnz, const double* l, const double* u,
                           const osqp_settings* settings, double* x, double* y, osqp_info* info,
                           void* stream);

/* Status of the last solve that ran in the work array (a call of
 * osqp_solve_noalloc, or a replay of one captured in a CUDA graph) for a
 * problem with these sizes, nonzero counts and precision (OSQP_PRECISION_*):
 * fills *info (host) as osqp_solve_noalloc does and returns OSQP_ERR_CSC,
 * OSQP_ERR_LIMIT, OSQP_ERR_NONFINITE or OSQP_ERR_LGTU when the device rejected
 * that problem (a rejected replay leaves x and y unwritten).  The sizes locate
 * the status inside the work array; other sizes read unrelated bytes.
 * Waits for the stream; OSQP_ERR_ARG inside a stream capture. */
int32_t osqp_noalloc_get_info(int32_t n, int32_t m, int32_t P_nnz, int32_t A_nnz,
                              int32_t precision, osqp_info* info, void* stream);

#ifdef __cplusplus
}
#endif
#endif
