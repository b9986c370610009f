// Host-side helpers shared by the single-problem and batched entry points:
// input validation, settings → device parameters, the CSR structure of
// Kn = [P̄ Āᵀ] and Ā built from the CSC input (with gather maps from the CSC
// value arrays), and the SpMV row schedule.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "../../include/osqp_gb300.h"
#include "device.cuh"

namespace osqpgb {
namespace host {

// Row schedule from row-length statistics.  Rows longer than
// max(256, 8·mean) are split into kChunk-nonzero chunks handled by whole
// warps.  The group width G for the other rows is the largest power of two
// that still gives every group about one row (32·warps/rows), kept between
// the width that caps a lane at 16 nonzeros of a mean row and the smallest
// power of two ≥ the mean row length.  (A wider G would spread a row over
// more lanes, but on GB300 the serial chain of dependent loads per group
// costs more: measured on the Lasso, portfolio, random-QP and MPC
// workloads.)  The short rows are then laid out in slices (see Sched).
struct SchedHost {
  int group = 1, long_thresh = 256, npos = 0;
  std::vector<int2> slices;
  std::vector<int> srow;
  std::vector<int4> chunks;  // (row, begin, end, long-row index)
  std::vector<int> long_rows;
  std::vector<int2> lrange;  // per long row: (first chunk, number of chunks)
  std::vector<int> lidx;     // per row: long-row index, −1 for a short row
  std::vector<int> pos;      // CSR index → position in the sliced layout
};

inline int sched_group(double mean_short, long long nshort, long long nwarps) {
  int g_mean = 1;
  while (g_mean < 32 && (double)g_mean < mean_short) g_mean <<= 1;
  int g_min = 1;
  while (g_min < 32 && (double)g_min * 16.0 < mean_short) g_min <<= 1;
  int g_occ = 1;
  while (g_occ < 32 && (long long)(g_occ * 2) * nshort <= 32LL * nwarps) g_occ <<= 1;
  return std::max(g_min, std::min(g_mean, g_occ));
}

// force_group > 0 replaces the rule's group width (the batch autotuner's
// measured choice).
inline SchedHost make_sched(const std::vector<int>& rp, long long nwarps, int force_group = 0) {
  SchedHost S;
  const int nrows = (int)rp.size() - 1;
  const long long nnz = nrows > 0 ? rp[nrows] : 0;
  const double mean_all = nrows > 0 ? (double)nnz / nrows : 0.0;
  S.long_thresh = std::max(256, (int)(8.0 * std::ceil(mean_all)));
  std::vector<int> shortr;
  long long sn = 0;
  for (int r = 0; r < nrows; ++r) {
    const int len = rp[r + 1] - rp[r];
    if (len <= S.long_thresh) {
      sn += len;
      shortr.push_back(r);
    } else {
      S.long_rows.push_back(r);
    }
  }
  const long long scount = (long long)shortr.size();
  const double ms = scount ? (double)sn / (double)scount : 1.0;
  S.group = force_group > 0 ? force_group : sched_group(ms, scount, nwarps);
  const int G = S.group, spw = 32 / G;
  std::stable_sort(shortr.begin(), shortr.end(),
                   [&](int a, int b) { return rp[a + 1] - rp[a] > rp[b + 1] - rp[b]; });
  S.pos.assign(nnz, -1);
  S.lidx.assign(nrows, -1);
  const int nsl = (int)((scount + spw - 1) / spw);
  S.srow.assign((size_t)nsl * spw, -1);
  int p = 0;
  for (int sl = 0; sl < nsl; ++sl) {
    int W = 0;
    for (int r = 0; r < spw && sl * spw + r < scount; ++r) {
      const int row = shortr[sl * spw + r];
      S.srow[sl * spw + r] = row;
      W = std::max(W, (rp[row + 1] - rp[row] + G - 1) / G);
    }
    S.slices.push_back(make_int2(p, W));
    for (int r = 0; r < spw; ++r) {
      const int row = S.srow[sl * spw + r];
      if (row < 0) continue;
      for (int j = 0; j < rp[row + 1] - rp[row]; ++j) S.pos[rp[row] + j] = p + 32 * (j / G) + r * G + j % G;
    }
    p += 32 * W;
  }
  for (int lr = 0; lr < (int)S.long_rows.size(); ++lr) {
    const int r = S.long_rows[lr];
    const int c0 = (int)S.chunks.size();
    for (int b = rp[r]; b < rp[r + 1]; b += kChunk) {
      const int e = std::min(b + kChunk, rp[r + 1]);
      S.chunks.push_back(make_int4(r, p + (b - rp[r]), p + (e - rp[r]), lr));
    }
    S.lrange.push_back(make_int2(c0, (int)S.chunks.size() - c0));
    S.lidx[r] = lr;
    for (int k = rp[r]; k < rp[r + 1]; ++k) S.pos[k] = p + (k - rp[r]);
    p += rp[r + 1] - rp[r];
  }
  S.npos = p;
  return S;
}

// v in CSR order → the sliced layout (fill at padding positions).
template <typename V>
std::vector<V> to_positions(const SchedHost& S, const std::vector<V>& v, V fill) {
  std::vector<V> out(S.npos, fill);
  for (size_t k = 0; k < v.size(); ++k) out[S.pos[k]] = v[k];
  return out;
}

struct Arena {
  char* base = nullptr;
  size_t off = 0;
  template <typename V>
  V* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    V* p = reinterpret_cast<V*>(base ? base + off : nullptr);
    off += std::max<size_t>(count, 1) * sizeof(V);
    return p;
  }
};

inline Params make_params(const osqp_settings& s) {
  Params P;
  P.sigma = s.sigma;
  P.alpha = s.alpha;
  P.eps_abs = s.eps_abs;
  P.eps_rel = s.eps_rel;
  P.eps_pinf = s.eps_pinf;
  P.eps_dinf = s.eps_dinf;
  P.rho_tol = s.adaptive_rho_tolerance;
  P.eps_equil = s.eps_equil;
  P.pcg_kappa = s.pcg_tol_fraction;
  P.pcg_floor = s.pcg_tol_floor;
  // FP32 PCG can only shrink the residual by a few orders per ADMM
  // iteration; the next iteration restarts from an FP64 residual.
  P.pcg_reduce = s.precision == OSQP_PRECISION_FP32_MIXED ? 1e-5 : 0.0;
  P.time_limit_ns = s.time_limit > 0 ? s.time_limit * 1e9 : 0.0;
  P.max_iter = s.max_iter;
  P.check_interval = s.check_interval;
  P.adaptive_rho = s.adaptive_rho;
  P.scaling_iters = s.scaling_iters;
  P.max_rho_updates = s.max_rho_updates;
  P.pcg_max_iter = s.pcg_max_iter;
  P.barrier_timeout_ns = 2000000000ull;
  P.polish = s.polish;
  P.polish_refine = s.polish_refine_iter;
  P.delta = s.delta;
  return P;
}

inline bool valid_csc(const osqp_csc* M, int rows, int cols, bool upper) {
  if (!M || M->n_rows != rows || M->n_cols != cols || M->nnz < 0) return false;
  if (!M->colptr || (M->nnz > 0 && (!M->rowind || !M->val))) return false;
  if (M->colptr[0] != 0 || M->colptr[cols] != M->nnz) return false;
  for (int j = 0; j < cols; ++j) {
    if (M->colptr[j + 1] < M->colptr[j]) return false;
    for (int k = M->colptr[j]; k < M->colptr[j + 1]; ++k) {
      const int i = M->rowind[k];
      if (i < 0 || i >= rows) return false;
      if (k > M->colptr[j] && i <= M->rowind[k - 1]) return false;
      if (upper && i > j) return false;
    }
  }
  return true;
}

inline bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

inline int check_settings(const osqp_settings& s) {
  if (!(s.rho > 0) || !(s.sigma > 0) || !(s.alpha > 0 && s.alpha < 2)) return OSQP_ERR_SETTINGS;
  if (!(s.eps_abs >= 0) || !(s.eps_rel >= 0) || !(s.eps_pinf > 0) || !(s.eps_dinf > 0))
    return OSQP_ERR_SETTINGS;
  if (!(s.adaptive_rho_tolerance >= 1) || !(s.eps_equil >= 0) || !(s.pcg_tol_fraction >= 0) ||
      !(s.pcg_tol_floor >= 0) || !(s.time_limit >= 0))
    return OSQP_ERR_SETTINGS;
  if (s.max_iter < 0 || s.check_interval < 1 || s.scaling_iters < 0 || s.max_rho_updates < 0 ||
      s.pcg_max_iter < 1)
    return OSQP_ERR_SETTINGS;
  if (s.precision != OSQP_PRECISION_FP64 && s.precision != OSQP_PRECISION_FP32_MIXED)
    return OSQP_ERR_SETTINGS;
  if (s.launch < 0 || s.launch > 3) return OSQP_ERR_SETTINGS;
  if (s.polish < 0 || s.polish > 1 || s.polish_refine_iter < 0 || !(s.delta > 0))
    return OSQP_ERR_SETTINGS;
  if (s.autotune < 0 || s.autotune > 1) return OSQP_ERR_SETTINGS;
  return OSQP_OK;
}


// CSR structure of one problem.  kn_src / a_src index the concatenated CSC
// value arrays [P_upper values | A values].
struct HostStructure {
  int n = 0, m = 0, nnz_p = 0, nnz_a = 0, nnz_kn = 0;
  std::vector<int> kn_rp, kn_ci, kn_src, a_rp, a_ci, a_src;
};

inline void build_host_structure(const osqp_csc* P, const osqp_csc* A, HostStructure* h) {
  const int n = P->n_cols, m = A->n_rows;
  h->n = n;
  h->m = m;
  h->nnz_p = P->nnz;
  h->nnz_a = A->nnz;
  // Full symmetric P rows (row j of P̄ = column j), each entry → index in P_upper.
  std::vector<int> plen(n, 0);
  for (int j = 0; j < n; ++j)
    for (int k = P->colptr[j]; k < P->colptr[j + 1]; ++k) {
      const int i = P->rowind[k];
      plen[j]++;
      if (i != j) plen[i]++;
    }
  h->kn_rp.assign(n + 1, 0);
  for (int j = 0; j < n; ++j) h->kn_rp[j + 1] = h->kn_rp[j] + plen[j] + (A->colptr[j + 1] - A->colptr[j]);
  h->nnz_kn = h->kn_rp[n];
  h->kn_ci.assign(h->nnz_kn, 0);
  h->kn_src.assign(h->nnz_kn, 0);
  // P part of row j in increasing column order: entries (j, c ≤ j) come from
  // column j of the upper triangle, entries (j, c > j) from the rows j of
  // later columns, visited in column order.
  std::vector<int> fill(n, 0);
  for (int j = 0; j < n; ++j)
    for (int k = P->colptr[j]; k < P->colptr[j + 1]; ++k) {
      const int i = P->rowind[k];
      // row j, column i (i ≤ j): appended in increasing i while scanning column j
      const int pos = h->kn_rp[j] + fill[j]++;
      h->kn_ci[pos] = i;
      h->kn_src[pos] = k;
      if (i != j) {
        // row i, column j (j > i): columns are scanned in increasing j
        const int pos2 = h->kn_rp[i] + fill[i]++;
        h->kn_ci[pos2] = j;
        h->kn_src[pos2] = k;
      }
    }
  for (int j = 0; j < n; ++j) {
    // entries of row j arrive as (c ≤ j from column j) interleaved with
    // (c > j from later columns); sort the P part by column
    const int b = h->kn_rp[j], e = b + fill[j];
    std::vector<std::pair<int, int>> tmp;
    tmp.reserve(e - b);
    for (int q = b; q < e; ++q) tmp.push_back({h->kn_ci[q], h->kn_src[q]});
    std::sort(tmp.begin(), tmp.end());
    for (int q = b; q < e; ++q) {
      h->kn_ci[q] = tmp[q - b].first;
      h->kn_src[q] = tmp[q - b].second;
    }
    int pos = e;
    for (int k = A->colptr[j]; k < A->colptr[j + 1]; ++k) {
      h->kn_ci[pos] = n + A->rowind[k];
      h->kn_src[pos] = h->nnz_p + k;
      ++pos;
    }
  }
  // Ā in CSR by a counting sort of the CSC entries (columns in order).
  h->a_rp.assign(m + 1, 0);
  for (int k = 0; k < h->nnz_a; ++k) h->a_rp[A->rowind[k] + 1]++;
  for (int i = 0; i < m; ++i) h->a_rp[i + 1] += h->a_rp[i];
  h->a_ci.assign(h->nnz_a, 0);
  h->a_src.assign(h->nnz_a, 0);
  std::vector<int> next(h->a_rp.begin(), h->a_rp.end() - 1);
  for (int j = 0; j < n; ++j)
    for (int k = A->colptr[j]; k < A->colptr[j + 1]; ++k) {
      const int d = next[A->rowind[k]]++;
      h->a_ci[d] = j;
      h->a_src[d] = h->nnz_p + k;
    }
}

}  // namespace host
}  // namespace osqpgb
