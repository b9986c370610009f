// CPU oracle for the OSQP ADMM (arXiv:1711.08013) — TEST INFRASTRUCTURE ONLY.
//
// Plain, slow, FP64.  Only the tests, the package smoke check and the
// benchmark's CPU-baseline / reference leg load this file's library.  It
// shares no code with the CUDA path.  Every function names the passage of the
// paper it follows; the readings taken where the paper is silent are listed
// next to the code that takes them.
//
// Linear solve: the direct method of §3.1 (Eq. kkt): a minimum-degree
// ordering of the quasi-definite KKT matrix, its elimination tree and column
// counts (symbolic factorisation), an up-looking numeric LDLᵀ storing D, and
// forward / diagonal / backward solves.  The ADMM steps follow Algorithm 1
// literally, including  z̃ = z + ρ⁻¹(ν − y)  (so agreement with an indirect
// solver that forms z̃ = Ax̃ comes only through the mathematics of §3.1).
//
// Parity unpinned: the magnitude of a ρ̄ update (§5.2; the tests pin its
// direction and the gate that decides it, not the square-root law of the
// new value) and exact iteration counts, which follow from the readings of
// §5.2 and §3.1 taken here.
#include "osqp_oracle.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <set>
#include <utility>
#include <vector>

namespace {

constexpr double kInfBound = 1e20;   // |bound| ≥ 1e20 is read as infinite
constexpr double kNormMin = 1e-4;    // Ruiz norm clamp (reading of Alg. 2)
constexpr double kNormMax = 1e4;
constexpr double kRhoMin = 1e-6;     // ρ̄ clamp for the adaptive rule (reading of §5.2)
constexpr double kRhoMax = 1e6;
constexpr double kEqRhoFactor = 1e3; // ρ_i = 10³ρ̄ on equality rows (§5.2)
constexpr double kTiny = 1e-30;

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Csc {
  int nr = 0, nc = 0;
  std::vector<int> p, i;
  std::vector<double> x;
  int nnz() const { return p.empty() ? 0 : p[nc]; }
};

Csc transpose(const Csc& A) {
  Csc T;
  T.nr = A.nc;
  T.nc = A.nr;
  T.p.assign(A.nr + 1, 0);
  for (int k = 0; k < A.nnz(); ++k) T.p[A.i[k] + 1]++;
  for (int r = 0; r < A.nr; ++r) T.p[r + 1] += T.p[r];
  T.i.resize(A.nnz());
  T.x.resize(A.nnz());
  std::vector<int> next(T.p.begin(), T.p.end() - 1);
  for (int j = 0; j < A.nc; ++j)
    for (int k = A.p[j]; k < A.p[j + 1]; ++k) {
      int d = next[A.i[k]]++;
      T.i[d] = j;
      T.x[d] = A.x[k];
    }
  return T;
}

// y = M v (M in CSC)
void csc_matvec(const Csc& M, const double* v, double* y) {
  std::fill(y, y + M.nr, 0.0);
  for (int j = 0; j < M.nc; ++j)
    for (int k = M.p[j]; k < M.p[j + 1]; ++k) y[M.i[k]] += M.x[k] * v[j];
}

double inf_norm(const std::vector<double>& v) {
  double r = 0.0;
  for (double a : v) r = std::max(r, std::fabs(a));
  return r;
}

// Full symmetric P from its upper triangle (the input convention of the boundary).
Csc full_from_upper(int n, const int* Pp, const int* Pi, const double* Px) {
  std::vector<std::vector<std::pair<int, double>>> cols(n);
  for (int j = 0; j < n; ++j)
    for (int k = Pp[j]; k < Pp[j + 1]; ++k) {
      int i = Pi[k];
      cols[j].push_back({i, Px[k]});
      if (i != j) cols[i].push_back({j, Px[k]});
    }
  Csc F;
  F.nr = F.nc = n;
  F.p.assign(n + 1, 0);
  for (int j = 0; j < n; ++j) {
    std::sort(cols[j].begin(), cols[j].end());
    F.p[j + 1] = F.p[j] + (int)cols[j].size();
    for (auto& e : cols[j]) {
      F.i.push_back(e.first);
      F.x.push_back(e.second);
    }
  }
  return F;
}

// ---------------------------------------------------------------------------
// Modified Ruiz equilibration, Alg. 2 (§5.1), on M = [P Aᵀ; A 0] (Eq. equil_matrix).
// Readings: at most `iters` passes, stopping early once ‖1 − δ‖∞ ≤ ε_equil;
// a norm of exactly 0 gives δ = 1, other norms are clamped to [1e-4, 1e4];
// γ uses the mean over all n columns of P̄; in γ's max a norm below 1e-4
// counts as 1 (a vanishing norm carries no scale, as for δ), and the max is
// clamped to [1e-4, 1e4].  (Taken literally with q̄ = 0 and mostly-zero P̄
// columns, 1/max grows c geometrically pass after pass, which inflates the
// cost and the duals that the step exists to normalise.)
// ---------------------------------------------------------------------------
struct Scaling {
  std::vector<double> D, E;
  double c = 1.0;
  int passes = 0;
};

Scaling ruiz(Csc& P, std::vector<double>& q, Csc& A, std::vector<double>& l,
             std::vector<double>& u, int iters, double eps_equil) {
  const int n = P.nc, m = A.nr;
  Scaling S;
  S.D.assign(n, 1.0);
  S.E.assign(m, 1.0);
  std::vector<double> dx(n), dz(m);
  for (int pass = 0; pass < iters; ++pass) {
    // δ_i = 1/√‖M_i‖∞ for every column of M
    for (int j = 0; j < n; ++j) {
      double nrm = 0.0;
      for (int k = P.p[j]; k < P.p[j + 1]; ++k) nrm = std::max(nrm, std::fabs(P.x[k]));
      for (int k = A.p[j]; k < A.p[j + 1]; ++k) nrm = std::max(nrm, std::fabs(A.x[k]));
      dx[j] = nrm == 0.0 ? 1.0 : 1.0 / std::sqrt(std::min(std::max(nrm, kNormMin), kNormMax));
    }
    std::vector<double> rown(m, 0.0);
    for (int j = 0; j < n; ++j)
      for (int k = A.p[j]; k < A.p[j + 1]; ++k)
        rown[A.i[k]] = std::max(rown[A.i[k]], std::fabs(A.x[k]));
    for (int i = 0; i < m; ++i)
      dz[i] = rown[i] == 0.0 ? 1.0
                             : 1.0 / std::sqrt(std::min(std::max(rown[i], kNormMin), kNormMax));
    // Scale P̄, q̄, Ā, C̄ using diag(δ)
    for (int j = 0; j < n; ++j)
      for (int k = P.p[j]; k < P.p[j + 1]; ++k) P.x[k] *= dx[P.i[k]] * dx[j];
    for (int j = 0; j < n; ++j)
      for (int k = A.p[j]; k < A.p[j + 1]; ++k) A.x[k] *= dz[A.i[k]] * dx[j];
    for (int j = 0; j < n; ++j) q[j] *= dx[j];
    for (int i = 0; i < m; ++i) {
      l[i] *= dz[i];  // ±∞ stays ±∞
      u[i] *= dz[i];
    }
    // Cost scaling γ = 1/max{mean(‖P̄_i‖∞), ‖q̄‖∞}
    double mean = 0.0;
    for (int j = 0; j < n; ++j) {
      double nrm = 0.0;
      for (int k = P.p[j]; k < P.p[j + 1]; ++k) nrm = std::max(nrm, std::fabs(P.x[k]));
      mean += nrm;
    }
    mean /= std::max(n, 1);
    double qn = inf_norm(q);
    if (mean < kNormMin) mean = 1.0;
    if (qn < kNormMin) qn = 1.0;
    const double mx = std::min(std::max(std::max(mean, qn), kNormMin), kNormMax);
    const double gamma = 1.0 / mx;
    for (double& v : P.x) v *= gamma;
    for (double& v : q) v *= gamma;
    // S ← diag(δ)S, c ← γc
    for (int j = 0; j < n; ++j) S.D[j] *= dx[j];
    for (int i = 0; i < m; ++i) S.E[i] *= dz[i];
    S.c *= gamma;
    S.passes++;
    double dev = 0.0;
    for (double d : dx) dev = std::max(dev, std::fabs(1.0 - d));
    for (double d : dz) dev = std::max(dev, std::fabs(1.0 - d));
    if (dev <= eps_equil) break;
  }
  return S;
}

// ---------------------------------------------------------------------------
// Fill-reducing minimum-degree ordering (§3.1 cites AMD for this role).
// A quotient-graph minimum degree: eliminated nodes become elements that
// stand for the clique they create; elements adjacent to a pivot are absorbed
// into the pivot's element; a variable's degree is the upper bound
// |variable neighbours| + Σ_e (|e| − 1), capped by the number of remaining
// variables.  Ties go to the smallest index.  The ordering only affects fill,
// never the value of the solution.
// ---------------------------------------------------------------------------
std::vector<int> min_degree(int N, const std::vector<std::vector<int>>& adj) {
  std::vector<std::vector<int>> vadj = adj;  // variable neighbours (stale entries skipped)
  std::vector<std::vector<int>> elen(N);     // adjacent elements (absorbed ones skipped)
  std::vector<std::vector<int>> evars(N);    // variables of an element, fixed at creation
  std::vector<char> state(N, 0);             // 0 variable, 1 element, 2 absorbed
  std::vector<long long> vcount(N), esum(N, 0), deg(N);
  std::vector<int> mark(N, -1);
  std::set<std::pair<long long, int>> pq;
  for (int i = 0; i < N; ++i) {
    vcount[i] = (long long)adj[i].size();
    deg[i] = vcount[i];
    pq.insert({deg[i], i});
  }
  std::vector<int> order;
  order.reserve(N);
  std::vector<int> Lp;
  for (int step = 0; step < N; ++step) {
    int p = pq.begin()->second;
    pq.erase(pq.begin());
    order.push_back(p);
    state[p] = 1;
    mark[p] = step;
    Lp.clear();
    for (int j : vadj[p])
      if (state[j] == 0 && mark[j] != step) {
        mark[j] = step;
        Lp.push_back(j);
      }
    for (int e : elen[p]) {
      if (state[e] != 1) continue;
      long long contrib = (long long)evars[e].size() - 1;
      for (int j : evars[e]) {
        if (state[j] != 0) continue;
        esum[j] -= contrib;
        if (mark[j] != step) {
          mark[j] = step;
          Lp.push_back(j);
        }
      }
      state[e] = 2;  // absorbed into p
      std::vector<int>().swap(evars[e]);
    }
    for (int j : vadj[p])
      if (state[j] == 0) vcount[j]--;
    std::vector<int>().swap(vadj[p]);
    std::vector<int>().swap(elen[p]);
    evars[p] = Lp;
    const long long s = (long long)Lp.size();
    const long long remaining = N - step - 1;
    for (int j : Lp) {
      esum[j] += s - 1;
      elen[j].push_back(p);
      long long d = std::min(vcount[j] + esum[j], std::max(remaining - 1, 0LL));
      if (d != deg[j]) {
        pq.erase({deg[j], j});
        deg[j] = d;
        pq.insert({d, j});
      }
    }
  }
  return order;
}

// ---------------------------------------------------------------------------
// Sparse LDLᵀ of a symmetric quasi-definite matrix (§3.1, "Direct method"):
// symbolic phase = elimination tree + column counts of L; numeric phase =
// up-looking factorisation in which row k of L solves a sparse triangular
// system whose pattern is the reach of column k's entries in the tree.
// C is the permuted matrix, upper triangle in CSC (diagonal present).
// ---------------------------------------------------------------------------
struct Ldl {
  int N = 0;
  std::vector<int> perm, parent, Lp, Li, Lnz;
  std::vector<double> Lx, D, Dinv;
};

void ldl_symbolic(const Csc& C, Ldl& F) {
  const int N = C.nc;
  F.N = N;
  F.parent.assign(N, -1);
  F.Lnz.assign(N, 0);
  std::vector<int> flag(N, -1);
  for (int k = 0; k < N; ++k) {
    flag[k] = k;
    for (int p = C.p[k]; p < C.p[k + 1]; ++p) {
      int i = C.i[p];
      if (i >= k) continue;
      for (; flag[i] != k; i = F.parent[i]) {
        if (F.parent[i] == -1) F.parent[i] = k;
        F.Lnz[i]++;
        flag[i] = k;
      }
    }
  }
  F.Lp.assign(N + 1, 0);
  for (int k = 0; k < N; ++k) F.Lp[k + 1] = F.Lp[k] + F.Lnz[k];
  F.Li.assign(F.Lp[N], 0);
  F.Lx.assign(F.Lp[N], 0.0);
  F.D.assign(N, 0.0);
  F.Dinv.assign(N, 0.0);
}

bool ldl_numeric(const Csc& C, Ldl& F) {
  const int N = F.N;
  std::vector<double> Y(N, 0.0);
  std::vector<int> flag(N, -1), pattern(N), stack(N);
  std::fill(F.Lnz.begin(), F.Lnz.end(), 0);
  for (int k = 0; k < N; ++k) {
    int top = N;
    flag[k] = k;
    for (int p = C.p[k]; p < C.p[k + 1]; ++p) {
      int i = C.i[p];
      if (i > k) continue;
      Y[i] += C.x[p];
      int len = 0;
      for (; flag[i] != k; i = F.parent[i]) {
        stack[len++] = i;
        flag[i] = k;
      }
      while (len > 0) pattern[--top] = stack[--len];
    }
    double dk = Y[k];
    Y[k] = 0.0;
    for (; top < N; ++top) {
      int j = pattern[top];
      double yj = Y[j];
      Y[j] = 0.0;
      int end = F.Lp[j] + F.Lnz[j];
      for (int p = F.Lp[j]; p < end; ++p) Y[F.Li[p]] -= F.Lx[p] * yj;
      double lkj = yj / F.D[j];
      dk -= lkj * yj;
      F.Li[end] = k;
      F.Lx[end] = lkj;
      F.Lnz[j]++;
    }
    if (dk == 0.0 || !std::isfinite(dk)) return false;
    F.D[k] = dk;
    F.Dinv[k] = 1.0 / dk;
  }
  return true;
}

// t = K⁻¹ g with C = K(perm, perm) = L D Lᵀ.
void ldl_solve(const Ldl& F, const double* g, double* t, std::vector<double>& w) {
  const int N = F.N;
  w.resize(N);
  for (int a = 0; a < N; ++a) w[a] = g[F.perm[a]];
  for (int j = 0; j < N; ++j)
    for (int p = F.Lp[j]; p < F.Lp[j + 1]; ++p) w[F.Li[p]] -= F.Lx[p] * w[j];
  for (int j = 0; j < N; ++j) w[j] *= F.Dinv[j];
  for (int j = N - 1; j >= 0; --j)
    for (int p = F.Lp[j]; p < F.Lp[j + 1]; ++p) w[j] -= F.Lx[p] * w[F.Li[p]];
  for (int a = 0; a < N; ++a) t[F.perm[a]] = w[a];
}

// Permuted upper triangle C = (PKPᵀ) from an upper-triangle K; kmap[k] = C slot of K entry k.
Csc permute_upper(const Csc& K, const std::vector<int>& perm, std::vector<int>& kmap) {
  const int N = K.nc;
  std::vector<int> pinv(N);
  for (int a = 0; a < N; ++a) pinv[perm[a]] = a;
  Csc C;
  C.nr = C.nc = N;
  C.p.assign(N + 1, 0);
  for (int j = 0; j < N; ++j)
    for (int k = K.p[j]; k < K.p[j + 1]; ++k) {
      int a = pinv[K.i[k]], b = pinv[j];
      C.p[std::max(a, b) + 1]++;
    }
  for (int j = 0; j < N; ++j) C.p[j + 1] += C.p[j];
  C.i.resize(K.nnz());
  C.x.resize(K.nnz());
  kmap.resize(K.nnz());
  std::vector<int> next(C.p.begin(), C.p.end() - 1);
  for (int j = 0; j < N; ++j)
    for (int k = K.p[j]; k < K.p[j + 1]; ++k) {
      int a = pinv[K.i[k]], b = pinv[j];
      int d = next[std::max(a, b)]++;
      C.i[d] = std::min(a, b);
      C.x[d] = K.x[k];
      kmap[k] = d;
    }
  return C;
}

std::vector<std::vector<int>> sym_adjacency_from_upper(const Csc& K) {
  std::vector<std::vector<int>> adj(K.nc);
  for (int j = 0; j < K.nc; ++j)
    for (int k = K.p[j]; k < K.p[j + 1]; ++k) {
      int i = K.i[k];
      if (i == j) continue;
      adj[i].push_back(j);
      adj[j].push_back(i);
    }
  for (auto& a : adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  return adj;
}

bool valid_csc(int nr, int nc, const int* p, const int* i, const double* x, bool upper) {
  if (p[0] != 0) return false;
  for (int j = 0; j < nc; ++j) {
    if (p[j + 1] < p[j]) return false;
    for (int k = p[j]; k < p[j + 1]; ++k) {
      if (i[k] < 0 || i[k] >= nr) return false;
      if (k > p[j] && i[k] <= i[k - 1]) return false;
      if (upper && i[k] > j) return false;
      if (!std::isfinite(x[k])) return false;
    }
  }
  return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// The solver: scaling (§5.1), ρ vector (§5.2), KKT factorisation (§3.1),
// Algorithm 1 (§3.2), unscaled termination and infeasibility tests (§5.1 in
// scaled form of §3.4), ρ̄ adaptation (§5.2), unscaling (Eq. pb:scaled_qp).
// ---------------------------------------------------------------------------
extern "C" int oracle_solve(int n, int m, const int* Pp, const int* Pi, const double* Px,
                            const double* q_in, const int* Ap, const int* Ai, const double* Ax,
                            const double* l_in, const double* u_in, const oracle_settings* s,
                            double* x_out, double* y_out, double* z_out, double* prim_cert,
                            double* dual_cert, oracle_info* info) {
  const double t0 = now_s();
  std::memset(info, 0, sizeof(*info));
  if (n <= 0 || m < 0) return -1;
  if (!valid_csc(n, n, Pp, Pi, Px, true) || !valid_csc(m, n, Ap, Ai, Ax, false)) return -2;
  for (int j = 0; j < n; ++j)
    if (!std::isfinite(q_in[j])) return -3;
  for (int i = 0; i < m; ++i) {
    if (std::isnan(l_in[i]) || std::isnan(u_in[i])) return -3;
    if (l_in[i] > u_in[i]) return -4;
  }
  if (!(s->alpha > 0 && s->alpha < 2) || !(s->rho > 0) || !(s->sigma > 0) || s->max_iter < 0 ||
      s->check_interval < 1)
    return -5;

  // Problem data (full P, A) and bound types from the unscaled input.
  Csc P = full_from_upper(n, Pp, Pi, Px);
  Csc A;
  A.nr = m;
  A.nc = n;
  A.p.assign(Ap, Ap + n + 1);
  A.i.assign(Ai, Ai + Ap[n]);
  A.x.assign(Ax, Ax + Ap[n]);
  const Csc P0 = P;
  std::vector<double> q(q_in, q_in + n), l(m), u(m);
  std::vector<char> linf(m), uinf(m), is_eq(m);
  for (int i = 0; i < m; ++i) {
    linf[i] = l_in[i] <= -kInfBound;
    uinf[i] = u_in[i] >= kInfBound;
    l[i] = linf[i] ? -INFINITY : l_in[i];
    u[i] = uinf[i] ? INFINITY : u_in[i];
    is_eq[i] = l_in[i] == u_in[i];  // equality row: l_i = u_i in the input data
  }

  Scaling S = ruiz(P, q, A, l, u, s->scaling_iters, s->eps_equil);
  info->ruiz_passes = S.passes;
  const std::vector<double>& D = S.D;
  const std::vector<double>& E = S.E;
  const double c = S.c;
  Csc At = transpose(A);

  // ρ = diag(ρ_i): ρ̄ on inequality rows, 10³ρ̄ on equality rows (§5.2).
  double rho_bar = s->rho;
  std::vector<double> rho(m), rho_inv(m);
  auto set_rho = [&]() {
    for (int i = 0; i < m; ++i) {
      rho[i] = is_eq[i] ? kEqRhoFactor * rho_bar : rho_bar;
      rho_inv[i] = 1.0 / rho[i];
    }
  };
  set_rho();

  // KKT matrix of Eq. (kkt), upper triangle: [P̄+σI, Āᵀ; ·, −diag(ρ)⁻¹].
  const int N = n + m;
  Csc K;
  K.nr = K.nc = N;
  K.p.assign(N + 1, 0);
  std::vector<int> diag_slot(N, -1);
  for (int j = 0; j < n; ++j) {
    bool has_diag = false;
    for (int k = P.p[j]; k < P.p[j + 1] && P.i[k] <= j; ++k) {
      K.i.push_back(P.i[k]);
      K.x.push_back(P.i[k] == j ? P.x[k] + s->sigma : P.x[k]);
      if (P.i[k] == j) {
        has_diag = true;
        diag_slot[j] = (int)K.x.size() - 1;
      }
    }
    if (!has_diag) {
      K.i.push_back(j);
      K.x.push_back(s->sigma);
      diag_slot[j] = (int)K.x.size() - 1;
    }
    K.p[j + 1] = (int)K.i.size();
  }
  for (int r = 0; r < m; ++r) {
    for (int k = At.p[r]; k < At.p[r + 1]; ++k) {
      K.i.push_back(At.i[k]);
      K.x.push_back(At.x[k]);
    }
    K.i.push_back(n + r);
    K.x.push_back(-rho_inv[r]);
    diag_slot[n + r] = (int)K.x.size() - 1;
    K.p[n + r + 1] = (int)K.i.size();
  }

  Ldl F;
  F.perm = min_degree(N, sym_adjacency_from_upper(K));
  std::vector<int> kmap;
  Csc C = permute_upper(K, F.perm, kmap);
  ldl_symbolic(C, F);
  if (!ldl_numeric(C, F)) return -6;
  info->nnz_L = F.Lp[N];
  auto refactor = [&]() -> bool {
    for (int r = 0; r < m; ++r) C.x[kmap[diag_slot[n + r]]] = -rho_inv[r];
    return ldl_numeric(C, F);
  };

  // Iterates in the scaled problem.  Cold start: zeros.  Warm start (§6):
  // (x⁰, z⁰, y⁰) = (D⁻¹x, Āx⁰, cE⁻¹y).
  std::vector<double> x(n, 0.0), z(m, 0.0), y(m, 0.0);
  if (s->warm_start) {
    for (int j = 0; j < n; ++j) x[j] = x_out[j] / D[j];
    for (int i = 0; i < m; ++i) y[i] = c * y_out[i] / E[i];
    csc_matvec(A, x.data(), z.data());
  }
  info->setup_time = now_s() - t0;
  const double t1 = now_s();

  std::vector<double> rhs(N), sol(N), w, xt(n), zt(m), xn(n), zn(m), yn(m), dx(n), dy(m);
  std::vector<double> Axv(m), Pxv(n), Aty(n), tmp_n(n), tmp_m(m);
  std::vector<double> cert_y(m, 0.0), cert_x(n, 0.0);
  int status = ORACLE_UNSOLVED;
  int k = 0;
  const double alpha = s->alpha, sigma = s->sigma;
  for (k = 1; k <= s->max_iter; ++k) {
    // Alg. 1 step 3: solve the KKT system of Eq. (kkt)
    for (int j = 0; j < n; ++j) rhs[j] = sigma * x[j] - q[j];
    for (int i = 0; i < m; ++i) rhs[n + i] = z[i] - rho_inv[i] * y[i];
    ldl_solve(F, rhs.data(), sol.data(), w);
    for (int j = 0; j < n; ++j) xt[j] = sol[j];
    // step 4: z̃ = z + ρ⁻¹(ν − y)
    for (int i = 0; i < m; ++i) zt[i] = z[i] + rho_inv[i] * (sol[n + i] - y[i]);
    // step 5: x ← αx̃ + (1−α)x
    for (int j = 0; j < n; ++j) xn[j] = alpha * xt[j] + (1.0 - alpha) * x[j];
    // steps 6–7: z ← Π(v), v = αz̃ + (1−α)z + ρ⁻¹y;  y ← y + ρ(αz̃ + (1−α)z − z⁺),
    // evaluated in the equal form y ← ρ(v − Π(v)) of Eq. (zy-update), which
    // keeps y ∈ N_C(z) exact in floating point (§3.3).
    for (int i = 0; i < m; ++i) {
      double v = alpha * zt[i] + (1.0 - alpha) * z[i] + rho_inv[i] * y[i];
      zn[i] = std::min(std::max(v, l[i]), u[i]);
      yn[i] = rho[i] * (v - zn[i]);
    }
    for (int j = 0; j < n; ++j) dx[j] = xn[j] - x[j];
    for (int i = 0; i < m; ++i) dy[i] = yn[i] - y[i];
    x.swap(xn);
    z.swap(zn);
    y.swap(yn);

    if (k % s->check_interval != 0 && k != s->max_iter) continue;

    // Unscaled termination criteria in scaled quantities (§5.1).
    csc_matvec(A, x.data(), Axv.data());
    csc_matvec(P, x.data(), Pxv.data());
    csc_matvec(At, y.data(), Aty.data());
    double prim_res = 0, ax_n = 0, z_n = 0, rp_bar = 0, axb = 0, zb = 0;
    for (int i = 0; i < m; ++i) {
      prim_res = std::max(prim_res, std::fabs((Axv[i] - z[i]) / E[i]));
      ax_n = std::max(ax_n, std::fabs(Axv[i] / E[i]));
      z_n = std::max(z_n, std::fabs(z[i] / E[i]));
      rp_bar = std::max(rp_bar, std::fabs(Axv[i] - z[i]));
      axb = std::max(axb, std::fabs(Axv[i]));
      zb = std::max(zb, std::fabs(z[i]));
    }
    double dual_res = 0, px_n = 0, aty_n = 0, q_n = 0, rd_bar = 0, pxb = 0, atyb = 0, qb = 0;
    for (int j = 0; j < n; ++j) {
      double r = Pxv[j] + q[j] + Aty[j];
      dual_res = std::max(dual_res, std::fabs(r / D[j]));
      px_n = std::max(px_n, std::fabs(Pxv[j] / D[j]));
      aty_n = std::max(aty_n, std::fabs(Aty[j] / D[j]));
      q_n = std::max(q_n, std::fabs(q[j] / D[j]));
      rd_bar = std::max(rd_bar, std::fabs(r));
      pxb = std::max(pxb, std::fabs(Pxv[j]));
      atyb = std::max(atyb, std::fabs(Aty[j]));
      qb = std::max(qb, std::fabs(q[j]));
    }
    dual_res /= c;
    const double eps_prim = s->eps_abs + s->eps_rel * std::max(ax_n, z_n);
    const double eps_dual = s->eps_abs + s->eps_rel * std::max({px_n, aty_n, q_n}) / c;
    info->prim_res = prim_res;
    info->dual_res = dual_res;
    if (!std::isfinite(prim_res) || !std::isfinite(dual_res)) {
      status = ORACLE_NUMERICAL_ERROR;
      break;
    }
    if (prim_res <= eps_prim && dual_res <= eps_dual) {
      status = ORACLE_SOLVED;
      break;
    }

    // Primal infeasibility (§5.1 scaled form of §3.4).  Reading: δȳ is first
    // projected so that no component pairs with an infinite bound (a positive
    // component on u_i = +∞ or a negative one on l_i = −∞ would make the
    // support function infinite), and the bound test is read as strict
    // negativity, ūᵀ(δȳ)₊ + l̄ᵀ(δȳ)₋ < −ε_pinf‖Eδȳ‖∞, as the certificate of
    // Eq. (prim-infeas-linear) requires.
    for (int i = 0; i < m; ++i) {
      double d = dy[i];
      if ((uinf[i] && d > 0) || (linf[i] && d < 0)) d = 0.0;
      tmp_m[i] = d;
    }
    double edy = 0.0, supp = 0.0;
    for (int i = 0; i < m; ++i) {
      edy = std::max(edy, std::fabs(E[i] * tmp_m[i]));
      if (tmp_m[i] > 0) supp += u[i] * tmp_m[i];
      else if (tmp_m[i] < 0) supp += l[i] * tmp_m[i];
    }
    csc_matvec(At, tmp_m.data(), tmp_n.data());
    double atdy = 0.0;
    for (int j = 0; j < n; ++j) atdy = std::max(atdy, std::fabs(tmp_n[j] / D[j]));
    if (atdy <= s->eps_pinf * edy && supp < -s->eps_pinf * edy) {
      for (int i = 0; i < m; ++i) cert_y[i] = E[i] * tmp_m[i] / c;
      status = ORACLE_PRIMAL_INFEASIBLE;
      break;
    }

    // Dual infeasibility (§5.1).  Readings: q̄ᵀδx̄ < −cε_dinf‖Dδx̄‖∞ (strict,
    // negative, as Eq. dual-infeas-linear requires); rows with both bounds
    // infinite impose no condition.
    double ddx = 0.0, qdx = 0.0;
    for (int j = 0; j < n; ++j) {
      ddx = std::max(ddx, std::fabs(D[j] * dx[j]));
      qdx += q[j] * dx[j];
    }
    csc_matvec(P, dx.data(), tmp_n.data());
    double pdx = 0.0;
    for (int j = 0; j < n; ++j) pdx = std::max(pdx, std::fabs(tmp_n[j] / D[j]));
    bool dinf = pdx <= c * s->eps_dinf * ddx && qdx < -c * s->eps_dinf * ddx;
    if (dinf) {
      csc_matvec(A, dx.data(), tmp_m.data());
      const double tol = s->eps_dinf * ddx;
      for (int i = 0; i < m && dinf; ++i) {
        double a = tmp_m[i] / E[i];
        if (!linf[i] && !uinf[i]) dinf = std::fabs(a) <= tol;
        else if (uinf[i] && !linf[i]) dinf = a >= -tol;
        else if (linf[i] && !uinf[i]) dinf = a <= tol;
      }
    }
    if (dinf) {
      for (int j = 0; j < n; ++j) cert_x[j] = D[j] * dx[j];
      status = ORACLE_DUAL_INFEASIBLE;
      break;
    }

    // ρ̄ adaptation (§5.2) in scaled norms.  Reading: evaluated at every
    // termination check, applied when the new value is more than the
    // tolerance factor away, ρ̄ clamped to [1e-6, 1e6], at most
    // max_rho_updates updates per solve.
    if (s->adaptive_rho && info->rho_updates < s->max_rho_updates && k < s->max_iter) {
      double pr = rp_bar / (std::max(axb, zb) + kTiny);
      double dr = rd_bar / (std::max({pxb, atyb, qb}) + kTiny);
      double rn = rho_bar * std::sqrt(pr / (dr + kTiny));
      rn = std::min(std::max(rn, kRhoMin), kRhoMax);
      if (rn > s->adaptive_rho_tolerance * rho_bar || rn < rho_bar / s->adaptive_rho_tolerance) {
        rho_bar = rn;
        set_rho();
        if (!refactor()) return -6;
        info->rho_updates++;
      }
    }
  }
  if (status == ORACLE_UNSOLVED && s->max_iter > 0) status = ORACLE_MAX_ITER;
  info->iter = std::min(k, s->max_iter);
  info->status = status;
  info->rho_bar = rho_bar;

  // Solution polishing (§4) in the scaled problem, after a solved run.
  // Active sets from the sign of ȳ (lower: ȳ_i < 0, upper: ȳ_i > 0); the
  // δ-regularised reduced KKT matrix of Eq. (kkt_polish_reg) is factored
  // once and iterative refinement (Eq. iterative_refinement) against the
  // unregularised matrix of Eq. (kkt_polish) runs a fixed number of passes.
  // The candidate replaces the ADMM solution when it satisfies the sign
  // conditions y ∈ N_C(z) of Eq. (compl_slack) on the active rows and its
  // unscaled residuals are no larger than the ADMM ones (reading: the paper
  // asks for the optimality conditions to hold; residual tolerances make
  // "hold" the comparison with the iterate the solver would return).
  if (s->polish && status == ORACLE_SOLVED) {
    std::vector<int> act;
    std::vector<double> bnd;
    for (int i = 0; i < m; ++i) {
      if (y[i] < 0.0 && !linf[i]) {
        act.push_back(i);
        bnd.push_back(l[i]);
      } else if (y[i] > 0.0 && !uinf[i]) {
        act.push_back(i);
        bnd.push_back(u[i]);
      }
    }
    const int na = (int)act.size(), NP = n + na;
    const double delta = s->delta;
    // upper triangle of [P̄ + δI, Ā_actᵀ; Ā_act, −δI]; the same pattern
    // without δ is the unregularised matrix used for the refinement residual
    Csc Kp;
    Kp.nr = Kp.nc = NP;
    Kp.p.assign(NP + 1, 0);
    for (int j = 0; j < n; ++j) {
      bool has_diag = false;
      for (int kk = P.p[j]; kk < P.p[j + 1] && P.i[kk] <= j; ++kk) {
        Kp.i.push_back(P.i[kk]);
        Kp.x.push_back(P.i[kk] == j ? P.x[kk] + delta : P.x[kk]);
        has_diag |= P.i[kk] == j;
      }
      if (!has_diag) {
        Kp.i.push_back(j);
        Kp.x.push_back(delta);
      }
      Kp.p[j + 1] = (int)Kp.i.size();
    }
    for (int a = 0; a < na; ++a) {
      const int r = act[a];
      for (int kk = At.p[r]; kk < At.p[r + 1]; ++kk) {
        Kp.i.push_back(At.i[kk]);
        Kp.x.push_back(At.x[kk]);
      }
      Kp.i.push_back(n + a);
      Kp.x.push_back(-delta);
      Kp.p[n + a + 1] = (int)Kp.i.size();
    }
    Ldl G;
    G.perm = min_degree(NP, sym_adjacency_from_upper(Kp));
    std::vector<int> kmap2;
    Csc Cp = permute_upper(Kp, G.perm, kmap2);
    ldl_symbolic(Cp, G);
    bool ok = ldl_numeric(Cp, G);
    std::vector<double> t(NP, 0.0), g(NP), res(NP), dt(NP), w2;
    for (int j = 0; j < n; ++j) g[j] = -q[j];
    for (int a = 0; a < na; ++a) g[n + a] = bnd[a];
    for (int pass = 0; ok && pass <= s->polish_refine_iter; ++pass) {
      // res = g − K t with K the unregularised matrix: K t = (P̄x + Ā_actᵀy, Ā_act x)
      std::vector<double> xs(t.begin(), t.begin() + n), ya(m, 0.0);
      for (int a = 0; a < na; ++a) ya[act[a]] = t[n + a];
      csc_matvec(P, xs.data(), Pxv.data());
      csc_matvec(At, ya.data(), Aty.data());
      csc_matvec(A, xs.data(), Axv.data());
      for (int j = 0; j < n; ++j) res[j] = g[j] - Pxv[j] - Aty[j];
      for (int a = 0; a < na; ++a) res[n + a] = g[n + a] - Axv[act[a]];
      ldl_solve(G, res.data(), dt.data(), w2);
      for (int q2 = 0; q2 < NP; ++q2) t[q2] += dt[q2];
    }
    if (ok) {
      std::vector<double> xp(t.begin(), t.begin() + n), yp(m, 0.0), zp(m);
      bool signs = true;
      for (int a = 0; a < na; ++a) {
        const int r = act[a];
        yp[r] = t[n + a];
        if (bnd[a] == l[r] && !(bnd[a] == u[r]) && yp[r] > 0.0) signs = false;
        if (bnd[a] == u[r] && !(bnd[a] == l[r]) && yp[r] < 0.0) signs = false;
      }
      csc_matvec(A, xp.data(), Axv.data());
      csc_matvec(P, xp.data(), Pxv.data());
      csc_matvec(At, yp.data(), Aty.data());
      double pr = 0.0, dr = 0.0;
      for (int i = 0; i < m; ++i) {
        zp[i] = std::min(std::max(Axv[i], l[i]), u[i]);
        pr = std::max(pr, std::fabs((Axv[i] - zp[i]) / E[i]));
      }
      for (int j = 0; j < n; ++j) dr = std::max(dr, std::fabs((Pxv[j] + q[j] + Aty[j]) / D[j]));
      dr /= c;
      if (signs && std::isfinite(pr) && std::isfinite(dr) && pr <= info->prim_res &&
          dr <= info->dual_res) {
        x = xp;
        y = yp;
        z = zp;
        info->prim_res = pr;
        info->dual_res = dr;
        info->polished = 1;
      } else {
        info->polished = -1;
      }
    } else {
      info->polished = -1;
    }
  }

  // Unscale (Eq. pb:scaled_qp): x = Dx̄, z = E⁻¹z̄, y = c⁻¹Eȳ.
  for (int j = 0; j < n; ++j) x_out[j] = D[j] * x[j];
  for (int i = 0; i < m; ++i) {
    z_out[i] = z[i] / E[i];
    y_out[i] = E[i] * y[i] / c;
  }
  if (prim_cert) std::copy(cert_y.begin(), cert_y.end(), prim_cert);
  if (dual_cert) std::copy(cert_x.begin(), cert_x.end(), dual_cert);
  // Objective ½xᵀPx + qᵀx on the unscaled data.
  std::vector<double> px(n);
  csc_matvec(P0, x_out, px.data());
  double obj = 0.0;
  for (int j = 0; j < n; ++j) obj += 0.5 * x_out[j] * px[j] + q_in[j] * x_out[j];
  info->obj_val = obj;
  info->solve_time = now_s() - t1;
  return 0;
}

extern "C" int oracle_ruiz(int n, int m, const int* Pfp, const int* Pfi, const double* Pfx,
                           const double* q_in, const int* Ap, const int* Ai, const double* Ax,
                           const double* l_in, const double* u_in, int scaling_iters,
                           double eps_equil, double* D, double* E, double* c, double* Pbar_x,
                           double* qbar, double* Abar_x, double* lbar, double* ubar) {
  Csc P;
  P.nr = P.nc = n;
  P.p.assign(Pfp, Pfp + n + 1);
  P.i.assign(Pfi, Pfi + Pfp[n]);
  P.x.assign(Pfx, Pfx + Pfp[n]);
  Csc A;
  A.nr = m;
  A.nc = n;
  A.p.assign(Ap, Ap + n + 1);
  A.i.assign(Ai, Ai + Ap[n]);
  A.x.assign(Ax, Ax + Ap[n]);
  std::vector<double> q(q_in, q_in + n), l(m), u(m);
  for (int i = 0; i < m; ++i) {
    l[i] = l_in[i] <= -kInfBound ? -INFINITY : l_in[i];
    u[i] = u_in[i] >= kInfBound ? INFINITY : u_in[i];
  }
  Scaling S = ruiz(P, q, A, l, u, scaling_iters, eps_equil);
  std::copy(S.D.begin(), S.D.end(), D);
  std::copy(S.E.begin(), S.E.end(), E);
  *c = S.c;
  std::copy(P.x.begin(), P.x.end(), Pbar_x);
  std::copy(q.begin(), q.end(), qbar);
  std::copy(A.x.begin(), A.x.end(), Abar_x);
  std::copy(l.begin(), l.end(), lbar);
  std::copy(u.begin(), u.end(), ubar);
  return S.passes;
}

extern "C" int oracle_min_degree(int N, const int* Kp, const int* Ki, int* perm) {
  std::vector<std::vector<int>> adj(N);
  for (int j = 0; j < N; ++j)
    for (int k = Kp[j]; k < Kp[j + 1]; ++k) {
      int i = Ki[k];
      if (i == j) continue;
      adj[i].push_back(j);
      adj[j].push_back(i);
    }
  for (auto& a : adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  std::vector<int> order = min_degree(N, adj);
  std::copy(order.begin(), order.end(), perm);
  return 0;
}

extern "C" long long oracle_ldl_solve(int N, const int* Kp, const int* Ki, const double* Kx,
                                      int nrhs, const double* g, double* t, double* Dout) {
  Csc K;
  K.nr = K.nc = N;
  K.p.assign(Kp, Kp + N + 1);
  K.i.assign(Ki, Ki + Kp[N]);
  K.x.assign(Kx, Kx + Kp[N]);
  for (int j = 0; j < N; ++j)
    for (int k = Kp[j]; k < Kp[j + 1]; ++k)
      if (Ki[k] > j) return -2;
  Ldl F;
  F.perm = min_degree(N, sym_adjacency_from_upper(K));
  std::vector<int> kmap;
  Csc C = permute_upper(K, F.perm, kmap);
  ldl_symbolic(C, F);
  if (!ldl_numeric(C, F)) return -6;
  std::vector<double> w;
  for (int r = 0; r < nrhs; ++r) ldl_solve(F, g + (size_t)r * N, t + (size_t)r * N, w);
  if (Dout)
    for (int a = 0; a < N; ++a) Dout[F.perm[a]] = F.D[a];
  return F.Lp[N];
}
