// Batched solve of many independent QPs in one persistent launch.
//
// Every problem keeps its own sizes, sparsity pattern, scaling, ρ̄ and
// iterates resident in one device allocation.  k_batch runs a grid of
// persistent CTAs (two per SM); each CTA takes the next problem from a device
// work counter — problems are queued largest first — and runs the whole
// solve for it with the one-CTA team: Ruiz scaling or a vector refresh when
// requested, then Algorithm 1 with PCG, termination and unscaling.  Problems
// never share a reduction, so each result is bit-for-bit the same whether
// the problem is solved alone or among others.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/osqp_gb300.h"
#include "device.cuh"
#include "host_common.h"

using namespace osqpgb;
using namespace osqpgb::host;

namespace {

constexpr int kBatchThreads = 512;
constexpr long long kBatchWarps = kBatchThreads / 32;
constexpr int kBatchCluster = 8;      // CTAs of a heavy-problem cluster
constexpr int kMaxHeavyClusters = 4;  // clusters a launch may take for heavy problems
constexpr int kMaxHeavy = 32;         // heavy problems per launch at most
constexpr long long kClusterWork = 1 << 17;  // nonzeros of Kn + Ā from which a slot launch
                                             // solves its problems on clusters
constexpr size_t kPoolCap = 160 << 10;  // shared memory for one problem's PCG vectors at most

enum : int { kModeScale = 1, kModeRefresh = 2, kModeReset = 4 };

// order[k] = problem index | (mode << kModeShift): the mode bits of a
// problem travel with the launch that solves it, so concurrent launches on
// different streams never share mutable per-problem flags.
constexpr int kModeShift = 28;

// One problem of a batch launch on a team: the mode bits of its queue entry
// (first scaling, data refresh, iterate reset), then Algorithm 1.
template <class Team, typename T>
__device__ void batch_solve_one(Team& tm, const Dev<T>& d, const Params& P, int md) {
  const double rho_bar = d.sc->rho_bar;
  if (md & kModeScale) {
    if (!scale_stage(tm, d, P, rho_bar, true)) return;
  } else {
    if ((md & kModeRefresh) && !refresh_stage(tm, d, P, rho_bar)) return;
    if (md & kModeReset) {
      if (tm.leader()) {
        d.sc->rp_last = 0.0;
        d.sc->rd_last = 0.0;
      }
      for (int j = tm.tid(); j < d.n; j += tm.nthreads()) {
        d.x[j] = 0.0;
        d.dx[j] = 0.0;
        d.xt[j] = 0.0;
      }
      for (int i = tm.tid(); i < d.m; i += tm.nthreads()) {
        d.z[i] = 0.0;
        d.y[i] = 0.0;
        d.dy[i] = 0.0;
        d.zt[i] = 0.0;
      }
      if (!tm.sync()) return;
    }
  }
  admm_stage(tm, d, P);
}

// As batch_solve_one, with the PCG vectors in the CTA's shared memory (one
// CTA per problem; the problem's vectors fit in `pool`).
template <typename T>
__device__ void batch_solve_one_smem(BlockTeam& tm, const Dev<T>& d, const Params& P, int md,
                                     Dev<T>& sd, unsigned char* pool, bool with_mat) {
  const double rho_bar = d.sc->rho_bar;
  if (md & kModeScale) {
    if (!scale_stage(tm, d, P, rho_bar, true)) return;
  } else {
    if ((md & kModeRefresh) && !refresh_stage(tm, d, P, rho_bar)) return;
    if (md & kModeReset) {
      if (tm.leader()) {
        d.sc->rp_last = 0.0;
        d.sc->rd_last = 0.0;
      }
      for (int j = tm.tid(); j < d.n; j += tm.nthreads()) {
        d.x[j] = 0.0;
        d.dx[j] = 0.0;
        d.xt[j] = 0.0;
      }
      for (int i = tm.tid(); i < d.m; i += tm.nthreads()) {
        d.z[i] = 0.0;
        d.y[i] = 0.0;
        d.dy[i] = 0.0;
        d.zt[i] = 0.0;
      }
    }
  }
  stage_in(d, sd, pool, with_mat);
  admm_stage(tm, sd, P);
  stage_out(d, sd);
}

template <typename T>
__global__ void __launch_bounds__(kBatchThreads, 1)
    k_batch(const Dev<T>* __restrict__ devs, const int* __restrict__ order, int count,
            const __grid_constant__ Params P, int* queue, unsigned long long* times,
            int pool_bytes) {
  __shared__ double sm[kSmemDoubles];
  __shared__ int sidx;
  __shared__ Dev<T> sdev;
  extern __shared__ __align__(16) unsigned char pool[];
  BlockTeam tm{sm};
  for (;;) {
    if (threadIdx.x == 0) sidx = atomicAdd(queue, 1);
    __syncthreads();
    const int idx = sidx;
    __syncthreads();
    if (idx >= count) break;
    const int code = order[idx];
    const int p = code & ((1 << kModeShift) - 1);
    const Dev<T>& d = devs[p];
    const unsigned long long t0 = gtimer();
    const int plan = smem_plan(d, (size_t)pool_bytes);
    if (plan > 0)
      batch_solve_one_smem(tm, d, P, code >> kModeShift, sdev, pool, plan == 2);
    else
      batch_solve_one(tm, d, P, code >> kModeShift);
    __syncthreads();
    if (threadIdx.x == 0) {
      times[2 * p] = t0;
      times[2 * p + 1] = gtimer();
    }
  }
}

// Clusters of kBatchCluster CTAs for the heaviest problems of a launch:
// each cluster takes problems from the heavy queue, then joins the queue of
// the one-CTA kernel running beside it (shared counter), so no SM idles
// once the heavy problems are done.  Rank 0 takes the index and the others
// read it through distributed shared memory; every decision is taken on
// values identical in all CTAs, so all CTAs leave the loop together.
template <typename T>
__global__ void __launch_bounds__(kBatchThreads, 1)
    k_batch_cluster(const Dev<T>* __restrict__ devs, const int* __restrict__ order_h, int count_h,
                    int* queue_h, const int* __restrict__ order_l, int count_l, int* queue_l,
                    const __grid_constant__ Params P, unsigned long long* times, int* err) {
  __shared__ double sm[kSmemDoubles];
  __shared__ double cpart[2 * kMaxRed];
  __shared__ unsigned ctr;
  __shared__ int sidx;
  if (threadIdx.x == 0) ctr = 0u;
  cluster_sync_all();
  ClusterTeam tm{sm, cpart, &ctr, err, P.barrier_timeout_ns, cluster_rank(), cluster_size(), 0u, 0};
  for (int phase = 0; phase < 2; ++phase) {
    const int* order = phase == 0 ? order_h : order_l;
    const int count = phase == 0 ? count_h : count_l;
    int* queue = phase == 0 ? queue_h : queue_l;
    bool ok = true;
    for (;;) {
      if (tm.leader()) sidx = atomicAdd(queue, 1);
      if (!tm.sync()) {
        ok = false;
        break;
      }
      const int idx = *cluster_map(&sidx, 0u);
      if (!tm.sync()) {  // every CTA has read rank 0's index before the next take
        ok = false;
        break;
      }
      if (idx >= count) break;
      const int code = order[idx];
      const int p = code & ((1 << kModeShift) - 1);
      const Dev<T>& d = devs[p];
      const unsigned long long t0 = gtimer();
      batch_solve_one(tm, d, P, code >> kModeShift);
      if (!tm.sync()) {
        ok = false;
        break;
      }
      if (tm.leader()) {
        times[2 * p] = t0;
        times[2 * p + 1] = gtimer();
      }
    }
    if (!ok) break;
  }
  cluster_sync_all();
}

// ---------------------------------------------------------------------------
// Autotuner of the row partition.  For every class of matrices of similar
// shape (rows, mean and longest row, in powers of two), one representative
// matrix is laid out with each candidate group width G and one CTA per
// (class, candidate) times `reps` products y = M x on the batch kernel's team
// shape, with x in shared memory as in the batched solve; the fastest G of
// each class is used for every matrix of the class.
// ---------------------------------------------------------------------------
constexpr int kTuneGroups[] = {1, 2, 4, 8, 16, 32};
constexpr int kTuneCandidates = 6;
constexpr int kTuneReps = 40;

template <typename T>
struct TuneCase {
  Sched S;
  const int* ci;
  const T* va;
  T* xg;   // x in global memory when it does not fit the shared pool
  T* y;
  int ncols, pad;
  unsigned long long* cycles;
};

template <typename T>
__global__ void __launch_bounds__(kBatchThreads, 1)
    k_tune(const TuneCase<T>* __restrict__ cases, int reps, int pool_bytes) {
  __shared__ double sm[kSmemDoubles];
  extern __shared__ __align__(16) unsigned char pool[];
  const TuneCase<T>& c = cases[blockIdx.x];
  T* x = (size_t)c.ncols * sizeof(T) <= (size_t)pool_bytes ? reinterpret_cast<T*>(pool) : c.xg;
  for (int j = threadIdx.x; j < c.ncols; j += blockDim.x) x[j] = T(1) + T(j & 7) * T(0.125);
  __syncthreads();
  BlockTeam tm{sm};
  T* __restrict__ y = c.y;
  auto store = [&](int row, T* acc) { y[row] = acc[0]; };
  const long long t0 = clock64();
  for (int r = 0; r < reps; ++r) {
    spmv<1, false, T, T>(tm, c.S, c.ci, c.va, [&](int col, T v, T* acc) { acc[0] += v * x[col]; },
                         store, NoChunk{}, store);
    __syncthreads();
  }
  const long long t1 = clock64();
  if (threadIdx.x == 0) *c.cycles = (unsigned long long)(t1 - t0);
}

// Whole-batch vector transfers: one CTA per problem moves its segment of
// the concatenated vectors.  Scatter: stage → raw q, l, u (each may be
// absent).  Gather: unscaled x, y → stage.
template <typename T>
__global__ void k_scatter_vectors(const Dev<T>* __restrict__ devs, int count,
                                  const long long* __restrict__ off, const double* __restrict__ q,
                                  const double* __restrict__ l, const double* __restrict__ u) {
  const long long* off_n = off;
  const long long* off_m = off + count + 1;
  for (int p = blockIdx.x; p < count; p += gridDim.x) {
    const Dev<T>& d = devs[p];
    for (int j = threadIdx.x; j < d.n; j += blockDim.x)
      if (q) const_cast<double*>(d.q_raw)[j] = q[off_n[p] + j];
    for (int i = threadIdx.x; i < d.m; i += blockDim.x) {
      if (l) const_cast<double*>(d.l_raw)[i] = l[off_m[p] + i];
      if (u) const_cast<double*>(d.u_raw)[i] = u[off_m[p] + i];
    }
  }
}

template <typename T>
__global__ void k_gather_solutions(const Dev<T>* __restrict__ devs, int count,
                                   const long long* __restrict__ off, double* __restrict__ x,
                                   double* __restrict__ y) {
  const long long* off_n = off;
  const long long* off_m = off + count + 1;
  for (int p = blockIdx.x; p < count; p += gridDim.x) {
    const Dev<T>& d = devs[p];
    for (int j = threadIdx.x; j < d.n; j += blockDim.x) x[off_n[p] + j] = d.x_out[j];
    for (int i = threadIdx.x; i < d.m; i += blockDim.x) y[off_m[p] + i] = d.y_out[i];
  }
}

// Per-problem sizes and offsets.
struct ProblemLayout {
  int n = 0, m = 0, nnz_kn = 0, nnz_a = 0;
  SchedHost kn_s, a_s;
  size_t s_off = 0;  // offset of this problem's static block
  size_t v_off = 0;  // offset of this problem's dynamic block
};

struct Bump {
  size_t off = 0;
  template <typename V>
  size_t take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    const size_t at = off;
    off += std::max<size_t>(count, 1) * sizeof(V);
    return at;
  }
};

// Static block (uploaded once): sliced structure, raw values, schedules,
// raw vectors.
struct SchedOffsets {
  size_t sl, sr, ch, lr, rng, li;
};

struct StaticOffsets {
  size_t kn_ci, kn_raw, a_ci, a_raw, q, l, u, end;
  SchedOffsets kn, a;
};

SchedOffsets sched_offsets(Bump& b, const SchedHost& h) {
  SchedOffsets o;
  o.sl = b.take<int2>(h.slices.size());
  o.sr = b.take<int>(h.srow.size());
  o.ch = b.take<int4>(h.chunks.size());
  o.lr = b.take<int>(h.long_rows.size());
  o.rng = b.take<int2>(h.lrange.size());
  o.li = b.take<int>(h.lidx.size());
  return o;
}

StaticOffsets static_offsets(const ProblemLayout& L) {
  Bump b;
  StaticOffsets o;
  o.kn_ci = b.take<int>(L.kn_s.npos);
  o.kn_raw = b.take<double>(L.kn_s.npos);
  o.a_ci = b.take<int>(L.a_s.npos);
  o.a_raw = b.take<double>(L.a_s.npos);
  o.kn = sched_offsets(b, L.kn_s);
  o.a = sched_offsets(b, L.a_s);
  o.q = b.take<double>(L.n);
  o.l = b.take<double>(L.m);
  o.u = b.take<double>(L.m);
  o.end = (b.off + 255) & ~(size_t)255;
  return o;
}

// Dynamic block: working matrices, the long-row partials and counters of
// both products, and every vector of Dev<T>.
template <typename T>
size_t dynamic_carve(const ProblemLayout& L, char* base, Dev<T>* d) {
  Bump b;
  const size_t n = L.n, m = L.m;
  const size_t kn_v = b.take<T>(L.kn_s.npos);
  const size_t a_v = b.take<T>(L.a_s.npos);
  const size_t kn_cp = b.take<double>(L.kn_s.chunks.size() * kMaxNV);
  const size_t kn_cc = b.take<unsigned>(L.kn_s.lrange.size());
  const size_t a_cp = b.take<double>(L.a_s.chunks.size() * kMaxNV);
  const size_t a_cc = b.take<unsigned>(L.a_s.lrange.size());
  const size_t rt = b.take<uint8_t>(m);
  const size_t pact = b.take<uint8_t>(m);
  size_t on[22], om[22], otn[10], otm[4], out[2];
  for (auto& v : on) v = b.take<double>(n);
  for (auto& v : om) v = b.take<double>(m);
  for (auto& v : otn) v = b.take<T>(n);
  for (auto& v : otm) v = b.take<T>(m);
  for (auto& v : out) v = b.take<T>(n + m);
  const size_t sc = b.take<Scalars>(1);
  if (base && d) {
    d->kn_v = (T*)(base + kn_v);
    d->a_v = (T*)(base + a_v);
    d->kn.cpart = (double*)(base + kn_cp);
    d->kn.ccount = (unsigned*)(base + kn_cc);
    d->as.cpart = (double*)(base + a_cp);
    d->as.ccount = (unsigned*)(base + a_cc);
    d->rtype = (uint8_t*)(base + rt);
    d->pol_act = (uint8_t*)(base + pact);
    double** nv[] = {&d->D, &d->q, &d->pdiag, &d->dg, &d->nrm_n, &d->x, &d->dx, &d->px,
                     &d->aty, &d->pdx, &d->atdy, &d->x_out, &d->dcert, &d->xt, &d->Dinv,
                     &d->pol_x, &d->pol_dx, &d->pol_r, &d->pol_z, &d->pol_p, &d->pol_kp,
                     &d->pol_dg};
    for (int k = 0; k < 22; ++k) *nv[k] = (double*)(base + on[k]);
    double** mv[] = {&d->E, &d->l, &d->u, &d->rho, &d->rho_inv, &d->nrm_m, &d->z, &d->y,
                     &d->dy, &d->ax, &d->adx, &d->azt, &d->z_out, &d->y_out, &d->pcert,
                     &d->zt, &d->wm, &d->um, &d->Einv, &d->pol_y, &d->pol_t, &d->pol_r2};
    for (int k = 0; k < 22; ++k) *mv[k] = (double*)(base + om[k]);
    T** tn[] = {&d->dinv, &d->b, &d->p, &d->r0, &d->r1, &d->s0, &d->s1, &d->w0, &d->w1, &d->dxt};
    for (int k = 0; k < 10; ++k) *tn[k] = (T*)(base + otn[k]);
    T** tmv[] = {&d->ap, &d->dzt, &d->rhoT, &d->rho_invT};
    for (int k = 0; k < 4; ++k) *tmv[k] = (T*)(base + otm[k]);
    d->ut0 = (T*)(base + out[0]);
    d->ut1 = (T*)(base + out[1]);
    d->sc = (Scalars*)(base + sc);
  }
  return (b.off + 255) & ~(size_t)255;
}

}  // namespace

struct osqp_batch {
  int count = 0, device = 0, num_sms = 0, grid = 0;
  int pool = 0;  // dynamic shared memory of k_batch: PCG vectors of problems that fit
  // autotuner: per class (matrix kind 0 = Kn, 1 = Ā; shape key; representative
  // problem), the cycles of each candidate group width and the choice
  struct TuneClass {
    int kind, rows_b, mean_b, max_b, rep, chosen;
    double cycles[kTuneCandidates];
  };
  std::vector<TuneClass> tune;
  std::vector<int2> groups;  // per problem: group width of Kn and of Ā
  cudaStream_t stream = nullptr;
  osqp_settings set{};
  Params P{};
  std::vector<ProblemLayout> L;
  std::vector<int> order;           // problems sorted by work, largest first
  std::vector<int> mode;            // per-problem kernel mode for the next launch
  std::vector<unsigned long long> times_host;
  std::vector<double> last_dur;     // device seconds of problem i in its last launch (0: none)
  std::vector<char> on_cluster;     // problem i was solved by a cluster in its last launch
  // heavy-problem clusters beside the one-CTA kernel (whole-batch launches)
  int cluster_ok = 0;               // the device can host a kBatchCluster-CTA cluster
  cudaStream_t cstream = nullptr;
  int* corder = nullptr;
  int* cqueue = nullptr;
  int* cerr = nullptr;
  cudaEvent_t cfork = nullptr, cjoin = nullptr;
  bool cused = false;
  bool unrecorded = false;          // a whole-batch launch whose times are not in last_dur
  char* arena = nullptr;
  size_t static_bytes = 0, arena_bytes = 0;
  void* devs = nullptr;             // Dev<T>[count]
  std::vector<char> devs_host;      // host copy of the Dev<T> array
  int* order_d = nullptr;
  int* queue = nullptr;
  // launch slots for overlapping subset solves (serving)
  struct Slot {
    cudaStream_t stream = nullptr;
    int* order = nullptr;
    int* queue = nullptr;
    int* err = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<int> members;
  } slots[OSQP_BATCH_MAX_SLOTS];
  std::vector<int> inflight;        // slot holding problem i, or -1
  std::vector<size_t> footprint;    // device bytes of problem i
  unsigned long long* times_d = nullptr;
  // whole-batch vector transfers: offsets of problem i in the concatenated
  // n- and m-vectors (host and device), and a device staging buffer of
  // Σn + 2Σm values (allocated on first use)
  std::vector<long long> off_n, off_m;
  long long* off_d = nullptr;
  double* stage_d = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double last_time = 0.0;
  bool solved = false;
};

namespace {

template <typename T>
Dev<T>* dev_at(osqp_batch* b, int i) {
  return reinterpret_cast<Dev<T>*>(b->devs_host.data()) + i;
}

template <typename T>
void fill_batch_devs(osqp_batch* b) {
  b->devs_host.assign(sizeof(Dev<T>) * b->count, 0);
  for (int i = 0; i < b->count; ++i) {
    const ProblemLayout& L = b->L[i];
    Dev<T>* d = dev_at<T>(b, i);
    std::memset((void*)d, 0, sizeof(Dev<T>));
    const StaticOffsets o = static_offsets(L);
    char* sb = b->arena + L.s_off;
    d->n = L.n;
    d->m = L.m;
    d->kn_ci = (const int*)(sb + o.kn_ci);
    d->kn_raw = (const double*)(sb + o.kn_raw);
    d->a_ci = (const int*)(sb + o.a_ci);
    d->a_raw = (const double*)(sb + o.a_raw);
    d->q_raw = (const double*)(sb + o.q);
    d->l_raw = (const double*)(sb + o.l);
    d->u_raw = (const double*)(sb + o.u);
    auto sched = [&](const SchedHost& h, const SchedOffsets& so, int nrows) {
      return Sched{nrows,
                   h.group,
                   h.long_thresh,
                   (int)h.chunks.size(),
                   (int)h.long_rows.size(),
                   (int)h.slices.size(),
                   (const int2*)(sb + so.sl),
                   (const int*)(sb + so.sr),
                   (const int4*)(sb + so.ch),
                   (const int*)(sb + so.lr),
                   (const int2*)(sb + so.rng),
                   (const int*)(sb + so.li),
                   nullptr,   // cpart, ccount: carved in the dynamic block below
                   nullptr};
    };
    d->kn = sched(L.kn_s, o.kn, L.n);
    d->as = sched(L.a_s, o.a, L.m);
    d->kn.npos = L.kn_s.npos;
    d->as.npos = L.a_s.npos;
    dynamic_carve<T>(L, b->arena + L.v_off, d);
  }
}

// Heavy problems of a whole-batch launch: with every problem's device time
// from its previous launch known and more problems than CTAs, a problem
// whose time exceeds the fair share (total time / CTAs, the wall time of a
// perfectly balanced launch) would set the wall time on one SM; such
// problems (longest first, at most kMaxHeavy) go to clusters.
void pick_heavy(const osqp_batch* b, const std::vector<int>& sel, cudaStream_t st,
                std::vector<int>& heavy, std::vector<int>& light) {
  heavy.clear();
  light = sel;
  if (!b->cluster_ok || b->set.launch == 1 || st != b->stream || (int)sel.size() <= b->grid) return;
  double total = 0.0;
  for (int v : sel) {
    if (!(b->last_dur[v] > 0.0)) return;
    total += b->last_dur[v];
  }
  const double fair = total / b->grid;
  light.clear();
  for (int v : sel) {
    if ((int)heavy.size() < kMaxHeavy && b->last_dur[v] > fair) heavy.push_back(v);
    else light.push_back(v);
  }
}

// A slot launch (serving) solves its problems on clusters when one of them
// is large: one CTA would hold such a problem for seconds.
bool large_problem(const osqp_batch* b, int i) {
  return (long long)b->L[i].nnz_kn + b->L[i].nnz_a >= kClusterWork;
}

template <typename T>
int launch_slot_clusters(osqp_batch* b, const std::vector<int>& sel, int* order_d, int* queue,
                         int* err, cudaStream_t st) {
  const int k = (int)sel.size();
  std::vector<int> code(k);
  for (int j = 0; j < k; ++j) code[j] = sel[j] | (b->mode[sel[j]] << kModeShift);
  if (cudaMemcpyAsync(order_d, code.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess ||
      cudaMemsetAsync(queue, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
    return OSQP_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::min(k, kMaxHeavyClusters) * kBatchCluster);
  cfg.blockDim = dim3(kBatchThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kBatchCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_batch_cluster<T>, (const Dev<T>*)b->devs, (const int*)order_d, k,
                         queue, (const int*)order_d, 0, queue, b->P, b->times_d, err) !=
      cudaSuccess)
    return OSQP_ERR_CUDA;
  for (int v : sel) {
    b->mode[v] = 0;
    b->on_cluster[v] = 1;
  }
  return OSQP_OK;
}

template <typename T>
int launch_batch(osqp_batch* b, const std::vector<int>& sel, int* order_d, int* queue,
                 cudaStream_t st, int* slot_err = nullptr) {
  if (slot_err && b->cluster_ok && b->set.launch != 1) {
    for (int v : sel)
      if (large_problem(b, v)) return launch_slot_clusters<T>(b, sel, order_d, queue, slot_err, st);
  }
  std::vector<int> heavy, light;
  pick_heavy(b, sel, st, heavy, light);
  const int nl = (int)light.size(), nh = (int)heavy.size();
  const int nclusters = std::min(nh, kMaxHeavyClusters);
  std::vector<int> code(nl), hcode(nh);
  for (int k = 0; k < nl; ++k) code[k] = light[k] | (b->mode[light[k]] << kModeShift);
  for (int k = 0; k < nh; ++k) hcode[k] = heavy[k] | (b->mode[heavy[k]] << kModeShift);
  if (nl && cudaMemcpyAsync(order_d, code.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, st) !=
                cudaSuccess)
    return OSQP_ERR_CUDA;
  // the host vector must outlive the copy: wait for it (small, pageable)
  if (cudaStreamSynchronize(st) != cudaSuccess) return OSQP_ERR_CUDA;
  if (cudaMemsetAsync(queue, 0, sizeof(int), st) != cudaSuccess) return OSQP_ERR_CUDA;
  if (nh) {
    if (!b->cstream) {
      if (cudaStreamCreateWithFlags(&b->cstream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaMalloc((void**)&b->corder, sizeof(int) * b->count) != cudaSuccess ||
          cudaMalloc((void**)&b->cqueue, sizeof(int)) != cudaSuccess ||
          cudaMalloc((void**)&b->cerr, sizeof(int)) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->cfork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->cjoin, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return OSQP_ERR_CUDA;
      }
    }
    // the cluster kernel also reads the light queue: fork after it is reset
    if (cudaEventRecord(b->cfork, st) != cudaSuccess ||
        cudaStreamWaitEvent(b->cstream, b->cfork, 0) != cudaSuccess ||
        cudaMemcpyAsync(b->corder, hcode.data(), sizeof(int) * nh, cudaMemcpyHostToDevice,
                        b->cstream) != cudaSuccess ||
        cudaMemsetAsync(b->cqueue, 0, sizeof(int), b->cstream) != cudaSuccess ||
        cudaMemsetAsync(b->cerr, 0, sizeof(int), b->cstream) != cudaSuccess ||
        cudaStreamSynchronize(b->cstream) != cudaSuccess)
      return OSQP_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nclusters * kBatchCluster);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.stream = b->cstream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kBatchCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_batch_cluster<T>, (const Dev<T>*)b->devs, (const int*)b->corder,
                           nh, b->cqueue, (const int*)order_d, nl, queue, b->P, b->times_d,
                           b->cerr) != cudaSuccess ||
        cudaEventRecord(b->cjoin, b->cstream) != cudaSuccess)
      return OSQP_ERR_CUDA;
  }
  if (nl) {
    // leave the clusters' SMs to them whichever kernel the GPU starts first
    const int grid = std::max(1, std::min(b->grid - nclusters * kBatchCluster, nl));
    k_batch<T><<<grid, kBatchThreads, b->pool, st>>>((const Dev<T>*)b->devs, order_d, nl, b->P,
                                                      queue, b->times_d, b->pool);
    if (cudaGetLastError() != cudaSuccess) return OSQP_ERR_CUDA;
  }
  if (nh && cudaStreamWaitEvent(st, b->cjoin, 0) != cudaSuccess) return OSQP_ERR_CUDA;
  for (int v : sel) {
    b->mode[v] = 0;
    b->on_cluster[v] = 0;
  }
  for (int v : heavy) b->on_cluster[v] = 1;
  if (st == b->stream) b->cused = nh > 0;
  return OSQP_OK;
}

// Shape class of a matrix given by its CSR row pointers.
std::array<int, 3> tune_key(const std::vector<int>& rp) {
  const int nrows = (int)rp.size() - 1;
  int maxlen = 0;
  for (int r = 0; r < nrows; ++r) maxlen = std::max(maxlen, rp[r + 1] - rp[r]);
  const double mean = nrows > 0 ? (double)rp[nrows] / nrows : 0.0;
  auto lg = [](double v) { return (int)std::floor(std::log2(v + 1.0)); };
  return {lg(nrows), (int)std::floor(2.0 * std::log2(mean + 1.0)), lg(maxlen)};
}

// Measure every candidate group width on one representative matrix per
// shape class (one launch of k_tune, one CTA per case) and set each
// problem's widths to its classes' fastest.  Returns OSQP_OK or a CUDA error
// code; on any failure the rule's widths stay in force.
template <typename T>
int autotune_groups(osqp_batch* b, const std::vector<HostStructure>& hs) {
  const int count = b->count;
  std::map<std::array<int, 4>, int> cls;  // (kind, key) → class index
  std::vector<int> cls_of(2 * (size_t)count);
  b->tune.clear();
  for (int i = 0; i < count; ++i)
    for (int kind = 0; kind < 2; ++kind) {
      const auto k = tune_key(kind == 0 ? hs[i].kn_rp : hs[i].a_rp);
      const std::array<int, 4> key{kind, k[0], k[1], k[2]};
      auto it = cls.find(key);
      if (it == cls.end()) {
        osqp_batch::TuneClass tc{};
        tc.kind = kind;
        tc.rows_b = k[0];
        tc.mean_b = k[1];
        tc.max_b = k[2];
        tc.rep = i;
        tc.chosen = 0;
        it = cls.emplace(key, (int)b->tune.size()).first;
        b->tune.push_back(tc);
      }
      cls_of[2 * (size_t)i + kind] = it->second;
    }
  // candidate layouts of each representative, packed into one device buffer
  struct Cand {
    SchedHost S;
    std::vector<int> ci;
    int nrows, ncols;
  };
  std::vector<Cand> cands;
  for (const auto& tc : b->tune) {
    const HostStructure& h = hs[tc.rep];
    const std::vector<int>& rp = tc.kind == 0 ? h.kn_rp : h.a_rp;
    const std::vector<int>& ci = tc.kind == 0 ? h.kn_ci : h.a_ci;
    for (int g : kTuneGroups) {
      Cand c;
      c.S = make_sched(rp, kBatchWarps, g);
      c.ci = to_positions(c.S, ci, -1);
      c.S.pos = {};
      c.nrows = (int)rp.size() - 1;
      c.ncols = tc.kind == 0 ? h.n + h.m : h.n;
      cands.push_back(std::move(c));
    }
  }
  Bump bump;
  struct Off {
    size_t ci, va, sl, sr, ch, lr, rng, li, cp, cc, xg, y, cyc;
  };
  std::vector<Off> off(cands.size());
  int max_cols = 0;
  for (size_t k = 0; k < cands.size(); ++k) {
    const Cand& c = cands[k];
    Off& o = off[k];
    o.ci = bump.take<int>(c.S.npos);
    o.va = bump.take<T>(c.S.npos);
    o.sl = bump.take<int2>(c.S.slices.size());
    o.sr = bump.take<int>(c.S.srow.size());
    o.ch = bump.take<int4>(c.S.chunks.size());
    o.lr = bump.take<int>(c.S.long_rows.size());
    o.rng = bump.take<int2>(c.S.lrange.size());
    o.li = bump.take<int>(c.S.lidx.size());
    o.cp = bump.take<double>(c.S.chunks.size() * kMaxNV);
    o.cc = bump.take<unsigned>(c.S.lrange.size());
    o.xg = bump.take<T>(c.ncols);
    o.y = bump.take<T>(c.nrows);
    o.cyc = bump.take<unsigned long long>(1);
    max_cols = std::max(max_cols, c.ncols);
  }
  const size_t cases_off = bump.take<TuneCase<T>>(cands.size());
  const size_t total = bump.off;
  std::vector<char> hbuf(total, 0);
  char* dbuf = nullptr;
  if (cudaMalloc((void**)&dbuf, total) != cudaSuccess) {
    cudaGetLastError();
    return OSQP_ERR_OOM;
  }
  std::vector<TuneCase<T>> tcs(cands.size());
  for (size_t k = 0; k < cands.size(); ++k) {
    const Cand& c = cands[k];
    const Off& o = off[k];
    auto put = [&](size_t at, const void* src, size_t bytes) {
      if (bytes) std::memcpy(hbuf.data() + at, src, bytes);
    };
    put(o.ci, c.ci.data(), sizeof(int) * c.ci.size());
    T* va = reinterpret_cast<T*>(hbuf.data() + o.va);
    for (int q = 0; q < c.S.npos; ++q) va[q] = c.ci[q] >= 0 ? T(1) : T(0);
    put(o.sl, c.S.slices.data(), sizeof(int2) * c.S.slices.size());
    put(o.sr, c.S.srow.data(), sizeof(int) * c.S.srow.size());
    put(o.ch, c.S.chunks.data(), sizeof(int4) * c.S.chunks.size());
    put(o.lr, c.S.long_rows.data(), sizeof(int) * c.S.long_rows.size());
    put(o.rng, c.S.lrange.data(), sizeof(int2) * c.S.lrange.size());
    put(o.li, c.S.lidx.data(), sizeof(int) * c.S.lidx.size());
    TuneCase<T>& t = tcs[k];
    t.S = Sched{c.nrows,
                c.S.group,
                c.S.long_thresh,
                (int)c.S.chunks.size(),
                (int)c.S.long_rows.size(),
                (int)c.S.slices.size(),
                (const int2*)(dbuf + o.sl),
                (const int*)(dbuf + o.sr),
                (const int4*)(dbuf + o.ch),
                (const int*)(dbuf + o.lr),
                (const int2*)(dbuf + o.rng),
                (const int*)(dbuf + o.li),
                (double*)(dbuf + o.cp),
                (unsigned*)(dbuf + o.cc)};
    t.S.npos = c.S.npos;
    t.ci = (const int*)(dbuf + o.ci);
    t.va = (const T*)(dbuf + o.va);
    t.xg = (T*)(dbuf + o.xg);
    t.y = (T*)(dbuf + o.y);
    t.ncols = c.ncols;
    t.pad = 0;
    t.cycles = (unsigned long long*)(dbuf + o.cyc);
  }
  std::memcpy(hbuf.data() + cases_off, tcs.data(), sizeof(TuneCase<T>) * tcs.size());
  const int xpool = (int)std::min<size_t>(kPoolCap, (size_t)max_cols * sizeof(T));
  int rc = OSQP_OK;
  if (cudaMemcpy(dbuf, hbuf.data(), total, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaFuncSetAttribute(k_tune<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kPoolCap) != cudaSuccess)
    rc = OSQP_ERR_CUDA;
  std::vector<unsigned long long> best(cands.size(), ~0ull);
  // two timed launches after a warm one; the faster of the two per case
  for (int pass = 0; rc == OSQP_OK && pass < 3; ++pass) {
    k_tune<T><<<(int)cands.size(), kBatchThreads, xpool, b->stream>>>(
        (const TuneCase<T>*)(dbuf + cases_off), kTuneReps, xpool);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess) {
      rc = OSQP_ERR_CUDA;
      break;
    }
    if (pass == 0) continue;
    for (size_t k = 0; k < cands.size(); ++k) {
      unsigned long long cy = 0;
      if (cudaMemcpy(&cy, dbuf + off[k].cyc, sizeof(cy), cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = OSQP_ERR_CUDA;
        break;
      }
      best[k] = std::min(best[k], cy);
    }
  }
  cudaFree(dbuf);
  if (rc != OSQP_OK) {
    cudaGetLastError();
    b->tune.clear();
    return rc;
  }
  for (size_t c = 0; c < b->tune.size(); ++c) {
    osqp_batch::TuneClass& tc = b->tune[c];
    int bi = 0;
    for (int g = 0; g < kTuneCandidates; ++g) {
      tc.cycles[g] = (double)best[c * kTuneCandidates + g];
      if (best[c * kTuneCandidates + g] < best[c * kTuneCandidates + bi]) bi = g;
    }
    tc.chosen = kTuneGroups[bi];
  }
  b->groups.assign(count, make_int2(0, 0));
  for (int i = 0; i < count; ++i)
    b->groups[i] = make_int2(b->tune[cls_of[2 * (size_t)i]].chosen,
                             b->tune[cls_of[2 * (size_t)i + 1]].chosen);
  return OSQP_OK;
}

int batch_launch(osqp_batch* b, const std::vector<int>& sel) {
  if (cudaEventRecord(b->ev[0], b->stream) != cudaSuccess) return OSQP_ERR_CUDA;
  const int rc = b->set.precision == OSQP_PRECISION_FP64
                     ? launch_batch<double>(b, sel, b->order_d, b->queue, b->stream)
                     : launch_batch<float>(b, sel, b->order_d, b->queue, b->stream);
  if (rc) return rc;
  if (cudaEventRecord(b->ev[1], b->stream) != cudaSuccess) return OSQP_ERR_CUDA;
  b->solved = true;
  return OSQP_OK;
}

// Per-problem device times of the launch that just completed → last_dur.
void record_durations(osqp_batch* b, const std::vector<int>& sel) {
  if (sel.empty()) return;
  if (cudaMemcpy(b->times_host.data(), b->times_d, sizeof(unsigned long long) * b->times_host.size(),
                 cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  for (int v : sel) {
    const unsigned long long t0 = b->times_host[2 * (size_t)v], t1 = b->times_host[2 * (size_t)v + 1];
    if (t1 > t0) b->last_dur[v] = (double)(t1 - t0) * 1e-9;
  }
}

// Launch order, longest first (a longest-processing-time schedule of the
// problems over the persistent CTAs).  The key is each problem's device time
// in its last launch when every selected problem has one — a batch that is
// solved again and again (parametric MPC, serving) knows its slow problems,
// which depend on iteration counts more than on size — else the static work
// estimate.  The order changes only which CTA solves a problem, never a result.
void order_longest_first(const osqp_batch* b, std::vector<int>& sel) {
  bool hist = true;
  for (int v : sel)
    if (!(b->last_dur[v] > 0.0)) {
      hist = false;
      break;
    }
  if (hist) {
    std::stable_sort(sel.begin(), sel.end(),
                     [&](int a, int c) { return b->last_dur[a] > b->last_dur[c]; });
  } else {
    std::stable_sort(sel.begin(), sel.end(), [&](int a, int c) {
      return (long long)b->L[a].nnz_kn + b->L[a].nnz_a + b->L[a].n + b->L[a].m >
             (long long)b->L[c].nnz_kn + b->L[c].nnz_a + b->L[c].n + b->L[c].m;
    });
  }
}

int batch_wait(osqp_batch* b, const std::vector<int>& sel) {
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return OSQP_ERR_CUDA;
  float ms = 0.f;
  if (b->solved && cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) == cudaSuccess)
    b->last_time = ms * 1e-3;
  record_durations(b, sel);
  b->unrecorded = false;
  if (b->cused) {
    int e = 0;
    if (cudaMemcpy(&e, b->cerr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return OSQP_ERR_CUDA;
    if (e != kDevOk) return OSQP_ERR_DEVICE;
  }
  return OSQP_OK;
}

template <typename T>
const Scalars* scalars_of(osqp_batch* b, int i) {
  return dev_at<T>(b, i)->sc;
}

}  // namespace

extern "C" {

int32_t osqp_batch_setup(osqp_batch** out, int32_t count, const osqp_csc* P, const double* const* q,
                         const osqp_csc* A, const double* const* l, const double* const* u,
                         const osqp_settings* settings, void* stream) {
  if (!out || !P || !A || !q || !settings || count < 1) return OSQP_ERR_ARG;
  *out = nullptr;
  int rc = check_settings(*settings);
  if (rc) return rc;
  for (int i = 0; i < count; ++i) {
    const int n = P[i].n_cols, m = A[i].n_rows;
    if (n < 1 || m < 0 || P[i].n_rows != n || A[i].n_cols != n) return OSQP_ERR_DIMS;
    if (!q[i] || (m > 0 && (!l || !u || !l[i] || !u[i]))) return OSQP_ERR_ARG;
    if (!valid_csc(&P[i], n, n, true) || !valid_csc(&A[i], m, n, false)) return OSQP_ERR_CSC;
    if (!finite_all(P[i].val, P[i].nnz) || !finite_all(A[i].val, A[i].nnz) || !finite_all(q[i], n))
      return OSQP_ERR_NONFINITE;
    for (int r = 0; r < m; ++r) {
      if (std::isnan(l[i][r]) || std::isnan(u[i][r])) return OSQP_ERR_NONFINITE;
      if (l[i][r] > u[i][r]) return OSQP_ERR_LGTU;
    }
  }
  osqp_batch* b = new (std::nothrow) osqp_batch();
  if (!b) return OSQP_ERR_OOM;
  auto fail = [&](int code) {
    osqp_batch_cleanup(b);
    return code;
  };
  b->count = count;
  b->set = *settings;
  b->P = make_params(*settings);
  b->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&b->device) != cudaSuccess) return fail(OSQP_ERR_CUDA);
  if (cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
    return fail(OSQP_ERR_CUDA);
  // the attribute is the cap for every batch (a per-batch value would race
  // with other batches' launches)
  if ((settings->precision == OSQP_PRECISION_FP64
           ? cudaFuncSetAttribute(k_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kPoolCap)
           : cudaFuncSetAttribute(k_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kPoolCap)) != cudaSuccess)
    return fail(OSQP_ERR_CUDA);
  cudaError_t e = cudaSuccess;
  b->grid = b->num_sms;  // one persistent CTA per SM (set from the occupancy below)

  // Structure of every problem, its schedule and its place in the arena:
  // all static blocks first (one upload), then all dynamic blocks.
  std::vector<HostStructure> hs(count);
  b->L.resize(count);
  size_t s_total = 0;
  for (int i = 0; i < count; ++i) build_host_structure(&P[i], &A[i], &hs[i]);
  // row partition: measured per shape class (settings->autotune), else the rule
  b->groups.assign(count, make_int2(0, 0));
  if (settings->autotune) {
    const int rt = settings->precision == OSQP_PRECISION_FP64 ? autotune_groups<double>(b, hs)
                                                             : autotune_groups<float>(b, hs);
    if (rt == OSQP_ERR_CUDA) return fail(rt);
    if (rt != OSQP_OK) b->groups.assign(count, make_int2(0, 0));
  }
  for (int i = 0; i < count; ++i) {
    ProblemLayout& L = b->L[i];
    L.n = hs[i].n;
    L.m = hs[i].m;
    L.nnz_kn = hs[i].nnz_kn;
    L.nnz_a = hs[i].nnz_a;
    L.kn_s = make_sched(hs[i].kn_rp, kBatchWarps, b->groups[i].x);
    L.a_s = make_sched(hs[i].a_rp, kBatchWarps, b->groups[i].y);
    L.s_off = s_total;
    s_total += static_offsets(L).end;
  }
  b->static_bytes = s_total;
  // Shared memory of a one-CTA solve: the largest need of the batch, capped;
  // a problem's PCG vectors, and its matrices too when they fit beside them
  // (problems above the cap keep their vectors in HBM).
  {
    size_t need = 0;
    for (int i = 0; i < count; ++i) {
      const ProblemLayout& L = b->L[i];
      const bool f64 = settings->precision == OSQP_PRECISION_FP64;
      const size_t v = f64 ? smem_vec_bytes<double>(L.n, L.m) : smem_vec_bytes<float>(L.n, L.m);
      const size_t mb = f64 ? smem_mat_bytes<double>(L.kn_s.npos, L.a_s.npos)
                            : smem_mat_bytes<float>(L.kn_s.npos, L.a_s.npos);
      if (v + mb <= kPoolCap) need = std::max(need, v + mb);
      else if (v <= kPoolCap) need = std::max(need, v);
    }
    b->pool = (int)need;
  }
  size_t v_total = s_total;
  for (int i = 0; i < count; ++i) {
    b->L[i].v_off = v_total;
    v_total += settings->precision == OSQP_PRECISION_FP64
                   ? dynamic_carve<double>(b->L[i], nullptr, nullptr)
                   : dynamic_carve<float>(b->L[i], nullptr, nullptr);
  }
  b->arena_bytes = v_total;
  {
    int occ = 0;
    e = settings->precision == OSQP_PRECISION_FP64
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<double>, kBatchThreads,
                                                            b->pool)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<float>, kBatchThreads,
                                                            b->pool);
    if (e != cudaSuccess) return fail(OSQP_ERR_CUDA);
    b->grid = b->num_sms * std::max(1, occ);
  }
  const size_t dev_bytes = (settings->precision == OSQP_PRECISION_FP64 ? sizeof(Dev<double>)
                                                                       : sizeof(Dev<float>)) *
                           (size_t)count;
  e = cudaMalloc((void**)&b->arena, b->arena_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->arena = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? OSQP_ERR_OOM : OSQP_ERR_CUDA);
  }
  if (cudaMalloc(&b->devs, dev_bytes) != cudaSuccess ||
      cudaMalloc((void**)&b->order_d, sizeof(int) * count) != cudaSuccess ||
      cudaMalloc((void**)&b->queue, sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&b->times_d, sizeof(unsigned long long) * 2 * count) != cudaSuccess) {
    cudaGetLastError();
    return fail(OSQP_ERR_OOM);
  }
  for (auto& ev : b->ev)
    if (cudaEventCreate(&ev) != cudaSuccess) return fail(OSQP_ERR_CUDA);

  // Upload the static blocks in chunks of at most 256 MB of host staging.
  const size_t kChunkBytes = (size_t)256 << 20;
  std::vector<char> stage;
  size_t chunk_begin = 0;
  auto flush = [&](size_t upto) -> bool {
    if (upto <= chunk_begin) return true;
    if (cudaMemcpy(b->arena + chunk_begin, stage.data(), upto - chunk_begin,
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return false;
    chunk_begin = upto;
    stage.clear();
    return true;
  };
  for (int i = 0; i < count; ++i) {
    const ProblemLayout& L = b->L[i];
    const StaticOffsets o = static_offsets(L);
    if (L.s_off + o.end - chunk_begin > kChunkBytes && !flush(L.s_off)) return fail(OSQP_ERR_CUDA);
    stage.resize(L.s_off + o.end - chunk_begin, 0);
    char* base = stage.data() + (L.s_off - chunk_begin);
    const HostStructure& h = hs[i];
    auto put = [&](size_t off, const void* src, size_t bytes) {
      if (bytes) std::memcpy(base + off, src, bytes);
    };
    // column indices and raw values at their positions; padding: column −1, 0
    int* knc = reinterpret_cast<int*>(base + o.kn_ci);
    double* knr = reinterpret_cast<double*>(base + o.kn_raw);
    std::fill(knc, knc + L.kn_s.npos, -1);
    for (int k = 0; k < h.nnz_kn; ++k) {
      const int at = L.kn_s.pos[k], src = h.kn_src[k];
      knc[at] = h.kn_ci[k];
      knr[at] = src < h.nnz_p ? P[i].val[src] : A[i].val[src - h.nnz_p];
    }
    int* ac = reinterpret_cast<int*>(base + o.a_ci);
    double* ar = reinterpret_cast<double*>(base + o.a_raw);
    std::fill(ac, ac + L.a_s.npos, -1);
    for (int k = 0; k < h.nnz_a; ++k) {
      const int at = L.a_s.pos[k];
      ac[at] = h.a_ci[k];
      ar[at] = A[i].val[h.a_src[k] - h.nnz_p];
    }
    const std::pair<const SchedHost*, const SchedOffsets*> sch[] = {{&L.kn_s, &o.kn},
                                                                    {&L.a_s, &o.a}};
    for (const auto& so : sch) {
      put(so.second->sl, so.first->slices.data(), sizeof(int2) * so.first->slices.size());
      put(so.second->sr, so.first->srow.data(), sizeof(int) * so.first->srow.size());
      put(so.second->ch, so.first->chunks.data(), sizeof(int4) * so.first->chunks.size());
      put(so.second->lr, so.first->long_rows.data(), sizeof(int) * so.first->long_rows.size());
      put(so.second->rng, so.first->lrange.data(), sizeof(int2) * so.first->lrange.size());
      put(so.second->li, so.first->lidx.data(), sizeof(int) * so.first->lidx.size());
    }
    put(o.q, q[i], sizeof(double) * L.n);
    if (L.m) {
      put(o.l, l[i], sizeof(double) * L.m);
      put(o.u, u[i], sizeof(double) * L.m);
    }
    hs[i] = HostStructure();  // release host memory early
    b->L[i].kn_s.pos = {};
    b->L[i].a_s.pos = {};
  }
  if (!flush(b->static_bytes)) return fail(OSQP_ERR_CUDA);
  // dynamic blocks start zeroed: the long-row counters must be zero before
  // the first product
  if (b->arena_bytes > b->static_bytes &&
      cudaMemset(b->arena + b->static_bytes, 0, b->arena_bytes - b->static_bytes) != cudaSuccess)
    return fail(OSQP_ERR_CUDA);

  if (settings->precision == OSQP_PRECISION_FP64) fill_batch_devs<double>(b);
  else fill_batch_devs<float>(b);
  if (cudaMemcpy(b->devs, b->devs_host.data(), dev_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(OSQP_ERR_CUDA);
  // Scalars: ρ̄⁰ for every problem; the first launch scales every problem.
  {
    Scalars init{};
    init.rho_bar = settings->rho;
    for (int i = 0; i < count; ++i) {
      Scalars* dst = settings->precision == OSQP_PRECISION_FP64 ? dev_at<double>(b, i)->sc
                                                               : dev_at<float>(b, i)->sc;
      if (cudaMemcpy(dst, &init, sizeof(Scalars), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(OSQP_ERR_CUDA);
    }
  }
  b->inflight.assign(count, -1);
  b->footprint.resize(count);
  for (int i = 0; i < count; ++i) {
    const size_t dyn = settings->precision == OSQP_PRECISION_FP64
                           ? dynamic_carve<double>(b->L[i], nullptr, nullptr)
                           : dynamic_carve<float>(b->L[i], nullptr, nullptr);
    b->footprint[i] = static_offsets(b->L[i]).end + dyn;
  }
  b->mode.assign(count, kModeScale);
  b->times_host.assign(2 * (size_t)count, 0);
  b->last_dur.assign(count, 0.0);
  b->on_cluster.assign(count, 0);
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kBatchCluster);
    cfg.blockDim = dim3(kBatchThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kBatchCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    const cudaError_t ec = settings->precision == OSQP_PRECISION_FP64
                               ? cudaOccupancyMaxActiveClusters(&nc, k_batch_cluster<double>, &cfg)
                               : cudaOccupancyMaxActiveClusters(&nc, k_batch_cluster<float>, &cfg);
    if (ec != cudaSuccess) cudaGetLastError();
    b->cluster_ok = ec == cudaSuccess && nc >= 1;
  }
  if (cudaMemset(b->times_d, 0, sizeof(unsigned long long) * 2 * count) != cudaSuccess)
    return fail(OSQP_ERR_CUDA);
  b->order.resize(count);
  std::iota(b->order.begin(), b->order.end(), 0);
  *out = b;
  return OSQP_OK;
}

int32_t osqp_batch_solve_async(osqp_batch* b) {
  if (!b) return OSQP_ERR_ARG;
  for (int v : b->inflight)
    if (v >= 0) return OSQP_ERR_ARG;  // a slot launch is still in flight
  if (!b->set.warm_start)
    for (int i = 0; i < b->count; ++i) b->mode[i] |= kModeReset;
  // times of an earlier asynchronous launch, if it has finished (no wait)
  if (b->unrecorded && cudaStreamQuery(b->stream) == cudaSuccess) {
    record_durations(b, b->order);
    b->unrecorded = false;
  }
  cudaGetLastError();
  order_longest_first(b, b->order);
  const int rc = batch_launch(b, b->order);
  if (rc == OSQP_OK) b->unrecorded = true;
  return rc;
}

int32_t osqp_batch_solve(osqp_batch* b) {
  const int rc = osqp_batch_solve_async(b);
  if (rc) return rc;
  return batch_wait(b, b->order);
}

int32_t osqp_batch_solve_subset(osqp_batch* b, const int32_t* idx, int32_t k) {
  if (!b || (k > 0 && !idx) || k < 0 || k > b->count) return OSQP_ERR_ARG;
  if (k == 0) return OSQP_OK;
  std::vector<int> sel(idx, idx + k);
  for (int v : sel)
    if (v < 0 || v >= b->count || b->inflight[v] >= 0) return OSQP_ERR_ARG;
  order_longest_first(b, sel);
  if (!b->set.warm_start)
    for (int v : sel) b->mode[v] |= kModeReset;
  const int rc = batch_launch(b, sel);
  if (rc) return rc;
  return batch_wait(b, sel);
}

int32_t osqp_batch_reset(osqp_batch* b) {
  if (!b) return OSQP_ERR_ARG;
  std::fill(b->mode.begin(), b->mode.end(), (int)kModeScale);
  for (int i = 0; i < b->count; ++i) {
    Scalars* dst = b->set.precision == OSQP_PRECISION_FP64 ? dev_at<double>(b, i)->sc
                                                          : dev_at<float>(b, i)->sc;
    if (cudaMemcpyAsync(&dst->rho_bar, &b->set.rho, sizeof(double), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess)
      return OSQP_ERR_CUDA;
  }
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? OSQP_OK : OSQP_ERR_CUDA;
}

static int32_t copy_vectors(osqp_batch* b, int i, const double* q, const double* l,
                            const double* u, cudaStream_t st) {
  const ProblemLayout& L = b->L[i];
  if (q && !finite_all(q, L.n)) return OSQP_ERR_NONFINITE;
  const StaticOffsets o = static_offsets(L);
  char* sb = b->arena + L.s_off;
  if (l || u) {
    std::vector<double> lh(L.m), uh(L.m);
    if (!l && L.m && cudaMemcpy(lh.data(), sb + o.l, sizeof(double) * L.m, cudaMemcpyDeviceToHost) != cudaSuccess)
      return OSQP_ERR_CUDA;
    if (!u && L.m && cudaMemcpy(uh.data(), sb + o.u, sizeof(double) * L.m, cudaMemcpyDeviceToHost) != cudaSuccess)
      return OSQP_ERR_CUDA;
    const double* Lv = l ? l : lh.data();
    const double* Uv = u ? u : uh.data();
    for (int r = 0; r < L.m; ++r) {
      if (std::isnan(Lv[r]) || std::isnan(Uv[r])) return OSQP_ERR_NONFINITE;
      if (Lv[r] > Uv[r]) return OSQP_ERR_LGTU;
    }
  }
  if (q && cudaMemcpyAsync(sb + o.q, q, sizeof(double) * L.n, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return OSQP_ERR_CUDA;
  if (l && L.m && cudaMemcpyAsync(sb + o.l, l, sizeof(double) * L.m, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return OSQP_ERR_CUDA;
  if (u && L.m && cudaMemcpyAsync(sb + o.u, u, sizeof(double) * L.m, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return OSQP_ERR_CUDA;
  if (q || l || u)
    if (!(b->mode[i] & kModeScale)) b->mode[i] |= kModeRefresh;
  return OSQP_OK;
}

int32_t osqp_batch_update_vectors(osqp_batch* b, int32_t i, const double* q, const double* l,
                                  const double* u) {
  if (!b || i < 0 || i >= b->count || b->inflight[i] >= 0) return OSQP_ERR_ARG;
  const int rc = copy_vectors(b, i, q, l, u, b->stream);
  if (rc) return rc;
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? OSQP_OK : OSQP_ERR_CUDA;
}

// Offsets of the concatenated vectors and the staging buffer, on first use.
static int32_t whole_batch_buffers(osqp_batch* b) {
  if (b->stage_d) return OSQP_OK;
  const int count = b->count;
  b->off_n.assign(count + 1, 0);
  b->off_m.assign(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    b->off_n[i + 1] = b->off_n[i] + b->L[i].n;
    b->off_m[i + 1] = b->off_m[i] + b->L[i].m;
  }
  std::vector<long long> both(b->off_n);
  both.insert(both.end(), b->off_m.begin(), b->off_m.end());
  const size_t vals = (size_t)b->off_n[count] + 2 * (size_t)b->off_m[count];
  if (cudaMalloc((void**)&b->off_d, sizeof(long long) * both.size()) != cudaSuccess ||
      cudaMalloc((void**)&b->stage_d, sizeof(double) * std::max<size_t>(vals, 1)) != cudaSuccess) {
    cudaGetLastError();
    if (b->off_d) cudaFree(b->off_d);
    b->off_d = nullptr;
    b->stage_d = nullptr;
    return OSQP_ERR_OOM;
  }
  if (cudaMemcpy(b->off_d, both.data(), sizeof(long long) * both.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return OSQP_ERR_CUDA;
  return OSQP_OK;
}

int32_t osqp_batch_update_all(osqp_batch* b, const double* q_all, const double* l_all,
                              const double* u_all) {
  if (!b || ((l_all == nullptr) != (u_all == nullptr))) return OSQP_ERR_ARG;
  for (int v : b->inflight)
    if (v >= 0) return OSQP_ERR_ARG;
  if (!q_all && !l_all) return OSQP_OK;
  int rc = whole_batch_buffers(b);
  if (rc) return rc;
  const long long N = b->off_n[b->count], M = b->off_m[b->count];
  if (q_all)
    for (long long j = 0; j < N; ++j)
      if (!std::isfinite(q_all[j])) return OSQP_ERR_NONFINITE;
  if (l_all)
    for (long long r = 0; r < M; ++r) {
      if (std::isnan(l_all[r]) || std::isnan(u_all[r])) return OSQP_ERR_NONFINITE;
      if (l_all[r] > u_all[r]) return OSQP_ERR_LGTU;
    }
  double* sq = b->stage_d;
  double* sl = b->stage_d + N;
  double* su = sl + M;
  if ((q_all && N && cudaMemcpyAsync(sq, q_all, sizeof(double) * N, cudaMemcpyHostToDevice,
                                     b->stream) != cudaSuccess) ||
      (l_all && M && cudaMemcpyAsync(sl, l_all, sizeof(double) * M, cudaMemcpyHostToDevice,
                                     b->stream) != cudaSuccess) ||
      (u_all && M && cudaMemcpyAsync(su, u_all, sizeof(double) * M, cudaMemcpyHostToDevice,
                                     b->stream) != cudaSuccess))
    return OSQP_ERR_CUDA;
  const int grid = std::min(b->count, 4 * b->num_sms);
  if (b->set.precision == OSQP_PRECISION_FP64)
    k_scatter_vectors<double><<<grid, 256, 0, b->stream>>>((const Dev<double>*)b->devs, b->count,
                                                           b->off_d, q_all ? sq : nullptr,
                                                           l_all ? sl : nullptr,
                                                           u_all ? su : nullptr);
  else
    k_scatter_vectors<float><<<grid, 256, 0, b->stream>>>((const Dev<float>*)b->devs, b->count,
                                                          b->off_d, q_all ? sq : nullptr,
                                                          l_all ? sl : nullptr,
                                                          u_all ? su : nullptr);
  if (cudaGetLastError() != cudaSuccess) return OSQP_ERR_CUDA;
  for (int i = 0; i < b->count; ++i)
    if (!(b->mode[i] & kModeScale)) b->mode[i] |= kModeRefresh;
  return OSQP_OK;
}

int32_t osqp_batch_get_all(osqp_batch* b, double* x_all, double* y_all) {
  if (!b) return OSQP_ERR_ARG;
  for (int v : b->inflight)
    if (v >= 0) {
      const int rc = osqp_batch_slot_wait(b, v);
      if (rc) return rc;
    }
  int rc = whole_batch_buffers(b);
  if (rc) return rc;
  const long long N = b->off_n[b->count], M = b->off_m[b->count];
  double* sx = b->stage_d;
  double* sy = b->stage_d + N;
  const int grid = std::min(b->count, 4 * b->num_sms);
  if (b->set.precision == OSQP_PRECISION_FP64)
    k_gather_solutions<double><<<grid, 256, 0, b->stream>>>((const Dev<double>*)b->devs, b->count,
                                                            b->off_d, sx, sy);
  else
    k_gather_solutions<float><<<grid, 256, 0, b->stream>>>((const Dev<float>*)b->devs, b->count,
                                                           b->off_d, sx, sy);
  if (cudaGetLastError() != cudaSuccess) return OSQP_ERR_CUDA;
  if ((x_all && N && cudaMemcpyAsync(x_all, sx, sizeof(double) * N, cudaMemcpyDeviceToHost,
                                     b->stream) != cudaSuccess) ||
      (y_all && M && cudaMemcpyAsync(y_all, sy, sizeof(double) * M, cudaMemcpyDeviceToHost,
                                     b->stream) != cudaSuccess))
    return OSQP_ERR_CUDA;
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? OSQP_OK : OSQP_ERR_CUDA;
}

int32_t osqp_batch_launch(osqp_batch* b, int32_t slot, const int32_t* idx, int32_t k,
                          const double* const* q, const double* const* l, const double* const* u) {
  if (!b || slot < 0 || slot >= OSQP_BATCH_MAX_SLOTS || k < 1 || k > b->count || !idx)
    return OSQP_ERR_ARG;
  osqp_batch::Slot& S = b->slots[slot];
  if (!S.members.empty()) return OSQP_ERR_ARG;  // previous launch not retired
  std::vector<int> sel(idx, idx + k);
  for (int v : sel)
    if (v < 0 || v >= b->count || b->inflight[v] >= 0) return OSQP_ERR_ARG;
  if (!S.stream) {
    if (cudaStreamCreateWithFlags(&S.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc((void**)&S.order, sizeof(int) * b->count) != cudaSuccess ||
        cudaMalloc((void**)&S.queue, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&S.err, sizeof(int)) != cudaSuccess ||
        cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return OSQP_ERR_CUDA;
    }
  }
  for (int j = 0; j < k; ++j) {
    const int rc = copy_vectors(b, sel[j], q ? q[j] : nullptr, l ? l[j] : nullptr,
                                u ? u[j] : nullptr, S.stream);
    if (rc) return rc;
  }
  if (!b->set.warm_start)
    for (int v : sel) b->mode[v] |= kModeReset;
  order_longest_first(b, sel);
  const int rc = b->set.precision == OSQP_PRECISION_FP64
                     ? launch_batch<double>(b, sel, S.order, S.queue, S.stream, S.err)
                     : launch_batch<float>(b, sel, S.order, S.queue, S.stream, S.err);
  if (rc) return rc;
  if (cudaEventRecord(S.done, S.stream) != cudaSuccess) return OSQP_ERR_CUDA;
  for (int v : sel) b->inflight[v] = slot;
  S.members = sel;
  return OSQP_OK;
}

// Barrier timeout recorded by a cluster launch of the slot (0: none).
static int slot_error(const osqp_batch::Slot& S) {
  int e = 0;
  if (S.err && cudaMemcpy(&e, S.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return OSQP_ERR_CUDA;
  return e == kDevOk ? OSQP_OK : OSQP_ERR_DEVICE;
}

static void retire(osqp_batch* b, int slot) {
  osqp_batch::Slot& S = b->slots[slot];
  for (int v : S.members) {
    b->inflight[v] = -1;
    unsigned long long t[2];
    if (cudaMemcpy(t, b->times_d + 2 * (size_t)v, sizeof(t), cudaMemcpyDeviceToHost) == cudaSuccess &&
        t[1] > t[0])
      b->last_dur[v] = (double)(t[1] - t[0]) * 1e-9;
  }
  S.members.clear();
}

int32_t osqp_batch_slot_query(osqp_batch* b, int32_t slot) {
  if (!b || slot < 0 || slot >= OSQP_BATCH_MAX_SLOTS) return OSQP_ERR_ARG;
  osqp_batch::Slot& S = b->slots[slot];
  if (S.members.empty()) return 1;
  const cudaError_t e = cudaEventQuery(S.done);
  if (e == cudaErrorNotReady) return 0;
  if (e != cudaSuccess) return OSQP_ERR_CUDA;
  const int rc = slot_error(S);
  retire(b, slot);
  return rc ? rc : 1;
}

int32_t osqp_batch_slot_wait(osqp_batch* b, int32_t slot) {
  if (!b || slot < 0 || slot >= OSQP_BATCH_MAX_SLOTS) return OSQP_ERR_ARG;
  osqp_batch::Slot& S = b->slots[slot];
  if (S.members.empty()) return OSQP_OK;
  if (cudaEventSynchronize(S.done) != cudaSuccess) return OSQP_ERR_CUDA;
  const int rc = slot_error(S);
  retire(b, slot);
  return rc;
}

int32_t osqp_batch_uses_cluster(const osqp_batch* b, int32_t i) {
  if (!b || i < 0 || i >= b->count) return OSQP_ERR_ARG;
  return (b->cluster_ok && b->set.launch != 1 && large_problem(b, i)) ? 1 : 0;
}

int32_t osqp_batch_schedule(const osqp_batch* b, int32_t i, int32_t* groups) {
  if (!b || !groups || i < 0 || i >= b->count) return OSQP_ERR_ARG;
  groups[0] = b->L[i].kn_s.group;
  groups[1] = b->L[i].a_s.group;
  return OSQP_OK;
}

int32_t osqp_batch_tuning(const osqp_batch* b, int32_t cap, int32_t* info, double* cycles) {
  if (!b) return OSQP_ERR_ARG;
  const int nc = (int)b->tune.size();
  for (int k = 0; k < nc && k < cap; ++k) {
    const osqp_batch::TuneClass& t = b->tune[k];
    if (info) {
      const int32_t v[6] = {t.kind, t.rows_b, t.mean_b, t.max_b, t.rep, t.chosen};
      std::memcpy(info + 6 * k, v, sizeof(v));
    }
    if (cycles) std::memcpy(cycles + 6 * k, t.cycles, sizeof(t.cycles));
  }
  return nc;
}

int64_t osqp_batch_footprint(const osqp_batch* b, int32_t i) {
  if (!b || i < 0 || i >= b->count) return OSQP_ERR_ARG;
  return (int64_t)b->footprint[i];
}

int32_t osqp_batch_get(osqp_batch* b, int32_t i, double* x, double* y, double* z,
                       osqp_info* info) {
  if (!b || i < 0 || i >= b->count) return OSQP_ERR_ARG;
  if (b->inflight[i] >= 0) {
    const int rc = osqp_batch_slot_wait(b, b->inflight[i]);
    if (rc) return rc;
  }
  const ProblemLayout& L = b->L[i];
  const bool f64 = b->set.precision == OSQP_PRECISION_FP64;
  const double* xo = f64 ? dev_at<double>(b, i)->x_out : dev_at<float>(b, i)->x_out;
  const double* yo = f64 ? dev_at<double>(b, i)->y_out : dev_at<float>(b, i)->y_out;
  const double* zo = f64 ? dev_at<double>(b, i)->z_out : dev_at<float>(b, i)->z_out;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return OSQP_ERR_CUDA;
  if (x && cudaMemcpy(x, xo, sizeof(double) * L.n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return OSQP_ERR_CUDA;
  if (y && L.m && cudaMemcpy(y, yo, sizeof(double) * L.m, cudaMemcpyDeviceToHost) != cudaSuccess)
    return OSQP_ERR_CUDA;
  if (z && L.m && cudaMemcpy(z, zo, sizeof(double) * L.m, cudaMemcpyDeviceToHost) != cudaSuccess)
    return OSQP_ERR_CUDA;
  if (info) {
    Scalars s;
    unsigned long long t[2];
    const Scalars* src = f64 ? scalars_of<double>(b, i) : scalars_of<float>(b, i);
    if (cudaMemcpy(&s, src, sizeof(Scalars), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(t, b->times_d + 2 * (size_t)i, sizeof(t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return OSQP_ERR_CUDA;
    std::memset(info, 0, sizeof(*info));
    info->status = s.status;
    info->iter = s.iter;
    info->pcg_iters = s.pcg_iters;
    info->rho_updates = s.rho_updates;
    info->ruiz_passes = s.ruiz_passes;
    info->launch = b->on_cluster[i] ? 3 : 1;  // 3: solved by a cluster
    info->polished = s.polished;
    info->obj_val = s.obj;
    info->prim_res = s.prim_res;
    info->dual_res = s.dual_res;
    info->rho_estimate = s.rho_bar;
    info->solve_time = t[1] > t[0] ? (double)(t[1] - t[0]) * 1e-9 : 0.0;
    info->setup_time = b->last_time;  // device time of the last whole-batch launch
  }
  return OSQP_OK;
}

int32_t osqp_batch_cleanup(osqp_batch* b) {
  if (!b) return OSQP_ERR_ARG;
  int rc = OSQP_OK;
  if (b->arena && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = OSQP_ERR_CUDA;
  for (auto& S : b->slots) {
    if (S.stream) {
      if (cudaStreamSynchronize(S.stream) != cudaSuccess) rc = OSQP_ERR_CUDA;
      cudaStreamDestroy(S.stream);
    }
    if (S.order) cudaFree(S.order);
    if (S.queue) cudaFree(S.queue);
    if (S.err) cudaFree(S.err);
    if (S.done) cudaEventDestroy(S.done);
  }
  if (b->cstream) {
    if (cudaStreamSynchronize(b->cstream) != cudaSuccess) rc = OSQP_ERR_CUDA;
    cudaStreamDestroy(b->cstream);
  }
  if (b->cfork) cudaEventDestroy(b->cfork);
  if (b->cjoin) cudaEventDestroy(b->cjoin);
  void* ptrs[] = {b->arena, b->devs, b->order_d, b->queue, b->times_d, b->off_d, b->stage_d,
                  b->corder, b->cqueue,
                  b->cerr};
  for (void* p : ptrs)
    if (p && cudaFree(p) != cudaSuccess) rc = OSQP_ERR_CUDA;
  for (auto& ev : b->ev)
    if (ev) cudaEventDestroy(ev);
  delete b;
  return rc;
}

}  // extern "C"
