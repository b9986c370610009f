// Host driver and C ABI of the GB300 OSQP library (see include/osqp_gb300.h).
//
// Setup (symbolic, host): validate the CSC input, build the structure of
// Kn = [P̄ Āᵀ] (full symmetric P̄ followed by the column of A that row j of Āᵀ
// reads) and of Ā, lay both out in slices (see Sched in device.cuh) with
// gather maps from the CSC value arrays.  Everything numeric — scattering values, Ruiz
// scaling, ρ, the Jacobi diagonal, the ADMM/PCG iteration, residuals,
// unscaling — runs in the kernels of device.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/osqp_gb300.h"
#include "device.cuh"
#include "host_common.h"

using namespace osqpgb;
using namespace osqpgb::host;

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_scale_grid(const __grid_constant__ Dev<T> d,
                                                          const __grid_constant__ Params P,
                                                          Barrier* bar, int* err, double* part,
                                                          double rho_bar, int reset) {
  __shared__ double sm[kSmemDoubles];
  GridTeam tm{bar, err, part, sm, P.barrier_timeout_ns, 0, 0u};
  scale_stage(tm, d, P, rho_bar, reset != 0);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_scale_block(const __grid_constant__ Dev<T> d,
                                                           const __grid_constant__ Params P,
                                                           double rho_bar, int reset) {
  __shared__ double sm[kSmemDoubles];
  BlockTeam tm{sm};
  scale_stage(tm, d, P, rho_bar, reset != 0);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_refresh_grid(const __grid_constant__ Dev<T> d,
                                                            const __grid_constant__ Params P,
                                                            Barrier* bar, int* err, double* part,
                                                            double rho_bar) {
  __shared__ double sm[kSmemDoubles];
  GridTeam tm{bar, err, part, sm, P.barrier_timeout_ns, 0, 0u};
  refresh_stage(tm, d, P, rho_bar);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_refresh_block(const __grid_constant__ Dev<T> d,
                                                             const __grid_constant__ Params P,
                                                             double rho_bar) {
  __shared__ double sm[kSmemDoubles];
  BlockTeam tm{sm};
  refresh_stage(tm, d, P, rho_bar);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_admm_grid(const __grid_constant__ Dev<T> d,
                                                         const __grid_constant__ Params P,
                                                         Barrier* bar, int* err, double* part) {
  __shared__ double sm[kSmemDoubles];
  GridTeam tm{bar, err, part, sm, P.barrier_timeout_ns, 0, 0u};
  admm_stage(tm, d, P);
}

// Cluster-team kernels: one thread-block cluster of kClusterSize CTAs per
// problem.  The counter is zeroed and every CTA has started before anyone
// arrives at a team barrier, and no CTA leaves while another may still read
// its shared memory (the two hardware cluster barriers, reached
// unconditionally by every thread).
#define OSQP_CLUSTER_KERNEL(NAME, STAGE_CALL, ...)                                      \
  template <typename T>                                                                  \
  __global__ void __launch_bounds__(kThreads) NAME(const __grid_constant__ Dev<T> d,     \
                                                   const __grid_constant__ Params P,     \
                                                   int* err, ##__VA_ARGS__) {            \
    __shared__ double sm[kSmemDoubles];                                                  \
    __shared__ double cpart[2 * kMaxRed];                                                \
    __shared__ unsigned ctr;                                                             \
    if (threadIdx.x == 0) ctr = 0u;                                                      \
    cluster_sync_all();                                                                  \
    ClusterTeam tm{sm, cpart, &ctr, err, P.barrier_timeout_ns, cluster_rank(),           \
                   cluster_size(), 0u, 0};                                               \
    STAGE_CALL;                                                                          \
    cluster_sync_all();                                                                  \
  }

OSQP_CLUSTER_KERNEL(k_admm_cluster, admm_stage(tm, d, P))
OSQP_CLUSTER_KERNEL(k_scale_cluster, scale_stage(tm, d, P, rho_bar, reset != 0), double rho_bar,
                    int reset)
OSQP_CLUSTER_KERNEL(k_refresh_cluster, refresh_stage(tm, d, P, rho_bar), double rho_bar)
#undef OSQP_CLUSTER_KERNEL

// One-CTA solve; with a pool the PCG vectors, and the matrices when they fit
// too, live in the CTA's shared memory (smem_plan).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_admm_block(const __grid_constant__ Dev<T> d,
                                                          const __grid_constant__ Params P,
                                                          int pool_bytes) {
  __shared__ double sm[kSmemDoubles];
  __shared__ Dev<T> sdev;
  extern __shared__ __align__(16) unsigned char pool[];
  BlockTeam tm{sm};
  const int plan = smem_plan(d, (size_t)pool_bytes);
  if (plan > 0) {
    stage_in(d, sdev, pool, plan == 2);
    admm_stage(tm, sdev, P);
    stage_out(d, sdev);
  } else {
    admm_stage(tm, d, P);
  }
}

// raw value gather: dst[k] = src[idx[k]], 0 where idx[k] < 0 (layout padding)
__global__ void k_gather(double* __restrict__ dst, const int* __restrict__ idx,
                         const double* __restrict__ src, int count) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    const int i = idx[k];
    dst[k] = i >= 0 ? src[i] : 0.0;
  }
}

// Barrier diagnostic: CTA `absent` returns without arriving, so the others
// must time out, record the error and leave.
__global__ void __launch_bounds__(kThreads) k_barrier_probe(Barrier* bar, int* err, double* part,
                                                             unsigned long long timeout_ns,
                                                             int absent) {
  __shared__ double sm[kSmemDoubles];
  GridTeam tm{bar, err, part, sm, timeout_ns, 0, 0u};
  if ((int)blockIdx.x == absent) return;
  tm.sync();
}

// Autotuner of a single problem's row partition on the grid team: `reps`
// products shaped like the PCG loop's (Alg. 1, step 3), each followed by a
// grid reduction and barrier as in the solve.  KN: w = σu + Kn u with long
// rows left as chunk partials and the inner product (w, u) reduced; else
// t = ρ ∘ Ā (D⁻¹ r), the preconditioned residual gathered on the fly.  x and
// x2 hold ones (x: the gathered vector, x2: the diagonal factor).
template <typename T, bool KN>
__global__ void __launch_bounds__(kThreads)
    k_tune_grid(const __grid_constant__ Sched S, const int* __restrict__ ci,
                const T* __restrict__ va, const T* __restrict__ x, const T* __restrict__ x2,
                T* __restrict__ y, int reps, Barrier* bar, int* err, double* part,
                unsigned long long timeout_ns) {
  __shared__ double sm[kSmemDoubles];
  GridTeam tm{bar, err, part, sm, timeout_ns, 0, 0u};
  for (int r = 0; r < reps; ++r) {
    T acc1 = T(0);
    if constexpr (KN) {
      spmv<1, false, T, T>(
          tm, S, ci, va, [&](int col, T v, T* acc) { acc[0] += v * x[col]; },
          [&](int j, T* acc) {
            const T wj = x2[j] * x[j] + acc[0];
            y[j] = wj;
            acc1 += wj * x[j];
          },
          [&](int j, int first, T* acc) { acc1 += (acc[0] + (first ? x2[j] : T(0))) * x[j]; },
          NoLong{}, LazyTag{});
    } else {
      spmv<1, false, T, T>(
          tm, S, ci, va, [&](int col, T v, T* acc) { acc[0] += v * (x[col] * x2[col]); },
          [&](int i, T* acc) {
            y[i] = x2[i] * acc[0];
            acc1 += y[i];
          });
    }
    const T red_t[1] = {acc1};
    tm.template publish<1, 0u>(red_t);
    if (!tm.sync()) return;
    double red[1];
    tm.template collect<1, 0u>(red);
  }
}

// warm start, part 1: x̄ = D⁻¹x, ȳ = cE⁻¹y, x̃ = x̄, δ = 0
template <typename T>
__global__ void k_warm_xy(const __grid_constant__ Dev<T> d, const double* __restrict__ xw,
                          const double* __restrict__ yw) {
  const double c = d.sc->c;
  const int stride = gridDim.x * blockDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // new iterates: no check on them yet
    d.sc->rp_last = 0.0;
    d.sc->rd_last = 0.0;
  }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += stride) {
    const double xv = xw ? xw[j] / d.D[j] : 0.0;
    d.x[j] = xv;
    d.xt[j] = xv;
    d.dx[j] = 0.0;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) {
    d.y[i] = yw ? c * yw[i] / d.E[i] : 0.0;
    d.dy[i] = 0.0;
    d.z[i] = 0.0;
    d.zt[i] = 0.0;
  }
}

// warm start, part 2: z̄ = z̃ = Āx̄
template <typename T>
__global__ void k_warm_z(const __grid_constant__ Dev<T> d) {
  PlainTeam tm;
  spmv<1, false, double, T>(
      tm, d.as, d.a_ci, d.a_v, [&](int col, T v, double* acc) { acc[0] += (double)v * d.x[col]; },
      [&](int i, double* acc) {
        d.z[i] = acc[0];
        d.zt[i] = acc[0];
      });
}

template <typename T>
__global__ void k_zero_iterates(const __grid_constant__ Dev<T> d) {
  const int stride = gridDim.x * blockDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.sc->rp_last = 0.0;
    d.sc->rd_last = 0.0;
  }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += stride) {
    d.x[j] = 0.0;
    d.dx[j] = 0.0;
    d.xt[j] = 0.0;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) {
    d.z[i] = 0.0;
    d.y[i] = 0.0;
    d.dy[i] = 0.0;
    d.zt[i] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

constexpr int kClusterSize = 8;  // CTAs of a cluster team (portable maximum)
constexpr size_t kBlockPoolCap = 160 << 10;  // shared memory for a one-CTA solve's PCG vectors

struct osqp_solver {
  int device = 0, num_sms = 0, grid = 0, use_grid = 0, use_cluster = 0;
  int pool = 0;  // dynamic shared memory of the one-CTA solve (0: vectors in HBM)
  // grid-team autotuner: chosen group widths of Kn and Ā (0: the rule, -1:
  // the timing failed and the rule is in force) and
  // the measured milliseconds per launch of each candidate G = 1…32
  int tuned_kn = 0, tuned_a = 0;
  double tune_kn_ms[6] = {0, 0, 0, 0, 0, 0}, tune_a_ms[6] = {0, 0, 0, 0, 0, 0};
  cudaStream_t stream = nullptr;
  osqp_settings set{};
  Params P{};
  int n = 0, m = 0, nnzP = 0, nnzA = 0, nnzKn = 0;
  // CSR structure (setup only), then column indices and CSC sources of the
  // sliced layouts (−1 at padding)
  std::vector<int> kn_rp, kn_ci, kn_src, a_rp, a_ci, a_src;
  SchedHost kn_s, a_s;
  char* arena = nullptr;
  Dev<double> d64{};
  Dev<float> d32{};
  double* raw_in = nullptr;
  int *kn_src_d = nullptr, *a_src_d = nullptr;
  double *x_ws = nullptr, *y_ws = nullptr;
  Barrier* bar = nullptr;
  int* err = nullptr;
  double* part = nullptr;
  Scalars* sc = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  osqp_info info{};
  double rho_bar = 0.1;
  bool solved = false;
};

namespace {

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) {                      \
      if (e_ == cudaErrorMemoryAllocation) {      \
        cudaGetLastError();                       \
        return OSQP_ERR_OOM;                      \
      }                                           \
      return OSQP_ERR_CUDA;                       \
    }                                             \
  } while (0)

// Device copy of a schedule: arrays carved from the arena.
void take_sched(Arena& A, const SchedHost& h, int nrows, Sched& S) {
  S.nrows = nrows;
  S.group = h.group;
  S.long_thresh = h.long_thresh;
  S.nchunks = (int)h.chunks.size();
  S.nlong = (int)h.long_rows.size();
  S.nslices = (int)h.slices.size();
  S.slices = A.take<int2>(h.slices.size());
  S.srow = A.take<int>(h.srow.size());
  S.chunks = A.take<int4>(h.chunks.size());
  S.long_rows = A.take<int>(h.long_rows.size());
  S.lrange = A.take<int2>(h.lrange.size());
  S.lidx = A.take<int>(h.lidx.size());
  S.cpart = A.take<double>(h.chunks.size() * kMaxNV);
  S.ccount = A.take<unsigned>(h.lrange.size());
  S.npos = h.npos;
}

template <typename T>
void fill_dev(osqp_solver* s, Arena& A, Dev<T>& d) {
  const int n = s->n, m = s->m;
  d.n = n;
  d.m = m;
  d.kn_ci = A.take<int>(s->kn_s.npos);
  d.kn_v = A.take<T>(s->kn_s.npos);
  d.kn_raw = A.take<double>(s->kn_s.npos);
  d.a_ci = A.take<int>(s->a_s.npos);
  d.a_v = A.take<T>(s->a_s.npos);
  d.a_raw = A.take<double>(s->a_s.npos);
  take_sched(A, s->kn_s, n, d.kn);
  take_sched(A, s->a_s, m, d.as);
  d.q_raw = A.take<double>(n);
  d.l_raw = A.take<double>(m);
  d.u_raw = A.take<double>(m);
  d.rtype = A.take<uint8_t>(m);
  double** nvec[] = {&d.D, &d.q, &d.pdiag, &d.dg, &d.nrm_n, &d.x, &d.dx, &d.px,
                     &d.aty, &d.pdx, &d.atdy, &d.x_out, &d.dcert, &d.xt, &d.Dinv,
                     &d.pol_x, &d.pol_dx, &d.pol_r, &d.pol_z, &d.pol_p, &d.pol_kp,
                     &d.pol_dg};
  for (double** p : nvec) *p = A.take<double>(n);
  double** mvec[] = {&d.E, &d.l, &d.u, &d.rho, &d.rho_inv, &d.nrm_m, &d.z, &d.y,
                     &d.dy, &d.ax, &d.adx, &d.azt, &d.z_out, &d.y_out, &d.pcert,
                     &d.zt, &d.wm, &d.um, &d.Einv, &d.pol_y, &d.pol_t, &d.pol_r2};
  for (double** p : mvec) *p = A.take<double>(m);
  d.pol_act = A.take<uint8_t>(m);
  T** tn[] = {&d.dinv, &d.b, &d.p, &d.r0, &d.r1, &d.s0, &d.s1, &d.w0, &d.w1};
  for (T** p : tn) *p = A.take<T>(n);
  d.ut0 = A.take<T>((size_t)n + m);
  d.ut1 = A.take<T>((size_t)n + m);
  T** tmv[] = {&d.ap, &d.dzt, &d.rhoT, &d.rho_invT};
  for (T** p : tmv) *p = A.take<T>(m);
  d.dxt = A.take<T>(n);
}

template <typename T>
Dev<T>& dev_of(osqp_solver* s);
template <>
Dev<double>& dev_of<double>(osqp_solver* s) {
  return s->d64;
}
template <>
Dev<float>& dev_of<float>(osqp_solver* s) {
  return s->d32;
}

// Launch a cluster-team kernel: one cluster of kClusterSize CTAs.
template <typename... KArgs, typename... Args>
cudaError_t launch_cluster(osqp_solver* s, void (*kernel)(KArgs...), Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterSize);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterSize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename T>
int launch_scale(osqp_solver* s, int reset) {
  Dev<T>& d = dev_of<T>(s);
  if (s->use_cluster) {
    CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
    CK(launch_cluster(s, k_scale_cluster<T>, d, s->P, s->err, s->rho_bar, reset));
  } else if (s->use_grid) {
    CK(cudaMemsetAsync(s->bar, 0, sizeof(Barrier), s->stream));
    CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
    double rb = s->rho_bar;
    void* args[] = {(void*)&d, (void*)&s->P, (void*)&s->bar, (void*)&s->err, (void*)&s->part,
                    (void*)&rb, (void*)&reset};
    CK(cudaLaunchCooperativeKernel((const void*)k_scale_grid<T>, dim3(s->grid), dim3(kThreads), args,
                                   0, s->stream));
  } else {
    k_scale_block<T><<<1, kThreads, 0, s->stream>>>(d, s->P, s->rho_bar, reset);
    CK(cudaGetLastError());
  }
  return OSQP_OK;
}

template <typename T>
int launch_refresh(osqp_solver* s) {
  Dev<T>& d = dev_of<T>(s);
  if (s->use_cluster) {
    CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
    CK(launch_cluster(s, k_refresh_cluster<T>, d, s->P, s->err, s->rho_bar));
  } else if (s->use_grid) {
    CK(cudaMemsetAsync(s->bar, 0, sizeof(Barrier), s->stream));
    CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
    double rb = s->rho_bar;
    void* args[] = {(void*)&d, (void*)&s->P, (void*)&s->bar, (void*)&s->err, (void*)&s->part,
                    (void*)&rb};
    CK(cudaLaunchCooperativeKernel((const void*)k_refresh_grid<T>, dim3(s->grid), dim3(kThreads),
                                   args, 0, s->stream));
  } else {
    k_refresh_block<T><<<1, kThreads, 0, s->stream>>>(d, s->P, s->rho_bar);
    CK(cudaGetLastError());
  }
  return OSQP_OK;
}

template <typename T>
int launch_admm(osqp_solver* s) {
  Dev<T>& d = dev_of<T>(s);
  if (!s->set.warm_start) {
    k_zero_iterates<T><<<64, 256, 0, s->stream>>>(d);
    CK(cudaGetLastError());
  }
  if (s->use_cluster) {
    CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
    CK(launch_cluster(s, k_admm_cluster<T>, d, s->P, s->err));
  } else if (s->use_grid) {
    CK(cudaMemsetAsync(s->bar, 0, sizeof(Barrier), s->stream));
    CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
    void* args[] = {(void*)&d, (void*)&s->P, (void*)&s->bar, (void*)&s->err, (void*)&s->part};
    CK(cudaLaunchCooperativeKernel((const void*)k_admm_grid<T>, dim3(s->grid), dim3(kThreads), args,
                                   0, s->stream));
  } else {
    k_admm_block<T><<<1, kThreads, s->pool, s->stream>>>(d, s->P, s->pool);
    CK(cudaGetLastError());
  }
  return OSQP_OK;
}

template <typename T>
int launch_warm(osqp_solver* s, const double* xw, const double* yw) {
  Dev<T>& d = dev_of<T>(s);
  k_warm_xy<T><<<64, 256, 0, s->stream>>>(d, xw, yw);
  CK(cudaGetLastError());
  k_warm_z<T><<<std::max(1, std::min(1024, (s->m + 255) / 256)), 256, 0, s->stream>>>(d);
  CK(cudaGetLastError());
  return OSQP_OK;
}

int do_scale(osqp_solver* s, int reset) {
  return s->set.precision == OSQP_PRECISION_FP64 ? launch_scale<double>(s, reset)
                                                 : launch_scale<float>(s, reset);
}
int do_refresh(osqp_solver* s) {
  return s->set.precision == OSQP_PRECISION_FP64 ? launch_refresh<double>(s)
                                                 : launch_refresh<float>(s);
}
int do_admm(osqp_solver* s) {
  return s->set.precision == OSQP_PRECISION_FP64 ? launch_admm<double>(s) : launch_admm<float>(s);
}
int do_warm(osqp_solver* s, const double* xw, const double* yw) {
  return s->set.precision == OSQP_PRECISION_FP64 ? launch_warm<double>(s, xw, yw)
                                                 : launch_warm<float>(s, xw, yw);
}

template <typename T>
const Dev<T>& cdev(const osqp_solver* s) {
  return dev_of<T>(const_cast<osqp_solver*>(s));
}

// The double-precision arrays shared by both precisions are at the same
// places in d64 and d32; read them through whichever is live.
const double* out_x(const osqp_solver* s) {
  return s->set.precision == OSQP_PRECISION_FP64 ? s->d64.x_out : s->d32.x_out;
}
const double* out_y(const osqp_solver* s) {
  return s->set.precision == OSQP_PRECISION_FP64 ? s->d64.y_out : s->d32.y_out;
}
const double* out_z(const osqp_solver* s) {
  return s->set.precision == OSQP_PRECISION_FP64 ? s->d64.z_out : s->d32.z_out;
}
const double* out_pc(const osqp_solver* s) {
  return s->set.precision == OSQP_PRECISION_FP64 ? s->d64.pcert : s->d32.pcert;
}
const double* out_dc(const osqp_solver* s) {
  return s->set.precision == OSQP_PRECISION_FP64 ? s->d64.dcert : s->d32.dcert;
}

template <typename T>
void raw_ptrs(osqp_solver* s, double** kn_raw, double** a_raw, double** q, double** l, double** u) {
  Dev<T>& d = dev_of<T>(s);
  *kn_raw = const_cast<double*>(d.kn_raw);
  *a_raw = const_cast<double*>(d.a_raw);
  *q = const_cast<double*>(d.q_raw);
  *l = const_cast<double*>(d.l_raw);
  *u = const_cast<double*>(d.u_raw);
}

void get_raw(osqp_solver* s, double** kn_raw, double** a_raw, double** q, double** l, double** u) {
  if (s->set.precision == OSQP_PRECISION_FP64) raw_ptrs<double>(s, kn_raw, a_raw, q, l, u);
  else raw_ptrs<float>(s, kn_raw, a_raw, q, l, u);
}

// Values of raw_in (CSC order: P upper then A) → sliced layouts of Kn and Ā.
int scatter_raw(osqp_solver* s) {
  double *kn_raw, *a_raw, *q, *l, *u;
  get_raw(s, &kn_raw, &a_raw, &q, &l, &u);
  const int nk = s->kn_s.npos, na = s->a_s.npos;
  if (nk > 0) {
    k_gather<<<std::min(4096, (nk + 255) / 256), 256, 0, s->stream>>>(kn_raw, s->kn_src_d,
                                                                       s->raw_in, nk);
    CK(cudaGetLastError());
  }
  if (na > 0) {
    k_gather<<<std::min(4096, (na + 255) / 256), 256, 0, s->stream>>>(a_raw, s->a_src_d,
                                                                       s->raw_in, na);
    CK(cudaGetLastError());
  }
  return OSQP_OK;
}

int read_scalars(osqp_solver* s, Scalars* out) {
  CK(cudaMemcpyAsync(out, s->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return OSQP_OK;
}

int check_device_error(osqp_solver* s) {
  if (!s->use_grid && !s->use_cluster) return OSQP_OK;
  int e = 0;
  CK(cudaMemcpyAsync(&e, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return e == kDevOk ? OSQP_OK : OSQP_ERR_DEVICE;
}

// Group widths tried by the autotuner and its products per timed launch.
constexpr int kGridTuneGroups[] = {1, 2, 4, 8, 16, 32};
constexpr int kGridTuneReps = 20;
constexpr float kGridTuneMargin = 1.03f;

// Time every candidate group width of one matrix (kn: Kn, else Ā; CSR row
// pointers rp, columns ci, ncols gathered entries) on the grid team, with
// the product the PCG loop makes of it, and return the one
// to use: the fastest, unless the rule's width is within kGridTuneMargin of
// it (timing noise then does not move the choice); -1 when a CUDA call fails
// (the rule stays in force).  The device memory of each candidate is
// allocated and freed here, at setup.
template <typename T>
int tune_grid_matrix(osqp_solver* s, bool kn, const std::vector<int>& rp,
                     const std::vector<int>& ci, int ncols, long long nwarps, double* ms_out) {
  const int nrows = (int)rp.size() - 1;
  int best = 0;
  float best_ms = 0.f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return -1;
  }
  for (int k = 0; k < 6; ++k) {
    const int g = kGridTuneGroups[k];
    ms_out[k] = 0.0;
    SchedHost h = make_sched(rp, nwarps, g);
    std::vector<int> cpos = to_positions(h, ci, -1);
    std::vector<T> vpos(cpos.size());
    for (size_t q = 0; q < cpos.size(); ++q) vpos[q] = cpos[q] >= 0 ? T(1) : T(0);
    // arrays of the candidate: one pass over a null arena sizes the
    // allocation, a second carves it
    Sched S{};
    int* d_ci = nullptr;
    T *d_va = nullptr, *d_x = nullptr, *d_x2 = nullptr, *d_y = nullptr;
    Barrier* bar = nullptr;
    int* err = nullptr;
    double* part = nullptr;
    auto carve = [&](Arena& A) {
      take_sched(A, h, nrows, S);
      d_ci = A.take<int>(h.npos);
      d_va = A.take<T>(h.npos);
      d_x = A.take<T>(ncols);
      d_x2 = A.take<T>(std::max(nrows, ncols));
      d_y = A.take<T>(nrows);
      bar = A.take<Barrier>(1);
      err = A.take<int>(1);
      part = A.take<double>((size_t)2 * s->grid * kMaxRed);
    };
    Arena sizing;
    carve(sizing);
    const size_t bytes = sizing.off + 256;
    char* mem = nullptr;
    if (cudaMalloc((void**)&mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      best = -1;
      break;
    }
    Arena A{mem, 0};
    carve(A);
    std::vector<T> ones(std::max(ncols, 1), T(1)), ones2(std::max(std::max(nrows, ncols), 1), T(1));
    // host → device copy of a whole vector (nothing to do when it is empty)
    auto up = [](const void* dst, const auto& v) {
      return v.empty() || cudaMemcpy(const_cast<void*>(dst), v.data(), sizeof(v[0]) * v.size(),
                                     cudaMemcpyHostToDevice) == cudaSuccess;
    };
    bool ok = cudaMemset(mem, 0, bytes) == cudaSuccess && up(d_ci, cpos) && up(d_va, vpos) &&
              up(d_x, ones) && up(d_x2, ones2) && up(S.slices, h.slices) && up(S.srow, h.srow) &&
              up(S.chunks, h.chunks) && up(S.long_rows, h.long_rows) && up(S.lrange, h.lrange) &&
              up(S.lidx, h.lidx);
    float ms_min = 0.f;
    for (int pass = 0; ok && pass < 3; ++pass) {
      // barrier counter and error flag zeroed before every launch
      int reps = kGridTuneReps;
      unsigned long long tns = s->P.barrier_timeout_ns;
      ok = cudaMemsetAsync(bar, 0, sizeof(Barrier), s->stream) == cudaSuccess &&
           cudaMemsetAsync(err, 0, sizeof(int), s->stream) == cudaSuccess &&
           cudaEventRecord(e0, s->stream) == cudaSuccess;
      void* args[] = {(void*)&S,   (void*)&d_ci, (void*)&d_va, (void*)&d_x,
                      (void*)&d_x2, (void*)&d_y, (void*)&reps, (void*)&bar,
                      (void*)&err, (void*)&part, (void*)&tns};
      const void* fn = kn ? (const void*)k_tune_grid<T, true> : (const void*)k_tune_grid<T, false>;
      ok = ok && cudaLaunchCooperativeKernel(fn, dim3(s->grid), dim3(kThreads), args, 0,
                                             s->stream) == cudaSuccess;
      ok = ok && cudaEventRecord(e1, s->stream) == cudaSuccess &&
           cudaStreamSynchronize(s->stream) == cudaSuccess;
      int he = 0;
      ok = ok && cudaMemcpy(&he, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && he == 0;
      float ms = 0.f;
      ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      if (ok && pass > 0) ms_min = pass == 1 ? ms : std::min(ms_min, ms);
    }
    cudaFree(mem);
    if (!ok) {
      cudaGetLastError();
      best = -1;
      break;
    }
    ms_out[k] = ms_min;
    if (best == 0 || ms_min < best_ms) {
      best = g;
      best_ms = ms_min;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best > 0) {
    const int rule = make_sched(rp, nwarps).group;
    for (int k = 0; k < 6; ++k)
      if (kGridTuneGroups[k] == rule && ms_out[k] <= kGridTuneMargin * best_ms) best = rule;
  }
  return best;
}

int build_structure(osqp_solver* s, const osqp_csc* P, const osqp_csc* A) {
  HostStructure h;
  build_host_structure(P, A, &h);
  s->nnzKn = h.nnz_kn;
  s->kn_rp.swap(h.kn_rp);
  s->kn_ci.swap(h.kn_ci);
  s->kn_src.swap(h.kn_src);
  s->a_rp.swap(h.a_rp);
  s->a_ci.swap(h.a_ci);
  s->a_src.swap(h.a_src);
  return OSQP_OK;
}

template <typename T>
size_t arena_bytes_for(osqp_solver* s, size_t part_doubles) {
  Arena A;
  Dev<T> d{};
  fill_dev<T>(s, A, d);
  A.take<double>(s->nnzP + s->nnzA);  // raw_in
  A.take<int>(s->kn_s.npos);
  A.take<int>(s->a_s.npos);
  A.take<double>(s->n);
  A.take<double>(s->m);
  A.take<Barrier>(1);
  A.take<int>(1);
  A.take<double>(part_doubles);
  A.take<Scalars>(1);
  return A.off + 256;
}

template <typename T>
int carve_and_upload(osqp_solver* s, size_t part_doubles) {
  Arena A{s->arena, 0};
  Dev<T>& d = dev_of<T>(s);
  fill_dev<T>(s, A, d);
  s->raw_in = A.take<double>(s->nnzP + s->nnzA);
  s->kn_src_d = A.take<int>(s->kn_s.npos);
  s->a_src_d = A.take<int>(s->a_s.npos);
  s->x_ws = A.take<double>(s->n);
  s->y_ws = A.take<double>(s->m);
  s->bar = A.take<Barrier>(1);
  s->err = A.take<int>(1);
  s->part = A.take<double>(part_doubles);
  s->sc = A.take<Scalars>(1);
  d.sc = s->sc;
  auto up = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream);
  };
  CK(up((void*)d.kn_ci, s->kn_ci.data(), s->kn_ci.size() * sizeof(int)));
  CK(up((void*)d.a_ci, s->a_ci.data(), s->a_ci.size() * sizeof(int)));
  CK(up(s->kn_src_d, s->kn_src.data(), s->kn_src.size() * sizeof(int)));
  CK(up(s->a_src_d, s->a_src.data(), s->a_src.size() * sizeof(int)));
  const std::pair<const SchedHost*, const Sched*> sch[] = {{&s->kn_s, &d.kn}, {&s->a_s, &d.as}};
  for (const auto& hs : sch) {
    const SchedHost& h = *hs.first;
    const Sched& S = *hs.second;
    CK(up((void*)S.slices, h.slices.data(), h.slices.size() * sizeof(int2)));
    CK(up((void*)S.srow, h.srow.data(), h.srow.size() * sizeof(int)));
    CK(up((void*)S.chunks, h.chunks.data(), h.chunks.size() * sizeof(int4)));
    CK(up((void*)S.long_rows, h.long_rows.data(), h.long_rows.size() * sizeof(int)));
    CK(up((void*)S.lrange, h.lrange.data(), h.lrange.size() * sizeof(int2)));
    CK(up((void*)S.lidx, h.lidx.data(), h.lidx.size() * sizeof(int)));
    if (!h.lrange.empty())
      CK(cudaMemsetAsync(S.ccount, 0, h.lrange.size() * sizeof(unsigned), s->stream));
  }
  CK(cudaMemsetAsync(s->sc, 0, sizeof(Scalars), s->stream));
  return OSQP_OK;
}

int upload_vectors(osqp_solver* s, const double* q, const double* l, const double* u,
                   cudaMemcpyKind kind) {
  double *kn_raw, *a_raw, *qd, *ld, *ud;
  get_raw(s, &kn_raw, &a_raw, &qd, &ld, &ud);
  if (q) CK(cudaMemcpyAsync(qd, q, sizeof(double) * s->n, kind, s->stream));
  if (l && s->m) CK(cudaMemcpyAsync(ld, l, sizeof(double) * s->m, kind, s->stream));
  if (u && s->m) CK(cudaMemcpyAsync(ud, u, sizeof(double) * s->m, kind, s->stream));
  return OSQP_OK;
}

float elapsed_s(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return 0.f;
  return ms * 1e-3f;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void osqp_set_default_settings(osqp_settings* s) {
  if (!s) return;
  std::memset(s, 0, sizeof(*s));
  s->rho = 0.1;
  s->sigma = 1e-6;
  s->alpha = 1.6;
  s->eps_abs = 1e-3;
  s->eps_rel = 1e-3;
  s->eps_pinf = 1e-4;
  s->eps_dinf = 1e-4;
  s->adaptive_rho_tolerance = 5.0;
  s->eps_equil = 1e-3;
  s->pcg_tol_fraction = 0.15;
  s->pcg_tol_floor = 1e-10;
  s->time_limit = 0.0;
  s->max_iter = 4000;
  s->check_interval = 25;
  s->adaptive_rho = 1;
  s->scaling_iters = 10;
  s->max_rho_updates = 20;
  s->pcg_max_iter = 100;
  s->precision = OSQP_PRECISION_FP64;
  s->warm_start = 1;
  s->launch = 0;
  s->polish = 0;
  s->polish_refine_iter = 3;
  s->delta = 1e-6;
  s->autotune = 1;
}

const char* osqp_error_message(int32_t code) {
  switch (code) {
    case OSQP_OK: return "ok";
    case OSQP_ERR_DIMS: return "invalid dimensions";
    case OSQP_ERR_CSC: return "invalid CSC matrix (pointers, ordering, range or triangle)";
    case OSQP_ERR_NONFINITE: return "non-finite value in P, A or q, or NaN bound";
    case OSQP_ERR_LGTU: return "lower bound greater than upper bound";
    case OSQP_ERR_SETTINGS: return "invalid settings";
    case OSQP_ERR_CUDA: return "CUDA runtime error";
    case OSQP_ERR_OOM: return "device memory allocation failed";
    case OSQP_ERR_ARG: return "NULL solver or required argument";
    case OSQP_ERR_DEVICE: return "device-side wait timed out";
    case OSQP_ERR_LIMIT: return "problem size beyond this entry point's limit";
    default: return "unknown code";
  }
}

int32_t osqp_setup(osqp_solver** out, const osqp_csc* P, const double* q, const osqp_csc* A,
                   const double* l, const double* u, const osqp_settings* settings,
                   void* stream) {
  if (!out || !P || !A || !q || !settings) return OSQP_ERR_ARG;
  *out = nullptr;
  const int n = P->n_cols, m = A->n_rows;
  if (n < 1 || m < 0 || P->n_rows != n || A->n_cols != n) return OSQP_ERR_DIMS;
  if (m > 0 && (!l || !u)) return OSQP_ERR_ARG;
  if (!valid_csc(P, n, n, true) || !valid_csc(A, m, n, false)) return OSQP_ERR_CSC;
  if (!finite_all(P->val, P->nnz) || !finite_all(A->val, A->nnz) || !finite_all(q, n))
    return OSQP_ERR_NONFINITE;
  for (int i = 0; i < m; ++i) {
    if (std::isnan(l[i]) || std::isnan(u[i])) return OSQP_ERR_NONFINITE;
    if (l[i] > u[i]) return OSQP_ERR_LGTU;
  }
  int rc = check_settings(*settings);
  if (rc) return rc;

  osqp_solver* s = new (std::nothrow) osqp_solver();
  if (!s) return OSQP_ERR_OOM;
  s->set = *settings;
  s->P = make_params(*settings);
  s->stream = (cudaStream_t)stream;
  s->n = n;
  s->m = m;
  s->nnzP = P->nnz;
  s->nnzA = A->nnz;
  s->rho_bar = settings->rho;
  auto fail = [&](int code) {
    osqp_cleanup(s);
    return code;
  };
  if (cudaGetDevice(&s->device) != cudaSuccess) return fail(OSQP_ERR_CUDA);
  if (cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
    return fail(OSQP_ERR_CUDA);
  build_structure(s, P, A);

  // Launch shape: one persistent CTA for small problems, else a cooperative
  // grid of every SM slot the kernel can hold.
  const long long work = (long long)s->nnzKn + s->nnzA + n + m;
  s->use_grid = settings->launch == 2 || (settings->launch == 0 && work > 60000);
  s->use_cluster = settings->launch == 3;
  if (s->use_cluster) {
    s->use_grid = 0;
    // a cluster of kClusterSize one-SM CTAs must fit on the device
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterSize);
    cfg.blockDim = dim3(kThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterSize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    cudaError_t ec = settings->precision == OSQP_PRECISION_FP64
                         ? cudaOccupancyMaxActiveClusters(&nc, k_admm_cluster<double>, &cfg)
                         : cudaOccupancyMaxActiveClusters(&nc, k_admm_cluster<float>, &cfg);
    if (ec != cudaSuccess || nc < 1) {
      cudaGetLastError();
      return fail(OSQP_ERR_CUDA);
    }
  }
  int per_sm = 1;
  {
    int occ = 0;
    cudaError_t e = settings->precision == OSQP_PRECISION_FP64
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_admm_grid<double>,
                                                                        kThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_admm_grid<float>,
                                                                        kThreads, 0);
    if (e != cudaSuccess) return fail(OSQP_ERR_CUDA);
    int occ2 = 0;
    e = settings->precision == OSQP_PRECISION_FP64
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_scale_grid<double>, kThreads, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_scale_grid<float>, kThreads, 0);
    if (e != cudaSuccess) return fail(OSQP_ERR_CUDA);
    int occ3 = 0;
    e = settings->precision == OSQP_PRECISION_FP64
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ3, k_refresh_grid<double>, kThreads,
                                                            0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ3, k_refresh_grid<float>, kThreads,
                                                            0);
    if (e != cudaSuccess) return fail(OSQP_ERR_CUDA);
    per_sm = std::max(1, std::min(std::min(occ, occ2), std::min(occ3, 2)));
    // the grid reduction combines at most 512 per-CTA partials
    while (per_sm > 1 && s->num_sms * per_sm > 512) --per_sm;
  }
  s->grid = s->num_sms * per_sm;
  {
    const long long nwarps =
        (long long)(s->use_grid ? s->grid : (s->use_cluster ? kClusterSize : 1)) * (kThreads / 32);
    // grid team: time the candidate row partitions of both matrices on
    // the device (settings->autotune) and keep the fastest
    if (s->use_grid && settings->autotune) {
      const bool f64 = settings->precision == OSQP_PRECISION_FP64;
      s->tuned_kn =
          f64 ? tune_grid_matrix<double>(s, true, s->kn_rp, s->kn_ci, n + m, nwarps, s->tune_kn_ms)
              : tune_grid_matrix<float>(s, true, s->kn_rp, s->kn_ci, n + m, nwarps, s->tune_kn_ms);
      s->tuned_a =
          f64 ? tune_grid_matrix<double>(s, false, s->a_rp, s->a_ci, n, nwarps, s->tune_a_ms)
              : tune_grid_matrix<float>(s, false, s->a_rp, s->a_ci, n, nwarps, s->tune_a_ms);
    }
    s->kn_s = make_sched(s->kn_rp, nwarps, std::max(s->tuned_kn, 0));
    s->a_s = make_sched(s->a_rp, nwarps, std::max(s->tuned_a, 0));
    s->kn_ci = to_positions(s->kn_s, s->kn_ci, -1);
    s->kn_src = to_positions(s->kn_s, s->kn_src, -1);
    s->a_ci = to_positions(s->a_s, s->a_ci, -1);
    s->a_src = to_positions(s->a_s, s->a_src, -1);
    s->kn_s.pos = {};
    s->a_s.pos = {};
  }
  if (!s->use_grid && !s->use_cluster) {
    const bool f64 = settings->precision == OSQP_PRECISION_FP64;
    const size_t v = f64 ? smem_vec_bytes<double>(n, m) : smem_vec_bytes<float>(n, m);
    const size_t mb = f64 ? smem_mat_bytes<double>(s->kn_s.npos, s->a_s.npos)
                          : smem_mat_bytes<float>(s->kn_s.npos, s->a_s.npos);
    const size_t need = v + mb <= kBlockPoolCap ? v + mb : v;
    if (need <= kBlockPoolCap) {
      // the attribute is the cap for every solver (a per-solver value would
      // race with other solvers' launches)
      const cudaError_t ea =
          settings->precision == OSQP_PRECISION_FP64
              ? cudaFuncSetAttribute(k_admm_block<double>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlockPoolCap)
              : cudaFuncSetAttribute(k_admm_block<float>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlockPoolCap);
      if (ea == cudaSuccess) s->pool = (int)need;
      else cudaGetLastError();
    }
  }
  const size_t part_doubles = (size_t)2 * s->grid * kMaxRed;
  const size_t bytes = settings->precision == OSQP_PRECISION_FP64
                           ? arena_bytes_for<double>(s, part_doubles)
                           : arena_bytes_for<float>(s, part_doubles);
  cudaError_t e = cudaMalloc((void**)&s->arena, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->arena = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? OSQP_ERR_OOM : OSQP_ERR_CUDA);
  }
  for (auto& ev : s->ev)
    if (cudaEventCreate(&ev) != cudaSuccess) return fail(OSQP_ERR_CUDA);
  rc = settings->precision == OSQP_PRECISION_FP64 ? carve_and_upload<double>(s, part_doubles)
                                                  : carve_and_upload<float>(s, part_doubles);
  if (rc) return fail(rc);
  if (s->nnzP && cudaMemcpyAsync(s->raw_in, P->val, sizeof(double) * s->nnzP,
                                 cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
    return fail(OSQP_ERR_CUDA);
  if (s->nnzA && cudaMemcpyAsync(s->raw_in + s->nnzP, A->val, sizeof(double) * s->nnzA,
                                 cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
    return fail(OSQP_ERR_CUDA);
  if ((rc = upload_vectors(s, q, l, u, cudaMemcpyHostToDevice))) return fail(rc);
  if ((rc = scatter_raw(s))) return fail(rc);
  if (cudaEventRecord(s->ev[0], s->stream) != cudaSuccess) return fail(OSQP_ERR_CUDA);
  if ((rc = do_scale(s, 1))) return fail(rc);
  if (cudaEventRecord(s->ev[1], s->stream) != cudaSuccess) return fail(OSQP_ERR_CUDA);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(OSQP_ERR_CUDA);
  if ((rc = check_device_error(s))) return fail(rc);
  s->info.setup_time = elapsed_s(s->ev[0], s->ev[1]);
  s->info.launch = s->use_cluster ? 3 : (s->use_grid ? 2 : 1);
  *out = s;
  return OSQP_OK;
}

int32_t osqp_solve_async(osqp_solver* s) {
  if (!s) return OSQP_ERR_ARG;
  CK(cudaEventRecord(s->ev[2], s->stream));
  int rc = do_admm(s);
  if (rc) return rc;
  CK(cudaEventRecord(s->ev[3], s->stream));
  s->solved = true;
  return OSQP_OK;
}

static int32_t refresh_info(osqp_solver* s) {
  Scalars sc;
  int rc;
  if ((rc = read_scalars(s, &sc))) return rc;
  if ((rc = check_device_error(s))) return rc;
  s->info.status = sc.status;
  s->info.iter = sc.iter;
  s->info.pcg_iters = sc.pcg_iters;
  s->info.rho_updates = sc.rho_updates;
  s->info.ruiz_passes = sc.ruiz_passes;
  s->info.obj_val = sc.obj;
  s->info.prim_res = sc.prim_res;
  s->info.dual_res = sc.dual_res;
  s->info.polished = sc.polished;
  s->info.rho_estimate = sc.rho_bar;
  s->info.solve_time = s->solved ? elapsed_s(s->ev[2], s->ev[3]) : 0.0;
  s->rho_bar = sc.rho_bar;
  return OSQP_OK;
}

int32_t osqp_solve(osqp_solver* s) {
  if (!s) return OSQP_ERR_ARG;
  int rc = osqp_solve_async(s);
  if (rc) return rc;
  return refresh_info(s);
}

int32_t osqp_update_vectors(osqp_solver* s, const double* q, const double* l, const double* u) {
  if (!s) return OSQP_ERR_ARG;
  if (q && !finite_all(q, s->n)) return OSQP_ERR_NONFINITE;
  // Check l ≤ u against the stored value of whichever side is not replaced.
  if (l || u) {
    std::vector<double> lh(s->m), uh(s->m);
    double *kn_raw, *a_raw, *qd, *ld, *ud;
    get_raw(s, &kn_raw, &a_raw, &qd, &ld, &ud);
    if (!l && s->m) CK(cudaMemcpyAsync(lh.data(), ld, sizeof(double) * s->m, cudaMemcpyDeviceToHost, s->stream));
    if (!u && s->m) CK(cudaMemcpyAsync(uh.data(), ud, sizeof(double) * s->m, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    const double* L = l ? l : lh.data();
    const double* U = u ? u : uh.data();
    for (int i = 0; i < s->m; ++i) {
      if (std::isnan(L[i]) || std::isnan(U[i])) return OSQP_ERR_NONFINITE;
      if (L[i] > U[i]) return OSQP_ERR_LGTU;
    }
  }
  int rc = upload_vectors(s, q, l, u, cudaMemcpyHostToDevice);
  if (rc) return rc;
  if ((rc = do_refresh(s))) return rc;
  CK(cudaStreamSynchronize(s->stream));
  return check_device_error(s);
}

int32_t osqp_update_matrices(osqp_solver* s, const double* Pv, const double* Av) {
  if (!s) return OSQP_ERR_ARG;
  if (Pv && !finite_all(Pv, s->nnzP)) return OSQP_ERR_NONFINITE;
  if (Av && !finite_all(Av, s->nnzA)) return OSQP_ERR_NONFINITE;
  if (Pv && s->nnzP)
    CK(cudaMemcpyAsync(s->raw_in, Pv, sizeof(double) * s->nnzP, cudaMemcpyHostToDevice, s->stream));
  if (Av && s->nnzA)
    CK(cudaMemcpyAsync(s->raw_in + s->nnzP, Av, sizeof(double) * s->nnzA, cudaMemcpyHostToDevice,
                       s->stream));
  int rc = scatter_raw(s);
  if (rc) return rc;
  CK(cudaEventRecord(s->ev[0], s->stream));
  if ((rc = do_scale(s, 0))) return rc;
  CK(cudaEventRecord(s->ev[1], s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->info.setup_time = elapsed_s(s->ev[0], s->ev[1]);
  return check_device_error(s);
}

static int32_t load_data(osqp_solver* s, const double* Pv, const double* q, const double* Av,
                         const double* l, const double* u, cudaMemcpyKind kind) {
  if (!s || !q || (s->nnzP && !Pv) || (s->nnzA && !Av) || (s->m && (!l || !u)))
    return OSQP_ERR_ARG;
  if (s->nnzP) CK(cudaMemcpyAsync(s->raw_in, Pv, sizeof(double) * s->nnzP, kind, s->stream));
  if (s->nnzA)
    CK(cudaMemcpyAsync(s->raw_in + s->nnzP, Av, sizeof(double) * s->nnzA, kind, s->stream));
  int rc = upload_vectors(s, q, l, u, kind);
  if (rc) return rc;
  if ((rc = scatter_raw(s))) return rc;
  s->rho_bar = s->set.rho;
  return do_scale(s, 1);
}

int32_t osqp_load_data(osqp_solver* s, const double* Pv, const double* q, const double* Av,
                       const double* l, const double* u) {
  return load_data(s, Pv, q, Av, l, u, cudaMemcpyHostToDevice);
}

int32_t osqp_load_data_device(osqp_solver* s, const double* Pv, const double* q, const double* Av,
                              const double* l, const double* u) {
  return load_data(s, Pv, q, Av, l, u, cudaMemcpyDeviceToDevice);
}

int32_t osqp_update_rho(osqp_solver* s, double rho_bar) {
  if (!s) return OSQP_ERR_ARG;
  if (!(rho_bar > 0) || !std::isfinite(rho_bar)) return OSQP_ERR_SETTINGS;
  s->rho_bar = rho_bar;
  int rc = do_refresh(s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s->stream));
  return check_device_error(s);
}

int32_t osqp_warm_start(osqp_solver* s, const double* x, const double* y) {
  if (!s) return OSQP_ERR_ARG;
  if (x && !finite_all(x, s->n)) return OSQP_ERR_NONFINITE;
  if (y && !finite_all(y, s->m)) return OSQP_ERR_NONFINITE;
  if (x) CK(cudaMemcpyAsync(s->x_ws, x, sizeof(double) * s->n, cudaMemcpyHostToDevice, s->stream));
  if (y && s->m)
    CK(cudaMemcpyAsync(s->y_ws, y, sizeof(double) * s->m, cudaMemcpyHostToDevice, s->stream));
  int rc = do_warm(s, x ? s->x_ws : nullptr, y ? s->y_ws : nullptr);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s->stream));
  return OSQP_OK;
}

int32_t osqp_get_solution(osqp_solver* s, double* x, double* y, double* z, osqp_info* info) {
  if (!s) return OSQP_ERR_ARG;
  if (x) CK(cudaMemcpyAsync(x, out_x(s), sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
  if (y && s->m)
    CK(cudaMemcpyAsync(y, out_y(s), sizeof(double) * s->m, cudaMemcpyDeviceToHost, s->stream));
  if (z && s->m)
    CK(cudaMemcpyAsync(z, out_z(s), sizeof(double) * s->m, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (info) {
    int rc = refresh_info(s);
    if (rc) return rc;
    *info = s->info;
  }
  return OSQP_OK;
}

int32_t osqp_get_solution_device(osqp_solver* s, double* x, double* y) {
  if (!s) return OSQP_ERR_ARG;
  if (x) CK(cudaMemcpyAsync(x, out_x(s), sizeof(double) * s->n, cudaMemcpyDeviceToDevice, s->stream));
  if (y && s->m)
    CK(cudaMemcpyAsync(y, out_y(s), sizeof(double) * s->m, cudaMemcpyDeviceToDevice, s->stream));
  return OSQP_OK;
}

int32_t osqp_get_certificate(osqp_solver* s, double* py, double* dx) {
  if (!s) return OSQP_ERR_ARG;
  if (py && s->m)
    CK(cudaMemcpyAsync(py, out_pc(s), sizeof(double) * s->m, cudaMemcpyDeviceToHost, s->stream));
  if (dx) CK(cudaMemcpyAsync(dx, out_dc(s), sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return OSQP_OK;
}

int32_t osqp_diag_scaling(osqp_solver* s, double* D, double* E, double* c, double* jacobi) {
  if (!s) return OSQP_ERR_ARG;
  const bool f64 = s->set.precision == OSQP_PRECISION_FP64;
  const double* Dd = f64 ? s->d64.D : s->d32.D;
  const double* Ed = f64 ? s->d64.E : s->d32.E;
  const double* gd = f64 ? s->d64.dg : s->d32.dg;
  if (D) CK(cudaMemcpyAsync(D, Dd, sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
  if (E && s->m)
    CK(cudaMemcpyAsync(E, Ed, sizeof(double) * s->m, cudaMemcpyDeviceToHost, s->stream));
  if (jacobi)
    CK(cudaMemcpyAsync(jacobi, gd, sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
  if (c) CK(cudaMemcpyAsync(c, &s->sc->c, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return OSQP_OK;
}

int32_t osqp_diag_schedule(osqp_solver* s, int32_t* groups, double* ms) {
  if (!s || !groups) return OSQP_ERR_ARG;
  groups[0] = s->kn_s.group;
  groups[1] = s->a_s.group;
  groups[2] = s->tuned_kn < 0 || s->tuned_a < 0 ? -1 : (s->tuned_kn > 0 || s->tuned_a > 0 ? 1 : 0);
  if (ms) {
    for (int k = 0; k < 6; ++k) {
      ms[k] = s->tune_kn_ms[k];
      ms[6 + k] = s->tune_a_ms[k];
    }
  }
  return OSQP_OK;
}

int32_t osqp_diag_barrier_timeout(double timeout_s) {
  if (!(timeout_s > 0.0) || !(timeout_s <= 10.0)) return OSQP_ERR_ARG;
  constexpr int kBlocks = 4;
  char* mem = nullptr;
  const size_t bytes = 256 + 256 + sizeof(double) * 2 * kBlocks * kMaxRed;
  if (cudaMalloc((void**)&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return OSQP_ERR_CUDA;
  }
  Barrier* bar = (Barrier*)mem;
  int* err = (int*)(mem + 256);
  double* part = (double*)(mem + 512);
  int rc = OSQP_OK;
  if (cudaMemset(mem, 0, 512) != cudaSuccess) rc = OSQP_ERR_CUDA;
  unsigned long long tns = (unsigned long long)(timeout_s * 1e9);
  int absent = 1;
  void* args[] = {&bar, &err, &part, &tns, &absent};
  if (rc == OSQP_OK &&
      cudaLaunchCooperativeKernel((const void*)k_barrier_probe, dim3(kBlocks), dim3(kThreads), args,
                                  0, (cudaStream_t)0) != cudaSuccess)
    rc = OSQP_ERR_CUDA;
  if (rc == OSQP_OK && cudaDeviceSynchronize() != cudaSuccess) rc = OSQP_ERR_CUDA;
  int e = 0;
  if (rc == OSQP_OK && cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = OSQP_ERR_CUDA;
  if (rc == OSQP_OK && e != kDevBarrierTimeout) rc = OSQP_ERR_DEVICE;
  cudaGetLastError();
  cudaFree(mem);
  return rc;
}

int32_t osqp_diag_sliced_layout(int32_t nrows, const int32_t* rowptr, int64_t nwarps,
                                int32_t* pos, int32_t* chunks, int32_t* stats) {
  if (nrows < 0 || !rowptr || nwarps < 1 || !stats) return OSQP_ERR_ARG;
  if (rowptr[0] != 0) return OSQP_ERR_CSC;
  for (int32_t r = 0; r < nrows; ++r)
    if (rowptr[r + 1] < rowptr[r]) return OSQP_ERR_CSC;
  const std::vector<int> rp(rowptr, rowptr + nrows + 1);
  const host::SchedHost S = host::make_sched(rp, nwarps);
  stats[0] = S.group;
  stats[1] = S.long_thresh;
  stats[2] = (int32_t)S.slices.size();
  stats[3] = S.npos;
  stats[4] = (int32_t)S.long_rows.size();
  stats[5] = (int32_t)S.chunks.size();
  if (pos) std::copy(S.pos.begin(), S.pos.end(), pos);
  if (chunks)
    for (size_t c = 0; c < S.chunks.size(); ++c) {
      chunks[4 * c + 0] = S.chunks[c].x;
      chunks[4 * c + 1] = S.chunks[c].y;
      chunks[4 * c + 2] = S.chunks[c].z;
      chunks[4 * c + 3] = S.lrange[S.chunks[c].w].x == (int)c ? 1 : 0;
    }
  return OSQP_OK;
}

int32_t osqp_cleanup(osqp_solver* s) {
  if (!s) return OSQP_ERR_ARG;
  int rc = OSQP_OK;
  if (s->stream || s->arena) {
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) rc = OSQP_ERR_CUDA;
  }
  if (s->arena && cudaFree(s->arena) != cudaSuccess) rc = OSQP_ERR_CUDA;
  for (auto& ev : s->ev)
    if (ev) cudaEventDestroy(ev);
  delete s;
  return rc;
}

}  // extern "C"
