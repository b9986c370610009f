// Device code of the OSQP ADMM hot path for sm_103a.
//
// One implementation of every stage, templated on a "team" that executes it:
//   GridTeam    — all CTAs of a cooperative launch, one persistent CTA per SM
//                 slot, synchronised by a bounded grid barrier;
//   ClusterTeam — the CTAs of one thread-block cluster, synchronised through
//                 distributed shared memory (heavy problems of a batch,
//                 large serving requests, launch = 3);
//   BlockTeam   — one CTA (small problems and the batched kernel, where every
//                 CTA owns one problem at a time);
//   PlainTeam   — an ordinary launch without barriers (warm start).
// Stages are separated by team-wide barriers; reductions are published by
// each CTA and combined after the next barrier in a fixed order, so every
// thread of every CTA derives bit-identical scalars (α, β, residual norms,
// termination decisions) without a second barrier or a host round trip.
//
// Matrices: Kn = [P̄ Āᵀ] (n rows; column c < n addresses P̄, column n + i
// addresses Āᵀ) and Ā (m rows), each in the sliced layout described at
// Sched: short rows in coalesced 32-lane slices sorted by length, rows
// longer than `long_thresh` in 256-nonzero chunks that whole warps reduce;
// the chunk partials of a long row are summed in chunk order by whichever
// warp stores the row's last partial, so every product is deterministic.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include "dfloat.cuh"  // double-float arithmetic of the FP32-mixed CG scalars

namespace osqpgb {

constexpr int kThreads = 512;   // threads per CTA of every team kernel
constexpr int kMaxRed = 32;     // reduction slots
constexpr int kMaxSumSlots = 4; // sum slots staged through shared memory per reduction
// Shared memory of every team kernel: reduction partials and results
// (34·kMaxRed), the sum-slot staging area, and the scalars of the PCG
// recurrence that one warp updates for the whole CTA (kScalSlots).  In the
// FP32-mixed mode five more slots hold the results of the last
// working-precision reduction as unevaluated sums of two floats (kScalMirror,
// one (high, low) pair per result, four results) and the PCG tolerance
// (kScalTolF), from which every thread runs the CG scalar recurrence itself.
constexpr int kScalMirror = 8;
constexpr int kScalTolF = 12;
constexpr int kScalSlots = 13;
constexpr int kScalOff = 34 * kMaxRed + kMaxSumSlots * kThreads;
constexpr int kSmemDoubles = kScalOff + kScalSlots;
constexpr int kChunk = 256;     // nonzeros per long-row chunk
constexpr int kMaxNV = 4;       // partial values stored per long-row chunk

constexpr uint8_t kLInf = 1, kUInf = 2, kEq = 4;  // row-type bits
constexpr double kInfBound = 1e20;
constexpr double kNormMin = 1e-4, kNormMax = 1e4;  // Ruiz norm clamp
constexpr double kRhoMin = 1e-6, kRhoMax = 1e6;    // ρ̄ clamp of the adaptive rule
constexpr double kEqRhoFactor = 1e3;               // ρ_i = 10³ρ̄ on equality rows
constexpr double kTiny = 1e-30;

enum DevStatus : int { kUnsolved = 0, kSolved = 1, kMaxIter = 2, kPrimInf = 3, kDualInf = 4,
                       kTimeLimit = 5, kNumErr = 6 };
enum DevError : int { kDevOk = 0, kDevBarrierTimeout = 1 };

// Sliced layout of a sparse matrix (rows of Kn = [P̄ Āᵀ] or of Ā).  Rows of
// at most long_thresh nonzeros, stably sorted by decreasing length, form
// slices of 32/group rows; a row's nonzeros are dealt to `group` lanes, and
// step t of a slice stores one nonzero per lane at first + 32·t + lane, so
// every warp load of column indices or values is one coalesced 128-byte
// line.  Padding positions hold column −1.  Longer rows follow in CSR order
// and are split into kChunk-nonzero chunks, each taken by a whole warp; a
// chunk stores its partial result in cpart and counts itself in the row's
// ccount, and the warp whose count completes the row sums the row's
// partials in chunk order (a fixed order, whoever arrives last).
struct Sched {
  int nrows, group, long_thresh, nchunks, nlong, nslices;
  const int2* slices;   // (first position, steps)
  const int* srow;      // row of local row r of slice s at s·(32/group) + r; −1 = none
  const int4* chunks;   // (row, begin, end, long-row index) in positions
  const int* long_rows;
  const int2* lrange;   // per long row: (first chunk, number of chunks)
  const int* lidx;      // per row: its long-row index, −1 for a short row
  double* cpart;        // per chunk: kMaxNV partial values of the current product
  unsigned* ccount;     // per long row: chunks stored in the current product
                        // (zero between products: the completing warp resets it)
  int npos;             // positions of the layout (nonzeros and padding)
};

struct Barrier {
  unsigned int count, gen;
};

// Per-problem scalars shared between launches (global memory).
struct Scalars {
  double c, rho_bar;
  double obj, prim_res, dual_res;
  int status, iter, pcg_iters, rho_updates, ruiz_passes, checks;
  int dev_error, pad;
  // scaled primal/dual residuals of the last termination check; a solve that
  // continues from the current iterates takes its first PCG tolerance from
  // them (0: no check since the iterates were last reset)
  double rp_last, rd_last;
  int polished, pad2;  // 1 polished, -1 rejected, 0 not run (§4)
};

struct Params {
  double sigma, alpha, eps_abs, eps_rel, eps_pinf, eps_dinf, rho_tol, eps_equil;
  double pcg_kappa, pcg_floor, pcg_reduce, time_limit_ns;
  int max_iter, check_interval, adaptive_rho, scaling_iters, max_rho_updates, pcg_max_iter;
  unsigned long long barrier_timeout_ns;
  int polish, polish_refine;  // §4 solution polishing
  double delta;
};

template <typename T>
struct Dev {
  int n, m;
  const int* kn_ci;
  T* kn_v;
  const double* kn_raw;
  Sched kn;
  const int* a_ci;
  T* a_v;
  const double* a_raw;
  Sched as;
  const double *q_raw, *l_raw, *u_raw;
  uint8_t* rtype;
  double *D, *E, *Dinv, *Einv, *q, *l, *u, *rho, *rho_inv, *pdiag, *dg, *nrm_n, *nrm_m;
  T* dinv;
  double *x, *z, *y, *dx, *dy;
  double *xt, *zt, *wm, *um;  // x̃, z̃ and the RHS inputs stay FP64 in both modes
  // PCG vectors (working precision): b, p; r, s = Kp and w = Ku
  // double-buffered; u = M⁻¹r and t = RĀu double-buffered as one array
  // [u | t] of n + m values each (ut0, ut1), so that a product with
  // Kn = [P̄ Āᵀ] gathers both from one base; ap = Āp (for z̃ = Āx̃)
  T *b, *p, *r0, *r1, *s0, *s1, *w0, *w1;
  T *ut0, *ut1, *ap;
  // PCG corrections of x̃ and z̃ in working precision, folded into the FP64
  // x̃, z̃ once per ADMM iteration; working-precision copies of ρ and ρ⁻¹
  T *dxt, *dzt, *rhoT, *rho_invT;
  double *px, *aty, *pdx, *atdy, *ax, *adx, *azt;
  // solution polishing (§4): n-vectors x, r, M⁻¹r, p, Kp, Jacobi diagonal;
  // m-vectors y, Āp/δ (or the refinement's Ā-side terms), r₂; row states
  double *pol_x, *pol_dx, *pol_r, *pol_z, *pol_p, *pol_kp, *pol_dg;
  double *pol_y, *pol_t, *pol_r2;
  uint8_t* pol_act;
  double *x_out, *y_out, *z_out, *pcert, *dcert;
  Scalars* sc;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <bool MAX>
__device__ __forceinline__ double rop(double a, double b) {
  return MAX ? fmax(a, b) : a + b;
}

__device__ __forceinline__ double red_identity(unsigned maxmask, int k) {
  return ((maxmask >> k) & 1u) ? -INFINITY : 0.0;
}

// Order-preserving 64-bit key of a double: max reductions run on integers,
// off the narrow FP64 pipe.  NaN keys above +∞, so a NaN propagates.
__device__ __forceinline__ unsigned long long dkey(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dunkey(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// Block-wide reduction of K slots; slot k is a max when bit k of MAXMASK is
// set, else a sum.  Max slots: integer keys combined by warp shuffles.  Sum
// slots (at most kMaxSumSlots): every thread stages its value in shared
// memory and one warp per slot adds the column (16 values per lane, then a
// 5-level shuffle tree), about a quarter of the FP64 instructions of a
// per-warp shuffle tree.  Result left in sm[32*kMaxRed + k].  All threads
// call it.
template <int K, unsigned MAXMASK>
__device__ __forceinline__ void block_reduce(const double (&v)[K], double* sm) {
  static_assert(K <= kMaxRed, "too many reduction slots");
  constexpr int S = K - __builtin_popcount(MAXMASK & ((1u << K) - 1u));
  static_assert(S <= kMaxSumSlots, "too many sum slots");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long* smk = reinterpret_cast<unsigned long long*>(sm);
  double* stage = sm + 34 * kMaxRed;
  int sidx = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if ((MAXMASK >> k) & 1u) {
      unsigned long long x = dkey(v[k]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x = umax64(x, __shfl_xor_sync(0xffffffffu, x, off));
      if (lane == 0) smk[wid * kMaxRed + k] = x;
    } else {
      stage[sidx * blockDim.x + threadIdx.x] = v[k];
      ++sidx;
    }
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if ((MAXMASK >> k) & 1u) {
        unsigned long long x = lane < nw ? smk[lane * kMaxRed + k] : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x = umax64(x, __shfl_xor_sync(0xffffffffu, x, off));
        if (lane == 0) sm[32 * kMaxRed + k] = dunkey(x);
      }
    }
  }
  // sum slot j is reduced by warp j (slot k is the j-th sum slot)
  if (S > 0 && wid < S) {
    int kk = -1, j = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (!((MAXMASK >> k) & 1u)) {
        if (j == wid) kk = k;
        ++j;
      }
    const double* col = stage + wid * blockDim.x;
    double t[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) t[u] = lane + 32 * u < (int)blockDim.x ? col[lane + 32 * u] : 0.0;
#pragma unroll
    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
      for (int u = 0; u < w; ++u) t[u] += t[u + w];
    double x = t[0];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) sm[32 * kMaxRed + kk] = x;
  }
  __syncthreads();
}

// Order-preserving 32-bit key of a float (NaN above +∞).
__device__ __forceinline__ unsigned fkey(float v) {
  const unsigned b = __float_as_uint(v);
  return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float funkey(unsigned k) {
  return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k);
}

// result k of the last reduction as a double-float pair at kScalMirror
__device__ __forceinline__ void mirror_store(double* sm, int k, ff v) {
  float* m = reinterpret_cast<float*>(sm + kScalOff + kScalMirror);
  m[2 * k] = v.h;
  m[2 * k + 1] = v.l;
}

// One level of a warp's shuffle tree over (sum, error) pairs of FP32 terms:
// the partner's pair is added by Knuth's TwoSum, whose rounding error joins
// the error term.
__device__ __forceinline__ void two_sum_level(float& hi, float& lo, int off) {
  const float b = __shfl_xor_sync(0xffffffffu, hi, off);
  const float bl = __shfl_xor_sync(0xffffffffu, lo, off);
  const float s = __fadd_rn(hi, b);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(bl, err));
}

// Block-wide reduction of K working-precision (FP32) slots with the result
// in FP64, for the FP32-mixed mode: each warp sums its lanes' values by a
// shuffle tree of error-free FP32 additions (Knuth's TwoSum, the rounding
// errors carried in a second FP32 term) and stores the (sum, error) pair;
// one warp per slot then converts the warps' pairs to FP64 and adds them,
// so the narrow FP64 pipe sees one instruction per slot rather than one per
// warp.  Max slots combine order-preserving keys.  Result in
// sm[32*kMaxRed + k], as block_reduce, and as a double-float pair at
// kScalMirror.
// With DBL false only the double-float result is formed, without FP64
// instructions: the warps' pairs are combined by the same TwoSum tree.  All
// threads call it.
template <int K, unsigned MAXMASK, bool DBL = true>
__device__ __forceinline__ void block_reduce(const float (&v)[K], double* sm) {
  static_assert(K <= kMaxSumSlots, "too many slots");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float2* pw = reinterpret_cast<float2*>(sm);  // [warp · kMaxRed + slot]
  float* mirror = reinterpret_cast<float*>(sm + kScalOff + kScalMirror);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if ((MAXMASK >> k) & 1u) {
      unsigned x = fkey(v[k]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned o = __shfl_xor_sync(0xffffffffu, x, off);
        x = x > o ? x : o;
      }
      if (lane == 0) pw[wid * kMaxRed + k] = make_float2(funkey(x), 0.0f);
    } else {
      float hi = v[k], lo = 0.0f;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) two_sum_level(hi, lo, off);
      if (lane == 0) pw[wid * kMaxRed + k] = make_float2(hi, lo);
    }
  }
  __syncthreads();
  if (wid < K) {
    const int k = wid;
    const bool mx = (MAXMASK >> k) & 1u;
    const float2 e = lane < nw ? pw[lane * kMaxRed + k] : make_float2(mx ? -INFINITY : 0.0f, 0.0f);
    if (mx) {
      unsigned x = fkey(e.x);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned o = __shfl_xor_sync(0xffffffffu, x, off);
        x = x > o ? x : o;
      }
      if (lane == 0) {
        const float f = funkey(x);
        if (DBL) sm[32 * kMaxRed + k] = (double)f;
        mirror[2 * k] = f;
        mirror[2 * k + 1] = 0.0f;
      }
    } else if (DBL) {
      double x = (double)e.x + (double)e.y;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      if (lane == 0) {
        sm[32 * kMaxRed + k] = x;
        const ff f = ff_of(x);
        mirror[2 * k] = f.h;
        mirror[2 * k + 1] = f.l;
      }
    } else {
      // FP32 result only: the warps' pairs combined by the same TwoSum tree
      float hi = e.x, lo = e.y;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) two_sum_level(hi, lo, off);
      if (lane == 0) {
        const ff f = ff_two_sum(hi, lo);
        mirror[2 * k] = f.h;
        mirror[2 * k + 1] = f.l;
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Teams
// ---------------------------------------------------------------------------
struct GridTeam {
  static constexpr bool kCtaScope = false;  // products span CTAs
  Barrier* bar;
  int* err;
  double* part;  // [2][gridDim.x][kMaxRed]
  double* sm;
  unsigned long long timeout_ns;
  int buf;
  unsigned int target;  // barrier count × gridDim.x reached so far (thread 0)

  __device__ int nthreads() const { return gridDim.x * blockDim.x; }
  __device__ int tid() const { return blockIdx.x * blockDim.x + threadIdx.x; }
  __device__ int nwarps() const { return gridDim.x * (blockDim.x >> 5); }
  __device__ int warp() const { return blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); }
  __device__ bool leader() const { return blockIdx.x == 0 && threadIdx.x == 0; }

  // Grid barrier with a bounded wait.  The arrival counter only grows
  // during a launch (the host zeroes it before every launch), so barrier
  // number k is complete once it reaches k·gridDim.x.  Thread 0 arrives with
  // an acquire-release atomic and spins with acquire loads, so the CTA's
  // writes before the barrier are visible to every CTA after it.  A CTA that
  // waits longer than timeout_ns records kDevBarrierTimeout and adds
  // kBarrierPoison to the counter, which releases every waiter at once; a
  // counter at or above kBarrierPoison makes every CTA stop at its barrier.
  static constexpr unsigned int kBarrierPoison = 0x80000000u;
  __device__ bool sync() {
    __syncthreads();
    int* flag = reinterpret_cast<int*>(sm + 34 * kMaxRed - 1);
    if (threadIdx.x == 0) {
      target += gridDim.x;
      unsigned int c;
      asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(c) : "l"(&bar->count) : "memory");
      c += 1u;
      if (c < target) {
        const unsigned long long t0 = gtimer();
        unsigned int spins = 0;
        for (;;) {
          asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(c) : "l"(&bar->count) : "memory");
          if (c >= target) break;
          if ((++spins & 255u) == 0 && gtimer() - t0 > timeout_ns) {
            atomicExch(err, kDevBarrierTimeout);
            atomicAdd(&bar->count, kBarrierPoison);
            c = kBarrierPoison;
            break;
          }
        }
      }
      *flag = c < kBarrierPoison ? 1 : 0;
    }
    __syncthreads();
    return *flag != 0;
  }

  // publish, then a team barrier (DBL is ignored: the CTAs' partials are
  // combined in FP64)
  template <int K, unsigned MAXMASK, bool DBL = true, typename V>
  __device__ bool publish_sync(const V (&v)[K]) {
    publish<K, MAXMASK>(v);
    return sync();
  }

  template <int K, unsigned MAXMASK, typename V>
  __device__ void publish(const V (&v)[K]) {
    block_reduce<K, MAXMASK>(v, sm);
    if (threadIdx.x < K)
      part[((size_t)buf * gridDim.x + blockIdx.x) * kMaxRed + threadIdx.x] =
          sm[32 * kMaxRed + threadIdx.x];
  }

  // Combine the partials of the last publish (after a sync).  Every CTA runs
  // the same fixed-order combination, so all threads see identical values.
  // Each lane issues all of its (≤ 16) partial loads before combining them.
  // MIRROR: also leave the results as double-float pairs at kScalMirror.
  template <int K, unsigned MAXMASK, bool MIRROR = false>
  __device__ void collect(double (&out)[K]) {
    static_assert(!MIRROR || K <= 4, "four mirrored results at most");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nb = gridDim.x;
    for (int k = wid; k < K; k += nw) {
      const bool mx = (MAXMASK >> k) & 1u;
      const double* src = part + (size_t)buf * nb * kMaxRed + k;
      // the ⌈nb/32⌉ partials of a lane, loaded together, then combined in
      // lane order (no FP64 work on absent partials)
      const int per = (nb + 31) >> 5;
      double y[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int b = lane + 32 * u;
        y[u] = (u < per && b < nb) ? __ldcg(src + (size_t)b * kMaxRed) : (mx ? -INFINITY : 0.0);
      }
      if (mx) {
        unsigned long long x = dkey(y[0]);
#pragma unroll
        for (int u = 1; u < 16; ++u)
          if (u < per) x = umax64(x, dkey(y[u]));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x = umax64(x, __shfl_xor_sync(0xffffffffu, x, off));
        if (lane == 0) {
          sm[33 * kMaxRed + k] = dunkey(x);
          if (MIRROR) mirror_store(sm, k, ff{(float)dunkey(x), 0.0f});
        }
      } else {
        double x = y[0];
#pragma unroll
        for (int u = 1; u < 16; ++u)
          if (u < per) x += y[u];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) {
          sm[33 * kMaxRed + k] = x;
          if (MIRROR) mirror_store(sm, k, ff_of(x));
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = sm[33 * kMaxRed + k];
    buf ^= 1;
  }
};

// Generic address of `p` (a shared variable of this CTA) in CTA `rank` of
// the thread-block cluster (distributed shared memory).
template <typename V>
__device__ __forceinline__ V* cluster_map(V* p, unsigned rank) {
  unsigned long long out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(p), "r"(rank));
  return reinterpret_cast<V*>(out);
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// Hardware barrier over every thread of the cluster.  Used only where all
// CTAs reach it unconditionally (kernel entry and exit).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

// One thread-block cluster as a team (a problem too large for one SM and
// too small to pay for whole-GPU barriers).  The barrier is a counter in
// the shared memory of CTA 0 of the cluster, reached through distributed
// shared memory: thread 0 of each CTA arrives with an acquire-release atomic
// and spins with acquire loads, bounded by timeout_ns exactly like the grid
// barrier (timeout → kDevBarrierTimeout and a poison add that releases every
// waiter).  Reductions: each CTA reduces its block into its own shared
// memory (double-buffered), and after the barrier every CTA combines the
// cluster's partials in rank order, so all CTAs hold identical values.
struct ClusterTeam {
  static constexpr bool kCtaScope = false;
  static constexpr unsigned int kBarrierPoison = 0x80000000u;
  double* sm;
  double* cpart;  // [2][kMaxRed] this CTA's published block results
  unsigned* ctr;  // barrier counter (CTA 0's is the one used)
  int* err;
  unsigned long long timeout_ns;
  unsigned rank, csize, target;
  int buf;

  __device__ int nthreads() const { return (int)csize * blockDim.x; }
  __device__ int tid() const { return (int)rank * blockDim.x + threadIdx.x; }
  __device__ int nwarps() const { return (int)csize * (blockDim.x >> 5); }
  __device__ int warp() const { return (int)rank * (blockDim.x >> 5) + (threadIdx.x >> 5); }
  __device__ bool leader() const { return rank == 0 && threadIdx.x == 0; }

  __device__ bool sync() {
    __syncthreads();
    int* flag = reinterpret_cast<int*>(sm + 34 * kMaxRed - 1);
    if (threadIdx.x == 0) {
      target += csize;
      unsigned* c0 = cluster_map(ctr, 0u);
      unsigned c;
      asm volatile("atom.acq_rel.gpu.add.u32 %0, [%1], 1;" : "=r"(c) : "l"(c0) : "memory");
      c += 1u;
      if (c < target) {
        const unsigned long long t0 = gtimer();
        unsigned int spins = 0;
        for (;;) {
          asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(c) : "l"(c0) : "memory");
          if (c >= target) break;
          if ((++spins & 255u) == 0 && gtimer() - t0 > timeout_ns) {
            atomicExch(err, kDevBarrierTimeout);
            atomicAdd(c0, kBarrierPoison);
            c = kBarrierPoison;
            break;
          }
        }
      }
      *flag = c < kBarrierPoison ? 1 : 0;
    }
    __syncthreads();
    return *flag != 0;
  }

  // publish, then a team barrier (DBL is ignored: the CTAs' partials are
  // combined in FP64)
  template <int K, unsigned MAXMASK, bool DBL = true, typename V>
  __device__ bool publish_sync(const V (&v)[K]) {
    publish<K, MAXMASK>(v);
    return sync();
  }

  template <int K, unsigned MAXMASK, typename V>
  __device__ void publish(const V (&v)[K]) {
    block_reduce<K, MAXMASK>(v, sm);
    if (threadIdx.x < K) cpart[buf * kMaxRed + threadIdx.x] = sm[32 * kMaxRed + threadIdx.x];
  }

  // Combine the partials of the last publish (after a sync), in rank order.
  // MIRROR: also leave the results as double-float pairs at kScalMirror.
  template <int K, unsigned MAXMASK, bool MIRROR = false>
  __device__ void collect(double (&out)[K]) {
    static_assert(!MIRROR || K <= 4, "four mirrored results at most");
    if (threadIdx.x < K) {
      const int k = threadIdx.x;
      const bool mx = (MAXMASK >> k) & 1u;
      double y[16];
#pragma unroll
      for (int r = 0; r < 16; ++r)
        y[r] = r < (int)csize ? *cluster_map(cpart + buf * kMaxRed + k, (unsigned)r) : 0.0;
      if (mx) {
        unsigned long long x = dkey(y[0]);
#pragma unroll
        for (int r = 1; r < 16; ++r)
          if (r < (int)csize) x = umax64(x, dkey(y[r]));
        sm[33 * kMaxRed + k] = dunkey(x);
        if (MIRROR) mirror_store(sm, k, ff{(float)dunkey(x), 0.0f});
      } else {
        double x = y[0];
#pragma unroll
        for (int r = 1; r < 16; ++r)
          if (r < (int)csize) x += y[r];
        sm[33 * kMaxRed + k] = x;
        if (MIRROR) mirror_store(sm, k, ff_of(x));
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = sm[33 * kMaxRed + k];
    buf ^= 1;
  }
};

struct BlockTeam {
  static constexpr bool kCtaScope = true;  // every warp of a product is in this CTA
  double* sm;
  __device__ int nthreads() const { return blockDim.x; }
  __device__ int tid() const { return threadIdx.x; }
  __device__ int nwarps() const { return blockDim.x >> 5; }
  __device__ int warp() const { return threadIdx.x >> 5; }
  __device__ bool leader() const { return threadIdx.x == 0; }
  __device__ bool sync() {
    __syncthreads();
    return true;
  }
  template <int K, unsigned MAXMASK, typename V>
  __device__ void publish(const V (&v)[K]) {
    block_reduce<K, MAXMASK>(v, sm);
  }
  // publish, then a team barrier: block_reduce already ends with a CTA
  // barrier, which orders every write made before it.  DBL false (FP32
  // values only): the caller reads only the double-float results at
  // kScalMirror.
  template <int K, unsigned MAXMASK, bool DBL = true, typename V>
  __device__ bool publish_sync(const V (&v)[K]) {
    if constexpr (sizeof(V) == sizeof(float))
      block_reduce<K, MAXMASK, DBL>(v, sm);
    else
      block_reduce<K, MAXMASK>(v, sm);
    return true;
  }
  // the FP32 copies (MIRROR) are left by the FP32 block_reduce itself
  template <int K, unsigned MAXMASK, bool MIRROR = false>
  __device__ void collect(double (&out)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = sm[32 * kMaxRed + k];
  }
};

// A plain (non-cooperative) launch as a traversal team: no barriers.
struct PlainTeam {
  static constexpr bool kCtaScope = false;
  __device__ int nthreads() const { return gridDim.x * blockDim.x; }
  __device__ int tid() const { return blockIdx.x * blockDim.x + threadIdx.x; }
  __device__ int nwarps() const { return gridDim.x * (blockDim.x >> 5); }
  __device__ int warp() const { return blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); }
};

// ---------------------------------------------------------------------------
// Traversal of the sliced layout.  gather(col, val, acc) folds one nonzero
// into the NV accumulators; the group then combines its lanes (sum, or max
// when MAXR) and on_row(row, acc) runs once per short row.  A long row is
// reduced chunk by chunk: on_chunk(row, first, acc) runs once per chunk with
// that chunk's partial (for inner products that take the row piecewise), and
// on_long(row, acc) once per long row with the sum of its partials in chunk
// order.  A lane accumulates its nonzeros of a row in order and the group
// combines them by a fixed shuffle tree, so a row's result does not depend on
// where its slice sits, and a long row's result not on which warp finished it.
// ---------------------------------------------------------------------------
// Arrival of one chunk at its row's counter: a release add (the chunk's
// partial, stored just before by the same thread, is published with it).
// The warp that completes the count then takes an acquire fence before it
// reads the other partials (see chunk_acquire).  CTA scope when the whole
// product runs in one CTA.
template <bool CTA>
__device__ __forceinline__ unsigned chunk_arrive(unsigned* ctr) {
  unsigned old;
  if (CTA)
    asm volatile("atom.release.cta.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
  else
    asm volatile("atom.release.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
  return old;
}
template <bool CTA>
__device__ __forceinline__ void chunk_acquire() {
  if (CTA) asm volatile("fence.acq_rel.cta;" ::: "memory");
  else asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

struct NoChunk {
  template <typename A>
  __device__ __forceinline__ void operator()(int, int, A*) const {}
};
struct NoLong {
  template <typename A>
  __device__ __forceinline__ void operator()(int, A*) const {}
};
struct LazyTag {};

// With LAZY the chunks only store their partials: no arrivals, no on_long.
// The stage that consumes the product then sums a long row's partials itself
// (long_sum), which is possible where it reads the output only at the row's
// own index (elementwise).
template <int NV, bool MAXR, typename AT, typename MT, class Team, class G, class R, class C,
          class L, bool LAZY = false>
__device__ __forceinline__ void spmv(const Team& tm, const Sched& S, const int* __restrict__ ci,
                                     const MT* __restrict__ va, G gather, R on_row, C on_chunk,
                                     L on_long) {
  static_assert(NV <= kMaxNV, "too many partial values per chunk");
  constexpr int B = NV == 1 ? 8 : 4;  // steps whose loads are issued together
  const int lane = threadIdx.x & 31;
  const int nwt = tm.nwarps();
  // The warp whose arrival completes a long row sums the row's partials
  // (lane k takes chunks k, k+32, … in order, then a fixed shuffle tree)
  // and resets the count for the next product.
  auto finish = [&](int4 ch) {
    const int2 lr = S.lrange[ch.w];
    chunk_acquire<Team::kCtaScope>();
    __syncwarp();  // every lane's partial loads after lane 0's acquire
    AT acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = AT(0);
    for (int k = lane; k < lr.y; k += 32) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const AT o = (AT)__ldcg(S.cpart + (size_t)(lr.x + k) * kMaxNV + v);
        acc[v] = MAXR ? (acc[v] > o ? acc[v] : o) : acc[v] + o;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        AT o = __shfl_xor_sync(0xffffffffu, acc[v], off);
        acc[v] = MAXR ? (acc[v] > o ? acc[v] : o) : acc[v] + o;
      }
    }
    if (lane == 0) {
      on_long(ch.x, acc);
      S.ccount[ch.w] = 0u;
    }
  };
  // Long-row chunks first.  Each stores its partial and arrives at its row's
  // count; the count returned for the warp's first chunk is looked at only
  // after the short rows, so its round trip overlaps them.  A chunk holds at
  // most kChunk = 8·32 nonzeros: one batch of 8 per lane.
  int first_c = -1;
  unsigned first_old = 0u;
  for (int c = tm.warp(); c < S.nchunks; c += nwt) {
    const int4 ch = S.chunks[c];
    AT acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = AT(0);
    int cc[kChunk / 32];
    MT vv[kChunk / 32];
#pragma unroll
    for (int u = 0; u < kChunk / 32; ++u) {
      const int k = ch.y + lane + 32 * u;
      cc[u] = k < ch.z ? ci[k] : -1;
      vv[u] = k < ch.z ? va[k] : MT(0);
    }
#pragma unroll
    for (int u = 0; u < kChunk / 32; ++u)
      if (cc[u] >= 0) gather(cc[u], vv[u], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        AT o = __shfl_xor_sync(0xffffffffu, acc[v], off);
        acc[v] = MAXR ? (acc[v] > o ? acc[v] : o) : acc[v] + o;
      }
    }
    unsigned old = 0u;
    if (lane == 0) {
      on_chunk(ch.x, c == S.lrange[ch.w].x ? 1 : 0, acc);
#pragma unroll
      for (int v = 0; v < NV; ++v) S.cpart[(size_t)c * kMaxNV + v] = (double)acc[v];
      if (!LAZY) old = chunk_arrive<Team::kCtaScope>(&S.ccount[ch.w]);
    }
    if (LAZY) continue;
    if (first_c < 0) {
      first_c = c;
      first_old = old;
    } else {
      old = __shfl_sync(0xffffffffu, old, 0);
      if (old + 1 == (unsigned)S.lrange[ch.w].y) finish(ch);
    }
  }
  const int Gw = S.group;
  const int sub = lane & (Gw - 1);
  const int spw = 32 / Gw;
  const int gw = lane / Gw;
  const unsigned gmask = (Gw == 32) ? 0xffffffffu : (((1u << Gw) - 1u) << (gw * Gw));
  for (int s = tm.warp(); s < S.nslices; s += nwt) {
    const int2 sl = S.slices[s];
    const int row = S.srow[s * spw + gw];
    AT acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = AT(0);
    const int* __restrict__ cp = ci + sl.x + lane;
    const MT* __restrict__ vp = va + sl.x + lane;
    for (int t = 0; t < sl.y; t += B) {
      int cc[B];
      MT vv[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const bool in = t + u < sl.y;  // uniform across the warp
        cc[u] = in ? cp[(t + u) * 32] : -1;
        vv[u] = in ? vp[(t + u) * 32] : MT(0);
      }
#pragma unroll
      for (int u = 0; u < B; ++u)
        if (cc[u] >= 0) gather(cc[u], vv[u], acc);
    }
    for (int off = Gw >> 1; off > 0; off >>= 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        AT o = __shfl_xor_sync(gmask, acc[v], off, Gw);
        acc[v] = MAXR ? (acc[v] > o ? acc[v] : o) : acc[v] + o;
      }
    }
    if (sub == 0 && row >= 0) on_row(row, acc);
  }
  if (!LAZY && first_c >= 0) {
    first_old = __shfl_sync(0xffffffffu, first_old, 0);
    const int4 ch = S.chunks[first_c];
    if (first_old + 1 == (unsigned)S.lrange[ch.w].y) finish(ch);
  }
}

// Sum of long row lr's partial value v after the LAZY product that stored
// them (a team barrier in between), by one warp: lane k adds chunks k, k+32,
// … in order, then a fixed xor-shuffle tree, so every lane holds the same
// total.  All lanes of the warp call it.
template <typename AT>
__device__ __forceinline__ AT warp_long_sum(const Sched& S, int lr, int v) {
  const int lane = threadIdx.x & 31;
  const int2 r = S.lrange[lr];
  AT acc = AT(0);
  for (int k = lane; k < r.y; k += 32) acc += (AT)__ldcg(S.cpart + (size_t)(r.x + k) * kMaxNV + v);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  return acc;
}

// A product whose long rows are left as chunk partials (see LAZY).
template <int NV, bool MAXR, typename AT, typename MT, class Team, class G, class R, class C>
__device__ __forceinline__ void spmv(const Team& tm, const Sched& S, const int* __restrict__ ci,
                                     const MT* __restrict__ va, G gather, R on_row, C on_chunk,
                                     NoLong, LazyTag) {
  spmv<NV, MAXR, AT, MT, Team, G, R, C, NoLong, true>(tm, S, ci, va, gather, on_row, on_chunk,
                                                      NoLong{});
}

// The common case: a long row's total goes to the same handler as a short
// row (no piecewise inner products).
template <int NV, bool MAXR, typename AT, typename MT, class Team, class G, class R>
__device__ __forceinline__ void spmv(const Team& tm, const Sched& S, const int* __restrict__ ci,
                                     const MT* __restrict__ va, G gather, R on_row) {
  spmv<NV, MAXR, AT, MT>(tm, S, ci, va, gather, on_row, NoChunk{}, on_row);
}

// Per-entry pass: f(row, k) for every stored nonzero k (padding skipped).
template <class Team, class F>
__device__ __forceinline__ void foreach_entry(const Team& tm, const Sched& S,
                                              const int* __restrict__ ci, F f) {
  const int lane = threadIdx.x & 31;
  const int spw = 32 / S.group;
  const int gw = lane / S.group;
  for (int s = tm.warp(); s < S.nslices; s += tm.nwarps()) {
    const int2 sl = S.slices[s];
    const int row = S.srow[s * spw + gw];
    if (row < 0) continue;
    for (int t = 0; t < sl.y; ++t) {
      const int k = sl.x + 32 * t + lane;
      if (ci[k] >= 0) f(row, k);
    }
  }
  for (int c = tm.warp(); c < S.nchunks; c += tm.nwarps()) {
    const int4 ch = S.chunks[c];
    for (int k = ch.y + lane; k < ch.z; k += 32) f(ch.x, k);
  }
}

__device__ __forceinline__ double ruiz_delta(double nrm) {
  // δ = 1/√‖M_i‖∞ (Alg. 2); reading: a zero norm gives δ = 1, others are
  // clamped to [1e-4, 1e4].
  return nrm == 0.0 ? 1.0 : 1.0 / sqrt(fmin(fmax(nrm, kNormMin), kNormMax));
}

__device__ __forceinline__ double rho_of(uint8_t t, double rho_bar) {
  return (t & kEq) ? kEqRhoFactor * rho_bar : rho_bar;
}

// ---------------------------------------------------------------------------
// Jacobi diagonal of K = P̄ + σI + ĀᵀRĀ: dg_j = P̄_jj + σ + Σ_i ρ_i Ā_ij²,
// read from the Āᵀ half of Kn with ρ_i recomputed from the row types so that
// the stage may run while the ρ vector itself is rewritten; dg and its
// inverse in working precision are written for every row.
// ---------------------------------------------------------------------------
template <class Team, typename T>
__device__ __forceinline__ void jacobi_rows(const Team& tm, const Dev<T>& d, double sigma,
                                            double rho_bar) {
  const int n = d.n;
  const uint8_t* __restrict__ rtype = d.rtype;
  spmv<1, false, double, T>(
      tm, d.kn, d.kn_ci, d.kn_v,
      [&](int c, T v, double* acc) {
        if (c >= n) {
          double vv = (double)v;
          acc[0] += rho_of(rtype[c - n], rho_bar) * vv * vv;
        }
      },
      [&](int j, double* acc) {
        double g = d.pdiag[j] + sigma + acc[0];
        d.dg[j] = g;
        d.dinv[j] = T(1.0 / g);
      });
}

// ---------------------------------------------------------------------------
// Stage 1: modified Ruiz equilibration (Alg. 2, §5.1) computed from the raw
// data and the running D, E, c, then the scaled matrices and vectors
// (Eq. pb:scaled_qp), the ρ vector (§5.2) and the Jacobi diagonal.
// ---------------------------------------------------------------------------
template <class Team, typename T>
__device__ bool scale_stage(Team& tm, const Dev<T>& d, const Params& P, double rho_bar,
                            bool reset_iterates) {
  const int n = d.n, m = d.m, tid = tm.tid(), nth = tm.nthreads();
  double c = 1.0;
  for (int j = tid; j < n; j += nth) {
    d.D[j] = 1.0;
    d.nrm_n[j] = 0.0;
    d.pdiag[j] = 0.0;
    d.dg[j] = 0.0;
  }
  for (int i = tid; i < m; i += nth) {
    d.E[i] = 1.0;
    d.nrm_m[i] = 0.0;
    const double lr = d.l_raw[i], ur = d.u_raw[i];
    d.rtype[i] = (uint8_t)((lr <= -kInfBound ? kLInf : 0) | (ur >= kInfBound ? kUInf : 0) |
                           (lr == ur ? kEq : 0));
  }
  if (!tm.sync()) return false;
  int passes = 0;
  for (int pass = 0; pass < P.scaling_iters; ++pass) {
    // ‖M_j‖∞ for the first n columns of M = [P Aᵀ; A 0] through the rows of
    // Kn, and for the last m through the rows of Ā.
    const double cc = c;
    spmv<2, true, double, double>(
        tm, d.kn, d.kn_ci, d.kn_raw,
        [&](int col, double v, double* acc) {
          if (col < n) acc[0] = fmax(acc[0], fabs(v) * d.D[col]);
          else acc[1] = fmax(acc[1], fabs(v) * d.E[col - n]);
        },
        [&](int j, double* acc) { d.nrm_n[j] = d.D[j] * fmax(cc * acc[0], acc[1]); });
    spmv<1, true, double, double>(
        tm, d.as, d.a_ci, d.a_raw,
        [&](int col, double v, double* acc) { acc[0] = fmax(acc[0], fabs(v) * d.D[col]); },
        [&](int i, double* acc) { d.nrm_m[i] = d.E[i] * acc[0]; });
    if (!tm.sync()) return false;
    // δ, S ← diag(δ)S, and ‖1 − δ‖∞
    double dev[1] = {0.0};
    for (int j = tid; j < n; j += nth) {
      double dl = ruiz_delta(d.nrm_n[j]);
      d.nrm_n[j] = 0.0;
      d.D[j] *= dl;
      dev[0] = fmax(dev[0], fabs(1.0 - dl));
    }
    for (int i = tid; i < m; i += nth) {
      double dl = ruiz_delta(d.nrm_m[i]);
      d.nrm_m[i] = 0.0;
      d.E[i] *= dl;
      dev[0] = fmax(dev[0], fabs(1.0 - dl));
    }
    if (!tm.template publish_sync<1, 1u>(dev)) return false;
    tm.template collect<1, 1u>(dev);
    ++passes;
    // Cost scaling γ = 1/max{mean_j ‖P̄_:,j‖∞, ‖q̄‖∞} with the new D.
    spmv<1, true, double, double>(
        tm, d.kn, d.kn_ci, d.kn_raw,
        [&](int col, double v, double* acc) {
          if (col < n) acc[0] = fmax(acc[0], fabs(v) * d.D[col]);
        },
        [&](int j, double* acc) { d.nrm_n[j] = cc * d.D[j] * acc[0]; });
    double qn[1] = {0.0};
    for (int j = tid; j < n; j += nth) qn[0] = fmax(qn[0], fabs(cc * d.D[j] * d.q_raw[j]));
    if (!tm.template publish_sync<1, 1u>(qn)) return false;
    tm.template collect<1, 1u>(qn);
    double sum[1] = {0.0};
    for (int j = tid; j < n; j += nth) {
      sum[0] += d.nrm_n[j];
      d.nrm_n[j] = 0.0;
    }
    if (!tm.template publish_sync<1, 0u>(sum)) return false;
    tm.template collect<1, 0u>(sum);
    // In γ's max a norm below 1e-4 counts as 1 (a vanishing norm carries no
    // scale, as for δ), and the max is clamped like the other norms; taken
    // literally with q̄ = 0 and mostly-zero P̄ columns, 1/max would grow c
    // geometrically pass after pass.
    double mean = sum[0] / (double)n, qnv = qn[0];
    if (mean < kNormMin) mean = 1.0;
    if (qnv < kNormMin) qnv = 1.0;
    const double gamma = 1.0 / fmin(fmax(fmax(mean, qnv), kNormMin), kNormMax);
    c *= gamma;
    if (dev[0] <= P.eps_equil) break;
  }
  // Scaled data: P̄ = cDPD, Ā = EAD (in both Kn and Ā), q̄ = cDq, [El, Eu].
  foreach_entry(tm, d.kn, d.kn_ci, [&](int j, int k) {
    const int col = d.kn_ci[k];
    const double v = d.kn_raw[k];
    double s;
    if (col < n) {
      s = c * d.D[j] * v * d.D[col];
      if (col == j) d.pdiag[j] = s;
    } else {
      s = d.E[col - n] * v * d.D[j];
    }
    d.kn_v[k] = T(s);
  });
  foreach_entry(tm, d.as, d.a_ci,
                        [&](int i, int k) { d.a_v[k] = T(d.E[i] * d.a_raw[k] * d.D[d.a_ci[k]]); });
  for (int j = tid; j < n; j += nth) {
    d.q[j] = c * d.D[j] * d.q_raw[j];
    d.Dinv[j] = 1.0 / d.D[j];
  }
  for (int i = tid; i < m; i += nth) {
    d.Einv[i] = 1.0 / d.E[i];
    const uint8_t t = d.rtype[i];
    d.l[i] = (t & kLInf) ? -INFINITY : d.E[i] * d.l_raw[i];
    d.u[i] = (t & kUInf) ? INFINITY : d.E[i] * d.u_raw[i];
    const double rh = rho_of(t, rho_bar);
    d.rho[i] = rh;
    d.rho_inv[i] = 1.0 / rh;
    d.rhoT[i] = T(rh);
    d.rho_invT[i] = T(1.0 / rh);
  }
  if (!tm.sync()) return false;
  jacobi_rows(tm, d, P.sigma, rho_bar);
  if (tm.leader()) {  // no residuals on the new data yet: zero = none, −1 = recompute
    d.sc->rp_last = reset_iterates ? 0.0 : -1.0;
    d.sc->rd_last = reset_iterates ? 0.0 : -1.0;
  }
  if (reset_iterates) {
    for (int j = tid; j < n; j += nth) {
      d.x[j] = 0.0;
      d.dx[j] = 0.0;
      d.xt[j] = 0.0;
    }
    for (int i = tid; i < m; i += nth) {
      d.z[i] = 0.0;
      d.y[i] = 0.0;
      d.dy[i] = 0.0;
      d.zt[i] = 0.0;
    }
  }
  if (tm.leader()) {
    d.sc->c = c;
    d.sc->ruiz_passes = passes;
    d.sc->rho_bar = rho_bar;
  }
  return tm.sync();
}

// ---------------------------------------------------------------------------
// Vector update (§6): q̄ = cDq, l̄ = El, ū = Eu with the stored scaling, row
// types, ρ vector and Jacobi diagonal for the current ρ̄.
// ---------------------------------------------------------------------------
template <class Team, typename T>
__device__ bool refresh_stage(Team& tm, const Dev<T>& d, const Params& P, double rho_bar) {
  const int n = d.n, m = d.m, tid = tm.tid(), nth = tm.nthreads();
  const double c = d.sc->c;
  for (int j = tid; j < n; j += nth) d.q[j] = c * d.D[j] * d.q_raw[j];
  for (int i = tid; i < m; i += nth) {
    const double lr = d.l_raw[i], ur = d.u_raw[i];
    const uint8_t t = (uint8_t)((lr <= -kInfBound ? kLInf : 0) | (ur >= kInfBound ? kUInf : 0) |
                                (lr == ur ? kEq : 0));
    d.rtype[i] = t;
    d.l[i] = (t & kLInf) ? -INFINITY : d.E[i] * lr;
    d.u[i] = (t & kUInf) ? INFINITY : d.E[i] * ur;
    const double rh = rho_of(t, rho_bar);
    d.rho[i] = rh;
    d.rho_inv[i] = 1.0 / rh;
    d.rhoT[i] = T(rh);
    d.rho_invT[i] = T(1.0 / rh);
  }
  if (!tm.sync()) return false;
  jacobi_rows(tm, d, P.sigma, rho_bar);
  if (tm.leader()) {
    d.sc->rho_bar = rho_bar;
    // the last check's residuals belong to the old data: recompute them on
    // the current iterates when the next solve starts
    d.sc->rp_last = -1.0;
    d.sc->rd_last = -1.0;
  }
  return tm.sync();
}

// ---------------------------------------------------------------------------
// Solution polishing (§4) in the scaled problem, after a solved run.  Active
// sets from the sign of ȳ; the δ-regularised reduced KKT system of Eq.
// (kkt_polish_reg) is solved in eliminated form,
//   (P̄ + δI + δ⁻¹Ā_actᵀĀ_act) x = −q̄ + δ⁻¹Ā_actᵀ b,   y_act = (Ā_act x − b)/δ,
// by FP64 Jacobi-PCG, and iterative refinement (Eq. iterative_refinement)
// against the unregularised system runs polish_refine passes: with
// r₂ = b − Ā_act x the correction Δx solves the same matrix with right-hand
// side −q̄ − P̄x − Ā_actᵀ(y − r₂/δ), and Δy = (Ā_act Δx − r₂)/δ (formed from
// the small correction, not from Ā_act x⁺ − b, which would lose the digits
// that the division by δ magnifies).  Matrix
// values are the raw FP64 ones scaled on the fly (c·D·P·D, E·A·D), so both
// precision modes polish in FP64.  The candidate replaces the ADMM iterates
// only when y has the signs of Eq. (compl_slack) on the active rows and its
// unscaled residuals are no larger than the ADMM ones.  Returns false on a
// failed team barrier; *pr_io, *dr_io, *obj_io receive the accepted
// residuals and objective.
// ---------------------------------------------------------------------------
constexpr int kPolishPcgMax = 4000;
constexpr double kPolishPcgTol = 1e-10;

template <class Team, typename T>
__device__ __noinline__ bool polish_stage(Team& tm, const Dev<T>& d, const Params& P,
                                          double* pr_io, double* dr_io, double* obj_io) {
  const int n = d.n, m = d.m, tid = tm.tid(), nth = tm.nthreads();
  const double delta = P.delta, idelta = 1.0 / P.delta;
  const double c = d.sc->c;
  const double* __restrict__ D = d.D;
  const double* __restrict__ E = d.E;
  uint8_t* __restrict__ act = d.pol_act;
  double* __restrict__ x = d.pol_x;
  double* __restrict__ dxp = d.pol_dx;
  double* __restrict__ r = d.pol_r;
  double* __restrict__ zz = d.pol_z;
  double* __restrict__ p = d.pol_p;
  double* __restrict__ kp = d.pol_kp;
  double* __restrict__ dg = d.pol_dg;
  double* __restrict__ y = d.pol_y;
  double* __restrict__ t = d.pol_t;
  double* __restrict__ r2 = d.pol_r2;
  auto bnd = [&](int i) { return act[i] == 1 ? d.l[i] : d.u[i]; };
  // Ā v into out (row sums E_i Σ a_ij D_j v_j)
  auto a_times = [&](const double* v, double* out) {
    spmv<1, false, double, double>(
        tm, d.as, d.a_ci, d.a_raw, [&](int col, double a, double* acc) { acc[0] += a * D[col] * v[col]; },
        [&](int i, double* acc) { out[i] = E[i] * acc[0]; });
  };
  // Kn·[v; w] = P̄v + Āᵀw, handed per short row to emit_row(j, P̄v, Āᵀw), per
  // long-row chunk to emit_chunk(j, first, parts) and per long row to
  // emit_long(j, P̄v, Āᵀw)
  auto kn_times = [&](const double* v, const double* w, auto emit_row, auto emit_chunk,
                      auto emit_long) {
    spmv<2, false, double, double>(
        tm, d.kn, d.kn_ci, d.kn_raw,
        [&](int col, double a, double* acc) {
          if (col < n) acc[0] += a * D[col] * v[col];
          else acc[1] += a * E[col - n] * w[col - n];
        },
        [&](int j, double* acc) { emit_row(j, c * D[j] * acc[0], D[j] * acc[1]); },
        [&](int j, int first, double* acc) { emit_chunk(j, first, c * D[j] * acc[0], D[j] * acc[1]); },
        [&](int j, double* acc) { emit_long(j, c * D[j] * acc[0], D[j] * acc[1]); });
  };
  auto no_chunk = [](int, int, double, double) {};

  // active sets, zero start, Jacobi diagonal P̄_jj + δ + δ⁻¹Σ_act Ā_ij²
  for (int i = tid; i < m; i += nth) {
    const double yi = d.y[i];
    const uint8_t ty = d.rtype[i];
    act[i] = (yi < 0.0 && !(ty & kLInf)) ? 1 : ((yi > 0.0 && !(ty & kUInf)) ? 2 : 0);
    y[i] = 0.0;
  }
  for (int j = tid; j < n; j += nth) x[j] = 0.0;
  if (!tm.sync()) return false;
  spmv<1, false, double, double>(
      tm, d.kn, d.kn_ci, d.kn_raw,
      [&](int col, double a, double* acc) {
        if (col >= n && act[col - n]) {
          const double e = E[col - n] * a;
          acc[0] += e * e;
        }
      },
      [&](int j, double* acc) { dg[j] = d.pdiag[j] + delta + idelta * D[j] * D[j] * acc[0]; });
  if (!tm.sync()) return false;

  for (int pass = 0; pass <= P.polish_refine; ++pass) {
    // r₂ = b − Ā_act x and the weights y − r₂/δ of the right-hand side
    a_times(x, t);
    if (!tm.sync()) return false;
    for (int i = tid; i < m; i += nth) {
      const double ri = act[i] ? bnd(i) - t[i] : 0.0;
      r2[i] = ri;
      t[i] = act[i] ? y[i] - ri * idelta : 0.0;
    }
    if (!tm.sync()) return false;
    // rhs = −q̄ − P̄x − Āᵀ(y − r₂/δ) into r
    {
      auto rhs = [&](int j, double pv, double av) { r[j] = -d.q[j] - pv - av; };
      kn_times(x, t, rhs, no_chunk, rhs);
    }
    if (!tm.sync()) return false;
    // PCG for the correction Δx from zero
    double red[2] = {0.0, 0.0};  // (r, M⁻¹r), ‖r‖∞
    for (int j = tid; j < n; j += nth) {
      const double zj = r[j] / dg[j];
      dxp[j] = 0.0;
      zz[j] = zj;
      p[j] = zj;
      red[0] += r[j] * zj;
      red[1] = fmax(red[1], fabs(r[j]));
    }
    if (!tm.template publish_sync<2, 2u>(red)) return false;
    tm.template collect<2, 2u>(red);
    double rz = red[0];
    const double tol = kPolishPcgTol * red[1];
    bool done = !(red[1] > tol) || !(rz > 0.0);
    for (int it = 0; !done && it < kPolishPcgMax; ++it) {
      // t = δ⁻¹Ā_act p
      spmv<1, false, double, double>(
          tm, d.as, d.a_ci, d.a_raw,
          [&](int col, double a, double* acc) { acc[0] += a * D[col] * p[col]; },
          [&](int i, double* acc) { t[i] = act[i] ? idelta * E[i] * acc[0] : 0.0; });
      if (!tm.sync()) return false;
      // Kp = P̄p + δp + Āᵀt and pᵀKp = pᵀP̄p + δ‖p‖² + δ‖t‖²
      double g[1] = {0.0};
      kn_times(
          p, t,
          [&](int j, double pv, double av) {
            kp[j] = pv + av + delta * p[j];
            g[0] += p[j] * pv + delta * p[j] * p[j];
          },
          [&](int j, int first, double pv, double) {
            g[0] += p[j] * pv + (first ? delta * p[j] * p[j] : 0.0);
          },
          [&](int j, double pv, double av) { kp[j] = pv + av + delta * p[j]; });
      for (int i = tid; i < m; i += nth) g[0] += delta * t[i] * t[i];
      if (!tm.template publish_sync<1, 0u>(g)) return false;
      tm.template collect<1, 0u>(g);
      if (!(g[0] > 0.0)) break;
      const double alpha_c = rz / g[0];
      double red2[2] = {0.0, 0.0};
      for (int j = tid; j < n; j += nth) {
        dxp[j] += alpha_c * p[j];
        const double rj = r[j] - alpha_c * kp[j];
        r[j] = rj;
        const double zj = rj / dg[j];
        zz[j] = zj;
        red2[0] += rj * zj;
        red2[1] = fmax(red2[1], fabs(rj));
      }
      if (!tm.template publish_sync<2, 2u>(red2)) return false;
      tm.template collect<2, 2u>(red2);
      if (!(red2[1] > tol) || !(red2[0] > 0.0)) break;
      const double beta_c = red2[0] / rz;
      rz = red2[0];
      for (int j = tid; j < n; j += nth) p[j] = zz[j] + beta_c * p[j];
      if (!tm.sync()) return false;
    }
    if (!tm.sync()) return false;
    // x ← x + Δx, y ← y + (Ā_act Δx − r₂)/δ
    a_times(dxp, t);
    for (int j = tid; j < n; j += nth) x[j] += dxp[j];
    if (!tm.sync()) return false;
    for (int i = tid; i < m; i += nth)
      if (act[i]) y[i] += (t[i] - r2[i]) * idelta;
    if (!tm.sync()) return false;
  }

  // acceptance: signs of y on the active rows, unscaled residuals
  a_times(x, t);
  double chk[4] = {0.0, 0.0, 0.0, 0.0};  // prim, dual·c, sign violation, c·objective
  kn_times(
      x, y,
      [&](int j, double pv, double av) {
        kp[j] = pv + av;
        chk[3] += x[j] * (0.5 * pv + d.q[j]);
      },
      [&](int j, int first, double pv, double) {
        chk[3] += x[j] * (0.5 * pv + (first ? d.q[j] : 0.0));
      },
      [&](int j, double pv, double av) { kp[j] = pv + av; });
  if (!tm.sync()) return false;
  for (int i = tid; i < m; i += nth) {
    const double zi = fmin(fmax(t[i], d.l[i]), d.u[i]);
    chk[0] = fmax(chk[0], fabs((t[i] - zi) / E[i]));
    if (!(d.rtype[i] & kEq) && ((act[i] == 1 && y[i] > 0.0) || (act[i] == 2 && y[i] < 0.0)))
      chk[2] = 1.0;
  }
  for (int j = tid; j < n; j += nth) chk[1] = fmax(chk[1], fabs((kp[j] + d.q[j]) / D[j]));
  if (!tm.template publish_sync<4, 7u>(chk)) return false;
  tm.template collect<4, 7u>(chk);
  const double pr = chk[0], dr = chk[1] / c;
  const bool accept = chk[2] == 0.0 && pr <= *pr_io && dr <= *dr_io;
  if (accept) {
    for (int j = tid; j < n; j += nth) d.x[j] = x[j];
    for (int i = tid; i < m; i += nth) {
      d.z[i] = fmin(fmax(t[i], d.l[i]), d.u[i]);
      d.y[i] = y[i];
    }
    *pr_io = pr;
    *dr_io = dr;
    *obj_io = chk[3] / c;
  }
  if (tm.leader()) d.sc->polished = accept ? 1 : -1;
  return tm.sync();
}

// ---------------------------------------------------------------------------
// Working-precision vectors of a one-CTA solve in shared memory.  The PCG
// vectors (p, r, s, w, the x̃ correction, the Jacobi inverse; [u | t]; Āp,
// the z̃ correction, ρ and ρ⁻¹ in working precision) are read and written
// every PCG iteration and gathered by both sparse products; for a problem
// whose vectors fit, admm_stage runs on a copy of the problem's Dev whose
// pointers to them address the CTA's shared memory.  Only the Jacobi
// inverse and the ρ vectors carry values into and out of a solve.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

template <typename T>
__host__ __device__ constexpr size_t smem_vec_bytes(int n, int m) {
  return 9 * align16((size_t)n * sizeof(T)) + 2 * align16((size_t)(n + m) * sizeof(T)) +
         4 * align16((size_t)m * sizeof(T));
}

// Column indices and working values of both matrices, when they fit beside
// the vectors (small problems): the products then read shared memory only.
template <typename T>
__host__ __device__ constexpr size_t smem_mat_bytes(int npos_kn, int npos_a) {
  return align16((size_t)npos_kn * sizeof(int)) + align16((size_t)npos_kn * sizeof(T)) +
         align16((size_t)npos_a * sizeof(int)) + align16((size_t)npos_a * sizeof(T));
}

// Copy of `bytes` (a multiple of 4, both pointers 16-byte aligned) by one
// CTA, 16 bytes per thread and step, then the last words.
__device__ __forceinline__ void cta_copy(void* dst, const void* src, size_t bytes) {
  const size_t n16 = bytes / 16;
  const int4* s4 = reinterpret_cast<const int4*>(src);
  int4* d4 = reinterpret_cast<int4*>(dst);
  for (size_t k = threadIdx.x; k < n16; k += blockDim.x) d4[k] = s4[k];
  const int* s1 = reinterpret_cast<const int*>(src);
  int* d1 = reinterpret_cast<int*>(dst);
  for (size_t k = 4 * n16 + threadIdx.x; k < bytes / 4; k += blockDim.x) d1[k] = s1[k];
}

template <typename T>
__device__ void stage_in(const Dev<T>& d, Dev<T>& sd, unsigned char* pool, bool with_mat) {
  if (threadIdx.x == 0) {
    sd = d;
    size_t off = 0;
    auto take = [&](int count) {
      T* q = reinterpret_cast<T*>(pool + off);
      off += align16((size_t)count * sizeof(T));
      return q;
    };
    T** nv[] = {&sd.p, &sd.r0, &sd.r1, &sd.s0, &sd.s1, &sd.w0, &sd.w1, &sd.dxt, &sd.dinv};
    for (T** q : nv) *q = take(d.n);
    sd.ut0 = take(d.n + d.m);
    sd.ut1 = take(d.n + d.m);
    T** mv[] = {&sd.ap, &sd.dzt, &sd.rhoT, &sd.rho_invT};
    for (T** q : mv) *q = take(d.m);
    if (with_mat) {
      auto take_i = [&](int count) {
        int* q = reinterpret_cast<int*>(pool + off);
        off += align16((size_t)count * sizeof(int));
        return q;
      };
      sd.kn_ci = take_i(d.kn.npos);
      sd.kn_v = take(d.kn.npos);
      sd.a_ci = take_i(d.as.npos);
      sd.a_v = take(d.as.npos);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < d.n; j += blockDim.x) sd.dinv[j] = d.dinv[j];
  for (int i = threadIdx.x; i < d.m; i += blockDim.x) {
    sd.rhoT[i] = d.rhoT[i];
    sd.rho_invT[i] = d.rho_invT[i];
  }
  if (with_mat) {
    cta_copy((void*)sd.kn_ci, d.kn_ci, (size_t)d.kn.npos * sizeof(int));
    cta_copy((void*)sd.kn_v, d.kn_v, (size_t)d.kn.npos * sizeof(T));
    cta_copy((void*)sd.a_ci, d.a_ci, (size_t)d.as.npos * sizeof(int));
    cta_copy((void*)sd.a_v, d.a_v, (size_t)d.as.npos * sizeof(T));
  }
  __syncthreads();
}

// What a one-CTA solve of this problem keeps in a pool of pool_bytes:
// 2 = vectors and matrices, 1 = vectors only, 0 = nothing.
template <typename T>
__device__ __forceinline__ int smem_plan(const Dev<T>& d, size_t pool_bytes) {
  const size_t v = smem_vec_bytes<T>(d.n, d.m);
  if (v > pool_bytes) return 0;
  return v + smem_mat_bytes<T>(d.kn.npos, d.as.npos) <= pool_bytes ? 2 : 1;
}

template <typename T>
__device__ void stage_out(const Dev<T>& d, const Dev<T>& sd) {
  __syncthreads();
  for (int j = threadIdx.x; j < d.n; j += blockDim.x) d.dinv[j] = sd.dinv[j];
  for (int i = threadIdx.x; i < d.m; i += blockDim.x) {
    d.rhoT[i] = sd.rhoT[i];
    d.rho_invT[i] = sd.rho_invT[i];
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Stage 2: Algorithm 1 with the indirect linear solve of §3.1.
// ---------------------------------------------------------------------------
template <class Team, typename T>
__device__ bool admm_stage(Team& tm, const Dev<T>& d, const Params& P) {
  const int n = d.n, m = d.m, tid = tm.tid(), nth = tm.nthreads();
  const double sigma = P.sigma, alpha = P.alpha;
  const T sigT = T(sigma);
  const double c = d.sc->c;
  double rho_bar = d.sc->rho_bar;
  // FP64 mode: scalars of the PCG recurrence (γ, α, β, tolerance, and α, β
  // and the stop flag handed to every thread), updated by warp 0 of each CTA
  // after each reduction: every CTA derives the same values from the same
  // reduced inputs, and the narrow FP64 pipe runs the divisions once per CTA
  // rather than once per warp.
  double* scal = tm.sm + kScalOff;
  T* scalT = reinterpret_cast<T*>(scal + 5);
  int* sflag = reinterpret_cast<int*>(scal + 7);
  const bool warp0 = (threadIdx.x >> 5) == 0;
  // FP32-mixed mode: every thread runs the recurrence itself, in
  // double-float arithmetic on FP32 instructions, from the reduced values
  // that the reduction leaves as double-float pairs (identical inputs and
  // operations in every thread give identical scalars), and keeps 1/γ and
  // 1/α as pairs and α, β as floats in registers: no FP64 instruction and
  // no CTA barrier after the reduction.  The pairs keep the accuracy of the
  // FP64 reduction of the FP32 partial sums, which the denominator
  // (w,u) − β·γ'/α needs: it cancels when CG converges slowly, and with
  // both terms rounded to FP32 the ADMM iteration of the portfolio problem
  // at ε = 1e-7 diverged.
  constexpr bool kF32 = sizeof(T) == sizeof(float);
  const float* fmir = reinterpret_cast<const float*>(scal + kScalMirror);
  float* ftol = reinterpret_cast<float*>(scal + kScalTolF);
  ff cg_g{0.0f, 0.0f}, cg_ig{0.0f, 0.0f}, cg_ia{0.0f, 0.0f};
  float cg_tol = 0.0f;
  T cg_a = T(0), cg_b = T(0);
  const unsigned long long t_start = gtimer();
  // Pointers read once (restrict-qualified for the compiler).
  const int* __restrict__ kn_ci = d.kn_ci;
  const T* __restrict__ kn_v = d.kn_v;
  const int* __restrict__ a_ci = d.a_ci;
  const T* __restrict__ a_v = d.a_v;
  double* __restrict__ x = d.x;
  double* __restrict__ z = d.z;
  double* __restrict__ y = d.y;
  double* __restrict__ xt = d.xt;
  double* __restrict__ zt = d.zt;
  double* __restrict__ wm = d.wm;
  double* __restrict__ um = d.um;
  T* __restrict__ bv = d.b;
  T* __restrict__ pv = d.p;
  T* __restrict__ ap = d.ap;
  // double-buffer selection without a local-memory pointer table
  auto rbuf = [&](int i) { return i ? d.r1 : d.r0; };
  auto sbuf = [&](int i) { return i ? d.s1 : d.s0; };
  auto wbuf = [&](int i) { return i ? d.w1 : d.w0; };
  auto ubuf = [&](int i) { return i ? d.ut1 : d.ut0; };  // [u | t]
  T* __restrict__ dinv = d.dinv;
  T* __restrict__ dxt = d.dxt;
  T* __restrict__ dzt = d.dzt;
  const T* __restrict__ rhoT = d.rhoT;
  const T* __restrict__ rho_invT = d.rho_invT;
  const double* __restrict__ rho = d.rho;
  const double* __restrict__ rho_inv = d.rho_inv;

  int status = kUnsolved, k = 0, pcg_total = 0, rho_updates = 0, checks = 0;
  // PCG tolerance before this solve's first check: the scaled residuals of
  // the current iterates (a warm start) — those of the last check, or, when
  // the data changed since (marked −1), recomputed below — else a fraction
  // of ‖b‖ (zero iterates)
  double rp_bar = d.sc->rp_last, rd_bar = d.sc->rd_last;
  const bool stale = rp_bar < 0.0 || rd_bar < 0.0;
  double prim_res = NAN, dual_res = NAN, obj = NAN;
  int cur = 0;

  // Right-hand-side inputs of the first iteration from the current iterates.
  for (int i = tid; i < m; i += nth) {
    const double rh = rho[i];
    wm[i] = rh * z[i] - y[i];
    um[i] = rh * (z[i] - zt[i]) - y[i];
    dzt[i] = T(0);
  }
  for (int j = tid; j < n; j += nth) dxt[j] = T(0);
  if (!tm.sync()) return false;
  if (stale) {
    // ‖Āx̄ − z̄‖∞ and ‖P̄x̄ + q̄ + Āᵀȳ‖∞ on the current iterates (§5.1, scaled)
    spmv<2, false, double, T>(
        tm, d.kn, kn_ci, kn_v,
        [&](int col, T v, double* acc) {
          const double vv = (double)v;
          if (col < n) acc[0] += vv * x[col];
          else acc[1] += vv * y[col - n];
        },
        [&](int j, double* acc) {
          d.px[j] = acc[0];
          d.aty[j] = acc[1];
        });
    spmv<1, false, double, T>(
        tm, d.as, a_ci, a_v, [&](int col, T v, double* acc) { acc[0] += (double)v * x[col]; },
        [&](int i, double* acc) { d.ax[i] = acc[0]; });
    if (!tm.sync()) return false;
    double res[2] = {0.0, 0.0};
    for (int i = tid; i < m; i += nth) res[0] = fmax(res[0], fabs(d.ax[i] - z[i]));
    for (int j = tid; j < n; j += nth) res[1] = fmax(res[1], fabs(d.px[j] + d.q[j] + d.aty[j]));
    if (!tm.template publish_sync<2, 3u>(res)) return false;
    tm.template collect<2, 3u>(res);
    rp_bar = res[0];
    rd_bar = res[1];
  }
  bool have_check = rp_bar > 0.0 && rd_bar > 0.0;

  for (k = 1; k <= P.max_iter; ++k) {
    // --- R: initial PCG residual r⁰ = b − Kx̃ and b = σx − q̄ + Āᵀ(Rz − y),
    // using z̃ = Āx̃:  r⁰ = σ(x − x̃) − q̄ − P̄x̃ + Āᵀ(R(z − z̃) − y).  Formed
    // from FP64 vectors with FP64 accumulation in both modes, so that in the
    // FP32 mode every ADMM iteration restarts PCG from an accurate residual
    // (mixed-precision iterative refinement of the linear solve).
    {
      T* __restrict__ r = rbuf(cur);
      spmv<2, false, double, T>(
          tm, d.kn, kn_ci, kn_v,
          [&](int col, T v, double* acc) {
            const double vv = (double)v;
            if (col < n) {
              acc[0] -= vv * xt[col];
            } else {
              acc[0] += vv * um[col - n];
              acc[1] += vv * wm[col - n];
            }
          },
          [&](int j, double* acc) {
            const double bj = sigma * x[j] - d.q[j];
            r[j] = T(bj - sigma * xt[j] + acc[0]);
            bv[j] = T(bj + acc[1]);
          });
    }
    if (!tm.sync()) return false;

    // PCG on K = P̄ + σI + ĀᵀRĀ in the single-reduction form of Chronopoulos
    // and Gear: per iteration one stage that updates p, s = Kp, x̃, r, u = M⁻¹r
    // and computes t = RĀu with u formed on the fly, and one stage that forms
    // w = Ku and the two inner products (r,u), (w,u).  r, s, w and t are
    // double-buffered so that gathers never see a vector being rewritten.
    // --- A0: u = M⁻¹r, t = RĀu; (r,u), ‖r‖∞, ‖b‖∞
    double red3[3];
    T red3t[3];
    {
      const T* __restrict__ r = rbuf(cur);
      T* __restrict__ u = ubuf(cur);
      T* __restrict__ t = ubuf(cur) + n;
      T a0 = T(0), a1 = T(0), a2 = T(0);
      for (int j = tid; j < n; j += nth) {
        const T rj = r[j];
        const T uj = rj * dinv[j];
        u[j] = uj;
        a0 += rj * uj;
        a1 = fmax(a1, fabs(rj));
        a2 = fmax(a2, fabs(bv[j]));
      }
      red3t[0] = a0;
      red3t[1] = a1;
      red3t[2] = a2;
      spmv<1, false, T, T>(
          tm, d.as, a_ci, a_v,
          [&](int col, T v, T* acc) { acc[0] += v * (r[col] * dinv[col]); },
          [&](int i, T* acc) { t[i] = rhoT[i] * acc[0]; });
    }
    if (!tm.template publish_sync<3, 6u>(red3t)) return false;
    tm.template collect<3, 6u, kF32>(red3);
    if (warp0) {
      // PCG accuracy (reading of "up to some predefined accuracy", §3.1).
      const double bnorm = red3[2];
      const double tol = fmax(fmax(P.pcg_floor * bnorm, P.pcg_reduce * red3[1]),
                              have_check ? P.pcg_kappa * fmin(rp_bar, rd_bar)
                                         : 0.1 * P.pcg_kappa * bnorm);
      scal[0] = red3[0];  // γ = (r, M⁻¹r)
      scal[3] = tol;
      if (kF32 && threadIdx.x == 0) *ftol = (float)tol;
      if (threadIdx.x == 0) *sflag = !(red3[1] > tol);
    }
    __syncthreads();
    bool done = *sflag != 0;
    if constexpr (kF32) {
      cg_g = ff{fmir[0], fmir[1]};
      cg_tol = *ftol;
    }
    if (!done) {
      // --- W: w = Ku, (w,u)
      double red1[1] = {0.0};
      T wacc = T(0);
      T* __restrict__ w = wbuf(cur);
      const T* __restrict__ ut = ubuf(cur);
      const T* __restrict__ u = ut;
      // long rows of w stay as chunk partials: P1, the only reader, sums them
      spmv<1, false, T, T>(
          tm, d.kn, kn_ci, kn_v, [&](int col, T v, T* acc) { acc[0] += v * ut[col]; },
          [&](int j, T* acc) {
            const T wj = sigT * u[j] + acc[0];
            w[j] = wj;
            wacc += wj * u[j];
          },
          [&](int j, int first, T* acc) {
            wacc += (acc[0] + (first ? sigT * u[j] : T(0))) * u[j];
          },
          NoLong{}, LazyTag{});
      const T red1t[1] = {wacc};
      if (!tm.template publish_sync<1, 0u, !kF32>(red1t)) return false;
      tm.template collect<1, 0u, kF32>(red1);
      if constexpr (kF32) {
        // α = γ/(w,u), β = 0; every thread, from the pair of (w,u)
        const ff wu{fmir[0], fmir[1]};
        done = !(wu.h > 0.0f);
        if (!done) {
          cg_a = ff_div(cg_g, wu).h;
          cg_b = 0.0f;
          cg_ig = ff_div(ff{1.0f, 0.0f}, cg_g);
          cg_ia = ff_mul(wu, cg_ig);  // 1/α
        }
      } else {
        if (warp0) {
          const double a = red1[0] > 0.0 ? scal[0] / red1[0] : 0.0;
          scal[1] = a;
          scalT[0] = T(a);
          scalT[1] = T(0);
          if (threadIdx.x == 0) *sflag = !(red1[0] > 0.0);
        }
        __syncthreads();
        done = *sflag != 0;
      }
    }
    int j_it = 0;
    while (!done) {
      const int nxt = cur ^ 1;
      const bool first = j_it == 0;
      const T aT = kF32 ? cg_a : scalT[0], bT = kF32 ? cg_b : scalT[1];
      // --- P1: p = u + βp, s = w + βs, x̃ += αp, r −= αs, u = M⁻¹r,
      //         Āp = t/ρ + β·Āp, z̃ += α·Āp   (elementwise)
      {
        const T* __restrict__ rc = rbuf(cur);
        const T* __restrict__ sc = sbuf(cur);
        const T* __restrict__ wc = wbuf(cur);
        T* __restrict__ rn = rbuf(nxt);
        T* __restrict__ sn = sbuf(nxt);
        const T* __restrict__ tc = ubuf(cur) + n;
        const T* __restrict__ u = ubuf(cur);
        T* __restrict__ un = ubuf(nxt);
        auto upd = [&](int j, T wj) {
          const T pj = first ? u[j] : u[j] + bT * pv[j];
          const T sj = first ? wj : wj + bT * sc[j];
          pv[j] = pj;
          sn[j] = sj;
          dxt[j] += aT * pj;
          const T rj = rc[j] - aT * sj;
          rn[j] = rj;
          un[j] = rj * dinv[j];
        };
        // w = Ku; its long rows are left as the product's chunk partials and
        // summed here, one warp per row, taken from the last warp down: the
        // elements above go to the first threads, so on a wide team the two
        // chains run on different warps
        const bool lazy_w = d.kn.nlong > 0;
        for (int j = tid; j < n; j += nth)
          if (!lazy_w || d.kn.lidx[j] < 0) upd(j, wc[j]);
        for (int lr = tm.nwarps() - 1 - tm.warp(); lr < d.kn.nlong; lr += tm.nwarps()) {
          const T sum = warp_long_sum<T>(d.kn, lr, 0);
          const int j = d.kn.long_rows[lr];
          if ((threadIdx.x & 31) == 0) upd(j, sigT * u[j] + sum);
        }
        for (int i = tid; i < m; i += nth) {
          const T ti = rho_invT[i] * tc[i];
          const T api = first ? ti : ti + bT * ap[i];
          ap[i] = api;
          dzt[i] += aT * api;
        }
      }
      if (!tm.sync()) return false;
      // --- P1b: t' = RĀu
      {
        const T* __restrict__ u = ubuf(nxt);
        T* __restrict__ tn = ubuf(nxt) + n;
        spmv<1, false, T, T>(
            tm, d.as, a_ci, a_v, [&](int col, T v, T* acc) { acc[0] += v * u[col]; },
            [&](int i, T* acc) { tn[i] = rhoT[i] * acc[0]; });
      }
      if (!tm.sync()) return false;
      ++j_it;
      ++pcg_total;
      // --- P2: w = Ku, (r,u), (w,u), ‖r‖∞
      double red2[3];
      T red2t[3];
      {
        const T* __restrict__ rn = rbuf(nxt);
        T* __restrict__ wn = wbuf(nxt);
        const T* __restrict__ ut = ubuf(nxt);
        const T* __restrict__ u = ut;
        T g0 = T(0), g1 = T(0), g2 = T(0);
        for (int j = tid; j < n; j += nth) {
          const T rj = rn[j];
          g0 += rj * u[j];
          g2 = fmax(g2, fabs(rj));
        }
        spmv<1, false, T, T>(
            tm, d.kn, kn_ci, kn_v, [&](int col, T v, T* acc) { acc[0] += v * ut[col]; },
            [&](int j, T* acc) {
              const T wj = sigT * u[j] + acc[0];
              wn[j] = wj;
              g1 += wj * u[j];
            },
            [&](int j, int first2, T* acc) {
              g1 += (acc[0] + (first2 ? sigT * u[j] : T(0))) * u[j];
            },
            NoLong{}, LazyTag{});
        red2t[0] = g0;
        red2t[1] = g1;
        red2t[2] = g2;
      }
      if (!tm.template publish_sync<3, 4u, !kF32>(red2t)) return false;
      tm.template collect<3, 4u, kF32>(red2);
      cur = nxt;
      if constexpr (kF32) {
        // Chronopoulos–Gear update in every thread, in double-float (see
        // above): β = γ'·(1/γ), α = γ'/((w,u) − β·γ'·(1/α)); stop at the
        // tolerance, the iteration cap, or a breakdown
        bool stop = !(fmir[4] > cg_tol) || j_it >= P.pcg_max_iter;
        if (!stop) {
          const ff gn{fmir[0], fmir[1]};
          const ff beta = ff_mul(gn, cg_ig);
          const ff denom = ff_sub(ff{fmir[2], fmir[3]}, ff_mul(beta, ff_mul(gn, cg_ia)));
          if (!(denom.h > 0.0f) || !(gn.h > 0.0f)) {
            stop = true;
          } else {
            cg_a = ff_div(gn, denom).h;
            cg_b = beta.h;
            cg_ig = ff_div(ff{1.0f, 0.0f}, gn);
            cg_ia = ff_mul(denom, cg_ig);
          }
        }
        if (stop) break;
        continue;
      }
      if (warp0) {
        // Chronopoulos–Gear update: β = γ'/γ, α = γ'/((w,u) − βγ'/α); stop
        // at the tolerance, the iteration cap, or a breakdown (p vanished).
        // β = γ'/γ and γ'/α are independent of each other and correctly
        // rounded: the FP64 PCG iteration count follows the rounding of
        // these scalars.
        int stop = !(red2[2] > scal[3]) || j_it >= P.pcg_max_iter;
        if (!stop) {
          const double gamma_n = red2[0];
          const double beta_n = gamma_n / scal[0];
          const double denom = red2[1] - beta_n * (gamma_n / scal[1]);
          if (!(denom > 0.0) || !(gamma_n > 0.0)) {
            stop = 1;
          } else {
            const double a = gamma_n / denom;
            scal[0] = gamma_n;
            scal[1] = a;
            scal[2] = beta_n;
            scalT[0] = T(a);
            scalT[1] = T(beta_n);
          }
        }
        if (threadIdx.x == 0) *sflag = stop;
      }
      __syncthreads();
      if (*sflag) break;
    }

    // --- U: Algorithm 1 steps 5–7, y in the form ρ(v − Π(v)) of Eq. (zy-update)
    for (int j = tid; j < n; j += nth) {
      const double xtj = xt[j] + (double)dxt[j];
      xt[j] = xtj;
      dxt[j] = T(0);
      const double xn = alpha * xtj + (1.0 - alpha) * x[j];
      d.dx[j] = xn - x[j];
      x[j] = xn;
    }
    for (int i = tid; i < m; i += nth) {
      const double rh = rho[i];
      const double zti = zt[i] + (double)dzt[i];
      zt[i] = zti;
      dzt[i] = T(0);
      const double v = alpha * zti + (1.0 - alpha) * z[i] + rho_inv[i] * y[i];
      const double zn = fmin(fmax(v, d.l[i]), d.u[i]);
      const double yn = rh * (v - zn);
      d.dy[i] = yn - y[i];
      z[i] = zn;
      y[i] = yn;
      wm[i] = rh * zn - yn;
      um[i] = rh * (zn - zti) - yn;
    }
    const bool check = (k % P.check_interval == 0) || (k == P.max_iter);
    if (!tm.sync()) return false;
    if (!check) continue;

    // --- K1: P̄x̄, Āᵀȳ, P̄δx̄, Āᵀδȳ (δȳ projected), Āx̄, Āδx̄, Āx̃ in FP64
    ++checks;
    {
      const uint8_t* __restrict__ rtype = d.rtype;
      const double* __restrict__ dxp = d.dx;
      const double* __restrict__ dyp = d.dy;
      spmv<4, false, double, T>(
          tm, d.kn, kn_ci, kn_v,
          [&](int col, T v, double* acc) {
            const double vv = (double)v;
            if (col < n) {
              acc[0] += vv * x[col];
              acc[2] += vv * dxp[col];
            } else {
              const int i = col - n;
              acc[1] += vv * y[i];
              double dv = dyp[i];
              const uint8_t t = rtype[i];
              if (((t & kUInf) && dv > 0.0) || ((t & kLInf) && dv < 0.0)) dv = 0.0;
              acc[3] += vv * dv;
            }
          },
          [&](int j, double* acc) {
            d.px[j] = acc[0];
            d.aty[j] = acc[1];
            d.pdx[j] = acc[2];
            d.atdy[j] = acc[3];
          });
      spmv<3, false, double, T>(
          tm, d.as, a_ci, a_v,
          [&](int col, T v, double* acc) {
            const double vv = (double)v;
            acc[0] += vv * x[col];
            acc[1] += vv * dxp[col];
            acc[2] += vv * xt[col];
          },
          [&](int i, double* acc) {
            d.ax[i] = acc[0];
            d.adx[i] = acc[1];
            d.azt[i] = acc[2];
          });
    }
    if (!tm.sync()) return false;

    // --- K2: norms of §5.1 (termination, infeasibility) and §5.2 (ρ ratio)
    double R[24];
#pragma unroll
    for (int q = 0; q < 24; ++q) R[q] = 0.0;
    R[20] = -INFINITY;
    constexpr unsigned kMaxMask = 0xFFFFFFu & ~((1u << 15) | (1u << 18) | (1u << 21) | (1u << 22));
    for (int i = tid; i < m; i += nth) {
      const double Ei = d.E[i], Eii = d.Einv[i], axi = d.ax[i], zi = z[i];
      R[0] = fmax(R[0], fabs((axi - zi) * Eii));
      R[1] = fmax(R[1], fabs(axi * Eii));
      R[2] = fmax(R[2], fabs(zi * Eii));
      R[3] = fmax(R[3], fabs(axi - zi));
      R[4] = fmax(R[4], fabs(axi));
      R[5] = fmax(R[5], fabs(zi));
      const uint8_t t = d.rtype[i];
      double dv = d.dy[i];
      if (((t & kUInf) && dv > 0.0) || ((t & kLInf) && dv < 0.0)) dv = 0.0;
      R[14] = fmax(R[14], fabs(Ei * dv));
      if (dv > 0.0) R[15] += d.u[i] * dv;
      else if (dv < 0.0) R[15] += d.l[i] * dv;
      const double a = d.adx[i] * Eii;
      const bool lf = !(t & kLInf), uf = !(t & kUInf);
      const double viol = (lf && uf) ? fabs(a) : (lf ? -a : (uf ? a : -INFINITY));
      R[20] = fmax(R[20], viol);
      // refresh z̃ = Āx̃ and the right-hand-side input that depends on it
      const double azi = d.azt[i];
      zt[i] = azi;
      um[i] = rho[i] * (zi - azi) - y[i];
    }
    for (int j = tid; j < n; j += nth) {
      const double Dj = d.D[j], Dij = d.Dinv[j], pxj = d.px[j], atyj = d.aty[j], qj = d.q[j];
      const double rd = pxj + qj + atyj;
      R[6] = fmax(R[6], fabs(rd * Dij));
      R[7] = fmax(R[7], fabs(pxj * Dij));
      R[8] = fmax(R[8], fabs(atyj * Dij));
      R[9] = fmax(R[9], fabs(qj * Dij));
      R[10] = fmax(R[10], fabs(rd));
      R[11] = fmax(R[11], fabs(pxj));
      R[12] = fmax(R[12], fabs(atyj));
      R[13] = fmax(R[13], fabs(qj));
      R[16] = fmax(R[16], fabs(d.atdy[j] * Dij));
      const double dxj = d.dx[j];
      R[17] = fmax(R[17], fabs(Dj * dxj));
      R[18] += qj * dxj;
      R[19] = fmax(R[19], fabs(d.pdx[j] * Dij));
      R[21] += x[j] * pxj;
      R[22] += qj * x[j];
    }
    if (threadIdx.x == 0) R[23] = (double)(gtimer() - t_start);
    if (!tm.template publish_sync<24, kMaxMask>(R)) return false;
    tm.template collect<24, kMaxMask>(R);
    prim_res = R[0];
    dual_res = R[6] / c;
    obj = (0.5 * R[21] + R[22]) / c;
    const double eps_prim = P.eps_abs + P.eps_rel * fmax(R[1], R[2]);
    const double eps_dual = P.eps_abs + P.eps_rel * fmax(fmax(R[7], R[8]), R[9]) / c;
    if (!isfinite(prim_res) || !isfinite(dual_res)) {
      status = kNumErr;
    } else if (prim_res <= eps_prim && dual_res <= eps_dual) {
      status = kSolved;
    } else if (R[16] <= P.eps_pinf * R[14] && R[15] < -P.eps_pinf * R[14]) {
      status = kPrimInf;
    } else if (R[19] <= c * P.eps_dinf * R[17] && R[18] < -c * P.eps_dinf * R[17] &&
               R[20] <= P.eps_dinf * R[17]) {
      status = kDualInf;
    } else if (P.time_limit_ns > 0.0 && R[23] > P.time_limit_ns) {
      status = kTimeLimit;
    }
    if (tm.leader()) {
      d.sc->rp_last = R[3];
      d.sc->rd_last = R[10];
    }
    if (status != kUnsolved) break;
    rp_bar = R[3];
    rd_bar = R[10];
    have_check = true;
    // ρ̄ adaptation (§5.2) in scaled norms; the Jacobi diagonal is rebuilt
    // on the device in place of a refactorisation.
    if (P.adaptive_rho && rho_updates < P.max_rho_updates && k < P.max_iter) {
      const double pr = R[3] / (fmax(R[4], R[5]) + kTiny);
      const double dr = R[10] / (fmax(fmax(R[11], R[12]), R[13]) + kTiny);
      double rn = rho_bar * sqrt(pr / (dr + kTiny));
      rn = fmin(fmax(rn, kRhoMin), kRhoMax);
      if (rn > P.rho_tol * rho_bar || rn < rho_bar / P.rho_tol) {
        rho_bar = rn;
        ++rho_updates;
        for (int i = tid; i < m; i += nth) {
          const double rh = rho_of(d.rtype[i], rho_bar);
          d.rho[i] = rh;
          d.rho_inv[i] = 1.0 / rh;
          d.rhoT[i] = T(rh);
          d.rho_invT[i] = T(1.0 / rh);
          wm[i] = rh * z[i] - y[i];
          um[i] = rh * (z[i] - zt[i]) - y[i];
        }
        jacobi_rows(tm, d, sigma, rho_bar);
        if (!tm.sync()) return false;
      }
    }
  }
  if (status == kUnsolved && P.max_iter > 0) status = kMaxIter;

  // --- solution polishing (§4)
  if (P.polish && status == kSolved) {
    if (!polish_stage(tm, d, P, &prim_res, &dual_res, &obj)) return false;
  } else if (tm.leader()) {
    d.sc->polished = 0;
  }

  // --- unscale (Eq. pb:scaled_qp) and certificates (§5.1)
  for (int j = tid; j < n; j += nth) {
    d.x_out[j] = d.D[j] * x[j];
    d.dcert[j] = status == kDualInf ? d.D[j] * d.dx[j] : 0.0;
  }
  for (int i = tid; i < m; i += nth) {
    const double Ei = d.E[i];
    d.z_out[i] = z[i] * d.Einv[i];
    d.y_out[i] = Ei * y[i] / c;
    double dv = d.dy[i];
    const uint8_t t = d.rtype[i];
    if (((t & kUInf) && dv > 0.0) || ((t & kLInf) && dv < 0.0)) dv = 0.0;
    d.pcert[i] = status == kPrimInf ? Ei * dv / c : 0.0;
  }
  if (tm.leader()) {
    Scalars* sc = d.sc;
    sc->status = status;
    sc->iter = k > P.max_iter ? P.max_iter : k;
    sc->pcg_iters = pcg_total;
    sc->rho_updates = rho_updates;
    sc->checks = checks;
    sc->rho_bar = rho_bar;
    sc->obj = obj;
    sc->prim_res = prim_res;
    sc->dual_res = dual_res;
  }
  return true;
}

}  // namespace osqpgb
