// osqp_solve_noalloc: a whole small-QP solve that allocates no memory.
//
// Some callers cannot allocate device memory at solve time: code running
// inside a CUDA-graph capture that must not touch the allocator, plugins
// hosted by a framework that owns all device memory, or real-time loops that
// forbid cudaMalloc/cudaFree after start-up.  For them this entry point runs
// the same one-CTA solver as osqp_setup/osqp_solve with launch = 1 (Ruiz
// scaling, ρ and Jacobi, Algorithm 1 with PCG, termination, unscaling), but
// every intermediate array — including the CSR structure and the sliced
// layout that osqp_setup builds on the host — lives in one file-scope device
// array of kNoallocScratchBytes.  The caller passes device inputs and
// outputs.
//
// The array is statically allocated in every GPU that loads the library and
// stays there until the process exits.  Its device address is looked up once
// per device (cudaGetSymbolAddress) by the first call made with that device
// current; make that first call before any stream capture.  All calls share
// the array: two calls whose kernels overlap on the GPU race on it, so
// serialise them (one stream, or events).  The kernel clears every counter it
// relies on at its start; the rest of the array keeps the last call's data.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/osqp_gb300.h"
#include "../../include/osqp_gb300_noalloc.h"
#include "device.cuh"

using namespace osqpgb;

namespace {

constexpr size_t kNoallocScratchBytes = OSQP_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocMaxRow = 8192;  // rows longer than this are rejected (sort cost)
constexpr int kMaxBins = 16384;       // short-row lengths the layout sort can bin
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

enum : int { kNaOk = 0, kNaBadCsc = 1, kNaLongRow = 2, kNaNoRoom = 3, kNaNonFinite = 4,
             kNaLgtU = 5 };

struct NaInput {
  int n, m, nnzP, nnzA;
  const int* Pp;
  const int* Pi;
  const double* Px;
  const double* q;
  const int* Ap;
  const int* Ai;
  const double* Ax;
  const double* l;
  const double* u;
  double* x;
  double* y;
};

// Scratch layout shared by the host size check and the device carve.
template <typename T>
struct NaLayout {
  size_t total = 0;
  template <typename V>
  __host__ __device__ size_t take(size_t count) {
    total = (total + 255) & ~(size_t)255;
    size_t at = total;
    total += (count ? count : 1) * sizeof(V);
    return at;
  }
};

// Buffers of one matrix's layout build.
struct NaSched {
  int* rp;        // CSR row pointer
  int* cci;       // CSR columns
  double* craw;   // CSR raw values
  int2* slices;
  int* srow;
  int4* chunks;
  int* long_rows;
  int* lpos;      // first position of each long row
  int* order;     // short rows, stably sorted by decreasing length
  int2* lrange;   // per long row: first chunk, number of chunks
  int* lidx;      // per row: long-row index, −1 for a short row
  double* cpart;  // per chunk: partial values of a product
  unsigned* ccount;  // per long row: chunks stored (zeroed by the build)
};

template <typename T>
struct NaPtrs {
  Dev<T> d;
  NaSched kn, a;
  int *plen, *cur_n, *alen, *cur_m, *tmp_ci, *err, *flag;
  int *bin_cnt, *bin_rev, *bin_start, *wsum;
  double* tmp_raw;
  size_t fixed_end;  // first byte after the fixed carve
  size_t dyn;        // first free byte after the sliced arrays carved so far
};

// Carve the scratch array; base == nullptr only measures.  The sliced
// arrays (column, raw and working values), whose size depends on the
// structure, are placed after the fixed part by the kernel itself.
template <typename T>
__host__ __device__ size_t na_carve(const NaInput& in, char* base, NaPtrs<T>* p) {
  NaLayout<T> L;
  const size_t n = in.n, m = in.m;
  const size_t nkn = 2 * (size_t)in.nnzP + in.nnzA;  // full P ≤ twice its upper triangle
  const size_t na = in.nnzA;
  const size_t tmpn = nkn > na ? nkn : na;
  const size_t ch_kn = nkn / kChunk + nkn / 257 + 1, lr_kn = nkn / 257 + 1;
  const size_t ch_a = na / kChunk + na / 257 + 1, lr_a = na / 257 + 1;
  const size_t nr = n > m ? n : m;
  constexpr int kSlots = 104;  // ≥ the number of take() calls below (101)
  size_t o[kSlots];
  int c = 0;
  o[c++] = L.template take<int>(n + 1);       // 0 kn rp
  o[c++] = L.template take<int>(nkn);         // 1 kn CSR columns
  o[c++] = L.template take<double>(nkn);      // 2 kn CSR raw
  o[c++] = L.template take<int>(m + 1);       // 3 a rp
  o[c++] = L.template take<int>(na);          // 4 a CSR columns
  o[c++] = L.template take<double>(na);       // 5 a CSR raw
  o[c++] = L.template take<int>(tmpn);        // 6 tmp_ci
  o[c++] = L.template take<double>(tmpn);     // 7 tmp_raw
  o[c++] = L.template take<int>(n);           // 8 plen
  o[c++] = L.template take<int>(n);           // 9 cur_n
  o[c++] = L.template take<int>(m);           // 10 alen
  o[c++] = L.template take<int>(m);           // 11 cur_m
  o[c++] = L.template take<int4>(ch_kn);      // 12 kn chunks
  o[c++] = L.template take<int>(lr_kn);       // 13 kn long rows
  o[c++] = L.template take<int>(lr_kn);       // 14 kn long-row positions
  o[c++] = L.template take<int4>(ch_a);       // 15 a chunks
  o[c++] = L.template take<int>(lr_a);        // 16 a long rows
  o[c++] = L.template take<int>(lr_a);        // 17 a long-row positions
  o[c++] = L.template take<int2>(n + 1);      // 18 kn slices
  o[c++] = L.template take<int>(n + 32);      // 19 kn slice rows
  o[c++] = L.template take<int>(n);           // 20 kn order
  o[c++] = L.template take<int2>(m + 1);      // 21 a slices
  o[c++] = L.template take<int>(m + 32);      // 22 a slice rows
  o[c++] = L.template take<int>(m);           // 23 a order
  o[c++] = L.template take<int>(kMaxBins + 1);  // 24 bin counts
  o[c++] = L.template take<int>(kMaxBins + 1);  // 25 bin counts, longest first
  o[c++] = L.template take<int>(kMaxBins + 2);  // 26 bin starts
  o[c++] = L.template take<int>(nr + 2);      // 27 slice widths / starts
  o[c++] = L.template take<uint8_t>(m);       // 28 rtype
  const int at_lr = c;
  o[c++] = L.template take<int2>(lr_kn);      // kn long-row chunk ranges
  o[c++] = L.template take<double>(ch_kn * kMaxNV);  // kn chunk partials
  o[c++] = L.template take<unsigned>(lr_kn);  // kn long-row counters
  o[c++] = L.template take<int2>(lr_a);       // a long-row chunk ranges
  o[c++] = L.template take<double>(ch_a * kMaxNV);   // a chunk partials
  o[c++] = L.template take<unsigned>(lr_a);   // a long-row counters
  o[c++] = L.template take<int>(n);           // kn row → long-row index
  o[c++] = L.template take<int>(m);           // a row → long-row index
  const int at_pact = c;
  o[c++] = L.template take<uint8_t>(m);       // 29 polishing row states
  const int nvec_n = 22, nvec_m = 22;
  const int first_n = c;
  for (int k = 0; k < nvec_n; ++k) o[c++] = L.template take<double>(n);
  const int first_m = c;
  for (int k = 0; k < nvec_m; ++k) o[c++] = L.template take<double>(m);
  const int first_tn = c;
  for (int k = 0; k < 10; ++k) o[c++] = L.template take<T>(n);
  const int at_rt = c;
  for (int k = 0; k < 4; ++k) o[c++] = L.template take<T>(m);
  const int at_ut = c;
  for (int k = 0; k < 2; ++k) o[c++] = L.template take<T>(n + m);
  const int at_sc = c;
  o[c++] = L.template take<Scalars>(1);
  const int at_err = c;
  o[c++] = L.template take<int>(2);
  static_assert(38 + 22 + 22 + 10 + 4 + 2 + 2 <= kSlots, "scratch slot table too small");
  if (base && p) {
    Dev<T>& d = p->d;
    d.n = in.n;
    d.m = in.m;
    p->kn = NaSched{(int*)(base + o[0]),   (int*)(base + o[1]),   (double*)(base + o[2]),
                    (int2*)(base + o[18]), (int*)(base + o[19]),  (int4*)(base + o[12]),
                    (int*)(base + o[13]),  (int*)(base + o[14]),  (int*)(base + o[20]),
                    (int2*)(base + o[at_lr]), (int*)(base + o[at_lr + 6]),
                    (double*)(base + o[at_lr + 1]), (unsigned*)(base + o[at_lr + 2])};
    p->a = NaSched{(int*)(base + o[3]),   (int*)(base + o[4]),   (double*)(base + o[5]),
                   (int2*)(base + o[21]), (int*)(base + o[22]),  (int4*)(base + o[15]),
                   (int*)(base + o[16]),  (int*)(base + o[17]),  (int*)(base + o[23]),
                   (int2*)(base + o[at_lr + 3]), (int*)(base + o[at_lr + 7]),
                   (double*)(base + o[at_lr + 4]), (unsigned*)(base + o[at_lr + 5])};
    p->tmp_ci = (int*)(base + o[6]);
    p->tmp_raw = (double*)(base + o[7]);
    p->plen = (int*)(base + o[8]);
    p->cur_n = (int*)(base + o[9]);
    p->alen = (int*)(base + o[10]);
    p->cur_m = (int*)(base + o[11]);
    p->bin_cnt = (int*)(base + o[24]);
    p->bin_rev = (int*)(base + o[25]);
    p->bin_start = (int*)(base + o[26]);
    p->wsum = (int*)(base + o[27]);
    d.rtype = (uint8_t*)(base + o[28]);
    d.pol_act = (uint8_t*)(base + o[at_pact]);
    double** nv[] = {&d.D, &d.q, &d.pdiag, &d.dg, &d.nrm_n, &d.x, &d.dx, &d.px,
                     &d.aty, &d.pdx, &d.atdy, &d.x_out, &d.dcert, &d.xt, &d.Dinv,
                     &d.pol_x, &d.pol_dx, &d.pol_r, &d.pol_z, &d.pol_p, &d.pol_kp,
                     &d.pol_dg};
    for (int k = 0; k < nvec_n; ++k) *nv[k] = (double*)(base + o[first_n + k]);
    double** mv[] = {&d.E, &d.l, &d.u, &d.rho, &d.rho_inv, &d.nrm_m, &d.z, &d.y, &d.dy,
                     &d.ax, &d.adx, &d.azt, &d.z_out, &d.y_out, &d.pcert, &d.zt, &d.wm, &d.um,
                     &d.Einv, &d.pol_y, &d.pol_t, &d.pol_r2};
    for (int k = 0; k < nvec_m; ++k) *mv[k] = (double*)(base + o[first_m + k]);
    T** tv[] = {&d.dinv, &d.b, &d.p, &d.r0, &d.r1, &d.s0, &d.s1, &d.w0, &d.w1, &d.dxt};
    for (int k = 0; k < 10; ++k) *tv[k] = (T*)(base + o[first_tn + k]);
    T** tmv[] = {&d.ap, &d.dzt, &d.rhoT, &d.rho_invT};
    for (int k = 0; k < 4; ++k) *tmv[k] = (T*)(base + o[at_rt + k]);
    d.ut0 = (T*)(base + o[at_ut]);
    d.ut1 = (T*)(base + o[at_ut + 1]);
    d.sc = (Scalars*)(base + o[at_sc]);
    p->err = (int*)(base + o[at_err]);
    p->flag = p->err + 1;
    p->fixed_end = L.total;
    // the caller's inputs are read in place; x and y are written in place
    d.q_raw = in.q;
    d.l_raw = in.l;
    d.u_raw = in.u;
    d.x_out = in.x;
    d.y_out = in.y;
  }
  return L.total;
}

// Bytes of the sliced arrays of one matrix with npos positions.
template <typename T>
__host__ __device__ size_t sliced_bytes(size_t npos) {
  const size_t c = npos ? npos : 1;
  return ((c * sizeof(int) + 255) & ~(size_t)255) + ((c * sizeof(double) + 255) & ~(size_t)255) +
         ((c * sizeof(T) + 255) & ~(size_t)255);
}

// Exclusive prefix sum of v[0..count) into out[0..count] by one CTA.
__device__ void block_exclusive_scan(const int* v, int* out, int count, int* sh) {
  // sh: at least blockDim.x/32 + 1 ints
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int carry = 0;
  for (int base = 0; base < count; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int x = i < count ? v[i] : 0;
    int incl = x;
    for (int off = 1; off < 32; off <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    if (lane == 31) sh[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int w = lane < nw ? sh[lane] : 0;
      int wi = w;
      for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, wi, off);
        if (lane >= off) wi += y;
      }
      if (lane < nw) sh[lane] = wi - w;  // exclusive warp offsets
      if (lane == nw - 1) sh[32] = wi;   // chunk total
    }
    __syncthreads();
    if (i < count) out[i] = carry + sh[wid] + incl - x;
    carry += sh[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[count] = carry;
  __syncthreads();
}

// Sliced layout of one CSR matrix, built by one CTA: the layout the host
// builder of osqp_setup makes (same long-row threshold and group width, short
// rows stably sorted by decreasing length by a counting sort), so a solve
// here takes the same arithmetic path as osqp_solve with launch = 1.  The
// column, raw and working-value arrays are carved at sp.dyn; a layout that
// does not fit in the scratch array sets kNaNoRoom.
template <typename T>
__device__ bool build_sliced(Sched& S, const NaSched& B, NaPtrs<T>& sp, int nrows, char* base,
                             const int** ci_out, const double** raw_out, T** v_out, int* sh_int,
                             double* sm) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  const int* rp = B.rp;
  const int nnz = rp[nrows];
  const double mean_all = nrows > 0 ? (double)nnz / nrows : 0.0;
  const int thresh = max(256, (int)(8.0 * ceil(mean_all)));
  double red[2] = {0.0, 0.0};  // short nnz, short rows
  for (int r = tid; r < nrows; r += nth) {
    const int len = rp[r + 1] - rp[r];
    if (len <= thresh) {
      red[0] += len;
      red[1] += 1.0;
    }
  }
  block_reduce<2, 0u>(red, sm);
  const double sn = sm[32 * kMaxRed], sc = sm[32 * kMaxRed + 1];
  __syncthreads();
  if (thresh > kMaxBins) {
    if (tid == 0) atomicExch(sp.err, kNaNoRoom);
    __syncthreads();
    return false;
  }
  const double ms = sc > 0 ? sn / sc : 1.0;
  // same width rule as the host schedule builder of osqp_setup
  int g_mean = 1;
  while (g_mean < 32 && (double)g_mean < ms) g_mean <<= 1;
  int g_min = 1;
  while (g_min < 32 && (double)g_min * 16.0 < ms) g_min <<= 1;
  int g_occ = 1;
  const long long nshort_ll = (long long)sc, nwarps = nw;
  while (g_occ < 32 && (long long)(g_occ * 2) * nshort_ll <= 32LL * nwarps) g_occ <<= 1;
  const int G = max(g_min, min(g_mean, g_occ));
  const int spw = 32 / G;
  const int nshort = (int)sc;
  // counting sort of the short rows by decreasing length, stable in the row
  // index: bin starts from a scan of the counts taken longest first
  const int nb = thresh + 1;
  for (int i = tid; i < nb; i += nth) sp.bin_cnt[i] = 0;
  __syncthreads();
  for (int r = tid; r < nrows; r += nth) {
    const int len = rp[r + 1] - rp[r];
    if (len <= thresh) atomicAdd(&sp.bin_cnt[len], 1);
  }
  __syncthreads();
  for (int i = tid; i < nb; i += nth) sp.bin_rev[i] = sp.bin_cnt[thresh - i];
  __syncthreads();
  block_exclusive_scan(sp.bin_rev, sp.bin_start, nb, sh_int);
  for (int i = tid; i < nb; i += nth) sp.bin_cnt[i] = 0;
  __syncthreads();
  // rows in index order, one CTA-wide chunk at a time; within a chunk the
  // warps take their turn so that equal lengths keep their index order
  for (int r0 = 0; r0 < nrows; r0 += nth) {
    const int r = r0 + tid;
    int len = -1;
    if (r < nrows) {
      const int l = rp[r + 1] - rp[r];
      if (l <= thresh) len = l;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, len);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const bool leader = (__ffs(peers) - 1) == lane;
    for (int w = 0; w < nw; ++w) {
      if (wid == w) {
        int at = 0;
        if (len >= 0) at = sp.bin_start[thresh - len] + sp.bin_cnt[len] + rank;
        __syncwarp();
        if (len >= 0) {
          if (leader) sp.bin_cnt[len] += __popc(peers);
          B.order[at] = r;
        }
      }
      __syncthreads();
    }
  }
  // slices: widths from their first (longest) row, starts by a scan
  const int nsl = (nshort + spw - 1) / spw;
  for (int q = tid; q < nsl; q += nth) {
    const int r = B.order[q * spw];
    sp.wsum[q] = 32 * ((rp[r + 1] - rp[r] + G - 1) / G);
  }
  __syncthreads();
  block_exclusive_scan(sp.wsum, sp.wsum, nsl, sh_int);
  for (int q = tid; q < nsl; q += nth)
    B.slices[q] = make_int2(sp.wsum[q], (sp.wsum[q + 1] - sp.wsum[q]) / 32);
  for (int q = tid; q < nsl * spw; q += nth) B.srow[q] = q < nshort ? B.order[q] : -1;
  for (int r = tid; r < nrows; r += nth) B.lidx[r] = -1;
  __syncthreads();
  // long rows in row order after the slices, with their chunks (few long
  // rows: one thread), then the sliced arrays
  if (tid == 0) {
    int nl = 0, nc = 0, p = sp.wsum[nsl];
    for (int r = 0; r < nrows; ++r) {
      const int b = rp[r], e = rp[r + 1];
      if (e - b <= thresh) continue;
      B.long_rows[nl] = r;
      B.lpos[nl] = p;
      B.ccount[nl] = 0u;
      B.lidx[r] = nl;
      const int c0 = nc;
      for (int k = b; k < e; k += kChunk)
        B.chunks[nc++] = make_int4(r, p + (k - b), p + (min(k + kChunk, e) - b), nl);
      B.lrange[nl] = make_int2(c0, nc - c0);
      ++nl;
      p += e - b;
    }
    const size_t np = p;
    size_t off = (sp.dyn + 255) & ~(size_t)255;
    const size_t at_ci = off;
    off = (off + (np ? np : 1) * sizeof(int) + 255) & ~(size_t)255;
    const size_t at_raw = off;
    off = (off + (np ? np : 1) * sizeof(double) + 255) & ~(size_t)255;
    const size_t at_v = off;
    off += (np ? np : 1) * sizeof(T);
    if (off > kNoallocScratchBytes) {
      atomicExch(sp.err, kNaNoRoom);
    } else {
      sp.dyn = off;
      *ci_out = (const int*)(base + at_ci);
      *raw_out = (const double*)(base + at_raw);
      *v_out = (T*)(base + at_v);
      S.nrows = nrows;
      S.group = G;
      S.long_thresh = thresh;
      S.nlong = nl;
      S.nchunks = nc;
      S.nslices = nsl;
      S.slices = B.slices;
      S.srow = B.srow;
      S.chunks = B.chunks;
      S.long_rows = B.long_rows;
      S.lrange = B.lrange;
      S.lidx = B.lidx;
      S.cpart = B.cpart;
      S.ccount = B.ccount;
      S.npos = p;
    }
  }
  __syncthreads();
  if (*(volatile int*)sp.err != kNaOk) return false;
  int* ci = (int*)*ci_out;
  double* raw = (double*)*raw_out;
  const int pshort = sp.wsum[nsl];
  for (int q = tid; q < pshort; q += nth) {
    ci[q] = -1;
    raw[q] = 0.0;
  }
  __syncthreads();
  for (int q = tid; q < nshort; q += nth) {
    const int r = B.order[q], s0 = sp.wsum[q / spw], rr = q % spw;
    for (int j = 0; j < rp[r + 1] - rp[r]; ++j) {
      const int at = s0 + 32 * (j / G) + rr * G + j % G;
      ci[at] = B.cci[rp[r] + j];
      raw[at] = B.craw[rp[r] + j];
    }
  }
  for (int q = wid; q < S.nlong; q += nw) {
    const int r = B.long_rows[q], b = rp[r], p0 = B.lpos[q];
    for (int j = lane; j < rp[r + 1] - b; j += 32) {
      ci[p0 + j] = B.cci[b + j];
      raw[p0 + j] = B.craw[b + j];
    }
  }
  __syncthreads();
  return true;
}

// Column of CSC entry k (binary search in colptr).
__device__ __forceinline__ int col_of(const int* cp, int ncols, int k) {
  int lo = 0, hi = ncols;  // cp[lo] <= k < cp[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (cp[mid] <= k) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_noalloc(NaInput in, const __grid_constant__ Params P,
                                                       double rho0, char* scratch) {
  __shared__ double sm[kSmemDoubles];
  __shared__ NaPtrs<T> sp;
  __shared__ int sh_int[40];
  if (threadIdx.x == 0) na_carve<T>(in, scratch, &sp);
  __syncthreads();
  Dev<T>& d = sp.d;
  const int n = in.n, m = in.m, tid = threadIdx.x, nth = blockDim.x;
  if (tid == 0) {
    sp.err[0] = kNaOk;
    *d.sc = Scalars{};
  }
  for (int j = tid; j < n; j += nth) {
    sp.plen[j] = 0;
  }
  for (int i = tid; i < m; i += nth) sp.alen[i] = 0;
  __syncthreads();
  // --- validate the CSC input (bounds, order, upper triangle of P)
  for (int j = tid; j < n; j += nth) {
    const int b = in.Pp[j], e = in.Pp[j + 1];
    if (b > e || b < 0 || e > in.nnzP) atomicExch(sp.err, kNaBadCsc);
    const int ba = in.Ap[j], ea = in.Ap[j + 1];
    if (ba > ea || ba < 0 || ea > in.nnzA) atomicExch(sp.err, kNaBadCsc);
  }
  if (tid == 0 && (in.Pp[0] != 0 || in.Pp[n] != in.nnzP || in.Ap[0] != 0 || in.Ap[n] != in.nnzA))
    atomicExch(sp.err, kNaBadCsc);
  __syncthreads();
  if (*(volatile int*)sp.err != kNaOk) {
    if (tid == 0) d.sc->dev_error = sp.err[0];
    return;
  }
  for (int k = tid; k < in.nnzP; k += nth) {
    const int j = col_of(in.Pp, n, k), i = in.Pi[k];
    if (i < 0 || i > j || (k > in.Pp[j] && in.Pi[k - 1] >= i)) atomicExch(sp.err, kNaBadCsc);
  }
  for (int k = tid; k < in.nnzA; k += nth) {
    const int j = col_of(in.Ap, n, k), i = in.Ai[k];
    if (i < 0 || i >= m || (k > in.Ap[j] && in.Ai[k - 1] >= i)) atomicExch(sp.err, kNaBadCsc);
  }
  __syncthreads();
  if (*(volatile int*)sp.err != kNaOk) {
    if (tid == 0) d.sc->dev_error = sp.err[0];
    return;
  }
  // --- values, as osqp_setup checks them: P, A and q finite, l and u not
  // NaN, l ≤ u (bit 0: a non-finite value, bit 1: some l_i > u_i; the
  // non-finite report takes precedence, as on the host)
  if (tid == 0) *sp.flag = 0;
  __syncthreads();
  {
    int bad = 0;
    for (int k = tid; k < in.nnzP; k += nth)
      if (!isfinite(in.Px[k])) bad |= 1;
    for (int k = tid; k < in.nnzA; k += nth)
      if (!isfinite(in.Ax[k])) bad |= 1;
    for (int j = tid; j < n; j += nth)
      if (!isfinite(in.q[j])) bad |= 1;
    for (int i = tid; i < m; i += nth) {
      const double lo = in.l[i], hi = in.u[i];
      if (isnan(lo) || isnan(hi)) bad |= 1;
      else if (lo > hi) bad |= 2;
    }
    if (bad) atomicOr(sp.flag, bad);
  }
  __syncthreads();
  if (*(volatile int*)sp.flag != 0) {
    if (tid == 0) d.sc->dev_error = (*sp.flag & 1) ? kNaNonFinite : kNaLgtU;
    return;
  }
  // --- Kn = [P̄ Āᵀ] rows: full-P part by counting + atomic scatter + rank sort
  for (int k = tid; k < in.nnzP; k += nth) {
    const int j = col_of(in.Pp, n, k), i = in.Pi[k];
    atomicAdd(&sp.plen[i], 1);
    if (i != j) atomicAdd(&sp.plen[j], 1);
  }
  __syncthreads();
  for (int j = tid; j < n; j += nth) sp.cur_n[j] = sp.plen[j] + (in.Ap[j + 1] - in.Ap[j]);
  __syncthreads();
  block_exclusive_scan(sp.cur_n, sp.kn.rp, n, sh_int);
  for (int j = tid; j < n; j += nth) {
    sp.cur_n[j] = sp.kn.rp[j];
    if (sp.kn.rp[j + 1] - sp.kn.rp[j] > kNoallocMaxRow) atomicExch(sp.err, kNaLongRow);
  }
  __syncthreads();
  for (int k = tid; k < in.nnzP; k += nth) {
    const int j = col_of(in.Pp, n, k), i = in.Pi[k];
    int pos = atomicAdd(&sp.cur_n[i], 1);
    sp.tmp_ci[pos] = j;
    sp.tmp_raw[pos] = in.Px[k];
    if (i != j) {
      pos = atomicAdd(&sp.cur_n[j], 1);
      sp.tmp_ci[pos] = i;
      sp.tmp_raw[pos] = in.Px[k];
    }
  }
  for (int k = tid; k < in.nnzA; k += nth) {
    const int j = col_of(in.Ap, n, k);
    const int pos = sp.kn.rp[j] + sp.plen[j] + (k - in.Ap[j]);
    sp.kn.cci[pos] = n + in.Ai[k];
    sp.kn.craw[pos] = in.Ax[k];
  }
  __syncthreads();
  if (*(volatile int*)sp.err != kNaOk) {
    if (tid == 0) d.sc->dev_error = sp.err[0];
    return;
  }
  // rank sort of each row's P part by column (unique columns → unique order)
  for (int e = tid; e < sp.kn.rp[n]; e += nth) {
    const int r = col_of(sp.kn.rp, n, e);
    const int b = sp.kn.rp[r], len = sp.plen[r];
    if (e - b >= len) continue;
    const int c = sp.tmp_ci[e];
    int rank = 0;
    for (int f = b; f < b + len; ++f) rank += sp.tmp_ci[f] < c;
    sp.kn.cci[b + rank] = c;
    sp.kn.craw[b + rank] = sp.tmp_raw[e];
  }
  __syncthreads();
  // --- Ā rows: counting + atomic scatter + rank sort
  for (int k = tid; k < in.nnzA; k += nth) atomicAdd(&sp.alen[in.Ai[k]], 1);
  __syncthreads();
  block_exclusive_scan(sp.alen, sp.a.rp, m, sh_int);
  for (int i = tid; i < m; i += nth) {
    sp.cur_m[i] = sp.a.rp[i];
    if (sp.alen[i] > kNoallocMaxRow) atomicExch(sp.err, kNaLongRow);
  }
  __syncthreads();
  if (*(volatile int*)sp.err != kNaOk) {
    if (tid == 0) d.sc->dev_error = sp.err[0];
    return;
  }
  for (int k = tid; k < in.nnzA; k += nth) {
    const int j = col_of(in.Ap, n, k);
    const int pos = atomicAdd(&sp.cur_m[in.Ai[k]], 1);
    sp.tmp_ci[pos] = j;
    sp.tmp_raw[pos] = in.Ax[k];
  }
  __syncthreads();
  for (int e = tid; e < in.nnzA; e += nth) {
    const int r = col_of(sp.a.rp, m, e);
    const int b = sp.a.rp[r], len = sp.a.rp[r + 1] - b;
    const int c = sp.tmp_ci[e];
    int rank = 0;
    for (int f = b; f < b + len; ++f) rank += sp.tmp_ci[f] < c;
    sp.a.cci[b + rank] = c;
    sp.a.craw[b + rank] = sp.tmp_raw[e];
  }
  __syncthreads();
  // --- sliced layouts, then the same stages as the one-CTA solver
  if (tid == 0) sp.dyn = sp.fixed_end;
  __syncthreads();
  if (!build_sliced(d.kn, sp.kn, sp, n, scratch, &d.kn_ci, &d.kn_raw, &d.kn_v, sh_int, sm) ||
      !build_sliced(d.as, sp.a, sp, m, scratch, &d.a_ci, &d.a_raw, &d.a_v, sh_int, sm)) {
    if (tid == 0) d.sc->dev_error = sp.err[0];
    return;
  }
  BlockTeam tm{sm};
  if (!scale_stage(tm, d, P, rho0, true)) return;
  admm_stage(tm, d, P);
}

void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Per-device address of the scratch array (host code must not use the
// symbol's name as an address).
int scratch_address(char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OSQP_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return OSQP_ERR_LIMIT;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return OSQP_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = (char*)g_scratch_ptr[dev];
  return OSQP_OK;
}

// Status of the last solve in the work array for a problem of these sizes:
// the Scalars sit at a fixed offset of its layout.  Waits for the stream.
int read_info(const NaInput& in, int precision, char* base, cudaStream_t st, osqp_info* info) {
  Scalars sc;
  NaPtrs<double> probe64;
  NaPtrs<float> probe32;
  const Scalars* dsc = precision == OSQP_PRECISION_FP64
                           ? (na_carve<double>(in, base, &probe64), probe64.d.sc)
                           : (na_carve<float>(in, base, &probe32), probe32.d.sc);
  if (cudaMemcpyAsync(&sc, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return OSQP_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return OSQP_ERR_CUDA;
  if (sc.dev_error == kNaBadCsc) return OSQP_ERR_CSC;
  if (sc.dev_error == kNaLongRow || sc.dev_error == kNaNoRoom) return OSQP_ERR_LIMIT;
  if (sc.dev_error == kNaNonFinite) return OSQP_ERR_NONFINITE;
  if (sc.dev_error == kNaLgtU) return OSQP_ERR_LGTU;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = sc.status;
    info->iter = sc.iter;
    info->pcg_iters = sc.pcg_iters;
    info->rho_updates = sc.rho_updates;
    info->ruiz_passes = sc.ruiz_passes;
    info->launch = 1;
    info->obj_val = sc.obj;
    info->prim_res = sc.prim_res;
    info->dual_res = sc.dual_res;
    info->rho_estimate = sc.rho_bar;
    info->polished = sc.polished;
  }
  return OSQP_OK;
}

}  // namespace

extern "C" int32_t osqp_solve_noalloc(int32_t n, int32_t m, const int32_t* P_colptr,
                                      const int32_t* P_rowind, const double* P_val, int32_t P_nnz,
                                      const double* q, const int32_t* A_colptr,
                                      const int32_t* A_rowind, const double* A_val, int32_t A_nnz,
                                      const double* l, const double* u,
                                      const osqp_settings* settings, double* x, double* y,
                                      osqp_info* info, void* stream) {
  if (!settings || !P_colptr || !q || !A_colptr || !x) return OSQP_ERR_ARG;
  if (n < 1 || m < 0 || P_nnz < 0 || A_nnz < 0) return OSQP_ERR_DIMS;
  if ((P_nnz && (!P_rowind || !P_val)) || (A_nnz && (!A_rowind || !A_val))) return OSQP_ERR_ARG;
  if (m > 0 && (!l || !u || !y)) return OSQP_ERR_ARG;
  const osqp_settings& s = *settings;
  if (!(s.rho > 0) || !(s.sigma > 0) || !(s.alpha > 0 && s.alpha < 2) || s.max_iter < 0 ||
      s.check_interval < 1 || s.scaling_iters < 0 || s.pcg_max_iter < 1 ||
      !(s.eps_abs >= 0) || !(s.eps_rel >= 0) || !(s.eps_pinf > 0) || !(s.eps_dinf > 0) ||
      !(s.adaptive_rho_tolerance >= 1) || !(s.pcg_tol_fraction >= 0) || !(s.pcg_tol_floor >= 0) ||
      (s.precision != OSQP_PRECISION_FP64 && s.precision != OSQP_PRECISION_FP32_MIXED) ||
      s.polish < 0 || s.polish > 1 || s.polish_refine_iter < 0 || !(s.delta > 0))
    return OSQP_ERR_SETTINGS;
  NaInput in{n, m, P_nnz, A_nnz, P_colptr, P_rowind, P_val, q, A_colptr, A_rowind, A_val,
             l, u, x, y};
  // fixed part plus the smallest sliced arrays (no padding); the kernel
  // checks the exact layout
  const size_t nkn_min = (size_t)P_nnz + A_nnz, na_min = A_nnz;
  const size_t need = s.precision == OSQP_PRECISION_FP64
                          ? na_carve<double>(in, nullptr, nullptr) + sliced_bytes<double>(nkn_min) +
                                sliced_bytes<double>(na_min) + 512
                          : na_carve<float>(in, nullptr, nullptr) + sliced_bytes<float>(nkn_min) +
                                sliced_bytes<float>(na_min) + 512;
  if (need > kNoallocScratchBytes) return OSQP_ERR_LIMIT;
  cudaStream_t st = (cudaStream_t)stream;
  // Inside a stream capture nothing may wait: the call only enqueues the
  // solve, and osqp_noalloc_get_info reads its status after a replay.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return OSQP_ERR_CUDA;
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  if (capturing && info) return OSQP_ERR_ARG;
  char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  Params P;
  std::memset(&P, 0, sizeof(P));
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
  P.pcg_reduce = s.precision == OSQP_PRECISION_FP32_MIXED ? 1e-5 : 0.0;
  P.time_limit_ns = s.time_limit > 0 ? s.time_limit * 1e9 : 0.0;
  P.max_iter = s.max_iter;
  P.check_interval = s.check_interval;
  P.adaptive_rho = s.adaptive_rho;
  P.scaling_iters = s.scaling_iters;
  P.max_rho_updates = s.max_rho_updates;
  P.pcg_max_iter = s.pcg_max_iter;
  P.barrier_timeout_ns = 0;  // the one-CTA team waits on no grid or cluster barrier
  P.polish = s.polish;
  P.polish_refine = s.polish_refine_iter;
  P.delta = s.delta;
  if (s.precision == OSQP_PRECISION_FP64)
    k_noalloc<double><<<1, kThreads, 0, st>>>(in, P, s.rho, base);
  else
    k_noalloc<float><<<1, kThreads, 0, st>>>(in, P, s.rho, base);
  if (cudaGetLastError() != cudaSuccess) return OSQP_ERR_CUDA;
  if (capturing) return OSQP_OK;
  return read_info(in, s.precision, base, st, info);
}

extern "C" int32_t osqp_noalloc_get_info(int32_t n, int32_t m, int32_t P_nnz, int32_t A_nnz,
                                         int32_t precision, osqp_info* info, void* stream) {
  if (!info) return OSQP_ERR_ARG;
  if (n < 1 || m < 0 || P_nnz < 0 || A_nnz < 0) return OSQP_ERR_DIMS;
  if (precision != OSQP_PRECISION_FP64 && precision != OSQP_PRECISION_FP32_MIXED)
    return OSQP_ERR_SETTINGS;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return OSQP_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return OSQP_ERR_ARG;
  char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  NaInput in{n, m, P_nnz, A_nnz, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
             nullptr, nullptr, nullptr, nullptr};
  return read_info(in, precision, base, st, info);
}
