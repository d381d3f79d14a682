// Passes over the input CSR (degrees, the two SpMV chains, validation), the
// degree ordering, the oriented graph, scans and the epilogue.
//
// Rows of the input CSR are processed by 8-lane groups when their degree is at
// most HEAVY_DEGREE and by a whole block otherwise (degree-binned scheduling:
// power-law graphs have a few rows with 10^4-10^6 entries next to millions of
// rows with a handful).
#include <algorithm>

#include "fglt_device.cuh"
#include "fglt_kernels.h"

namespace fglt {

thread_local int64_t g_launches = 0;

namespace {

constexpr int G = 8;          // lanes per light row
constexpr int ROW_BLOCK = 256;

template <typename RP>
__device__ __forceinline__ int64_t ld_rp(const RP* rp, int64_t i) {
  return (int64_t)__ldg(rp + i);
}

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int64_t light_blocks(int64_t n) {
  int64_t want = (n * G + ROW_BLOCK - 1) / ROW_BLOCK;
  int64_t cap = (int64_t)num_sms() * 16;
  if (want < 1) want = 1;
  return want < cap ? want : cap;
}

// ---------------------------------------------------------------------------
// Generic row kernels. Op supplies
//   edge(v, j, k, s, e, a, b): one entry j = colidx[k] of row v = [s, e)
//   done(v, a, b): the row's reductions
// ---------------------------------------------------------------------------
template <typename RP, typename Op>
__global__ void __launch_bounds__(ROW_BLOCK) k_rows_light(const RP* __restrict__ rp,
                                                          const int32_t* __restrict__ ci, int64_t n, Op op) {
  const int lane = threadIdx.x & (G - 1);
  const unsigned gmask = 0xFFu << ((threadIdx.x & 31) & ~(G - 1));
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; v < n; v += stride) {
    const int64_t s = ld_rp(rp, v), e = ld_rp(rp, v + 1);
    if (e - s > HEAVY_DEGREE) continue;
    long long a = 0, b = 0;
    for (int64_t k = s + lane; k < e; k += G) op.edge(v, __ldg(ci + k), k, s, e, a, b);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      a += __shfl_xor_sync(gmask, a, o, G);
      b += __shfl_xor_sync(gmask, b, o, G);
    }
    if (lane == 0) op.done(v, a, b);
  }
}

template <typename RP, typename Op>
__global__ void __launch_bounds__(ROW_BLOCK) k_rows_heavy(const RP* __restrict__ rp,
                                                          const int32_t* __restrict__ ci,
                                                          const int32_t* __restrict__ heavy,
                                                          const int32_t* __restrict__ nheavy, Op op) {
  __shared__ long long red[32];
  const int nh = *nheavy;
  for (int h = blockIdx.x; h < nh; h += gridDim.x) {
    const int64_t v = heavy[h];
    const int64_t s = ld_rp(rp, v), e = ld_rp(rp, v + 1);
    long long a = 0, b = 0;
    for (int64_t k = s + threadIdx.x; k < e; k += blockDim.x) op.edge(v, __ldg(ci + k), k, s, e, a, b);
    a = block_sum(a, red);
    b = block_sum(b, red);
    if (threadIdx.x == 0) op.done(v, a, b);
  }
}

template <typename RP, typename Op>
cudaError_t run_rows(const Csr& g, const int32_t* heavy, const int32_t* nheavy, int64_t heavy_cap, Op op,
                     cudaStream_t st) {
  const RP* rp = static_cast<const RP*>(g.rowptr);
  if (g.n <= 0) return cudaSuccess;
  k_rows_light<RP, Op><<<(unsigned)light_blocks(g.n), ROW_BLOCK, 0, st>>>(rp, g.colidx, g.n, op);
  note_launch();
  if (heavy_cap > 0) {
    int64_t hb = heavy_cap < (int64_t)num_sms() * 4 ? heavy_cap : (int64_t)num_sms() * 4;
    if (hb < 1) hb = 1;
    k_rows_heavy<RP, Op><<<(unsigned)hb, ROW_BLOCK, 0, st>>>(rp, g.colidx, heavy, nheavy, op);
    note_launch();
  }
  return cudaGetLastError();
}

template <typename Op>
cudaError_t dispatch_rows(const Csr& g, const int32_t* heavy, const int32_t* nheavy, int64_t heavy_cap,
                          Op op, cudaStream_t st) {
  return g.rp64 ? run_rows<int64_t>(g, heavy, nheavy, heavy_cap, op, st)
                : run_rows<int32_t>(g, heavy, nheavy, heavy_cap, op, st);
}

// --- row operations ----------------------------------------------------------

struct Spmv1Op {  // p2 = A p1 - p1 (eq. p2), d^7 = A((p1-1) o (p1-2)) / 2
  const int32_t* d;
  int64_t* p2;
  int64_t* r7;
  int64_t n;
  int* err;
  __device__ __forceinline__ void edge(int64_t, int32_t j, int64_t, int64_t, int64_t, long long& a,
                                       long long& b) const {
    if ((uint32_t)j >= (uint64_t)n) {
      atomicOr(err, ERR_BAD_GRAPH);
      return;
    }
    const long long dj = __ldg(d + j);
    a += dj;
    b += (dj - 1) * (dj - 2) / 2;
  }
  __device__ __forceinline__ void done(int64_t v, long long a, long long b) const {
    p2[v] = a - __ldg(d + v);
    r7[v] = b;
  }
};

struct Spmv2Op {  // p3 = A p2 - p1 o (p1-1) - 2 c3, d^9 = A c3 - 2 c3
  const int32_t* d;
  const int64_t* p2;
  const int64_t* c3o;
  int64_t* p3;
  int64_t* r9;
  int64_t n;
  __device__ __forceinline__ void edge(int64_t, int32_t j, int64_t, int64_t, int64_t, long long& a,
                                       long long& b) const {
    if ((uint32_t)j >= (uint64_t)n) return;
    a += __ldg(p2 + j);
    b += __ldg(c3o + j);
  }
  __device__ __forceinline__ void done(int64_t v, long long a, long long b) const {
    const long long dv = __ldg(d + v), c = __ldg(c3o + v);
    p3[v] = a - dv * (dv - 1) - 2 * c;
    r9[v] = b - 2 * c;
  }
};

struct OrientCountOp {  // out-degree in the degree-ordered orientation
  const int32_t* rank;
  int32_t* opc;
  int32_t* dpmax;
  int64_t n;
  __device__ __forceinline__ void edge(int64_t v, int32_t j, int64_t, int64_t, int64_t, long long& a,
                                       long long&) const {
    if ((uint32_t)j >= (uint64_t)n) return;
    a += __ldg(rank + j) > __ldg(rank + v);
  }
  __device__ __forceinline__ void done(int64_t v, long long a, long long) const {
    opc[__ldg(rank + v)] = (int32_t)a;
    atomicMax(dpmax, (int32_t)a);
  }
};

struct OrientFillOp {  // appends rank(j) to the oriented row of rank(v)
  const int32_t* rank;
  const int64_t* orp;
  int32_t* cursor;
  int32_t* ocol;
  int64_t n;
  __device__ __forceinline__ void edge(int64_t v, int32_t j, int64_t, int64_t, int64_t, long long&,
                                       long long&) const {
    if ((uint32_t)j >= (uint64_t)n) return;
    const int32_t rv = __ldg(rank + v), rj = __ldg(rank + j);
    if (rj > rv) {
      const int64_t base = orp[rv];
      const int32_t pos = atomicAdd(cursor + rv, 1);
      if (base + pos < orp[rv + 1]) ocol[base + pos] = rj;
    }
  }
  __device__ __forceinline__ void done(int64_t, long long, long long) const {}
};

template <typename RP>
struct ValidateOp {  // simple, symmetric, strictly increasing rows
  const RP* rp;
  const int32_t* ci;
  int64_t n;
  int* err;
  __device__ __forceinline__ void edge(int64_t v, int32_t j, int64_t k, int64_t s, int64_t, long long&,
                                       long long&) const {
    bool bad = (j < 0) || ((int64_t)j >= n) || ((int64_t)j == v);
    if (!bad && k > s && __ldg(ci + k - 1) >= j) bad = true;
    if (!bad) {
      int64_t lo = ld_rp(rp, j), hi = ld_rp(rp, j + 1);
      bool found = false;
      while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        int32_t x = __ldg(ci + mid);
        if (x == (int32_t)v) { found = true; break; }
        if (x < (int32_t)v) lo = mid + 1; else hi = mid;
      }
      bad = !found;
    }
    if (bad) atomicOr(err, ERR_BAD_GRAPH);
  }
  __device__ __forceinline__ void done(int64_t, long long, long long) const {}
};

// Batched inputs: every neighbour of v lies in v's own graph [off[g], off[g+1]).
template <typename RP>
__global__ void k_validate_batch(const RP* __restrict__ rp, const int32_t* __restrict__ ci, int64_t n,
                                 const int64_t* __restrict__ off, int64_t num_graphs, int* err) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = num_graphs - 1;  // last g with off[g] <= v
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (off[mid] <= v) lo = mid; else hi = mid - 1;
    }
    const int64_t a = off[lo], b = off[lo + 1];
    bool bad = false;
    for (int64_t k = ld_rp(rp, v); k < ld_rp(rp, v + 1); ++k) {
      const int64_t j = __ldg(ci + k);
      bad |= (j < a) || (j >= b);
    }
    if (bad) atomicOr(err, ERR_BAD_GRAPH);
  }
}

// ---------------------------------------------------------------------------
// Degrees
// ---------------------------------------------------------------------------
template <typename RP>
__global__ void k_degree(const RP* __restrict__ rp, int64_t n, int64_t nnz, int32_t* d, int32_t* dmax,
                         int32_t* heavy, int32_t* nheavy, int64_t heavy_cap, int32_t dcap, int* err) {
  int local_max = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = ld_rp(rp, v), hi = ld_rp(rp, v + 1);
    int64_t dv = hi - lo;
    if (lo < 0 || hi > nnz || dv < 0 || dv > 0x7fffffff || (v == 0 && lo != 0)) {
      atomicOr(err, ERR_BAD_ROWPTR);
      dv = 0;
    }
    if (dv > dcap) {  // above the caller's bound (batched inputs): flag it and clamp
      atomicOr(err, ERR_BAD_GRAPH);
      dv = dcap;
    }
    const int32_t dd = (int32_t)dv;
    d[v] = dd;
    local_max = max(local_max, dd);
    if (dd > HEAVY_DEGREE) {
      int h = atomicAdd(nheavy, 1);
      if (h < heavy_cap) heavy[h] = (int32_t)v;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dmax, local_max);
}

// ---------------------------------------------------------------------------
// Degree ordering: a counting sort of the vertices by degree. rank(v) is the
// position of v in non-decreasing degree order (ties in any order); the
// oriented graph keeps the edge v -> u iff rank(v) < rank(u).
// ---------------------------------------------------------------------------
constexpr int SMALL_BINS = 1024;

__global__ void k_degree_hist(const int32_t* __restrict__ d, int64_t n, int32_t* hist) {
  __shared__ int32_t h[SMALL_BINS];
  for (int i = threadIdx.x; i < SMALL_BINS; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t dv = d[v];
    if (dv < SMALL_BINS) atomicAdd(&h[dv], 1);
    else atomicAdd(&hist[dv], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < SMALL_BINS; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

constexpr int RANK_T = 256, RANK_I = 8;

__global__ void __launch_bounds__(RANK_T) k_rank_assign(const int32_t* __restrict__ d, int64_t n,
                                                        const int64_t* __restrict__ base, int32_t* cursor,
                                                        int32_t* rank, int32_t* perm, int32_t* dr) {
  __shared__ int32_t cnt[SMALL_BINS];
  __shared__ int32_t off[SMALL_BINS];
  const int64_t chunk = (int64_t)RANK_T * RANK_I;
  for (int64_t c0 = (int64_t)blockIdx.x * chunk; c0 < n; c0 += (int64_t)gridDim.x * chunk) {
    for (int i = threadIdx.x; i < SMALL_BINS; i += RANK_T) cnt[i] = 0;
    __syncthreads();
    int32_t dv[RANK_I], loc[RANK_I];
#pragma unroll
    for (int t = 0; t < RANK_I; ++t) {
      const int64_t v = c0 + (int64_t)t * RANK_T + threadIdx.x;
      dv[t] = v < n ? d[v] : -1;
      loc[t] = (dv[t] >= 0 && dv[t] < SMALL_BINS) ? atomicAdd(&cnt[dv[t]], 1) : 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SMALL_BINS; i += RANK_T)
      if (cnt[i]) off[i] = atomicAdd(&cursor[i], cnt[i]);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < RANK_I; ++t) {
      const int64_t v = c0 + (int64_t)t * RANK_T + threadIdx.x;
      if (dv[t] < 0) continue;
      int64_t r;
      if (dv[t] < SMALL_BINS) r = base[dv[t]] + off[dv[t]] + loc[t];
      else r = base[dv[t]] + atomicAdd(&cursor[dv[t]], 1);
      rank[v] = (int32_t)r;
      perm[r] = (int32_t)v;
      dr[r] = dv[t];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Row sort of the oriented graph (ascending rank labels): bitonic networks in
// registers (rows of at most 32), shared memory (at most 16384) or global
// scratch (longer rows).
// ---------------------------------------------------------------------------
__global__ void k_sort_rows_warp(const int64_t* __restrict__ orp, int64_t n, int32_t* ocol) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    const int64_t b = orp[r];
    const int L = (int)(orp[r + 1] - b);
    if (L < 2 || L > 32) continue;
    int32_t x = lane < L ? ocol[b + lane] : 0x7fffffff;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const int32_t y = __shfl_xor_sync(0xffffffffu, x, j);
        const bool keep_min = ((lane & k) == 0) == ((lane & j) == 0);
        x = keep_min ? min(x, y) : max(x, y);
      }
    }
    if (lane < L) ocol[b + lane] = x;
  }
}

__device__ void bitonic_block(int32_t* buf, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int32_t a = buf[i], b = buf[ixj];
          const bool asc = (i & k) == 0;
          if ((a > b) == asc) { buf[i] = b; buf[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
}

constexpr int SORT_SMEM_MAX = 16384;

constexpr int SORT_BLOCK_T = 256;

// Rows of 33 .. SORT_SMEM_MAX entries, one block per row in shared memory.
// Block b owns rows b, b + grid, b + 2 grid, ... (rows of similar length sit
// together in rank order, so interleaving spreads them over the blocks); its
// threads test SORT_BLOCK_T of its rows at once, then it sorts the ones in
// range one after the other.
__global__ void __launch_bounds__(SORT_BLOCK_T) k_sort_rows_block(const int64_t* __restrict__ orp, int64_t n,
                                                                   int32_t* ocol) {
  extern __shared__ int32_t sbuf[];
  __shared__ int64_t rows[SORT_BLOCK_T];
  __shared__ int nrows;
  const int64_t G = gridDim.x;
  for (int64_t k0 = 0; (int64_t)blockIdx.x + k0 * G < n; k0 += SORT_BLOCK_T) {
    if (threadIdx.x == 0) nrows = 0;
    __syncthreads();
    const int64_t rr = (int64_t)blockIdx.x + (k0 + threadIdx.x) * G;
    if (rr < n) {
      const int64_t L = orp[rr + 1] - orp[rr];
      if (L > 32 && L <= SORT_SMEM_MAX) rows[atomicAdd(&nrows, 1)] = rr;
    }
    __syncthreads();
    const int count = nrows;
    for (int q = 0; q < count; ++q) {
      const int64_t r = rows[q];
      const int64_t b = orp[r];
      const int L = (int)(orp[r + 1] - b);
      int P = 64;
      while (P < L) P <<= 1;
      for (int i = threadIdx.x; i < P; i += blockDim.x) sbuf[i] = i < L ? ocol[b + i] : 0x7fffffff;
      __syncthreads();
      bitonic_block(sbuf, P);
      for (int i = threadIdx.x; i < L; i += blockDim.x) ocol[b + i] = sbuf[i];
      __syncthreads();
    }
  }
}

// Rows longer than the shared-memory sort holds, listed (at most cap of
// them; list[-1] is the count).
__global__ void k_long_rows(const int64_t* __restrict__ orp, int64_t n, int32_t* list, int64_t cap) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); r0 < n; r0 += stride) {
    const int64_t r = r0 + lane;
    const bool take = r < n && orp[r + 1] - orp[r] > SORT_SMEM_MAX;
    const unsigned m = __ballot_sync(0xffffffffu, take);
    int pos0 = 0;
    if (lane == 0 && m) pos0 = atomicAdd(list - 1, __popc(m));
    pos0 = __shfl_sync(0xffffffffu, pos0, 0);
    const int64_t pos = (int64_t)pos0 + __popc(m & ((1u << lane) - 1));
    if (take && pos < cap) list[pos] = (int32_t)r;
  }
}

// One listed row per block at a time, bitonic-sorted in the block's own
// power-of-two slot of scratch (P int32 per slot).
__global__ void k_sort_rows_global(const int64_t* __restrict__ orp, const int32_t* __restrict__ list, int64_t cap,
                                   int32_t* ocol, int32_t* scratch, int P) {
  int32_t* slot = scratch + (size_t)blockIdx.x * P;
  const int64_t count = min((int64_t)list[-1], cap);
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int64_t r = list[i];
    const int64_t b = orp[r];
    const int64_t L = orp[r + 1] - b;
    int Q = SORT_SMEM_MAX;
    while (Q < L) Q <<= 1;  // L <= the longest row, so Q <= P
    for (int j = threadIdx.x; j < Q; j += blockDim.x) slot[j] = j < L ? ocol[b + j] : 0x7fffffff;
    __syncthreads();
    bitonic_block(slot, Q);
    for (int j = threadIdx.x; j < L; j += blockDim.x) ocol[b + j] = slot[j];
    __syncthreads();
  }
}

__global__ void k_worklist_outdeg(const int32_t* __restrict__ opc, int64_t n, int min_out, int32_t* list,
                                  int32_t* count) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); r0 < n; r0 += stride) {
    const int64_t r = r0 + lane;
    const bool take = r < n && opc[r] >= min_out;
    const unsigned m = __ballot_sync(0xffffffffu, take);
    int pos0 = 0;
    if (lane == 0 && m) pos0 = atomicAdd(count, __popc(m));
    pos0 = __shfl_sync(0xffffffffu, pos0, 0);
    if (take) list[pos0 + __popc(m & ((1u << lane) - 1))] = (int32_t)r;
  }
}

// Five lists by out-degree: [min_out, tw], (tw, t0], (t0, t1], (t1, t2], (t2, ...).
__global__ void k_worklist_outdeg5(const int32_t* __restrict__ opc, int64_t n, int min_out, int tw, int t0, int t1,
                                   int t2, int32_t* lists, int64_t stride, int32_t* counts,
                                   const int32_t* __restrict__ indeg, int promote) {
  const int lane = threadIdx.x & 31;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); r0 < n; r0 += step) {
    const int64_t r = r0 + lane;
    const int d = r < n ? opc[r] : 0;
    int cls = d < min_out ? -1 : (d <= tw ? 0 : (d <= t0 ? 1 : (d <= t1 ? 2 : (d <= t2 ? 3 : 4))));
    if (cls == 0 && indeg && r < n && indeg[r] > promote) cls = 1;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const unsigned m = __ballot_sync(0xffffffffu, cls == c);
      int pos = 0;
      if (lane == 0 && m) pos = atomicAdd(&counts[c], __popc(m));
      pos = __shfl_sync(0xffffffffu, pos, 0);
      if (cls == c) lists[c * stride + pos + __popc(m & ((1u << lane) - 1))] = (int32_t)r;
    }
  }
}

// ---------------------------------------------------------------------------
// Exclusive scan int32 -> int64 (three phases).
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 256, SCAN_I = 8, SCAN_B = SCAN_T * SCAN_I;

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const int32_t* __restrict__ in, int64_t n, int64_t* bsum) {
  __shared__ long long red[32];
  const int64_t b0 = (int64_t)blockIdx.x * SCAN_B;
  long long s = 0;
  for (int i = threadIdx.x; i < SCAN_B; i += SCAN_T) {
    const int64_t k = b0 + i;
    if (k < n) s += in[k];
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) bsum[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_scan_bsums(int64_t* bsum, int64_t nb) {
  __shared__ long long wsum[32];
  __shared__ long long carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t c0 = 0; c0 < nb; c0 += 1024) {
    const int64_t k = c0 + threadIdx.x;
    long long x = k < nb ? bsum[k] : 0;
    long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      long long w = wsum[lane];
      long long wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      wsum[lane] = wi - w;  // exclusive over warps
    }
    __syncthreads();
    const long long carry = carry_s;
    if (k < nb) bsum[k] = carry + wsum[wid] + incl - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = carry + wsum[wid] + incl;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_down(const int32_t* __restrict__ in, int64_t n,
                                                      const int64_t* __restrict__ bsum, int64_t* out) {
  __shared__ long long wsum[SCAN_T / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t b0 = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * SCAN_I;
  long long v[SCAN_I];
  long long t = 0;
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i) {
    v[i] = (b0 + i < n) ? in[b0 + i] : 0;
    t += v[i];
  }
  long long incl = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  long long wpre = 0;
  for (int w = 0; w < wid; ++w) wpre += wsum[w];
  long long run = bsum[blockIdx.x] + wpre + incl - t;
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i) {
    if (b0 + i < n) out[b0 + i] = run;
    run += v[i];
  }
  if (b0 < n && b0 + SCAN_I >= n) out[n] = run;
}

// ---------------------------------------------------------------------------
// Edge terms of the final C3 (oriented edges a -> b, rank space):
// d^10 = C3 (p1 - 2) and d^14 = D4,3 e / 2 = sum_j C3(i,j)(C3(i,j)-1)/2, since
// P2(i,j) = C3(i,j) on an edge (Sec. 4.3, D4,3 = A o C4,2).
// ---------------------------------------------------------------------------
__global__ void k_c3_edge_terms(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol,
                                const int32_t* __restrict__ C3o, const int32_t* __restrict__ dr, int64_t n,
                                u64* r10r, u64* r14r) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n; a += warps) {
    const int64_t b0 = orp[a], b1 = orp[a + 1];
    if (b1 == b0) continue;
    const long long da = dr[a];
    long long s10 = 0, s14 = 0;
    for (int64_t k = b0 + lane; k < b1; k += 32) {
      const long long t = C3o[k];
      if (t) {
        const int32_t b = ocol[k];
        const long long pair = t * (t - 1) / 2;
        s10 += t * ((long long)dr[b] - 2);
        s14 += pair;
        atomicAdd(r10r + b, (u64)(t * (da - 2)));
        if (pair) atomicAdd(r14r + b, (u64)pair);
      }
    }
    s10 = warp_sum_i64(s10);
    s14 = warp_sum_i64(s14);
    if (lane == 0) {
      if (s10) atomicAdd(r10r + a, (u64)s10);
      if (s14) atomicAdd(r14r + a, (u64)s14);
    }
  }
}

__global__ void k_unrank_u64(const u64* __restrict__ src, const int32_t* __restrict__ perm, int64_t n,
                             int64_t* dst) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    dst[perm[r]] = (int64_t)src[r];
}

// ---------------------------------------------------------------------------
// Epilogue: Table I rows and f = U16^{-1} f^ (Table II), exact in int64.
// ---------------------------------------------------------------------------
template <bool VEC>
__global__ void k_epilogue(EpilogueIn in, int64_t n, int64_t* __restrict__ raw, int64_t* __restrict__ net) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = in.rank[v];
    long long f[16], g[16];
    table1_row(in.d[v], in.p2[v], in.p3[v], (long long)in.c3r[r], in.r7[v], in.r9[v], (long long)in.r10r[r],
               (long long)in.r12r[r], (long long)in.r13r[r], (long long)in.r14r[r], (long long)in.r15r[r], f);
    u16_inverse(f, g);
    if (VEC) {  // both outputs 16-byte aligned
      if (raw) {
        longlong2* o = reinterpret_cast<longlong2*>(raw + v * 16);
#pragma unroll
        for (int i = 0; i < 8; ++i) o[i] = make_longlong2(f[2 * i], f[2 * i + 1]);
      }
      if (net) {
        longlong2* o = reinterpret_cast<longlong2*>(net + v * 16);
#pragma unroll
        for (int i = 0; i < 8; ++i) o[i] = make_longlong2(g[2 * i], g[2 * i + 1]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (raw) raw[v * 16 + i] = f[i];
        if (net) net[v * 16 + i] = g[i];
      }
    }
  }
}

// Sub-dictionary epilogue: the Table I rows of the columns in s, and
// f(s) = U16(s,s)^{-1} f^(s) (Table II caption), exact in int64. Inputs of
// stages the sub-dictionary does not need are zero.
__global__ void k_epilogue_sub(EpilogueIn in, SubDict sd, int64_t n, int64_t* __restrict__ raw,
                               int64_t* __restrict__ net) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = in.rank[v];
    long long f[16];
    table1_row(in.d[v], in.p2[v], in.p3[v], (long long)in.c3r[r], in.r7[v], in.r9[v], (long long)in.r10r[r],
               (long long)in.r12r[r], (long long)in.r13r[r], (long long)in.r14r[r], (long long)in.r15r[r], f);
    long long fs[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      long long x = 0;
#pragma unroll
      for (int k = 0; k < 16; ++k) x = (sd.col[i] == k) ? f[k] : x;
      fs[i] = x;
    }
    for (int i = 0; i < sd.k; ++i) {
      if (raw) raw[v * sd.k + i] = fs[i];
      if (net) {
        long long g = 0;
        for (int j = i; j < sd.k; ++j) g += sd.uinv[i][j] * fs[j];
        net[v * sd.k + i] = g;
      }
    }
  }
}

unsigned grid_for(int64_t items, int threads, int per_sm = 8) {
  int64_t want = (items + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms() * per_sm;
  if (want < 1) want = 1;
  return (unsigned)(want < cap ? want : cap);
}

}  // namespace

// ===========================================================================
// Launchers
// ===========================================================================

cudaError_t launch_degree(const Csr& g, int32_t* d, int32_t* dmax, int32_t* heavy, int32_t* nheavy, int* err,
                          cudaStream_t st, int32_t dcap) {
  if (g.n <= 0) return cudaSuccess;
  const int64_t cap = g.nnz / HEAVY_DEGREE + 1;
  if (g.rp64)
    k_degree<int64_t><<<grid_for(g.n, 256), 256, 0, st>>>(static_cast<const int64_t*>(g.rowptr), g.n, g.nnz, d,
                                                          dmax, heavy, nheavy, cap, dcap, err);
  else
    k_degree<int32_t><<<grid_for(g.n, 256), 256, 0, st>>>(static_cast<const int32_t*>(g.rowptr), g.n, g.nnz, d,
                                                          dmax, heavy, nheavy, cap, dcap, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_validate(const Csr& g, const int32_t* heavy, const int32_t* nheavy, int64_t heavy_cap,
                            int* err, cudaStream_t st) {
  if (g.rp64) {
    ValidateOp<int64_t> op{static_cast<const int64_t*>(g.rowptr), g.colidx, g.n, err};
    return run_rows<int64_t>(g, heavy, nheavy, heavy_cap, op, st);
  }
  ValidateOp<int32_t> op{static_cast<const int32_t*>(g.rowptr), g.colidx, g.n, err};
  return run_rows<int32_t>(g, heavy, nheavy, heavy_cap, op, st);
}

cudaError_t launch_validate_batch(const Csr& g, const int64_t* off, int64_t num_graphs, int* err, cudaStream_t st) {
  if (g.n <= 0 || num_graphs <= 0) return cudaSuccess;
  if (g.rp64)
    k_validate_batch<int64_t><<<grid_for(g.n, 256), 256, 0, st>>>(static_cast<const int64_t*>(g.rowptr), g.colidx,
                                                                  g.n, off, num_graphs, err);
  else
    k_validate_batch<int32_t><<<grid_for(g.n, 256), 256, 0, st>>>(static_cast<const int32_t*>(g.rowptr), g.colidx,
                                                                  g.n, off, num_graphs, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_spmv1(const Csr& g, const int32_t* d, const int32_t* heavy, const int32_t* nheavy,
                         int64_t heavy_cap, int64_t* p2, int64_t* r7, int* err, cudaStream_t st) {
  return dispatch_rows(g, heavy, nheavy, heavy_cap, Spmv1Op{d, p2, r7, g.n, err}, st);
}

cudaError_t launch_spmv2(const Csr& g, const int32_t* d, const int64_t* p2, const int64_t* c3o,
                         const int32_t* heavy, const int32_t* nheavy, int64_t heavy_cap, int64_t* p3,
                         int64_t* r9, cudaStream_t st) {
  return dispatch_rows(g, heavy, nheavy, heavy_cap, Spmv2Op{d, p2, c3o, p3, r9, g.n}, st);
}

cudaError_t launch_degree_hist(const int32_t* d, int64_t n, int32_t* hist, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_degree_hist<<<grid_for(n, 256, 4), 256, 0, st>>>(d, n, hist);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_rank_assign(const int32_t* d, int64_t n, const int64_t* base, int32_t* cursor,
                               int32_t* rank, int32_t* perm, int32_t* dr, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_rank_assign<<<grid_for(n, RANK_T * RANK_I, 4), RANK_T, 0, st>>>(d, n, base, cursor, rank, perm, dr);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_orient_count(const Csr& g, const int32_t* rank, const int32_t* heavy,
                                const int32_t* nheavy, int64_t heavy_cap, int32_t* opc, int32_t* dpmax,
                                cudaStream_t st) {
  return dispatch_rows(g, heavy, nheavy, heavy_cap, OrientCountOp{rank, opc, dpmax, g.n}, st);
}

cudaError_t launch_orient_fill(const Csr& g, const int32_t* rank, const int64_t* orp, const int32_t* heavy,
                               const int32_t* nheavy, int64_t heavy_cap, int32_t* cursor, int32_t* ocol,
                               cudaStream_t st) {
  return dispatch_rows(g, heavy, nheavy, heavy_cap, OrientFillOp{rank, orp, cursor, ocol, g.n}, st);
}

namespace {
// Layout of the long-row scratch: [count][list of cap rows][pad][slots x P].
struct LongRowScratch {
  int64_t cap, slots, P, slot_off, total;
};
LongRowScratch long_row_scratch(int64_t entries, int32_t dpmax) {
  LongRowScratch x{0, 0, 0, 0, 0};
  if (dpmax <= SORT_SMEM_MAX) return x;
  x.P = SORT_SMEM_MAX;
  while (x.P < dpmax) x.P <<= 1;
  x.cap = entries / (SORT_SMEM_MAX + 1) + 1;
  // one slot per SM, at most 2^28 int32 in all
  x.slots = std::max<int64_t>(1, std::min<int64_t>(num_sms(), ((int64_t)1 << 28) / x.P));
  x.slot_off = ((1 + x.cap) + 3) & ~(int64_t)3;  // 16-byte aligned slots
  x.total = x.slot_off + x.slots * x.P;
  return x;
}
}  // namespace

int64_t sort_rows_scratch_ints(int64_t entries, int32_t dpmax) { return long_row_scratch(entries, dpmax).total; }

cudaError_t launch_sort_rows(const int64_t* orp, int64_t n, int32_t dpmax, int64_t entries, int32_t* ocol,
                             int32_t* gscratch, cudaStream_t st) {
  if (n <= 0 || dpmax < 2) return cudaSuccess;
  k_sort_rows_warp<<<grid_for(n * 32, 256), 256, 0, st>>>(orp, n, ocol);
  note_launch();
  if (dpmax > 32) {
    int P = 64;
    while (P < dpmax && P < SORT_SMEM_MAX) P <<= 1;
    const size_t smem = (size_t)P * sizeof(int32_t);
    allow_max_smem(k_sort_rows_block);
    k_sort_rows_block<<<grid_for(n, SORT_BLOCK_T, 4), SORT_BLOCK_T, smem, st>>>(orp, n, ocol);
    note_launch();
  }
  if (dpmax > SORT_SMEM_MAX) {
    const LongRowScratch x = long_row_scratch(entries, dpmax);
    if (!gscratch || x.P > ((int64_t)1 << 30)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(gscratch, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    k_long_rows<<<grid_for(n, 256), 256, 0, st>>>(orp, n, gscratch + 1, x.cap);
    note_launch();
    k_sort_rows_global<<<(unsigned)x.slots, 1024, 0, st>>>(orp, gscratch + 1, x.cap, ocol, gscratch + x.slot_off,
                                                           (int)x.P);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_worklist_outdeg(const int32_t* opc, int64_t n, int min_out, int32_t* list, int32_t* count,
                                   cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_worklist_outdeg<<<grid_for(n, 256), 256, 0, st>>>(opc, n, min_out, list, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_worklist_outdeg5(const int32_t* opc, int64_t n, int min_out, int tw, int t0, int t1, int t2,
                                    int32_t* lists, int64_t stride, int32_t* counts, cudaStream_t st,
                                    const int32_t* indeg, int promote) {
  if (n <= 0) return cudaSuccess;
  k_worklist_outdeg5<<<grid_for(n, 256), 256, 0, st>>>(opc, n, min_out, tw, t0, t1, t2, lists, stride, counts,
                                                       indeg, promote);
  note_launch();
  return cudaGetLastError();
}

size_t scan_temp_bytes(int64_t n) {
  const int64_t nb = (n + SCAN_B - 1) / SCAN_B + 1;
  return (size_t)nb * sizeof(int64_t);
}

cudaError_t launch_scan_i32_to_i64(const int32_t* in, int64_t n, int64_t* out, void* temp, cudaStream_t st) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), st);
  const int64_t nb = (n + SCAN_B - 1) / SCAN_B;
  int64_t* bsum = static_cast<int64_t*>(temp);
  k_scan_reduce<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, bsum);
  note_launch();
  k_scan_bsums<<<1, 1024, 0, st>>>(bsum, nb);
  note_launch();
  k_scan_down<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, bsum, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_c3_edge_terms(const int64_t* orp, const int32_t* ocol, const int32_t* C3o, const int32_t* dr,
                                 int64_t n, u64* r10r, u64* r14r, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_c3_edge_terms<<<grid_for(n * 32, 256), 256, 0, st>>>(orp, ocol, C3o, dr, n, r10r, r14r);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_unrank_u64(const u64* src_r, const int32_t* perm, int64_t n, int64_t* dst_o, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_unrank_u64<<<grid_for(n, 256), 256, 0, st>>>(src_r, perm, n, dst_o);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_epilogue_sub(const EpilogueIn& in, const SubDict& sd, int64_t n, int64_t* raw, int64_t* net,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_epilogue_sub<<<grid_for(n, 256), 256, 0, st>>>(in, sd, n, raw, net);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_epilogue(const EpilogueIn& in, int64_t n, int64_t* raw, int64_t* net, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const bool vec = ((uintptr_t)raw % 16 == 0) && ((uintptr_t)net % 16 == 0);
  if (vec) k_epilogue<true><<<grid_for(n, 256), 256, 0, st>>>(in, n, raw, net);
  else k_epilogue<false><<<grid_for(n, 256), 256, 0, st>>>(in, n, raw, net);
  note_launch();
  return cudaGetLastError();
}

}  // namespace fglt
