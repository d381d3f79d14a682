// Edge list -> the symmetric simple CSR the transform expects (Sec. 1 assumes
// a simple undirected graph): every pair is an undirected edge, self-loops are
// dropped, both directions are stored, repeated pairs merge, rows are sorted.
//
//   count   deg0[v] = stored entries of v before merging (both directions)
//   scan    rp0 = exclusive prefix of deg0
//   fill    tmp[rp0[v] ..] = the other ends, in arrival order
//   sort    every row of tmp ascending (the row sorts of the oriented graph)
//   unique  deg[v] = distinct entries of row v; rowptr = prefix of deg
//   compact colidx[rowptr[v] ..] = the distinct entries of row v
//
// Degree relabelling of a CSR (locality):
//   degree  d[v] from the row pointers, and its maximum
//   rank    counting sort by degree (the transform's own rank kernels)
//   ids     perm[v] = rank or n - 1 - rank; inv[perm[v]] = v; ndeg[perm[v]] = d[v]
//   scan    out_rowptr = exclusive prefix of ndeg
//   fill    out row perm[v] = perm of v's neighbours, then the row sorts
#include "fglt_device.cuh"
#include "fglt_kernels.h"

namespace fglt {

namespace {

int num_sms() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

unsigned grid_for(int64_t items, int threads, int per_sm = 8) {
  int64_t want = (items + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * per_sm;
  if (want < 1) want = 1;
  return (unsigned)(want < cap ? want : cap);
}

__global__ void k_edge_count(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t E,
                             int64_t n, int32_t* deg0, int* err) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = src[e], d = dst[e];
    if ((uint32_t)s >= (uint64_t)n || (uint32_t)d >= (uint64_t)n) {
      atomicOr(err, ERR_BAD_GRAPH);
      continue;
    }
    if (s == d) continue;
    atomicAdd(deg0 + s, 1);
    atomicAdd(deg0 + d, 1);
  }
}

__global__ void k_row_max(const int32_t* __restrict__ deg, int64_t n, int32_t* dmax) {
  int m = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    m = max(m, deg[v]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(dmax, m);
}

__global__ void k_edge_fill(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t E, int64_t n,
                            const int64_t* __restrict__ rp0, int32_t* cursor, int32_t* tmp) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = src[e], d = dst[e];
    if ((uint32_t)s >= (uint64_t)n || (uint32_t)d >= (uint64_t)n || s == d) continue;
    tmp[rp0[s] + atomicAdd(cursor + s, 1)] = d;
    tmp[rp0[d] + atomicAdd(cursor + d, 1)] = s;
  }
}

// One warp per row: distinct entries of the sorted row (count or compact).
template <bool WRITE>
__global__ void k_row_unique(const int64_t* __restrict__ rp0, const int32_t* __restrict__ tmp, int64_t n,
                             int32_t* deg, const int64_t* __restrict__ rowptr, int32_t* colidx) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int64_t b = rp0[v], e = rp0[v + 1];
    int64_t out = WRITE ? rowptr[v] : 0;
    int count = 0;
    for (int64_t k0 = b; k0 < e; k0 += 32) {
      const int64_t k = k0 + lane;
      bool keep = false;
      int32_t x = 0;
      if (k < e) {
        x = tmp[k];
        keep = k == b || tmp[k - 1] != x;
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (WRITE && keep) colidx[out + __popc(m & ((1u << lane) - 1u))] = x;
      out += __popc(m);
      count += __popc(m);
    }
    if (!WRITE && lane == 0) deg[v] = count;
  }
}

__global__ void k_row_degree(const void* __restrict__ rowptr, int rp64, int64_t n, int32_t* d) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = rp64 ? static_cast<const int64_t*>(rowptr)[v] : static_cast<const int32_t*>(rowptr)[v];
    const int64_t e = rp64 ? static_cast<const int64_t*>(rowptr)[v + 1] : static_cast<const int32_t*>(rowptr)[v + 1];
    d[v] = (int32_t)(e - b);
  }
}

__global__ void k_relabel_ids(const int32_t* __restrict__ rank, const int32_t* __restrict__ d, int64_t n, int desc,
                              int32_t* perm, int32_t* inv, int32_t* ndeg) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rank[v];
    const int32_t p = desc ? (int32_t)(n - 1 - r) : r;
    perm[v] = p;
    inv[p] = (int32_t)v;
    ndeg[p] = d[v];
  }
}

// One warp per new row: the new ids of the old row's entries (unsorted). An
// entry outside [0, n) is flagged and written as -1.
__global__ void k_relabel_fill(const void* __restrict__ rowptr, int rp64, const int32_t* __restrict__ colidx,
                               const int32_t* __restrict__ perm, const int32_t* __restrict__ inv, int64_t n,
                               const int64_t* __restrict__ out_rowptr, int32_t* out_colidx, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int32_t v = inv[i];
    const int64_t b = rp64 ? static_cast<const int64_t*>(rowptr)[v] : static_cast<const int32_t*>(rowptr)[v];
    const int64_t o = out_rowptr[i], len = out_rowptr[i + 1] - o;
    for (int64_t k = lane; k < len; k += 32) {
      const int32_t u = colidx[b + k];
      int32_t x = -1;
      if ((uint32_t)u < (uint64_t)n) x = perm[u];
      else atomicOr(err, ERR_BAD_GRAPH);
      out_colidx[o + k] = x;
    }
  }
}

}  // namespace

cudaError_t launch_row_degree(const void* rowptr, bool rp64, int64_t n, int32_t* d, int32_t* dmax, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_row_degree<<<grid_for(n, 256), 256, 0, st>>>(rowptr, rp64 ? 1 : 0, n, d);
  note_launch();
  k_row_max<<<grid_for(n, 256), 256, 0, st>>>(d, n, dmax);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_relabel_ids(const int32_t* rank, const int32_t* d, int64_t n, bool descending, int32_t* perm,
                               int32_t* inv, int32_t* ndeg, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_relabel_ids<<<grid_for(n, 256), 256, 0, st>>>(rank, d, n, descending ? 1 : 0, perm, inv, ndeg);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_relabel_fill(const void* rowptr, bool rp64, const int32_t* colidx, const int32_t* perm,
                                const int32_t* inv, int64_t n, const int64_t* out_rowptr, int32_t* out_colidx,
                                int* err, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_relabel_fill<<<grid_for(n * 32, 256, 16), 256, 0, st>>>(rowptr, rp64 ? 1 : 0, colidx, perm, inv, n, out_rowptr,
                                                             out_colidx, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_edge_count(const int32_t* src, const int32_t* dst, int64_t E, int64_t n, int32_t* deg0,
                              int32_t* dmax, int* err, cudaStream_t st) {
  if (E > 0) {
    k_edge_count<<<grid_for(E, 256), 256, 0, st>>>(src, dst, E, n, deg0, err);
    note_launch();
  }
  if (n > 0) {
    k_row_max<<<grid_for(n, 256), 256, 0, st>>>(deg0, n, dmax);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_edge_fill(const int32_t* src, const int32_t* dst, int64_t E, int64_t n, const int64_t* rp0,
                             int32_t* cursor, int32_t* tmp, cudaStream_t st) {
  if (E <= 0) return cudaSuccess;
  k_edge_fill<<<grid_for(E, 256), 256, 0, st>>>(src, dst, E, n, rp0, cursor, tmp);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_row_unique(const int64_t* rp0, const int32_t* tmp, int64_t n, int32_t* deg, const int64_t* rowptr,
                              int32_t* colidx, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (colidx)
    k_row_unique<true><<<grid_for(n * 32, 256, 16), 256, 0, st>>>(rp0, tmp, n, deg, rowptr, colidx);
  else
    k_row_unique<false><<<grid_for(n * 32, 256, 16), 256, 0, st>>>(rp0, tmp, n, deg, rowptr, colidx);
  note_launch();
  return cudaGetLastError();
}

}  // namespace fglt
