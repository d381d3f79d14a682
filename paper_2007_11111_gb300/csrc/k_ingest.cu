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

}  // namespace

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
