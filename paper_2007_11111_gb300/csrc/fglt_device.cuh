// Device-side helpers shared by the FGLT kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fglt {

typedef unsigned long long u64;

// Bits of the device error word (the host maps any set bit to a status).
enum : int {
  ERR_HASH_FULL = 1,      // a hash table ran out of probes (sizing bug)
  ERR_BAD_GRAPH = 2,      // validation found a non-simple / asymmetric CSR
  ERR_INTERNAL = 4,       // a consistency check failed
  ERR_BAD_ROWPTR = 8,     // row pointers not monotone / outside [0, nnz]
  ERR_TIMEOUT = 16,       // a bounded device wait ran out
};

constexpr uint32_t EMPTY_KEY = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t hash_slot(uint32_t key, int bits) {
  return (key * 0x9E3779B1u) >> (32 - bits);
}

__device__ __forceinline__ int warp_sum_i32(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ long long warp_sum_i64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ u64 warp_sum_u64(u64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// First index in sorted a[lo, hi) whose value is > key.
__device__ __forceinline__ int64_t upper_bound_i32(const int32_t* a, int64_t lo, int64_t hi, int32_t key) {
  while (lo < hi) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] <= key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Block-wide sum (blockDim.x a multiple of 32, at most 1024). `red` needs 32 slots.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T s = 0;
  if (wid == 0) {
    s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in warp 0
}

// Table I of one vertex from its per-vertex quantities: degree d = p1, p2, p3,
// c3, and the SpMV / listing sums d^7, d^9, d^10, d^12 .. d^15 (Sec. 4).
__device__ __forceinline__ void table1_row(long long d, long long p2, long long p3, long long c3, long long r7,
                                           long long r9, long long r10, long long r12, long long r13, long long r14,
                                           long long r15, long long f[16]) {
  f[0] = 1;
  f[1] = d;
  f[2] = p2;
  f[3] = d * (d - 1) / 2;
  f[4] = c3;
  f[5] = p3;
  f[6] = p2 * (d - 1) - 2 * c3;
  f[7] = r7;
  f[8] = (d * (d - 1) / 2) * (d - 2) / 3;
  f[9] = r9;
  f[10] = r10;
  f[11] = (d - 2) * c3;
  f[12] = r12;
  f[13] = r13;
  f[14] = r14;
  f[15] = r15;
}

// Net frequencies g = U16^{-1} f (Table II), the inverse written out; exact
// in int64.
__device__ __forceinline__ void u16_inverse(const long long f[16], long long g[16]) {
  g[0] = f[0];
  g[1] = f[1];
  g[2] = f[2] - 2 * f[4];
  g[3] = f[3] - f[4];
  g[4] = f[4];
  g[5] = f[5] - 2 * f[9] - f[10] - 2 * f[12] + 4 * f[13] + 2 * f[14] - 6 * f[15];
  g[6] = f[6] - f[10] - 2 * f[11] - 2 * f[12] + 2 * f[13] + 4 * f[14] - 6 * f[15];
  g[7] = f[7] - f[9] - f[10] + 2 * f[13] + f[14] - 3 * f[15];
  g[8] = f[8] - f[11] + f[14] - f[15];
  g[9] = f[9] - 2 * f[13] + 3 * f[15];
  g[10] = f[10] - 2 * f[13] - 2 * f[14] + 6 * f[15];
  g[11] = f[11] - 2 * f[14] + 3 * f[15];
  g[12] = f[12] - f[13] - f[14] + 3 * f[15];
  g[13] = f[13] - 3 * f[15];
  g[14] = f[14] - 3 * f[15];
  g[15] = f[15];
}

// Lets fn use the device's full opt-in shared memory per block. Every caller
// sets the same value, so concurrent host threads launching the kernel with
// different dynamic sizes cannot shrink the limit under one another.
template <typename F>
inline void allow_max_smem(F* fn) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return;
  const int dyn = optin - (int)fa.sharedSizeBytes;  // the limit covers static + dynamic
  if (dyn > 0) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
}

}  // namespace fglt
