// Batched transform of small graphs in one fused, persistent launch.
//
// A block takes one graph of at most SMALL_N_MAX vertices at a time from a
// work queue (largest graphs first) and computes its whole transform in
// shared memory. The graph's adjacency A is held as a bitmap (row i = N(i),
// W words); every product the formulas of Table I need is formed on the fly
// from the rows, so no auxiliary matrix (C3, P2, D4,c, T) is stored (Sec. 6
// notes that the auxiliary matrices need not be kept). Per graph:
//   1. the bitmap, the degrees, and checks of the structure the kernel relies
//      on (every neighbour inside its graph, no self-loop, no repeated entry,
//      a symmetric pattern; a violation sets ERR_BAD_GRAPH);
//   2. one warp per vertex i: the row P2(i, .) = sum_{k in N(i)} A(k, .) by a
//      walk over the neighbours' rows (each set bit adds one), giving
//        c4(i)   = sum_{l != i} binom(P2(i,l), 2)            (Lemma on c4)
//        C3(i,j) = P2(i,j) on the edges, c3(i) = sum_j C3(i,j) / 2 (Lemma 2)
//        d^7, d^10, d^14, p2 as sums over the edges of i    (Sec. 3.1-4.3)
//   3. one half-warp per edge j-k, the lanes over the words of
//      Q = A_j & A_k (|Q| = C3(j,k)): every i in Q gains C3(j,k) - 1 towards
//      d^13 = D4,c e / 2 and |Q & A_i| (4-cliques {i, j, k, .}, each counted
//      on three of its edges) towards d^15                 (Sec. 4.3)
//   4. one warp per vertex: p3 and d^9 from the neighbours' p2 and c3, then
//      Table I and U16^{-1} (Table II), exact.
// All per-graph quantities fit in 32 bits (n <= 512); the outputs are int64.
#include <algorithm>

#include "fglt_device.cuh"
#include "fglt_kernels.h"

namespace fglt {

namespace {

constexpr int SN = SMALL_N_MAX;  // vertices per graph at most
constexpr int SWD = SN / 32;     // bitmap words per row at most
constexpr int ST = 256;          // threads per block
constexpr int SW = ST / 32;      // warps per block

// Dynamic shared memory of a block (32-bit words).
enum : int {
  O_A = 0,                      // adjacency bitmap, rows of W words
  O_NB = O_A + SN * SWD,        // per warp: neighbour list (uint16)
  O_PROW = O_NB + SW * SN / 2,  // per warp: P2 row (int32, zero between vertices)
  O_D = O_PROW + SW * SN,       // per vertex: degree
  O_C3 = O_D + SN,
  O_P2 = O_C3 + SN,
  O_R7 = O_P2 + SN,
  O_R10 = O_R7 + SN,
  O_R14 = O_R10 + SN,
  O_C4 = O_R14 + SN,
  O_D13 = O_C4 + SN,
  O_K4 = O_D13 + SN,            // 3 x the 4-cliques at each vertex
  O_WORDS = O_K4 + SN
};

__device__ __forceinline__ int warp_excl_scan(int x, int lane) {
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  return incl - x;
}

template <typename RP>
__global__ void __launch_bounds__(ST) k_small_fglt(const RP* __restrict__ rp, const int32_t* __restrict__ ci,
                                                   const int64_t* __restrict__ off,
                                                   const int32_t* __restrict__ order, int64_t num_graphs,
                                                   int64_t nnz, int* next, int64_t* __restrict__ raw,
                                                   int64_t* __restrict__ net, SubDict sd, bool full, int* err) {
  extern __shared__ __align__(16) uint32_t smw[];
  __shared__ int s_item;
  uint32_t* A = smw + O_A;
  int32_t* dg = reinterpret_cast<int32_t*>(smw + O_D);
  int32_t* c3a = reinterpret_cast<int32_t*>(smw + O_C3);
  int32_t* p2a = reinterpret_cast<int32_t*>(smw + O_P2);
  int32_t* r7a = reinterpret_cast<int32_t*>(smw + O_R7);
  int32_t* r10a = reinterpret_cast<int32_t*>(smw + O_R10);
  int32_t* r14a = reinterpret_cast<int32_t*>(smw + O_R14);
  int32_t* c4a = reinterpret_cast<int32_t*>(smw + O_C4);
  int32_t* d13a = reinterpret_cast<int32_t*>(smw + O_D13);
  int32_t* k4a = reinterpret_cast<int32_t*>(smw + O_K4);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint16_t* nb = reinterpret_cast<uint16_t*>(smw + O_NB) + warp * SN;
  int32_t* prow = reinterpret_cast<int32_t*>(smw + O_PROW) + warp * SN;
  for (int l = lane; l < SN; l += 32) prow[l] = 0;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= num_graphs) break;
    const int g = order[item];
    const int64_t lo = off[g];
    const int n = (int)(off[g + 1] - lo);
    const int W = (n + 31) >> 5;
    for (int i = tid; i < n * W; i += ST) A[i] = 0u;
    for (int i = tid; i < n; i += ST) {
      d13a[i] = 0;
      k4a[i] = 0;
    }
    __syncthreads();
    // 1. Rows of the bitmap from the CSR, one warp per vertex.
    bool bad = false, bad_rp = false;
    for (int i = warp; i < n; i += SW) {
      int64_t b = (int64_t)rp[lo + i], e = (int64_t)rp[lo + i + 1];
      if (b < 0 || e < b || e > nnz) {  // malformed row pointers: the row is not read
        bad_rp = true;
        b = e = 0;
      }
      if (lane == 0) dg[i] = (int32_t)(e - b);
      for (int64_t k = b + lane; k < e; k += 32) {
        const int64_t j = (int64_t)ci[k] - lo;
        if (j < 0 || j >= n || j == i) bad = true;
        else atomicOr(&A[i * W + (j >> 5)], 1u << (j & 31));
      }
    }
    __syncthreads();
    // 2. One warp per vertex i: its neighbour list, the P2 row by column
    // counts, and the sums over its edges.
    for (int i = warp; i < n; i += SW) {
      const uint32_t* Ai = A + i * W;
      const uint32_t wi = lane < W ? Ai[lane] : 0u;
      const int pos = warp_excl_scan(__popc(wi), lane);
      const int d = __shfl_sync(0xffffffffu, pos + __popc(wi), 31);
      if (d != dg[i]) bad = true;  // a repeated entry (popcount below the stored degree)
      {
        uint32_t bits = wi;
        int q = pos;
        while (bits) {
          const int t = __ffs(bits) - 1;
          bits &= bits - 1;
          nb[q++] = (uint16_t)((lane << 5) + t);
        }
      }
      __syncwarp();
      // P2(i, l) for every l of the 2-hop set: the neighbours' rows are
      // walked WP lanes per row (one word each), each set bit l != i adding
      // one to prow[l]. An increment from p to p + 1 raises binom(P2, 2) by
      // p, so c4(i) is the sum of the old values.
      int c4 = 0;
      const int WP = W <= 1 ? 1 : (W <= 2 ? 2 : (W <= 4 ? 4 : (W <= 8 ? 8 : 16)));
      for (int q0 = 0; q0 < d; q0 += 32 / WP) {
        const int q = q0 + lane / WP, w = lane % WP;
        if (q < d && w < W) {
          uint32_t bits = A[nb[q] * W + w];
          while (bits) {
            const int l = (w << 5) + __ffs(bits) - 1;
            bits &= bits - 1;
            if (l != i) c4 += atomicAdd(&prow[l], 1);
          }
        }
      }
      __syncwarp();
      int c3x2 = 0, sdj = 0, r7 = 0, r10 = 0, r14 = 0;
      for (int q = lane; q < d; q += 32) {
        const int j = nb[q];
        const int c = prow[j];  // C3(i,j) = P2(i,j) on an edge
        const int dj = dg[j];
        const uint32_t* Aj = A + j * W;
        if (!((Aj[i >> 5] >> (i & 31)) & 1u)) bad = true;  // asymmetric pattern
        c3x2 += c;
        sdj += dj;
        r7 += (dj - 1) * (dj - 2) / 2;
        r10 += c * (dj - 2);
        r14 += c * (c - 1) / 2;
      }
      c4 = warp_sum_i32(c4);
      c3x2 = warp_sum_i32(c3x2);
      sdj = warp_sum_i32(sdj);
      r7 = warp_sum_i32(r7);
      r10 = warp_sum_i32(r10);
      r14 = warp_sum_i32(r14);
      if (lane == 0) {
        c3a[i] = c3x2 / 2;
        p2a[i] = sdj - d;
        r7a[i] = r7;
        r10a[i] = r10;
        r14a[i] = r14;
        c4a[i] = c4;
      }
      __syncwarp();
      for (int l = lane; l < n; l += 32) prow[l] = 0;
      __syncwarp();
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, ERR_BAD_GRAPH);
    if (__any_sync(0xffffffffu, bad_rp) && lane == 0) atomicOr(err, ERR_BAD_ROWPTR);
    // 3. One half-warp per edge j-k (j < k), lane w on word w of
    // Q = A_j & A_k: every i in Q gains C3(j,k) - 1 and |Q & A_i|.
    {
      const int hl = lane & 15;
      const unsigned hmask = 0xFFFFu << (lane & 16);
      for (int j = tid >> 4; j < n; j += ST / 16) {
        const uint32_t* Aj = A + j * W;
        uint32_t up = 0u;  // neighbours k > j, in word hl
        if (hl < W) {
          up = Aj[hl];
          const int base = hl << 5;
          if (base + 31 <= j) up = 0u;
          else if (base <= j) up &= ~((2u << (j - base)) - 1u);
        }
        for (;;) {
          const unsigned has = __ballot_sync(hmask, up != 0u) & hmask;
          if (!has) break;
          const int src = __ffs(has) - 1;  // lane holding the next k
          const uint32_t sw = __shfl_sync(hmask, up, src & 31);
          const int k = (((src & 15)) << 5) + __ffs(sw) - 1;
          if (lane == src) up &= up - 1;
          const uint32_t* Ak = A + k * W;
          uint32_t q = hl < W ? (Aj[hl] & Ak[hl]) : 0u;
          int c = __popc(q);
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) c += __shfl_xor_sync(hmask, c, o, 16);
          for (;;) {  // every i in Q
            const unsigned hi = __ballot_sync(hmask, q != 0u) & hmask;
            if (!hi) break;
            const int s2 = __ffs(hi) - 1;
            const uint32_t qw = __shfl_sync(hmask, q, s2 & 31);
            const int i = ((s2 & 15) << 5) + __ffs(qw) - 1;
            if (lane == s2) q &= q - 1;
            int t = hl < W ? __popc(Aj[hl] & Ak[hl] & A[i * W + hl]) : 0;
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(hmask, t, o, 16);
            if (hl == 0) {
              atomicAdd(&d13a[i], c - 1);
              if (t) atomicAdd(&k4a[i], t);
            }
          }
        }
      }
    }
    __syncthreads();
    // 4. One warp per vertex: p3, d^9, Table I and U16^{-1}.
    for (int i = warp; i < n; i += SW) {
      const uint32_t* Ai = A + i * W;
      int sp2 = 0, sc3 = 0;
      for (int w = lane; w < W; w += 32) {
        uint32_t bits = Ai[w];
        while (bits) {
          const int j = (w << 5) + __ffs(bits) - 1;
          bits &= bits - 1;
          sp2 += p2a[j];
          sc3 += c3a[j];
        }
      }
      sp2 = warp_sum_i32(sp2);
      sc3 = warp_sum_i32(sc3);
      // Every lane forms the row; lane c writes column c (coalesced stores).
      const long long d = dg[i], c3 = c3a[i];
      long long f[16];
      table1_row(d, p2a[i], sp2 - d * (d - 1) - 2 * c3, c3, r7a[i], sc3 - 2 * c3, r10a[i], c4a[i], d13a[i],
                 r14a[i], k4a[i] / 3, f);
      const int64_t v = lo + i;
      if (full) {
        long long u[16];
        u16_inverse(f, u);
        long long fr = f[0], ur = u[0];
#pragma unroll
        for (int c = 1; c < 16; ++c)
          if (lane == c) {
            fr = f[c];
            ur = u[c];
          }
        if (lane < 16) {
          if (raw) raw[v * 16 + lane] = fr;
          if (net) net[v * 16 + lane] = ur;
        }
      } else {
        long long fs[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          long long x = 0;
#pragma unroll
          for (int k = 0; k < 16; ++k) x = (sd.col[c] == k) ? f[k] : x;
          fs[c] = x;
        }
        if (lane < sd.k) {
          long long fr = 0, y = 0;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            if (k == lane) fr = fs[k];
            if (k >= lane && k < sd.k) y += sd.uinv[lane][k] * fs[k];
          }
          if (raw) raw[v * sd.k + lane] = fr;
          if (net) net[v * sd.k + lane] = y;
        }
      }
    }
    __syncthreads();
  }
}

int num_sms() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

cudaError_t launch_small_fglt(const Csr& g, const int64_t* off, const int32_t* order, int64_t num_graphs, int* next,
                              int64_t* raw, int64_t* net, const SubDict& sd, bool full, int* err, cudaStream_t st) {
  // g.nnz: stored entries (row pointers outside [0, nnz] flag ERR_BAD_ROWPTR)
  if (num_graphs <= 0) return cudaSuccess;
  auto* fn = g.rp64 ? (const void*)k_small_fglt<int64_t> : (const void*)k_small_fglt<int32_t>;
  const size_t smem = (size_t)O_WORDS * 4;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, ST, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t grid = std::min<int64_t>((int64_t)per_sm * num_sms(), num_graphs);
  if (g.rp64)
    k_small_fglt<int64_t><<<(int)grid, ST, smem, st>>>(static_cast<const int64_t*>(g.rowptr), g.colidx, off, order,
                                                     num_graphs, g.nnz, next, raw, net, sd, full, err);
  else
    k_small_fglt<int32_t><<<(int)grid, ST, smem, st>>>(static_cast<const int32_t*>(g.rowptr), g.colidx, off, order,
                                                     num_graphs, g.nnz, next, raw, net, sd, full, err);
  note_launch();
  return cudaGetLastError();
}

}  // namespace fglt
