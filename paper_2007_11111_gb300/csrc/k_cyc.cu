// 4-cycles per vertex (rank space).
//
// The paper's formula is c4 = C4,2 e / 2 with C4,2 = P2 o (P2 - 1) (Lemma on
// c4): for every vertex i, c4(i) = sum over l != i of binom(P2(i,l), 2), i.e.
// every 4-cycle through i is counted once via its vertex l opposite to i.
// Forming the P2 rows costs sum_k d_k^2 (Lemma 1). This kernel reaches the
// same integers by enumerating each 4-cycle once from its bottom-opposite pair:
// every 4-cycle has a unique top vertex u (highest rank) and u's opposite w;
// the two other vertices v, v' are common neighbours of u and w below u.
// For a vertex w, the wedges w - v - u with u in N+(v) and u above w are
// counted per u in a hash table (cnt[u] = number of such v). Then, for the
// pair (u, w), binom(cnt[u], 2) cycles have top u and bottom w; each of u and w
// gains that many cycles, and each middle v gains cnt[u] - 1 (one per other
// middle). Summed over all w this is exactly C4,2 e / 2 per vertex; the work
// is sum_v d_v * d+_v instead of sum_k d_k^2 (degree orientation, as in the
// cost analysis of Appendix A).
#include "fglt_device.cuh"
#include "fglt_kernels.h"

namespace fglt {

namespace {

constexpr int CYC_T = 256;
constexpr int SMEM_BITS = 13;  // 8192 slots x (key, count) = 64 KB

int num_sms() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <bool GMEM>
struct Table {
  uint32_t* keys;
  uint32_t* cnts;
  __device__ __forceinline__ uint32_t load_key(uint32_t h) const {
    if (GMEM) return __ldcg(keys + h);
    return *((volatile uint32_t*)keys + h);
  }
  __device__ __forceinline__ uint32_t load_cnt(uint32_t h) const {
    if (GMEM) return __ldcg(cnts + h);
    return cnts[h];
  }
  __device__ __forceinline__ void clear(uint32_t h) const {
    if (GMEM) {
      __stcg(keys + h, EMPTY_KEY);
      __stcg(cnts + h, 0u);
    } else {
      keys[h] = EMPTY_KEY;
      cnts[h] = 0u;
    }
  }
  __device__ __forceinline__ void increment(uint32_t key, int hb, int* err) const {
    const uint32_t mask = (1u << hb) - 1;
    uint32_t h = hash_slot(key, hb);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      uint32_t k = load_key(h);
      if (k == EMPTY_KEY) {
        k = atomicCAS(keys + h, EMPTY_KEY, key);
        if (k == EMPTY_KEY) k = key;
      }
      if (k == key) {
        atomicAdd(cnts + h, 1u);
        return;
      }
      h = (h + 1) & mask;
    }
    atomicOr(err, ERR_HASH_FULL);
  }
  __device__ __forceinline__ uint32_t count_of(uint32_t key, int hb) const {
    const uint32_t mask = (1u << hb) - 1;
    uint32_t h = hash_slot(key, hb);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      const uint32_t k = load_key(h);
      if (k == key) return load_cnt(h);
      if (k == EMPTY_KEY) return 0u;
      h = (h + 1) & mask;
    }
    return 0u;
  }
};

template <typename RP, bool GMEM>
__global__ void __launch_bounds__(CYC_T) k_cyc(const RP* __restrict__ rp, const int32_t* __restrict__ ci,
                                               const int32_t* __restrict__ rank, const int32_t* __restrict__ perm,
                                               const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol,
                                               const int64_t* __restrict__ wc, const int32_t* __restrict__ list,
                                               const int32_t* __restrict__ cnt, int* next, int gbits,
                                               uint32_t* gkeys, uint32_t* gcnt, u64* r12r, int64_t n, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ u64 red[32];
  Table<GMEM> T;
  if (GMEM) {
    T.keys = gkeys + ((size_t)blockIdx.x << gbits);
    T.cnts = gcnt + ((size_t)blockIdx.x << gbits);
  } else {
    T.keys = reinterpret_cast<uint32_t*>(smem);
    T.cnts = T.keys + (1 << SMEM_BITS);
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int total = *cnt;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    const int32_t w = list[item];
    int64_t cap = wc[w];
    if (cap > n - 1 - w) cap = n - 1 - w;
    int hb = 5;
    while ((1LL << hb) < 2 * cap) ++hb;
    const uint32_t H = 1u << hb;
    for (uint32_t i = tid; i < H; i += blockDim.x) T.clear(i);
    __syncthreads();

    const int64_t wo = perm[w];
    const int64_t s = (int64_t)rp[wo], e = (int64_t)rp[wo + 1];
    // Pass A: count wedges w - v - u per top vertex u.
    for (int64_t k = s + warp; k < e; k += nwarps) {
      const int32_t v = ci[k];
      if ((uint32_t)v >= (uint64_t)n) continue;
      const int32_t rv = rank[v];
      const int64_t ob = orp[rv], oe = orp[rv + 1];
      const int64_t st = upper_bound_i32(ocol, ob, oe, w);
      for (int64_t q = st + lane; q < oe; q += 32) T.increment((uint32_t)ocol[q], hb, err);
    }
    __syncthreads();
    // Pass B: every middle v of a wedge gains cnt[u] - 1.
    for (int64_t k = s + warp; k < e; k += nwarps) {
      const int32_t v = ci[k];
      if ((uint32_t)v >= (uint64_t)n) continue;
      const int32_t rv = rank[v];
      const int64_t ob = orp[rv], oe = orp[rv + 1];
      const int64_t st = upper_bound_i32(ocol, ob, oe, w);
      long long sum = 0;
      for (int64_t q = st + lane; q < oe; q += 32) sum += (long long)T.count_of((uint32_t)ocol[q], hb) - 1;
      sum = warp_sum_i64(sum);
      if (lane == 0 && sum) atomicAdd(&r12r[rv], (u64)sum);
    }
    // Pass C: top u and bottom w gain binom(cnt[u], 2) each.
    u64 accw = 0;
    for (uint32_t i = tid; i < H; i += blockDim.x) {
      const uint32_t key = T.load_key(i);
      if (key != EMPTY_KEY) {
        const u64 c = T.load_cnt(i);
        if (c >= 2) {
          const u64 v = c * (c - 1) / 2;
          atomicAdd(&r12r[key], v);
          accw += v;
        }
      }
    }
    accw = block_sum(accw, red);
    if (tid == 0 && accw) atomicAdd(&r12r[w], accw);
    __syncthreads();
  }
}

__global__ void k_cyc_worklists(const int64_t* __restrict__ wc, int64_t n, int64_t smem_cap, int32_t* list_s,
                                int32_t* cnt_s, int32_t* list_g, int32_t* cnt_g) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); r0 < n; r0 += stride) {
    const int64_t r = r0 + lane;
    int64_t cap = 0;
    if (r < n) {
      cap = wc[r];
      if (cap > n - 1 - r) cap = n - 1 - r;
    }
    const bool take = r < n && wc[r] >= 2;
    const bool small = cap <= smem_cap;
    const unsigned ms = __ballot_sync(0xffffffffu, take && small);
    const unsigned mg = __ballot_sync(0xffffffffu, take && !small);
    int ps = 0, pg = 0;
    if (lane == 0) {
      if (ms) ps = atomicAdd(cnt_s, __popc(ms));
      if (mg) pg = atomicAdd(cnt_g, __popc(mg));
    }
    ps = __shfl_sync(0xffffffffu, ps, 0);
    pg = __shfl_sync(0xffffffffu, pg, 0);
    const unsigned below = (1u << lane) - 1;
    if (take && small) list_s[ps + __popc(ms & below)] = (int32_t)r;
    if (take && !small) list_g[pg + __popc(mg & below)] = (int32_t)r;
  }
}

template <typename RP>
cudaError_t launch_cyc_rp(const Csr& g, const int32_t* rank, const int32_t* perm, const int64_t* orp,
                          const int32_t* ocol, const int64_t* wc, const int32_t* list, const int32_t* cnt, int* next,
                          bool gmem, int gbits, uint32_t* gkeys, uint32_t* gcnt, u64* r12r, int* err,
                          cudaStream_t st) {
  const RP* rp = static_cast<const RP*>(g.rowptr);
  if (gmem) {
    k_cyc<RP, true><<<cyc_grid_blocks_gmem(), CYC_T, 0, st>>>(rp, g.colidx, rank, perm, orp, ocol, wc, list, cnt,
                                                               next, gbits, gkeys, gcnt, r12r, g.n, err);
  } else {
    const size_t smem = (size_t)8 << SMEM_BITS;
    cudaFuncSetAttribute(k_cyc<RP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cyc<RP, false><<<cyc_grid_blocks_smem(), CYC_T, smem, st>>>(rp, g.colidx, rank, perm, orp, ocol, wc, list,
                                                                   cnt, next, 0, nullptr, nullptr, r12r, g.n, err);
  }
  return cudaGetLastError();
}

}  // namespace

int cyc_smem_hash_bits() { return SMEM_BITS; }
int cyc_grid_blocks_smem() { return num_sms() * 3; }
int cyc_grid_blocks_gmem() { return num_sms(); }

cudaError_t launch_cyc_worklists(const int64_t* wc, int64_t n, int64_t smem_cap, int32_t* list_s, int32_t* cnt_s,
                                 int32_t* list_g, int32_t* cnt_g, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
  k_cyc_worklists<<<(unsigned)blocks, 256, 0, st>>>(wc, n, smem_cap, list_s, cnt_s, list_g, cnt_g);
  return cudaGetLastError();
}

cudaError_t launch_cyc(const Csr& g, const int32_t* rank, const int32_t* perm, const int64_t* orp,
                       const int32_t* ocol, const int64_t* wc, const int32_t* list, const int32_t* cnt, int* next,
                       bool gmem, int gbits, uint32_t* gkeys, uint32_t* gcnt, u64* r12r, int* err,
                       cudaStream_t st) {
  if (g.n <= 0) return cudaSuccess;
  return g.rp64 ? launch_cyc_rp<int64_t>(g, rank, perm, orp, ocol, wc, list, cnt, next, gmem, gbits, gkeys, gcnt,
                                         r12r, err, st)
                : launch_cyc_rp<int32_t>(g, rank, perm, orp, ocol, wc, list, cnt, next, gmem, gbits, gkeys, gcnt,
                                         r12r, err, st);
}

}  // namespace fglt
