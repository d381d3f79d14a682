// 4-cycles per vertex (rank space).
//
// The paper's formula is c4 = C4,2 e / 2 with C4,2 = P2 o (P2 - 1) (Lemma on
// c4): for every vertex i, c4(i) = sum over l != i of binom(P2(i,l), 2), i.e.
// every 4-cycle through i is counted once via its vertex l opposite to i.
// Forming the P2 rows costs sum_k d_k^2 (Lemma 1). These kernels reach the
// same integers by enumerating each 4-cycle once: every 4-cycle has a unique
// top vertex u (highest rank) and u's opposite w; the two other vertices v, v'
// are common neighbours of u and w below u. For a vertex w, the wedges
// w - v - u with u in N+(v) and u above w are counted per u (cnt[u] = number
// of such v). Then binom(cnt[u], 2) cycles have top u and bottom w; each of u
// and w gains that many, and each middle v gains cnt[u] - 1 (one per other
// middle). Summed over all w this is C4,2 e / 2 per vertex; the work is the
// number of such wedges, at most sum_v d_v d+_v (degree orientation, the cost
// model of Appendix A), instead of sum_k d_k^2.
//
// Everything runs in rank space. The middles v of w are read from two lists:
// the in-list of w, entries (v, j) with w = N+(v)[j], whose tops are the
// entries of N+(v) after position j, and the out-list N+(w), whose middles v
// have every entry of N+(v) as a top (all above v > w). One load of v's row
// pointers gives each middle's segment of tops; no search is needed.
//
// Counters per w live in
//  - a per-warp shared-memory hash table (vertices with few wedges),
//  - a per-block shared-memory hash table, in three sizes (medium vertices;
//    each size class is launched with shared memory for its own tables),
//  - a dense shared-memory array of 16-bit counters over a window of the
//    top-ranked ("hub") vertices plus a small shared-memory hash table for the
//    other tops (heavy vertices: most wedges of a power-law graph end at a
//    hub; a count never exceeds the degree of w, so 16 bits suffice for every
//    w of degree below 65536, and the others take the global class),
//  - the dense window with the other tops in a per-block global-memory hash
//    table (heavy vertices with many tops outside the window),
//  - or a global-memory hash table alone (fallback).
// Wedges are walked cooperatively: in the warp class the segments of N+(v) of
// many middles v are concatenated and split evenly over the lanes; in the block
// classes long segments are cut into pieces walked one warp each and short ones
// are walked by groups of lanes.
#include "fglt_device.cuh"
#include "fglt_kernels.h"

namespace fglt {

namespace {

constexpr int WARP_T = 256;
constexpr int DENSE_SPAN_MAX = 90112;  // 16-bit counters: 176 KB of shared memory at most
// The dense class keeps the tops outside its window in a shared table of
// 2^spill_bits slots (11 .. 13, tunable).
constexpr int MID_BITS0 = 11, MID_BITS1 = 12, MID_BITS2 = 13;  // table sizes of the three hash-only block classes
constexpr int MID_BITS[3] = {MID_BITS0, MID_BITS1, MID_BITS2};

int num_sms() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Hash table of (top, count). In shared memory keys and counts are two
// arrays; in global memory slot h is one 8-byte word {keys[2h], keys[2h+1]},
// so that a lookup reads key and count in one access.
template <bool GMEM>
struct Table {
  uint32_t* keys;
  uint32_t* cnts;  // shared tables only
  // global tables: the slots claimed since the last pass C (so that pass C
  // visits only those), with room for tcap entries
  uint32_t* touched = nullptr;
  int* ntouched = nullptr;
  int tcap = 0;
  __device__ __forceinline__ uint32_t* key_at(uint32_t h) const { return GMEM ? keys + 2 * (size_t)h : keys + h; }
  __device__ __forceinline__ uint32_t* cnt_at(uint32_t h) const {
    return GMEM ? keys + 2 * (size_t)h + 1 : cnts + h;
  }
  __device__ __forceinline__ uint32_t load_key(uint32_t h) const {
    if (GMEM) return __ldcg(key_at(h));
    return *((volatile uint32_t*)keys + h);
  }
  __device__ __forceinline__ uint32_t load_cnt(uint32_t h) const {
    if (GMEM) return __ldcg(cnt_at(h));
    return cnts[h];
  }
  __device__ __forceinline__ void clear(uint32_t h) const {
    if (GMEM) {
      __stcg(reinterpret_cast<uint2*>(keys) + h, make_uint2(EMPTY_KEY, 0u));
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
        k = atomicCAS(key_at(h), EMPTY_KEY, key);
        if (k == EMPTY_KEY) {
          k = key;
          if (GMEM) {
            const int pos = atomicAdd(ntouched, 1);
            if (pos < tcap) touched[pos] = h;
            else atomicOr(err, ERR_HASH_FULL);
          }
        }
      }
      if (k == key) {
        atomicAdd(cnt_at(h), 1u);
        return;
      }
      h = (h + 1) & mask;
    }
    atomicOr(err, ERR_HASH_FULL);
  }
  // First level of a two-level table: the key is counted only within the
  // first `window` slots of its probe sequence; false if they all hold other
  // keys (the caller then counts it in the next level). Slots are never freed
  // while the vertex's passes run, so a key that went to the next level never
  // finds room here later, and no key is counted in both levels.
  __device__ __forceinline__ bool increment_window(uint32_t key, int hb, int window) const {
    const uint32_t mask = (1u << hb) - 1;
    uint32_t h = hash_slot(key, hb);
    for (int probe = 0; probe < window; ++probe) {
      uint32_t k = load_key(h);
      if (k == EMPTY_KEY) {
        k = atomicCAS(keys + h, EMPTY_KEY, key);
        if (k == EMPTY_KEY) k = key;
      }
      if (k == key) {
        atomicAdd(cnts + h, 1u);
        return true;
      }
      h = (h + 1) & mask;
    }
    return false;
  }
  // The key's count in the first level (0 if an empty slot ends its window),
  // or -1 if its window is full of other keys (the key is in the next level).
  __device__ __forceinline__ int count_in_window(uint32_t key, int hb, int window) const {
    const uint32_t mask = (1u << hb) - 1;
    uint32_t h = hash_slot(key, hb);
    for (int probe = 0; probe < window; ++probe) {
      const uint32_t k = load_key(h);
      if (k == key) return (int)load_cnt(h);
      if (k == EMPTY_KEY) return 0;
      h = (h + 1) & mask;
    }
    return -1;
  }
  __device__ __forceinline__ uint32_t count_of(uint32_t key, int hb) const {
    const uint32_t mask = (1u << hb) - 1;
    uint32_t h = hash_slot(key, hb);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      if (GMEM) {
        const uint2 e = __ldcg(reinterpret_cast<const uint2*>(keys) + h);
        if (e.x == key) return e.y;
        if (e.x == EMPTY_KEY) return 0u;
      } else {
        const uint32_t k = load_key(h);
        if (k == key) return load_cnt(h);
        if (k == EMPTY_KEY) return 0u;
      }
      h = (h + 1) & mask;
    }
    return 0u;
  }
};

// The middles of one vertex w (rank space): K = nin + nout middles; middle
// k < nin is the in-entry iin[ib + k] = (v, j), later ones are N+(w)[k - nin].
struct Mids {
  const int64_t* orp;
  const int32_t* ocol;
  const int2* iin;
  int64_t ib, nin, ob, K;
};

__device__ __forceinline__ Mids mids_of(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol,
                                        const int64_t* __restrict__ irp, const int2* __restrict__ iin, int32_t w) {
  Mids M;
  M.orp = orp;
  M.ocol = ocol;
  M.iin = iin;
  M.ib = irp[w];
  M.nin = irp[w + 1] - M.ib;
  M.ob = orp[w];
  M.K = M.nin + (orp[w + 1] - M.ob);
  return M;
}

// Middle k of w: its rank v and its segment [st, st + len) of tops in ocol.
// Entries of a malformed graph (never-written in-list slots) give v = -1 and
// an empty segment.
__device__ __forceinline__ void middle_seg(const Mids& M, int64_t k, int64_t n, int32_t& v, int64_t& st,
                                           int64_t& len) {
  int32_t j = -1;
  if (k < M.nin) {
    const int2 e = __ldg(M.iin + M.ib + k);
    v = e.x;
    j = e.y;
  } else {
    v = __ldg(M.ocol + M.ob + (k - M.nin));
  }
  st = 0;
  len = 0;
  if ((uint32_t)v >= (uint64_t)n) {
    v = -1;
    return;
  }
  const int64_t b = __ldg(M.orp + v), e = __ldg(M.orp + v + 1);
  st = b + (int64_t)j + 1;
  if (st < b) st = b;
  len = e > st ? e - st : 0;
}

// One group of up to 32 middles of w (middle k0 + lane per lane): each lane
// owns one v and its segment of tops; the concatenated segments are split over
// the lanes. f(u, owner_lane) is called for every wedge.
struct Group {
  int32_t rv;     // rank of this lane's v (-1 if none)
  int64_t st;     // segment start in ocol
  int64_t excl;   // exclusive prefix of segment lengths
  int64_t total;  // wedges in the group
};

__device__ __forceinline__ Group make_group(const Mids& M, int64_t k, int64_t n, int lane) {
  Group g;
  g.rv = -1;
  g.st = 0;
  int64_t len = 0;
  if (k < M.K) middle_seg(M, k, n, g.rv, g.st, len);
  int64_t incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  g.excl = incl - len;
  g.total = __shfl_sync(0xffffffffu, incl, 31);
  return g;
}

template <typename F>
__device__ __forceinline__ void walk_group(const Group& g, const int32_t* __restrict__ ocol, int lane, F f) {
  for (int64_t t0 = 0; t0 < g.total; t0 += 32) {
    const int64_t t = t0 + lane;
    // owner = last lane whose exclusive prefix is <= t (prefixes are non-decreasing)
    int j = 0;
#pragma unroll
    for (int b = 16; b >= 1; b >>= 1) {
      const int64_t p = __shfl_sync(0xffffffffu, g.excl, j + b);
      if (p <= t) j += b;
    }
    const int64_t ost = __shfl_sync(0xffffffffu, g.st, j);
    const int64_t oex = __shfl_sync(0xffffffffu, g.excl, j);
    const bool valid = t < g.total;
    f(valid ? (uint32_t)__ldg(ocol + ost + (t - oex)) : 0u, j, valid);
  }
}

// Sum of x over the lanes of each run of equal owners j (owners are
// non-decreasing over the lanes); the first lane of a run gets the run total.
// 32 bits suffice: one credit is below the degree limit of the library
// (2^21) and a run spans at most 32 lanes.
__device__ __forceinline__ uint32_t run_sum(uint32_t x, int j, bool& head) {
  const int lane = threadIdx.x & 31;
  const int jp = __shfl_up_sync(0xffffffffu, j, 1);
  head = lane == 0 || jp != j;
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const unsigned after = lane == 31 ? 0u : (heads >> (lane + 1));  // run heads after this lane
  const int end = after ? lane + __ffs(after) - 1 : 31;            // last lane of this run
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_down_sync(0xffffffffu, x, o);
    if (lane + o <= end) x += y;
  }
  return x;
}

// ---------------------------------------------------------------------------
// Small vertices: one warp per w, a 2^wbits-slot hash table per warp.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(WARP_T) k_cyc_warp(const int64_t* __restrict__ orp,
                                                     const int32_t* __restrict__ ocol,
                                                     const int64_t* __restrict__ irp, const int2* __restrict__ iin,
                                                     const int64_t* __restrict__ wc, const int32_t* __restrict__ list,
                                                     const int32_t* __restrict__ cnt, int* next, u64* r12r, int64_t n,
                                                     int64_t cap_bound, int wbits, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t WH = 1u << wbits;
  u64* acc = reinterpret_cast<u64*>(smem) + warp * 32;
  uint32_t* tables = reinterpret_cast<uint32_t*>(reinterpret_cast<u64*>(smem) + (WARP_T / 32) * 32);
  Table<false> T{tables + (size_t)warp * 2 * WH, tables + (size_t)warp * 2 * WH + WH};
  const int total = *cnt;
  // The table starts empty; pass C empties every slot it reads, so each
  // vertex finds it empty again.
  for (uint32_t i = lane; i < WH; i += 32) T.clear(i);
  __syncwarp();
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(next, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    const int32_t w = list[total - 1 - item];  // lists run in rising rank: the largest vertices first
    int64_t cap = wc[w];
    if (cap > n - 1 - w) cap = n - 1 - w;
    if (cap > cap_bound) cap = cap_bound;
    int hb = 5;
    while ((1LL << hb) < 2 * cap) ++hb;
    if (hb > wbits) hb = wbits;  // the class guarantees 2 * cap <= 2^wbits
    const uint32_t H = 1u << hb;
    acc[lane] = 0;
    __syncwarp();
    const Mids M = mids_of(orp, ocol, irp, iin, w);
    for (int64_t k0 = 0; k0 < M.K; k0 += 32) {
      const Group g = make_group(M, k0 + lane, n, lane);
      walk_group(g, ocol, lane, [&](uint32_t u, int, bool valid) {
        if (valid) T.increment(u, hb, err);
      });
    }
    __syncwarp();
    for (int64_t k0 = 0; k0 < M.K; k0 += 32) {
      const Group g = make_group(M, k0 + lane, n, lane);
      walk_group(g, ocol, lane, [&](uint32_t u, int j, bool valid) {
        u64 c = 0;
        if (valid) {
          c = T.count_of(u, hb);
          c = c > 1 ? c - 1 : 0;
        }
        bool head;
        const uint32_t sum = run_sum((uint32_t)c, valid ? j : -1, head);
        if (head && valid && sum) atomicAdd(&acc[j], (u64)sum);
      });
      __syncwarp();
      if (acc[lane]) {
        atomicAdd(&r12r[g.rv], acc[lane]);
        acc[lane] = 0;
      }
      __syncwarp();
    }
    u64 accw = 0;
    for (uint32_t i = lane; i < H; i += 32) {
      const uint32_t key = T.load_key(i);
      if (key != EMPTY_KEY) {
        const u64 c = T.load_cnt(i);
        if (c >= 2) {
          const u64 v = c * (c - 1) / 2;
          atomicAdd(&r12r[key], v);
          accw += v;
        }
        T.clear(i);
      }
    }
    accw = warp_sum_u64(accw);
    if (lane == 0 && accw) atomicAdd(&r12r[w], accw);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Larger vertices: one block per w. N(w) is taken CH middles at a time;
// the non-empty segments of the chunk are compacted into shared memory with
// their exclusive wedge prefix; long segments are cut into pieces walked one
// warp each, short ones are walked by groups of SHORT_LANES lanes.
//
// MODE 0: hash table in shared memory sized per w (at most 2^13 slots)
// MODE 1: dense 16-bit counters for tops >= hub_lo + a shared spill table
//         (2^sbits slots)
// MODE 3: hash table in global memory sized per w (fallback)
// MODE 4: dense 16-bit counters + a two-level spill table: a shared first
//         level of 2^sbits slots (keys kept within TWO_WINDOW probes), the
//         block's global table sized per w for the keys that find no room
// ---------------------------------------------------------------------------
constexpr int CHUNK_MAX = 512;  // middles per chunk: min(block size, 512)
constexpr int SHORT_LANES = 8;  // lanes per short segment
constexpr int TWO_WINDOW = 16;  // probe window of the shared first level (MODE 4)

// Segments at least long_seg long are cut into pieces of PIECE wedges, walked
// warp-per-piece (coalesced, one owner per piece), so one long segment is
// shared by several warps; shorter ones are walked by lane groups
// (walk_short). Measured at R-MAT s24: pieces of 256 wedges suit the
// shared-hash classes, 512 the dense window with a shared spill table, 2048
// the dense window with a global one (per-piece costs against the imbalance
// of whole segments).

struct Segs {
  int64_t* st;      // [chunk] short segments: start in ocol
  int32_t* pre;     // [chunk + 1] short segments: exclusive wedge prefix
  u64* acc;         // [chunk] short segments: middle credits
  long long* scan;  // [64] block-scan scratch
  int32_t* rv;      // [chunk] short segments: rank of the middle
  int64_t* lst;     // [chunk] long segments: start in ocol
  int32_t* llen;    // [chunk] long segments: length
  int32_t* lrv;     // [chunk] long segments: rank of the middle
  int32_t* lpp;     // [chunk + 1] long segments: exclusive piece prefix
  int* misc;        // [0] short count, [1] piece count, [2] piece cursor, [3] short cursor, [4] long count
};

// Block-wide exclusive scan; *total = sum.
__device__ __forceinline__ long long block_excl_scan(long long x, long long* scratch, long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const long long wv = lane < (int)(blockDim.x >> 5) ? scratch[lane] : 0;
    long long wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    scratch[32 + lane] = wi - wv;
    if (lane == 31) scratch[63] = wi;
  }
  __syncthreads();
  *total = scratch[63];
  const long long r = scratch[32 + warp] + incl - x;
  __syncthreads();
  return r;
}

// Segments of the middles c0 .. c0 + chunk of w: long ones listed with the
// prefix sums of their pieces for the warp-per-piece walk, short non-empty
// ones compacted with their wedge prefix for the group walk (one packed block
// scan).
template <int PIECE>
__device__ __forceinline__ void build_chunk(const Segs& S, const Mids& M, int64_t c0, int64_t n, int chunk,
                                            int long_seg) {
  const int64_t k = c0 + threadIdx.x;
  int32_t rv = -1;
  int64_t st = 0, len = 0;
  if ((int)threadIdx.x < chunk && k < M.K) middle_seg(M, k, n, rv, st, len);
  const bool is_long = len >= long_seg;
  const bool is_short = len > 0 && !is_long;
  // A segment lies in one out-list of the degree order, so len <= sqrt(2 nnz)
  // < 2^16 and a chunk holds fewer than 2^17 pieces and 2^18 short wedges.
  // packed: [short wedge sum : 20 | short count : 11 | long count : 11 | pieces : 22]
  const long long pieces = is_long ? (len + PIECE - 1) / PIECE : 0;
  const long long packed = ((is_short ? len : 0LL) << 44) | ((long long)is_short << 33) |
                           ((long long)is_long << 22) | pieces;
  long long tot;
  const long long ex = block_excl_scan(packed, S.scan, &tot);
  if (is_short) {
    const int pos = (int)((ex >> 33) & 0x7FF);
    S.st[pos] = st;
    S.pre[pos] = (int32_t)(ex >> 44);
    S.rv[pos] = rv;
    S.acc[pos] = 0;
  } else if (is_long) {
    const int pos = (int)((ex >> 22) & 0x7FF);
    S.lst[pos] = st;
    S.llen[pos] = (int32_t)len;
    S.lrv[pos] = rv;
    S.lpp[pos] = (int32_t)(ex & 0x3FFFFF);
  }
  if (threadIdx.x == 0) {
    const int ns = (int)((tot >> 33) & 0x7FF);
    const int nl = (int)((tot >> 22) & 0x7FF);
    S.misc[0] = ns;
    S.misc[1] = (int)(tot & 0x3FFFFF);
    S.misc[2] = 0;
    S.misc[3] = 0;
    S.misc[4] = nl;
    S.pre[ns] = (int32_t)(tot >> 44);
    S.lpp[nl] = (int32_t)(tot & 0x3FFFFF);
  }
  __syncthreads();
}

// Long segments: warps take pieces one at a time from the chunk's queue
// (S.misc[2]); the piece's segment is the last one whose piece prefix is at
// most the piece index (a two-level ballot search over at most 2^10
// prefixes). Lanes stride over the piece (coalesced, four loads in flight).
// g(u) per wedge; done(rv, lane_sum, len) after each piece of len wedges,
// lane_sum the lane's 32-bit sum of g's return values (the caller reduces).
template <int PIECE, typename G, typename D>
__device__ __forceinline__ void walk_long(const Segs& S, const int32_t* __restrict__ ocol, G g, D done) {
  const int lane = threadIdx.x & 31;
  const int np = S.misc[1], nl = S.misc[4];
  for (;;) {
    int i = 0;
    if (lane == 0) i = atomicAdd(&S.misc[2], 1);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= np) break;
    // coarse: lanes test every 32nd prefix; fine: the 32 prefixes after it
    const int c = lane * 32;
    const unsigned mc = __ballot_sync(0xffffffffu, c < nl && S.lpp[c] <= i);
    const int base = (31 - __clz(mc)) * 32;
    const unsigned mf = __ballot_sync(0xffffffffu, base + lane < nl && S.lpp[base + lane] <= i);
    const int sg = base + 31 - __clz(mf);
    const int off = (i - S.lpp[sg]) * PIECE;
    const int32_t* p = ocol + S.lst[sg] + off;
    const int len = min(PIECE, S.llen[sg] - off);
    uint32_t sum = 0;
    for (int q = lane; q < len; q += 128) {
      uint32_t x[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) x[r] = q + 32 * r < len ? (uint32_t)__ldg(p + q + 32 * r) : 0u;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (q + 32 * r < len) sum += g(x[r]);
    }
    done(S.lrv[sg], sum, len);
  }
}

// Short segments: groups of SG lanes take them one at a time from the
// chunk's queue (S.misc[3]); a group's lanes stride over one segment, two
// list loads in flight per lane. g(u) per wedge; with SUM, done(j, s, len) is
// called by the group's first lane with the group's 32-bit sum s of g over
// segment j of len wedges.
template <int SG, bool SUM, typename G, typename D>
__device__ __forceinline__ void walk_short(const Segs& S, const int32_t* __restrict__ ocol, G g, D done) {
  const int lane = threadIdx.x & 31, gl = lane % SG;
  const unsigned gmask = (SG == 32 ? 0xffffffffu : ((1u << SG) - 1u)) << (lane & ~(SG - 1));
  const int ns = S.misc[0];
  for (;;) {
    int j = 0;
    if (gl == 0) j = atomicAdd(&S.misc[3], 1);
    j = __shfl_sync(gmask, j, lane & ~(SG - 1));
    if (j >= ns) break;
    const int32_t* p = ocol + S.st[j];
    const int len = S.pre[j + 1] - S.pre[j];
    uint32_t sum = 0;
    for (int k = gl; k < len; k += 2 * SG) {
      const uint32_t u0 = (uint32_t)__ldg(p + k);
      const uint32_t u1 = k + SG < len ? (uint32_t)__ldg(p + k + SG) : 0u;
      sum += g(u0);
      if (k + SG < len) sum += g(u1);
    }
    if (SUM) {
#pragma unroll
      for (int o = SG / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(gmask, sum, o, SG);
      if (gl == 0) done(j, sum, len);
    }
  }
}

size_t seg_bytes(int ch) {
  return (size_t)ch * 8 * 3 + 64 * 8 + (size_t)(ch + 1) * 4 * 2 + (size_t)ch * 4 * 3 + 32;
}

template <int MODE, int BT>
__global__ void __launch_bounds__(BT) k_cyc_block(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol,
                                                  const int64_t* __restrict__ irp, const int2* __restrict__ iin,
                                                  const int64_t* __restrict__ wc, const int32_t* __restrict__ list,
                                                  const int32_t* __restrict__ cnt, int* next, u64* r12r, int64_t n,
                                                  const int64_t* __restrict__ wcn, int32_t hub_lo, int tbits,
                                                  int dense_words, int long_seg, uint32_t* gkeys, uint32_t* gtouch,
                                                  int64_t cap_bound, int sbits, int* err) {
  constexpr bool DENSE = MODE == 1 || MODE == 4;
  constexpr bool GMEM = MODE == 3 || MODE == 4;
  constexpr bool TWO = MODE == 4;
  constexpr int CH = BT < CHUNK_MAX ? BT : CHUNK_MAX;
  constexpr int PIECE = MODE == 0 ? 256 : (MODE == 4 ? 2048 : 512);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ u64 red[32];
  // dynamic layout: [segments][dense counters][hash keys][hash counts]
  Segs S;
  S.st = reinterpret_cast<int64_t*>(smem);
  S.acc = reinterpret_cast<u64*>(S.st + CH);
  S.lst = reinterpret_cast<int64_t*>(S.acc + CH);
  S.scan = reinterpret_cast<long long*>(S.lst + CH);
  S.pre = reinterpret_cast<int32_t*>(S.scan + 64);
  S.rv = S.pre + CH + 1;
  S.llen = S.rv + CH;
  S.lrv = S.llen + CH;
  S.lpp = S.lrv + CH;
  S.misc = S.lpp + CH + 1;
  uint32_t* after = reinterpret_cast<uint32_t*>(S.misc + 8);
  uint32_t* dense = after;
  uint32_t* hbase = DENSE ? after + dense_words : after;
  __shared__ int s_ntouched;
  Table<GMEM> T;
  if (GMEM) {
    T.keys = gkeys + ((size_t)blockIdx.x << (tbits + 1));  // 2^tbits slots of 8 bytes
    T.cnts = nullptr;
    T.touched = gtouch + ((size_t)blockIdx.x << (tbits - 1));
    T.ntouched = &s_ntouched;
    T.tcap = 1 << (tbits - 1);
  } else {
    T.keys = hbase;
    T.cnts = hbase + (1 << tbits);
  }
  Table<false> T1;  // MODE 4: the shared first level of the spill table
  if (TWO) {
    T1.keys = hbase;
    T1.cnts = hbase + (1 << sbits);
  }
  const int tid = threadIdx.x;
  const int total = *cnt;
  const int hub_n = DENSE ? (int)(n - hub_lo) : 0;

  auto dense_add = [&](uint32_t u) {
    const uint32_t i = u - (uint32_t)hub_lo;
    atomicAdd(&dense[i >> 1], 1u << ((i & 1u) << 4));
  };
  auto dense_get = [&](uint32_t u) -> uint32_t {
    const uint32_t i = u - (uint32_t)hub_lo;
    return (dense[i >> 1] >> ((i & 1u) << 4)) & 0xFFFFu;
  };

  // Every table and the dense window start empty; pass C empties what it
  // reads (for a global table: the slots listed as claimed), so each vertex
  // finds them empty again.
  for (uint32_t i = tid; i < (1u << tbits); i += blockDim.x) T.clear(i);
  for (uint32_t i = tid; TWO && i < (1u << sbits); i += blockDim.x) T1.clear(i);
  if (tid == 0) s_ntouched = 0;
  if (DENSE)
    for (int i = tid; i < (hub_n + 1) >> 1; i += blockDim.x) dense[i] = 0u;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    const int32_t w = list[total - 1 - item];  // lists run in rising rank: the largest vertices first
    int hb = tbits;
    if (!DENSE || GMEM) {
      // distinct tops the table must hold: all of them, or (dense window)
      // those below the window, at most the wedges that reach them
      int64_t cap = GMEM && DENSE ? wcn[w] : wc[w];
      if (cap > n - 1 - w) cap = n - 1 - w;
      if (cap > cap_bound) cap = cap_bound;
      hb = 5;
      while ((1LL << hb) < 2 * cap) ++hb;
      if (hb > tbits) hb = tbits;  // the class (or the table sizing) guarantees 2 * cap <= 2^tbits
    }
    const uint32_t H = 1u << hb;

    const Mids M = mids_of(orp, ocol, irp, iin, w);
    const bool single = M.K <= CH;
    auto count = [&](uint32_t u) {
      if (DENSE && (int32_t)u >= hub_lo) dense_add(u);
      else if (!TWO || !T1.increment_window(u, sbits, TWO_WINDOW)) T.increment(u, hb, err);
    };
    // Every top of a middle's segment was counted in pass A, so cnt[u] >= 1
    // and the credits cnt[u] - 1 of a segment sum to sum(cnt) - (its wedges).
    // The sums stay below 2^30: a piece or short segment has at most 512
    // wedges (2048 in the spill class, whose counts are below 2^16) and a
    // count never exceeds the degree of w (below 2^21).
    auto credit = [&](uint32_t u) -> uint32_t {
      if (DENSE && (int32_t)u >= hub_lo) return dense_get(u);
      const int c1 = TWO ? T1.count_in_window(u, sbits, TWO_WINDOW) : -1;
      return c1 >= 0 ? (uint32_t)c1 : T.count_of(u, hb);
    };
    // Pass A: count the wedges per top u.
    for (int64_t c0 = 0; c0 < M.K; c0 += CH) {
      build_chunk<PIECE>(S, M, c0, n, CH, long_seg);
      walk_long<PIECE>(S, ocol, [&](uint32_t u) -> uint32_t { count(u); return 0u; }, [](int32_t, uint32_t, int) {});
      walk_short<SHORT_LANES, false>(S, ocol, [&](uint32_t u) -> uint32_t { count(u); return 0u; },
                                     [](int, uint32_t, int) {});
      __syncthreads();
    }
    // Pass B: each middle gains cnt[u] - 1 per wedge.
    for (int64_t c0 = 0; c0 < M.K; c0 += CH) {
      if (!single) {
        build_chunk<PIECE>(S, M, c0, n, CH, long_seg);
      } else {
        if (tid == 0) S.misc[2] = S.misc[3] = 0;
        __syncthreads();
      }
      walk_long<PIECE>(S, ocol, credit, [&](int32_t rv, uint32_t sum, int len) {
        const uint32_t v = (uint32_t)warp_sum_i32((int)sum) - (uint32_t)len;
        if ((tid & 31) == 0 && v) atomicAdd(&r12r[rv], (u64)v);
      });
      walk_short<SHORT_LANES, true>(S, ocol, credit, [&](int j, uint32_t sum, int len) {
        const uint32_t v = sum - (uint32_t)len;
        if (v) S.acc[j] += v;  // one group per segment
      });
      __syncthreads();
      const int ns = S.misc[0];
      for (int j = tid; j < ns; j += blockDim.x)
        if (S.acc[j]) atomicAdd(&r12r[S.rv[j]], S.acc[j]);
      __syncthreads();
    }
    // Pass C: top u and bottom w gain binom(cnt[u], 2).
    u64 accw = 0;
    if (DENSE) {
      for (int i = tid; i < (hub_n + 1) >> 1; i += blockDim.x) {
        const uint32_t x = dense[i];  // counters of tops hub_lo + 2i and hub_lo + 2i + 1
        if (x) {
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const u64 c = (x >> (16 * half)) & 0xFFFFu;
            if (c >= 2) {
              const u64 v = c * (c - 1) / 2;
              atomicAdd(&r12r[hub_lo + 2 * i + half], v);
              accw += v;
            }
          }
          dense[i] = 0u;
        }
      }
    }
    if (TWO) {
      for (uint32_t i = tid; i < (1u << sbits); i += blockDim.x) {
        const uint32_t key = T1.load_key(i);
        if (key != EMPTY_KEY) {
          const u64 c = T1.load_cnt(i);
          if (c >= 2) {
            const u64 v = c * (c - 1) / 2;
            atomicAdd(&r12r[key], v);
            accw += v;
          }
          T1.clear(i);
        }
      }
    }
    if (GMEM) {
      const int nt = min(s_ntouched, T.tcap);
      for (int i = tid; i < nt; i += blockDim.x) {
        const uint32_t h = __ldcg(T.touched + i);
        const uint32_t key = T.load_key(h);
        const u64 c = T.load_cnt(h);
        if (c >= 2) {
          const u64 v = c * (c - 1) / 2;
          atomicAdd(&r12r[key], v);
          accw += v;
        }
        T.clear(h);
      }
    } else {
      for (uint32_t i = tid; i < H; i += blockDim.x) {
        const uint32_t key = T.load_key(i);
        if (key != EMPTY_KEY) {
          const u64 c = T.load_cnt(i);
          if (c >= 2) {
            const u64 v = c * (c - 1) / 2;
            atomicAdd(&r12r[key], v);
            accw += v;
          }
          T.clear(i);
        }
      }
    }
    accw = block_sum(accw, red);
    if (tid == 0) {
      if (accw) atomicAdd(&r12r[w], accw);
      if (GMEM) s_ntouched = 0;
    }
    __syncthreads();
  }
}

// Hub cut: hc[v] = entries of N+(v) below hub_lo (rows are sorted).
__global__ void k_hub_cut(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol, int64_t n,
                          int32_t hub_lo, int32_t* hc) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = orp[v], e = orp[v + 1];
    hc[v] = (int32_t)(upper_bound_i32(ocol, b, e, hub_lo - 1) - b);
  }
}

__global__ void k_in_degree(const int32_t* __restrict__ dr, const int32_t* __restrict__ opc, int64_t n,
                            int32_t* indeg) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = dr[v] - opc[v];
    indeg[v] = x > 0 ? x : 0;
  }
}

// In-lists and wedge counts, one warp per oriented row v. For the edge
// v -> w = N+(v)[j]: the in-list of w gets (v, j); w's in-part wedges are the
// d+(v) - j - 1 later entries of N+(v) (those below hub_lo: hc[v] - j - 1);
// v's out-part wedges are all of N+(w) (hc[w] of them below hub_lo).
// A slot beyond w's in-list capacity (only for a malformed graph) is dropped.
__global__ void k_in_fill(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol,
                          const int64_t* __restrict__ irp, const int32_t* __restrict__ hc, int64_t n, int32_t* icur,
                          int2* iin, unsigned long long* wc, unsigned long long* wcn) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int64_t b = orp[v];
    const int d = (int)(orp[v + 1] - b);
    if (d == 0) continue;
    const int hcv = hc[v];
    u64 a = 0, c = 0;
    for (int j = lane; j < d; j += 32) {
      const int32_t w = ocol[b + j];
      if ((uint32_t)w >= (uint64_t)n) continue;
      const int32_t pos = atomicAdd(icur + w, 1);
      if (irp[w] + pos < irp[w + 1]) iin[irp[w] + pos] = make_int2((int32_t)v, j);
      if (d - j - 1 > 0) atomicAdd(wc + w, (u64)(d - j - 1));
      if (hcv - j - 1 > 0) atomicAdd(wcn + w, (u64)(hcv - j - 1));
      a += (u64)(orp[w + 1] - orp[w]);
      c += (u64)hc[w];
    }
    a = warp_sum_u64(a);
    c = warp_sum_u64(c);
    if (lane == 0) {
      if (a) atomicAdd(wc + v, a);
      if (c) atomicAdd(wcn + v, c);
    }
  }
}

// Vertex classes (CYC_CLASSES lists): 0 = warp table, 1..3 = block + shared
// hash table of 2^MID_BITS[c-1] slots, 4 = block + dense hub counters + shared
// hash, 5 = block + dense hub counters + global hash, 6 = block + global hash. Also the stage's total and largest wedge
// counts (work counters).
__global__ void k_cyc_worklists(const int64_t* __restrict__ wc, const int64_t* __restrict__ wcn,
                                const int32_t* __restrict__ dr, int64_t n,
                                int32_t* lists, int64_t list_stride, int32_t* counts, u64* gcap_max, u64* wmax,
                                u64* wsum, u64* cls_wedges, int dense_ok, int64_t cap_bound, int wbits,
                                int64_t dense_min, int spill_bits) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  u64 lmax = 0, lsum = 0;
  u64 csum[CYC_CLASSES] = {};
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); r0 < n; r0 += stride) {
    const int64_t r = r0 + lane;
    int cls = -1;
    int64_t cap = 0;
    if (r < n) {
      lmax = max(lmax, (u64)wc[r]);
      lsum += (u64)wc[r];
    }
    if (r < n && wc[r] >= 2) {
      cap = wc[r];
      if (cap > n - 1 - r) cap = n - 1 - r;
      if (cap > cap_bound) cap = cap_bound;
      const bool dense_fit = dense_ok && dr[r] < 65536;
      if (wc[r] <= (1LL << (wbits - 1))) cls = 0;
      else if (cap > dense_min && dense_fit && wcn[r] <= (1 << (spill_bits - 1))) cls = 4;
      else if (cap <= (1LL << (MID_BITS0 - 1))) cls = 1;
      else if (cap <= (1LL << (MID_BITS1 - 1))) cls = 2;
      else if (cap <= (1LL << (MID_BITS2 - 1))) cls = 3;
      else if (dense_fit) cls = 5;
      else cls = 6;
    }
    if (cls == 5) atomicMax(gcap_max, (u64)min(cap, (int64_t)wcn[r]));
    if (cls == 6) atomicMax(gcap_max, (u64)cap);
#pragma unroll
    for (int c = 0; c < CYC_CLASSES; ++c) {
      if (cls == c) csum[c] += (u64)wc[r];
      const unsigned m = __ballot_sync(0xffffffffu, cls == c);
      int pos = 0;
      if (lane == 0 && m) pos = atomicAdd(&counts[c], __popc(m));
      pos = __shfl_sync(0xffffffffu, pos, 0);
      if (cls == c) lists[c * list_stride + pos + __popc(m & ((1u << lane) - 1))] = (int32_t)r;
    }
  }
  lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, 16));
  lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, 8));
  lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, 4));
  lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, 2));
  lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, 1));
  lsum = warp_sum_u64(lsum);
  if (lane == 0) {
    if (lmax) atomicMax(wmax, lmax);
    if (lsum) atomicAdd(wsum, lsum);
  }
#pragma unroll
  for (int c = 0; c < CYC_CLASSES; ++c) {
    const u64 x = warp_sum_u64(csum[c]);
    if (lane == 0 && x) atomicAdd(cls_wedges + c, x);
  }
}

int occupancy(const void* fn, int threads, size_t smem) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  return per_sm < 1 ? 1 : per_sm;
}

size_t block_smem(int mode, int bt, int tbits, int dense_words) {  // tbits: table bits of modes 0 and 1
  const size_t seg = seg_bytes(bt < CHUNK_MAX ? bt : CHUNK_MAX);
  if (mode == 0) return seg + ((size_t)8 << tbits);
  if (mode == 1) return seg + (size_t)dense_words * 4 + ((size_t)8 << tbits);
  return seg;
}

size_t block_smem_two(int bt, int sbits, int dense_words) {  // MODE 4: dense window + shared first level
  return seg_bytes(bt < CHUNK_MAX ? bt : CHUNK_MAX) + (size_t)dense_words * 4 + ((size_t)8 << sbits);
}

int gmem_blocks() { return num_sms(); }

template <int MODE, int BT>
void launch_block(const CycArgs& a, int cls, int tbits, int dense_words, cudaStream_t st) {
  const size_t smem = MODE == 4 ? block_smem_two(BT, a.spill_bits, dense_words) : block_smem(MODE, BT, tbits, dense_words);
  allow_max_smem(k_cyc_block<MODE, BT>);
  // global-table modes: one table per block, cyc_gmem_blocks() tables
  const int grid = MODE >= 3 ? gmem_blocks() : num_sms() * occupancy((const void*)k_cyc_block<MODE, BT>, BT, smem);
  k_cyc_block<MODE, BT><<<grid, BT, smem, st>>>(a.orp, a.ocol, a.irp, a.iin, a.wc, a.lists + cls * a.list_stride,
                                                a.counts + cls, a.next + cls, a.r12r, a.n, a.wcn, a.hub_lo, tbits,
                                                dense_words, a.long_seg, a.gkeys, a.gtouch, a.cap_bound,
                                                a.spill_bits, a.err);
  note_launch();
}

template <int MODE>
void launch_block_bt(const CycArgs& a, int cls, int tbits, int dense_words, int bt, cudaStream_t st) {
  if (bt >= 1024) launch_block<MODE, 1024>(a, cls, tbits, dense_words, st);
  else if (bt >= 512) launch_block<MODE, 512>(a, cls, tbits, dense_words, st);
  else if (bt >= 256) launch_block<MODE, 256>(a, cls, tbits, dense_words, st);
  else launch_block<MODE, 128>(a, cls, tbits, dense_words, st);
}

}  // namespace

int cyc_dense_span_max() { return DENSE_SPAN_MAX; }

int cyc_fit_spill_bits(int span, int spill_bits, int threads) {
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || optin <= 0)
    optin = 227 * 1024;
  const size_t limit = (size_t)optin - 1024;  // room for the kernel's static shared memory
  const int bt = threads >= 1024 ? 1024 : (threads >= 512 ? 512 : (threads >= 256 ? 256 : 128));
  int b = spill_bits;
  while (b > 11 && block_smem(1, bt, b, (span + 1) / 2) > limit) --b;
  return b;
}
int cyc_block_cap() { return 1 << (MID_BITS[2] - 1); }
int cyc_gmem_blocks() { return gmem_blocks(); }
int cyc_warp_bits_max() { return 10; }

cudaError_t launch_in_lists(const int64_t* orp, const int32_t* ocol, const int32_t* dr, const int32_t* opc,
                            int64_t n, int32_t hub_lo, int32_t* hc, int32_t* indeg, int64_t* irp, void* scan_tmp,
                            int32_t* icur, int2* iin, int64_t* wc, int64_t* wcn, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
  k_hub_cut<<<(unsigned)blocks, 256, 0, st>>>(orp, ocol, n, hub_lo, hc);
  note_launch();
  k_in_degree<<<(unsigned)blocks, 256, 0, st>>>(dr, opc, n, indeg);
  note_launch();
  cudaError_t e = launch_scan_i32_to_i64(indeg, n, irp, scan_tmp, st);
  if (e != cudaSuccess) return e;
  int64_t wblocks = (n * 32 + 255) / 256;
  if (wblocks > (int64_t)num_sms() * 16) wblocks = (int64_t)num_sms() * 16;
  k_in_fill<<<(unsigned)wblocks, 256, 0, st>>>(orp, ocol, irp, hc, n, icur, iin,
                                                reinterpret_cast<u64*>(wc), reinterpret_cast<u64*>(wcn));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_cyc_worklists(const int64_t* wc, const int64_t* wcn, const int32_t* dr, int64_t n, int32_t* lists,
                                 int64_t list_stride, int32_t* counts, u64* gcap_max, u64* wmax, u64* wsum,
                                 u64* cls_wedges, bool dense_ok, int64_t cap_bound, int wbits, int64_t dense_min,
                                 int spill_bits, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
  k_cyc_worklists<<<(unsigned)blocks, 256, 0, st>>>(wc, wcn, dr, n, lists, list_stride, counts, gcap_max, wmax, wsum,
                                                     cls_wedges, dense_ok ? 1 : 0, cap_bound, wbits, dense_min,
                                                     spill_bits);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_cyc(const CycArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  auto mark = [&](int c, int edge) {
    if (!a.ev) return;
    cudaEventRecord(a.ev[2 * c + edge], st);
    if (edge) a.ev_rec[c] = true;
  };
  const int sms = num_sms();
  const int wbits = a.wbits;
  const size_t wsmem = (size_t)(WARP_T / 32) * (32 * 8 + ((size_t)8 << wbits));
  allow_max_smem(k_cyc_warp);
  mark(0, 0);
  k_cyc_warp<<<sms * occupancy((const void*)k_cyc_warp, WARP_T, wsmem), WARP_T, wsmem, st>>>(
      a.orp, a.ocol, a.irp, a.iin, a.wc, a.lists, a.counts, a.next + 0, a.r12r, a.n, a.cap_bound, wbits, a.err);
  note_launch();
  mark(0, 1);
  for (int c = 0; c < 3; ++c) {
    mark(1 + c, 0);
    launch_block_bt<0>(a, 1 + c, MID_BITS[c], 0, a.mid_threads[c], st);
    mark(1 + c, 1);
  }
  const int span = (int)(a.n - a.hub_lo);
  if (span > 0) {
    mark(4, 0);
    launch_block_bt<1>(a, 4, a.spill_bits, (span + 1) / 2, a.heavy_threads, st);
    mark(4, 1);
  }
  if (a.gkeys && span > 0) {
    mark(5, 0);
    launch_block_bt<4>(a, 5, a.gbits, (span + 1) / 2, a.heavy_threads, st);
    mark(5, 1);
  }
  if (a.gkeys) {
    mark(6, 0);
    launch_block_bt<3>(a, 6, a.gbits, 0, a.heavy_threads, st);
    mark(6, 1);
  }
  return cudaGetLastError();
}

}  // namespace fglt
