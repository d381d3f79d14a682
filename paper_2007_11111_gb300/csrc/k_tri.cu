// Triangle passes over the degree-ordered orientation (rank space).
//
// Every triangle {a, b, c} with rank a < b < c is listed exactly once, while
// processing its lowest vertex a: b runs over N+(a), c over N+(b), and c is
// kept when it is also in N+(a). N+(a) lives in a shared-memory hash table
// (key = rank label, value = position in N+(a)). Both out-lists are sorted, so
// the scan of N+(b) stops at the largest element of N+(a).
//
// Pass 1 builds, per vertex a, the symmetric adjacency bitmap of the subgraph
// G_a induced on N+(a) and from it
//   C3(i,j) = |N(i) ∩ N(j)| per oriented edge           (Lemma 2: C3 = A o A^2)
//   c3(i)   = triangles at i = C3 e / 2                  (Lemma 2)
//   d^15(i) = 4-cliques at i = T e / 6, T(i,j) = q_ij^T A q_ij (Sec. 4.3):
//             the 4-cliques {a, x, y, z} with a lowest are the triangles
//             {x, y, z} of G_a, counted per vertex by popcounts of row ANDs
//             (bitmap in shared memory) or, for the largest out-degrees, from
//             the product S S of G_a's adjacency matrix on the tensor cores.
// Pass 2 re-lists the triangles once C3 is final, from their middle vertex
// (in-lists of the oriented graph), and adds, for a triangle {i,j,k},
// C3(j,k) - 1 to i (and likewise for j and k):
//   d^13 = D4,c e / 2 with D4,c = A o (A (C3 - A))       (Sec. 4.3)
#include "fglt_device.cuh"
#include "fglt_kernels.h"
#include "tcgen05.cuh"

namespace fglt {

namespace {

constexpr int TRI_T = 256;       // block size of the classes whose bitmap fits in shared memory
constexpr int TRI_T_BIG = 1024;  // block size of the class with the global-memory bitmap
constexpr size_t SMEM_LIMIT = 227 * 1024;

// Hash table of N+(a): hf slots per element (2 or 4), a power of two.
int hash_bits_for(int D, int hf) {
  int hb = 5;
  while ((1 << hb) < hf * D) ++hb;
  return hb;
}

int num_sms() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

__device__ __forceinline__ void table_insert(uint32_t* keys, int32_t* vals, uint32_t key, int32_t val, int hb,
                                             int* err) {
  const uint32_t mask = (1u << hb) - 1;
  uint32_t h = hash_slot(key, hb);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    if (atomicCAS(&keys[h], EMPTY_KEY, key) == EMPTY_KEY) {
      vals[h] = val;
      return;
    }
    h = (h + 1) & mask;
  }
  atomicOr(err, ERR_HASH_FULL);
}

__device__ __forceinline__ int table_find(const uint32_t* keys, const int32_t* vals, uint32_t key, int hb) {
  const uint32_t mask = (1u << hb) - 1;
  uint32_t h = hash_slot(key, hb);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const uint32_t k = keys[h];
    if (k == key) return vals[h];
    if (k == EMPTY_KEY) return -1;
    h = (h + 1) & mask;
  }
  return -1;
}

// Membership pre-filter: one bit per hashed key, about 16 bits per element
// of N+(a); a clear bit proves the key absent, so most probes of keys not in
// N+(a) cost one shared-memory load.
__device__ __forceinline__ int filter_bits_for(int D) {
  int fb = 5;
  while ((1 << fb) < 16 * D) ++fb;
  return fb;
}

__device__ __forceinline__ uint32_t filter_slot(uint32_t key, int fb) { return (key * 0x85EBCA6Bu) >> (32 - fb); }

__device__ __forceinline__ void filter_set(uint32_t* filt, uint32_t key, int fb) {
  const uint32_t b = filter_slot(key, fb);
  atomicOr(&filt[b >> 5], 1u << (b & 31));
}

__device__ __forceinline__ bool filter_test(const uint32_t* filt, uint32_t key, int fb) {
  const uint32_t b = filter_slot(key, fb);
  return (filt[b >> 5] >> (b & 31)) & 1u;
}

// Scan of the sorted list ocol[bb, be) by a group of G lanes (gl = lane in
// the group, gmask = the group's lanes) up to the first entry above last: PL
// loads per lane per step (G * PL entries), probe(c, k) for each entry
// c = ocol[k] (entries past the end read as INT_MAX). The next step's loads
// are issued before the current step's probes, so two steps' loads are in
// flight while the probes wait on shared memory.
template <int PL, int G, typename P>
__device__ __forceinline__ void scan_sorted(const int32_t* __restrict__ ocol, int64_t bb, int64_t be, int32_t last,
                                            int gl, unsigned gmask, P probe) {
  if (bb >= be) return;
  int32_t c[PL];
#pragma unroll
  for (int t = 0; t < PL; ++t) {
    const int64_t k = bb + gl + G * t;
    c[t] = k < be ? ocol[k] : 0x7fffffff;
  }
  for (int64_t k0 = bb;; k0 += G * PL) {
    // the step after this one is needed unless the list ends or this step
    // already passes last (the group's last entry decides, for all lanes)
    const bool more = k0 + G * PL < be && __shfl_sync(gmask, c[PL - 1], G - 1, G) <= last;
    int32_t nx[PL];
#pragma unroll
    for (int t = 0; t < PL; ++t) {
      const int64_t k = k0 + G * PL + gl + G * t;
      nx[t] = more && k < be ? ocol[k] : 0x7fffffff;
    }
#pragma unroll
    for (int t = 0; t < PL; ++t) probe(c[t], k0 + gl + G * t);
    if (!more) break;
#pragma unroll
    for (int t = 0; t < PL; ++t) c[t] = nx[t];
  }
}

// Lane groups of G lanes, one out-neighbour b of a per group.
template <int G>
struct Groups {
  int first, stride, gl;
  unsigned mask;
  __device__ __forceinline__ Groups(int warp, int nwarps, int lane) {
    first = warp * (32 / G) + lane / G;
    stride = nwarps * (32 / G);
    gl = lane % G;
    mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  }
};

// Tensor-core clique phase of the global-bitmap class (tcgen05, E4M3 inputs,
// f32 accumulators in tensor memory). With S the 0/1 adjacency matrix of G_a,
// k2loc[x] gains sum_y S_xy (S S)_xy: over the edges x-y of G_a, the
// triangles of G_a on each (the row-AND popcounts of the shared-memory
// classes give the same tallies). S is
// symmetric, so the block of S S for a row band X (128 rows) and a column
// span Y (512 columns) is S_X S_Y^T, both operands K-major rows of S, and
// only the blocks on or above the diagonal are formed: spans start at the
// band's first row; a pair (x, y) with y in a later 128-row block adds its
// count to the row tally of x and (by a cross-lane column reduction) to the
// tally of y, a pair in the band's own square block to the row tally only.
// Per chunk of 128 columns of K both bands are expanded from the bitmap to
// bytes (0 or 1.0 in E4M3) in shared memory, in core matrices of 8 rows x 16
// bytes; one thread issues 8 MMAs (two 128 x 256 accumulators, four K steps
// of 32) and commits them to the stage's barrier while the block expands the
// next chunk into the other stage (its bitmap words loaded a chunk ahead).
// The accumulators are read out (and restarted) after at most 4096 columns
// of K, so every f32 sum is an integer below 2^12, exact even for an adder
// that keeps only 14 mantissa bits. The epilogue reads the 128 x 512
// accumulators as 4 lane quarters x 8 column blocks: 32 warps.
constexpr int TC_M = 128, TC_N = 256, TC_SPAN = 2 * TC_N, TC_KC = 128;
constexpr int TC_A_BYTES = TC_M * TC_KC, TC_B_BYTES = TC_SPAN * TC_KC;
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_REGION_WORDS = 2 * TC_STAGE_BYTES / 4;
constexpr uint32_t TC_COLS = 512;                     // tensor-memory columns: two f32 accumulators of 256
constexpr uint64_t TC_WAIT_NS = 2000000000ull;        // default limit of one barrier wait (2 s)
constexpr uint32_t TC_IDESC = tc::idesc_e4m3_f32(TC_M, TC_N);
constexpr int TC_SEG_CHUNKS = 4096 / TC_KC;            // K chunks per accumulator read-out
constexpr int TC_ITEMS = (TC_M + TC_SPAN) * (TC_KC / 32);  // (operand row, bitmap word) pairs per chunk

struct TcState {
  uint64_t* bar;     // [2] stage barriers (one phase per committed chunk)
  uint32_t tmem;     // accumulator base address in tensor memory
  uint32_t g;        // chunks committed by this block so far
  int* abort;        // shared: a barrier wait ran out
  uint64_t wait_ns;  // limit of one barrier wait
};

// 16 bits of a bitmap row -> 16 bytes, bit b -> byte b (0 or 0x38 = 1.0 in E4M3).
__device__ __forceinline__ void expand16(uint32_t bits, uint4* dst) {
  auto nib = [](uint32_t n) { return ((n * 0x00204081u) & 0x01010101u) * 0x38u; };
  uint4 v;
  v.x = nib(bits & 15u);
  v.y = nib((bits >> 4) & 15u);
  v.z = nib((bits >> 8) & 15u);
  v.w = nib((bits >> 12) & 15u);
  *dst = v;
}

// Column sums across the warp (v holds f32 bit patterns): lane L ends with
// the sum over all 32 lanes of v[L % 16] (recursive halving, 16 shuffles).
__device__ __forceinline__ float warp_column_sums16(uint32_t (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool upper = lane & o;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const uint32_t give = upper ? v[k] : v[k + o];
      const uint32_t keep = upper ? v[k + o] : v[k];
      v[k] = __float_as_uint(__uint_as_float(keep) + __uint_as_float(__shfl_xor_sync(0xffffffffu, give, o)));
    }
  }
  return __uint_as_float(v[0]) + __uint_as_float(__shfl_xor_sync(0xffffffffu, v[0], 16));
}

// False if a barrier wait ran out (all threads return together).
template <int BT>
__device__ __forceinline__ bool hub_cliques_tc(const uint32_t* __restrict__ bm, int D, int W, int WS,
                                               uint32_t* k2loc, unsigned char* smem, TcState& T) {
  static_assert(BT == 1024, "the epilogue maps 32 warps onto the accumulators");
  constexpr int PER = (TC_ITEMS + BT - 1) / BT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nk = (D + TC_KC - 1) / TC_KC;
  const uint32_t sbase = tc::smem_addr(smem);
  // item i: operand row i / 4 (A rows, then B rows), word i % 4 of the chunk
  // This thread's items: operand rows (tid / 4) + 256 t, bitmap word tid % 4
  // of each chunk. Per span, each item's bitmap row (null past D, or in the
  // B rows of a second accumulator the span does not need) and its offset in
  // a stage are fixed.
  const int jw = tid & 3;
  const uint32_t* src[PER];
  uint32_t dst[PER];
  auto setup = [&](int x0, int y0, bool hi_on) {
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int i = tid + t * BT;
      const int r = i >> 2;
      const bool isA = r < TC_M;
      const int rr = isA ? r : r - TC_M;
      const int row = isA ? x0 + rr : y0 + rr;
      const bool need = i < TC_ITEMS && (isA || hi_on || rr < TC_N);
      src[t] = need && row < D ? bm + (size_t)row * WS + jw : nullptr;
      dst[t] = need ? (uint32_t)((isA ? 0 : TC_A_BYTES) + (rr >> 3) * (8 * TC_KC) + (rr & 7) * 16 + jw * 256)
                    : 0xFFFFFFFFu;
    }
  };
  auto load = [&](uint32_t (&v)[PER], int c) {
    const int kw = c * (TC_KC / 32) + jw;
#pragma unroll
    for (int t = 0; t < PER; ++t) v[t] = (src[t] && kw < W) ? __ldcg(src[t] + c * (TC_KC / 32)) : 0u;
  };
  auto store = [&](const uint32_t (&v)[PER], unsigned char* stage) {
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      if (dst[t] != 0xFFFFFFFFu) {
        unsigned char* op = stage + dst[t];
        expand16(v[t] & 0xFFFFu, reinterpret_cast<uint4*>(op));
        expand16(v[t] >> 16, reinterpret_cast<uint4*>(op + 128));
      }
    }
  };
  for (int x0 = 0; x0 < D; x0 += TC_M) {
    for (int y0 = x0; y0 < D; y0 += TC_SPAN) {
      // the second accumulator (span rows 256..511) only while they reach into D
      const bool hi_on = y0 + TC_N < D;
      setup(x0, y0, hi_on);
      for (int c0 = 0; c0 < nk; c0 += TC_SEG_CHUNKS) {
        const int c1 = min(nk, c0 + TC_SEG_CHUNKS);
        uint32_t v[PER];
        load(v, c0);
        for (int c = c0; c < c1; ++c, ++T.g) {
          const int s = T.g & 1;
          // the stage's previous chunk must be consumed before it is overwritten
          if (T.g >= 2 && !tc::mbar_wait(&T.bar[s], ((T.g - 2) >> 1) & 1u, T.wait_ns)) *T.abort = 1;
          store(v, smem + s * TC_STAGE_BYTES);
          if (c + 1 < c1) load(v, c + 1);
          tc::fence_async_smem();
          __syncthreads();
          if (*T.abort) return false;
          if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = sbase + s * TC_STAGE_BYTES, b0 = a0 + TC_A_BYTES;
#pragma unroll
            for (int ks = 0; ks < TC_KC / 32; ++ks) {
              // a K step of 32 bytes spans two core matrices along K (128 bytes apart)
              const uint64_t ad = tc::smem_desc(a0 + ks * 256, 128, 8 * TC_KC);
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                if (h == 1 && !hi_on) break;
                const uint64_t bd = tc::smem_desc(b0 + h * (TC_N * TC_KC) + ks * 256, 128, 8 * TC_KC);
                tc::mma_e4m3(T.tmem + h * TC_N, ad, bd, TC_IDESC, (c > c0 || ks > 0) ? 1u : 0u);
              }
            }
            tc::mma_commit(&T.bar[s]);
          }
        }
        // the last commit completes after every MMA of the segment
        const uint32_t gl = T.g - 1;
        // every thread leaves before reading the accumulators if any wait ran out
        const bool done = tc::mbar_wait(&T.bar[gl & 1], (gl >> 1) & 1u, T.wait_ns);
        if (__syncthreads_or(!done)) {
          *T.abort = 1;
          return false;
        }
        tc::fence_after_sync();
        const int q = warp & 3, cb = warp >> 2;
        const int x = x0 + 32 * q + lane;
        float kx = 0.f;
        // column groups at or past D (and so every column of a second
        // accumulator the span skipped) hold nothing to read
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) {
          const int col = cb * 64 + hh * 16;
          if (y0 + col >= D) break;
          uint32_t r[16];
          tc::tmem_ld16(T.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col, r);
          tc::tmem_ld_wait();
          const int yw = (y0 + col) >> 5;
          const uint32_t bits = (x < D && yw < W) ? __ldcg(bm + (size_t)x * WS + yw) >> (col & 16) : 0u;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float f = ((bits >> j) & 1u) ? __uint_as_float(r[j]) : 0.f;
            kx += f;
            r[j] = __float_as_uint(f);
          }
          if (y0 + col >= x0 + TC_M) {  // beyond the band's square block: the pairs (y, x) too
            const float cy = warp_column_sums16(r);
            const int y = y0 + col + lane;
            if (lane < 16 && y < D && cy != 0.f) atomicAdd(&k2loc[y], (uint32_t)cy);
          }
        }
        if (x < D && kx != 0.f) atomicAdd(&k2loc[x], (uint32_t)kx);
        tc::fence_before_sync();
        __syncthreads();
        if (*T.abort) return false;
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Pass 1
//
// S is the symmetric adjacency bitmap of the subgraph G_a induced on N+(a)
// (row x = local neighbours of x inside N+(a)). From it, per local vertex x:
//   popc(S_x)                      triangles {a, x, .}  -> C3(a,x), c3(x)
//   sum_{y in S_x} popc(S_x & S_y) twice the triangles of G_a through x,
//                                  i.e. twice the 4-cliques {a, x, ., .}
// and a's own counts are the sums over x divided by 2 and 6.
// ---------------------------------------------------------------------------
// Shared-memory words of the region of the global-bitmap class that holds,
// in turn, the probe tables of N+(a) (hash keys and values, filter) with one
// row of scratch bits per lane group (the class scans with 32-lane groups:
// one per warp of its 1024-thread blocks), and the two operand stages of the
// tensor-core clique phase; the clique tallies follow it.
constexpr int HUB_GROUPS_MAX = TRI_T_BIG / 32;
__host__ __device__ __forceinline__ size_t hub_region_words(int Hbits, int fwords, int Wmax) {
  const size_t table = 2 * ((size_t)1 << Hbits) + (size_t)fwords + (size_t)HUB_GROUPS_MAX * (size_t)Wmax;
  return table > (size_t)TC_REGION_WORDS ? table : (size_t)TC_REGION_WORDS;
}

constexpr int TRI_YL = 256;  // y-list entries per warp in the clique phase of the shared-memory classes

template <bool SMEM_BM, bool K4, int PL, int G, int BT>
__global__ void __launch_bounds__(BT)
    k_tri1(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol, const int32_t* __restrict__ work,
           const int32_t* __restrict__ nwork, int* next, int Dmax, int Hbits, int hf, int32_t* C3o, u64* c3r,
           u64* k4r, uint32_t* gbm, u64* work_ctr, int* err, uint64_t wait_ns) {
  static_assert(SMEM_BM || G == 32, "the global-bitmap class keeps one scratch row per warp");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ u64 red[32];
  const int Hmax = 1 << Hbits, Wmax = (Dmax + 31) >> 5;
  const int FWmax = (1 << filter_bits_for(Dmax)) >> 5;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  uint32_t* keys = reinterpret_cast<uint32_t*>(smem);
  int32_t* vals = reinterpret_cast<int32_t*>(keys + Hmax);
  uint32_t* filt = reinterpret_cast<uint32_t*>(vals + Hmax);
  // Shared-memory bitmap: [per-warp lists][bitmap][tallies] in shared memory.
  // Otherwise the bitmap lives in this block's slot of gbm, and shared memory
  // holds [probe tables | tensor-core operand stages][tallies].
  int32_t* lists_base = nullptr;
  uint32_t* bm;
  uint32_t* k2loc;  // [Dmax] per-vertex 4-clique tallies
  if (SMEM_BM) {
    lists_base = reinterpret_cast<int32_t*>(filt + FWmax);
    bm = reinterpret_cast<uint32_t*>(lists_base + nwarps * (TRI_YL + Wmax));
    k2loc = bm + (size_t)Dmax * (Wmax + 1);
  } else {
    bm = gbm + (size_t)blockIdx.x * ((size_t)Dmax * (Wmax + 1));
    k2loc = reinterpret_cast<uint32_t*>(smem) + hub_region_words(Hbits, FWmax, Wmax);
  }
  int32_t* ylist = SMEM_BM ? lists_base + warp * (TRI_YL + Wmax) : nullptr;
  int32_t* wlist = SMEM_BM ? ylist + TRI_YL : nullptr;
  const int total = *nwork;
  const unsigned below = (1u << lane) - 1u;

  // Global-bitmap class: each lane group collects the row of its b in shared
  // memory (the upper triangle of S: c after b), stores it to the bitmap in
  // global memory once, and a transpose pass fills the lower triangle. The
  // scratch rows are cleared per vertex (the clique phase's operand stages
  // overwrite them) and after each use.
  uint32_t* gscr = SMEM_BM ? nullptr : filt + FWmax;

  // Global-bitmap class with cliques: tensor memory for the accumulators and
  // the two stage barriers of the tensor-core clique phase.
  constexpr bool TCP = !SMEM_BM && K4;
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  TcState T{s_bar, 0u, 0u, &s_abort, wait_ns};
  if (TCP) {
    if (tid == 0) {
      tc::mbar_init(&s_bar[0], 1);
      tc::mbar_init(&s_bar[1], 1);
      tc::mbar_init_fence();
      s_abort = 0;
    }
    if (warp == 0) {
      tc::tmem_alloc(&s_tmem, TC_COLS);
      tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    T.tmem = s_tmem;
  }

  for (;;) {
    if (tid == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    const int a = work[total - 1 - item];  // lists run in rising rank: the largest vertices first
    const int64_t base = orp[a];
    const int D = (int)(orp[a + 1] - base);
    int hb = 5;
    while ((1 << hb) < hf * D) ++hb;
    const int fb = filter_bits_for(D);
    const int W = (D + 31) >> 5;

    for (int i = tid; i < (1 << hb); i += blockDim.x) keys[i] = EMPTY_KEY;
    for (int i = tid; i < (1 << (fb - 5)); i += blockDim.x) filt[i] = 0u;
    // bitmap rows at an odd stride of words: lanes reading different rows
    // at the same word offset hit different shared-memory banks
    const int WS = W | 1;
    for (int i = tid; SMEM_BM && i < D * WS; i += blockDim.x) bm[i] = 0u;  // global rows are stored whole
    for (int i = tid; !SMEM_BM && i < HUB_GROUPS_MAX * W; i += blockDim.x) gscr[(i / W) * Wmax + i % W] = 0u;
    for (int i = tid; K4 && i < D; i += blockDim.x) k2loc[i] = 0u;
    __syncthreads();
    for (int x = tid; x < D; x += blockDim.x) {
      const uint32_t key = (uint32_t)ocol[base + x];
      table_insert(keys, vals, key, x, hb, err);
      filter_set(filt, key, fb);
    }
    __syncthreads();

    // Triangles {a, b, c}: c in N+(b) ∩ N+(a); N+(b) is sorted, so the scan
    // stops at the first step beyond the largest element of N+(a).
    const int32_t lastA = ocol[base + D - 1];
    uint32_t probes = 0;  // this vertex's scanned entries (32 bits: bounded by D times an out-degree)
    const Groups<G> grp(warp, nwarps, lane);
    for (int ib = grp.first; ib < D; ib += grp.stride) {
      const int32_t b = ocol[base + ib];
      const int64_t bb = orp[b], be = orp[b + 1];
      uint32_t* row = bm + (size_t)ib * WS;
      uint32_t* srow = SMEM_BM ? row : gscr + (size_t)grp.first * Wmax;
      auto probe = [&](int32_t c, int64_t k) {
        if (c <= lastA) {
          ++probes;
          if (filter_test(filt, (uint32_t)c, fb)) {
            const int ic = table_find(keys, vals, (uint32_t)c, hb);
            if (ic >= 0) {
              atomicOr(&srow[ic >> 5], 1u << (ic & 31));
              if (SMEM_BM) atomicOr(&bm[(size_t)ic * WS + (ib >> 5)], 1u << (ib & 31));
              atomicAdd(&C3o[k], 1);  // edge b -> c
            }
          }
        }
      };
      scan_sorted<PL, G>(ocol, bb, be, lastA, grp.gl, grp.mask, probe);
      if (!SMEM_BM) {  // row ib (upper triangle) to global memory, scratch back to zero
        __syncwarp(grp.mask);
        for (int w = grp.gl; w < W; w += G) {
          __stcg(row + w, srow[w]);
          srow[w] = 0u;
        }
        __syncwarp(grp.mask);
      }
    }
    __syncthreads();
    if (!SMEM_BM) {
      // Lower triangle: the 32 x 32 tile (J, I) of S is the transpose of the
      // upper tile (I, J), J >= I; a diagonal tile is ORed with its transpose.
      // Tile row r of (I, J) is lane r's word; ballot b gathers column b.
      for (int t = warp; t < W * W; t += nwarps) {
        const int I = t / W, J = t % W;
        if (J < I) continue;
        const int r0 = 32 * I + lane;
        const uint32_t wv = r0 < D ? __ldcg(bm + (size_t)r0 * WS + J) : 0u;
        uint32_t mine = 0u;
#pragma unroll
        for (int b2 = 0; b2 < 32; ++b2) {
          const uint32_t col = __ballot_sync(0xffffffffu, (wv >> b2) & 1u);
          if (lane == b2) mine = col;
        }
        const int r1 = 32 * J + lane;
        if (r1 < D) __stcg(bm + (size_t)r1 * WS + I, I == J ? (wv | mine) : mine);
      }
      __syncthreads();
    }

    // Per local vertex x: triangles through edge a-x (popc S_x). Per edge x-y
    // of G_a: t = |S_x ∩ S_y| triangles of G_a on that edge, added to both
    // ends, so k2loc[x] ends as twice the triangles of G_a at x, i.e. twice
    // the 4-cliques {a, x, ., .} (tensor-core products in the global-bitmap
    // class, row-AND popcounts over y > x otherwise).
    u64 tri2x = 0;
    if (!SMEM_BM) {
      for (int x = warp; x < D; x += nwarps) {
        const uint32_t* Sx = bm + (size_t)x * WS;
        int deg = 0;
        for (int w = lane; w < W; w += 32) deg += __popc(__ldcg(Sx + w));
        deg = warp_sum_i32(deg);
        if (lane == 0) {
          if (deg) {
            atomicAdd(&C3o[base + x], deg);
            atomicAdd(&c3r[ocol[base + x]], (u64)deg);
          }
          tri2x += (u64)deg;
        }
      }
      if constexpr (TCP) {
        if (!hub_cliques_tc<BT>(bm, D, W, WS, k2loc, smem, T)) break;
      }
    }
    for (int x = warp; SMEM_BM && x < D; x += nwarps) {
      const uint32_t* Sx = bm + (size_t)x * WS;
      int deg = 0, nzw = 0;
      const int xw = x >> 5;
      const uint32_t above = ~((2u << (x & 31)) - 1u);  // bits of the word of x above x
      for (int w0 = 0; w0 < W; w0 += 32) {
        const int w = w0 + lane;
        const uint32_t bits = w < W ? Sx[w] : 0u;
        const unsigned mz = __ballot_sync(0xffffffffu, bits != 0u);
        if (bits) wlist[nzw + __popc(mz & below)] = w;
        nzw += __popc(mz);
        deg += warp_sum_i32(__popc(bits));
      }
      __syncwarp();
      if (K4) {
        // neighbours y > x of x, TRI_YL columns at a time
        uint32_t kx = 0;
        for (int yw0 = xw; yw0 < W; yw0 += TRI_YL / 32) {
          const int w = yw0 + lane;
          uint32_t ub = 0u;
          if (lane < TRI_YL / 32 && w < W) {
            const uint32_t bits = Sx[w];
            ub = w > xw ? bits : (w == xw ? bits & above : 0u);
          }
          const int c = __popc(ub);
          int incl = c;
#pragma unroll
          for (int o = 1; o < TRI_YL / 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          int p = incl - c;
          while (ub) {
            const int t = __ffs(ub) - 1;
            ub &= ub - 1;
            ylist[p++] = (w << 5) + t;
          }
          const int nyl = __shfl_sync(0xffffffffu, incl, TRI_YL / 32 - 1);
          __syncwarp();
          for (int i = lane; i < nyl; i += 32) {
            const int y = ylist[i];
            const uint32_t* Sy = bm + (size_t)y * WS;
            uint32_t t = 0;
            for (int q = 0; q < nzw; ++q) {
              const int ww = wlist[q];
              t += __popc(Sx[ww] & Sy[ww]);
            }
            if (t) {
              atomicAdd(&k2loc[y], t);
              kx += t;
            }
          }
          __syncwarp();
        }
        kx = (uint32_t)warp_sum_i32((int)kx);
        if (lane == 0 && kx) atomicAdd(&k2loc[x], kx);
      }
      if (lane == 0) {
        if (deg) {
          const int32_t vx = ocol[base + x];
          atomicAdd(&C3o[base + x], deg);
          atomicAdd(&c3r[vx], (u64)deg);
        }
        tri2x += (u64)deg;
      }
      __syncwarp();
    }
    u64 k4_6x = 0;
    if (K4) {
      __syncthreads();
      for (int x = tid; x < D; x += blockDim.x) {
        const uint32_t k2 = k2loc[x];
        if (k2) {
          atomicAdd(&k4r[ocol[base + x]], (u64)(k2 / 2));
          k4_6x += k2;
        }
      }
    }
    const u64 tri_sum = block_sum(tri2x, red) / 2;
    const u64 k4_sum = block_sum(k4_6x, red) / 6;
    const u64 probe_sum = block_sum((u64)probes, red);
    if (tid == 0) {
      if (tri_sum) atomicAdd(&c3r[a], tri_sum);
      if (k4_sum) atomicAdd(&k4r[a], k4_sum);
      atomicAdd(&work_ctr[0], probe_sum);
      atomicAdd(&work_ctr[1], tri_sum);
      atomicAdd(&work_ctr[2], k4_sum);
    }
    __syncthreads();
  }
  if (TCP) {
    // after a wait ran out: wait (bounded) for the block's last MMAs before
    // the tensor memory is released
    if (s_abort) {
      if (tid == 0) atomicOr(err, ERR_TIMEOUT);
      if (T.g > 0) tc::mbar_wait(&s_bar[(T.g - 1) & 1], ((T.g - 1) >> 1) & 1u, TC_WAIT_NS);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
      tc::fence_after_sync();
      tc::tmem_dealloc(T.tmem, TC_COLS);
    }
  }
}

// ---------------------------------------------------------------------------
// Pass 2, listed from the middle vertex: a block takes a vertex b and holds
// N+(b) in a shared hash table, with C3(b, c) beside each entry. For every
// in-entry (a, j) of b (b = N+(a)[j], so C3(a, b) = C3o[orp[a] + j]) a lane
// group scans the tail of N+(a) after position j up to max N+(b); a hit c
// closes the triangle {a, b, c} with a < b < c, found once. Its three
// corners gain the opposite edge's C3 - 1: a gains C3(b, c) - 1 (summed per
// scan), b gains C3(a, c) - 1 (C3o at the scanned position, summed per
// block), c gains C3(a, b) - 1 (shared tally per entry of N+(b)). The scans
// cover sum_a binom(d+(a), 2) entries at most, against the per-a listing of
// pass 1, which scans N+(b) for every b in N+(a).
// ---------------------------------------------------------------------------
template <int PL, int BT, int G>
__global__ void __launch_bounds__(BT) k_tri2(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol,
                                                const int64_t* __restrict__ irp, const int2* __restrict__ iin,
                                                const int32_t* __restrict__ work, const int32_t* __restrict__ nwork,
                                                int* next, int Dmax, int Hbits, int hf,
                                                const int32_t* __restrict__ C3o, u64* r13r, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ u64 red[32];
  const int Hmax = 1 << Hbits;
  u64* acc = reinterpret_cast<u64*>(smem);
  uint32_t* keys = reinterpret_cast<uint32_t*>(acc + Dmax);
  int32_t* vals = reinterpret_cast<int32_t*>(keys + Hmax);
  int32_t* tv = vals + Hmax;
  uint32_t* filt = reinterpret_cast<uint32_t*>(tv + Dmax);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int total = *nwork;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    const int b = work[total - 1 - item];  // lists run in rising rank: the largest vertices first
    const int64_t base = orp[b];
    const int D = (int)(orp[b + 1] - base);
    int hb = 5;
    while ((1 << hb) < hf * D) ++hb;
    const int fb = filter_bits_for(D);

    for (int i = tid; i < (1 << hb); i += blockDim.x) keys[i] = EMPTY_KEY;
    for (int i = tid; i < (1 << (fb - 5)); i += blockDim.x) filt[i] = 0u;
    for (int i = tid; i < D; i += blockDim.x) { acc[i] = 0; tv[i] = C3o[base + i]; }
    __syncthreads();
    for (int x = tid; x < D; x += blockDim.x) {
      const uint32_t key = (uint32_t)ocol[base + x];
      table_insert(keys, vals, key, x, hb, err);
      filter_set(filt, key, fb);
    }
    __syncthreads();

    const int32_t lastB = ocol[base + D - 1];
    const int64_t ib0 = irp[b], nin = irp[b + 1] - ib0;
    long long acc_b = 0;
    const Groups<G> grp(warp, nwarps, lane);
    for (int64_t e = grp.first; e < nin; e += grp.stride) {
      const int2 ent = __ldg(iin + ib0 + e);
      const int32_t a = ent.x;
      if (a < 0) continue;  // never-written slot (malformed graph only)
      const int64_t ab = orp[a], ae = orp[a + 1];
      const long long tab = C3o[ab + ent.y];  // C3(a, b)
      long long acca = 0;
      auto probe = [&](int32_t c, int64_t k) {
        if (c <= lastB && filter_test(filt, (uint32_t)c, fb)) {
          const int32_t c3ac = C3o[k];  // issued before the table probe so that the two overlap
          const int ic = table_find(keys, vals, (uint32_t)c, hb);
          if (ic >= 0) {
            acca += (long long)tv[ic] - 1;   // a: opposite edge b-c
            acc_b += (long long)c3ac - 1;    // b: opposite edge a-c
            if (tab > 1) atomicAdd(&acc[ic], (u64)(tab - 1));  // c: opposite edge a-b
          }
        }
      };
      scan_sorted<PL, G>(ocol, ab + ent.y + 1, ae, lastB, grp.gl, grp.mask, probe);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acca += __shfl_xor_sync(grp.mask, acca, o, G);
      if (grp.gl == 0 && acca) atomicAdd(&r13r[a], (u64)acca);
    }
    __syncthreads();
    for (int x = tid; x < D; x += blockDim.x)
      if (acc[x]) atomicAdd(&r13r[ocol[base + x]], acc[x]);
    const u64 sb = block_sum((u64)acc_b, red);
    if (tid == 0 && sb) atomicAdd(&r13r[b], sb);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Small out-degree (|N+(a)| <= 32): one warp per vertex a, no block barriers.
// Each bitmap row of G_a is one word, so the 4-clique tallies are per-lane
// popcounts. Per warp: a 128-slot hash table of N+(a) (at most 4 slots per
// element), a 512-bit filter, the bitmap rows and the tallies.
// ---------------------------------------------------------------------------
constexpr int TW_MAX = 32;      // largest out-degree of the warp class
constexpr int TW_HBITS = 7;     // 128 slots
constexpr int TW_FBITS = 9;     // 512-bit filter
constexpr int TW_T = 256;       // 8 warps per block
struct WarpTri {                // per-warp shared memory
  uint32_t keys[1 << TW_HBITS];
  int32_t vals[1 << TW_HBITS];
  uint32_t filt[(1 << TW_FBITS) / 32];
  uint32_t S[TW_MAX];
  uint32_t k2[TW_MAX];
  u64 acc[TW_MAX];
  int32_t tv[TW_MAX];
};

// Loads N+(a) into the warp's table and filter; returns the lane's element
// (or 0x7fffffff past D) and sets *D, *base.
__device__ __forceinline__ int32_t warp_load_out(WarpTri& w, const int64_t* __restrict__ orp,
                                                 const int32_t* __restrict__ ocol, int32_t a, int lane, int* D,
                                                 int64_t* base, int* hb, int* err) {
  *base = orp[a];
  *D = (int)(orp[a + 1] - *base);
  if (*D > TW_MAX || *D < 1) {  // outside the class (a sizing bug): flag it, skip the vertex
    if (lane == 0) atomicOr(err, ERR_INTERNAL);
    *D = 0;
    return 0x7fffffff;
  }
  int b = 5;
  while ((1 << b) < 4 * *D) ++b;
  *hb = b;
  for (int i = lane; i < (1 << b); i += 32) w.keys[i] = EMPTY_KEY;
  if (lane < (1 << TW_FBITS) / 32) w.filt[lane] = 0u;
  __syncwarp();
  const int32_t x = lane < *D ? ocol[*base + lane] : 0x7fffffff;
  if (lane < *D) {
    table_insert(w.keys, w.vals, (uint32_t)x, lane, b, err);
    filter_set(w.filt, (uint32_t)x, TW_FBITS);
  }
  __syncwarp();
  return x;
}

template <int PL, bool K4>
__global__ void __launch_bounds__(TW_T) k_tri1_warp(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol,
                                                    const int32_t* __restrict__ work,
                                                    const int32_t* __restrict__ nwork, int* next, int32_t* C3o,
                                                    u64* c3r, u64* k4r, u64* work_ctr, int* err) {
  __shared__ WarpTri sw[TW_T / 32];
  const int lane = threadIdx.x & 31;
  WarpTri& w = sw[threadIdx.x >> 5];
  const int total = *nwork;
  u64 probes = 0, tri_total = 0, k4_total = 0;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(next, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    const int32_t a = work[total - 1 - item];  // the largest vertices first
    int D, hb;
    int64_t base;
    const int32_t x = warp_load_out(w, orp, ocol, a, lane, &D, &base, &hb, err);
    if (D < 2) continue;  // a single out-neighbour closes no triangle with a lowest
    w.S[lane] = 0u;
    w.k2[lane] = 0u;
    __syncwarp();
    const int32_t lastA = __shfl_sync(0xffffffffu, x, D - 1);
    uint32_t vprobes = 0;  // this vertex's scanned entries
    for (int ib = 0; ib < D; ++ib) {
      const int32_t b = __shfl_sync(0xffffffffu, x, ib);
      const int64_t bb = orp[b], be = orp[b + 1];
      auto probe = [&](int32_t c, int64_t k) {
        if (c <= lastA) {
          ++vprobes;
          if (filter_test(w.filt, (uint32_t)c, TW_FBITS)) {
            const int ic = table_find(w.keys, w.vals, (uint32_t)c, hb);
            if (ic >= 0) {
              atomicOr(&w.S[ib], 1u << ic);
              atomicOr(&w.S[ic], 1u << ib);
              atomicAdd(&C3o[k], 1);  // edge b -> c
            }
          }
        }
      };
      scan_sorted<PL, 32>(ocol, bb, be, lastA, lane, 0xffffffffu, probe);
    }
    probes += vprobes;
    __syncwarp();
    const uint32_t Sx = lane < D ? w.S[lane] : 0u;
    const int deg = __popc(Sx);
    if (deg) {
      atomicAdd(&C3o[base + lane], deg);
      atomicAdd(&c3r[x], (u64)deg);
    }
    const u64 tri_a = (u64)warp_sum_i32(deg) / 2;
    if (K4) {
      // per edge x-y of G_a with y > x: t = |S_x ∩ S_y|, added to both ends
      uint32_t up = lane < 31 ? (Sx & ~((2u << lane) - 1u)) : 0u;
      uint32_t kx = 0;
      while (up) {
        const int y = __ffs(up) - 1;
        up &= up - 1;
        const uint32_t t = __popc(Sx & w.S[y]);
        if (t) {
          atomicAdd(&w.k2[y], t);
          kx += t;
        }
      }
      if (kx) atomicAdd(&w.k2[lane], kx);
      __syncwarp();
      const uint32_t k2 = lane < D ? w.k2[lane] : 0u;
      if (k2) atomicAdd(&k4r[x], (u64)(k2 / 2));
      const u64 k4_a = (u64)warp_sum_i32((int)k2) / 6;
      if (lane == 0 && k4_a) atomicAdd(&k4r[a], k4_a);
      k4_total += k4_a;
    }
    if (lane == 0 && tri_a) atomicAdd(&c3r[a], tri_a);
    tri_total += tri_a;
    __syncwarp();
  }
  probes = warp_sum_u64(probes);
  if (lane == 0) {
    if (probes) atomicAdd(&work_ctr[0], probes);
    if (tri_total) atomicAdd(&work_ctr[1], tri_total);
    if (k4_total) atomicAdd(&work_ctr[2], k4_total);
  }
}

// Pass 2 for out-degrees up to 32, from the middle vertex (see k_tri2): one
// warp per b, groups of 8 lanes per in-entry of b.
template <int PL>
__global__ void __launch_bounds__(TW_T) k_tri2_warp(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol,
                                                    const int64_t* __restrict__ irp, const int2* __restrict__ iin,
                                                    const int32_t* __restrict__ work,
                                                    const int32_t* __restrict__ nwork, int* next,
                                                    const int32_t* __restrict__ C3o, u64* r13r, int* err) {
  constexpr int G = 8;
  __shared__ WarpTri sw[TW_T / 32];
  const int lane = threadIdx.x & 31;
  WarpTri& w = sw[threadIdx.x >> 5];
  const int total = *nwork;
  const Groups<G> grp(0, 1, lane);
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(next, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    const int32_t b = work[total - 1 - item];  // the largest vertices first
    int D, hb;
    int64_t base;
    const int32_t x = warp_load_out(w, orp, ocol, b, lane, &D, &base, &hb, err);
    if (D == 0) continue;
    w.acc[lane] = 0;
    w.tv[lane] = lane < D ? C3o[base + lane] : 0;
    __syncwarp();
    const int32_t lastB = __shfl_sync(0xffffffffu, x, D - 1);
    const int64_t ib0 = irp[b], nin = irp[b + 1] - ib0;
    long long acc_b = 0;
    for (int64_t e0 = 0; e0 < nin; e0 += 32 / G) {
      const int64_t e = e0 + grp.first;
      int32_t a = -1;
      int64_t ab = 0, ae = 0;
      long long tab = 0;
      if (e < nin) {
        const int2 ent = __ldg(iin + ib0 + e);
        a = ent.x;
        if (a >= 0) {
          ab = orp[a] + ent.y + 1;
          ae = orp[a + 1];
          tab = C3o[ab - 1];  // C3(a, b)
        }
      }
      long long acca = 0;
      auto probe = [&](int32_t c, int64_t k) {
        if (c <= lastB && filter_test(w.filt, (uint32_t)c, TW_FBITS)) {
          const int32_t c3ac = C3o[k];  // issued before the table probe so that the two overlap
          const int ic = table_find(w.keys, w.vals, (uint32_t)c, hb);
          if (ic >= 0) {
            acca += (long long)w.tv[ic] - 1;  // a: opposite edge b-c
            acc_b += (long long)c3ac - 1;     // b: opposite edge a-c
            if (tab > 1) atomicAdd(&w.acc[ic], (u64)(tab - 1));  // c: opposite edge a-b
          }
        }
      };
      scan_sorted<PL, G>(ocol, ab, ae, lastB, grp.gl, grp.mask, probe);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acca += __shfl_xor_sync(grp.mask, acca, o, G);
      if (grp.gl == 0 && acca) atomicAdd(&r13r[a], (u64)acca);
    }
    __syncwarp();
    if (lane < D && w.acc[lane]) atomicAdd(&r13r[x], w.acc[lane]);
    const u64 sb = (u64)warp_sum_i64(acc_b);
    if (lane == 0 && sb) atomicAdd(&r13r[b], sb);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Pass 2, listed from the lowest vertex a like pass 1 (the scans of N+(b) for
// every b in N+(a)); on graphs whose out-lists mostly stay in L2 this costs
// less than the listing from the middle vertex, whose scans are shorter but
// each needs an in-entry and two row pointers.
// ---------------------------------------------------------------------------
template <int PL, int BT, int G>
__global__ void __launch_bounds__(BT) k_tri2_low(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol,
                                                const int32_t* __restrict__ work, const int32_t* __restrict__ nwork,
                                                int* next, int Dmax, int Hbits, int hf,
                                                const int32_t* __restrict__ C3o,
                                                u64* r13r, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ u64 red[32];
  const int Hmax = 1 << Hbits;
  u64* acc = reinterpret_cast<u64*>(smem);
  uint32_t* keys = reinterpret_cast<uint32_t*>(acc + Dmax);
  int32_t* vals = reinterpret_cast<int32_t*>(keys + Hmax);
  int32_t* tv = vals + Hmax;
  uint32_t* filt = reinterpret_cast<uint32_t*>(tv + Dmax);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int total = *nwork;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    const int a = work[total - 1 - item];  // lists run in rising rank: the largest vertices first
    const int64_t base = orp[a];
    const int D = (int)(orp[a + 1] - base);
    int hb = 5;
    while ((1 << hb) < hf * D) ++hb;
    const int fb = filter_bits_for(D);

    for (int i = tid; i < (1 << hb); i += blockDim.x) keys[i] = EMPTY_KEY;
    for (int i = tid; i < (1 << (fb - 5)); i += blockDim.x) filt[i] = 0u;
    for (int i = tid; i < D; i += blockDim.x) { acc[i] = 0; tv[i] = C3o[base + i]; }
    __syncthreads();
    for (int x = tid; x < D; x += blockDim.x) {
      const uint32_t key = (uint32_t)ocol[base + x];
      table_insert(keys, vals, key, x, hb, err);
      filter_set(filt, key, fb);
    }
    __syncthreads();

    const int32_t lastA = ocol[base + D - 1];
    long long acc_a = 0;
    const Groups<G> grp(warp, nwarps, lane);
    for (int ib = grp.first; ib < D; ib += grp.stride) {
      const int32_t b = ocol[base + ib];
      const int64_t bb = orp[b], be = orp[b + 1];
      const long long tab = tv[ib];
      long long accb = 0;
      auto probe = [&](int32_t c, int64_t k) {
        if (c <= lastA && filter_test(filt, (uint32_t)c, fb)) {
          const int32_t c3bc = C3o[k];  // issued before the table probe so that the two overlap
          const int ic = table_find(keys, vals, (uint32_t)c, hb);
          if (ic >= 0) {
            acc_a += (long long)c3bc - 1;  // a: opposite edge b-c
            accb += (long long)tv[ic] - 1;   // b: opposite edge a-c
            if (tab > 1) atomicAdd(&acc[ic], (u64)(tab - 1));  // c: opposite edge a-b
          }
        }
      };
      scan_sorted<PL, G>(ocol, bb, be, lastA, grp.gl, grp.mask, probe);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) accb += __shfl_xor_sync(grp.mask, accb, o, G);
      if (grp.gl == 0 && accb) atomicAdd(&acc[ib], (u64)accb);
    }
    __syncthreads();
    for (int x = tid; x < D; x += blockDim.x)
      if (acc[x]) atomicAdd(&r13r[ocol[base + x]], acc[x]);
    const u64 sa = block_sum((u64)acc_a, red);
    if (tid == 0 && sa) atomicAdd(&r13r[a], sa);
    __syncthreads();
  }
}

// Pass 2 from the lowest vertex for out-degrees up to 32 (see k_tri2_low).
template <int PL>
__global__ void __launch_bounds__(TW_T) k_tri2_warp_low(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol,
                                                    const int32_t* __restrict__ work,
                                                    const int32_t* __restrict__ nwork, int* next,
                                                    const int32_t* __restrict__ C3o, u64* r13r, int* err) {
  __shared__ WarpTri sw[TW_T / 32];
  const int lane = threadIdx.x & 31;
  WarpTri& w = sw[threadIdx.x >> 5];
  const int total = *nwork;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(next, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    const int32_t a = work[total - 1 - item];  // the largest vertices first
    int D, hb;
    int64_t base;
    const int32_t x = warp_load_out(w, orp, ocol, a, lane, &D, &base, &hb, err);
    if (D == 0) continue;
    w.acc[lane] = 0;
    w.tv[lane] = lane < D ? C3o[base + lane] : 0;
    __syncwarp();
    const int32_t lastA = __shfl_sync(0xffffffffu, x, D - 1);
    long long acc_a = 0;
    for (int ib = 0; ib < D; ++ib) {
      const int32_t b = __shfl_sync(0xffffffffu, x, ib);
      const int64_t bb = orp[b], be = orp[b + 1];
      const long long tab = w.tv[ib];
      long long accb = 0;
      auto probe = [&](int32_t c, int64_t k) {
        if (c <= lastA && filter_test(w.filt, (uint32_t)c, TW_FBITS)) {
          const int32_t c3bc = C3o[k];  // issued before the table probe so that the two overlap
          const int ic = table_find(w.keys, w.vals, (uint32_t)c, hb);
          if (ic >= 0) {
            acc_a += (long long)c3bc - 1;   // a: opposite edge b-c
            accb += (long long)w.tv[ic] - 1;  // b: opposite edge a-c
            if (tab > 1) atomicAdd(&w.acc[ic], (u64)(tab - 1));  // c: opposite edge a-b
          }
        }
      };
      scan_sorted<PL, 32>(ocol, bb, be, lastA, lane, 0xffffffffu, probe);
      accb = warp_sum_i64(accb);
      if (lane == 0 && accb) atomicAdd(&w.acc[ib], (u64)accb);
    }
    __syncwarp();
    if (lane < D && w.acc[lane]) atomicAdd(&r13r[x], w.acc[lane]);
    const u64 sa = (u64)warp_sum_i64(acc_a);
    if (lane == 0 && sa) atomicAdd(&r13r[a], sa);
    __syncwarp();
  }
}

int host_filter_words(int D) {
  int fb = 5;
  while ((1 << fb) < 16 * D) ++fb;
  return (1 << fb) >> 5;
}

size_t tri1_smem_impl(int D, bool smem_bm, int hf, int bt = TRI_T) {
  const int H = 1 << hash_bits_for(D, hf);
  const size_t W = (size_t)(D + 31) / 32;
  if (!smem_bm) {  // [probe tables | tensor-core operand stages][tallies]
    const size_t words = hub_region_words(hash_bits_for(D, hf), host_filter_words(D), (int)W) + (size_t)D;
    return (words * 4 + 15) & ~(size_t)15;
  }
  size_t bytes = (size_t)H * 8 + (size_t)host_filter_words(D) * 4;
  bytes += (size_t)D * 4;  // per-vertex 4-clique tallies
  bytes += (size_t)(bt / 32) * (TRI_YL + W) * 4 + (size_t)D * (W + 1) * 4;  // per-warp lists and bitmap
  return (bytes + 15) & ~(size_t)15;
}

int occupancy_grid(const void* fn, size_t smem, int threads = TRI_T) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (per_sm < 1) per_sm = 1;
  return per_sm * num_sms();
}

}  // namespace

size_t tri_smem_limit() { return SMEM_LIMIT - 1024; }  // room for the kernels' static shared memory

bool tri1_bitmap_fits_smem(int dpmax, int hf) { return tri1_smem_impl(dpmax, true, hf) <= tri_smem_limit(); }

int tri1_smem_bitmap_max(int hf) {
  int lo = 2, hi = 1 << 14;  // fits(lo), !fits(hi)
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (tri1_bitmap_fits_smem(mid, hf)) lo = mid; else hi = mid;
  }
  return lo;
}

size_t tri1_smem_bytes(int dpmax, bool bitmap_in_smem, int hf) { return tri1_smem_impl(dpmax, bitmap_in_smem, hf); }

size_t tri2_smem_bytes(int dpmax, int hf) {
  const int H = 1 << hash_bits_for(dpmax, hf);
  return (((size_t)dpmax * 12 + (size_t)H * 8 + (size_t)host_filter_words(dpmax) * 4) + 15) & ~(size_t)15;
}

int tri_grid_blocks() { return num_sms(); }

// Kernel instance for (bitmap in shared memory, cliques, loads, group lanes,
// block size).
template <bool SMEM_BM, bool K4, int BT>
auto tri1_fn(int loads, int g) {
  // the global-bitmap class scans with 32-lane groups (one scratch row per warp)
  if constexpr (!SMEM_BM) {
    return loads >= 4 ? k_tri1<SMEM_BM, K4, 4, 32, BT> : k_tri1<SMEM_BM, K4, 2, 32, BT>;
  } else {
    if (loads >= 4)
      return g >= 32 ? k_tri1<SMEM_BM, K4, 4, 32, BT>
                     : (g >= 16 ? k_tri1<SMEM_BM, K4, 4, 16, BT> : k_tri1<SMEM_BM, K4, 4, 8, BT>);
    return g >= 32 ? k_tri1<SMEM_BM, K4, 2, 32, BT>
                   : (g >= 16 ? k_tri1<SMEM_BM, K4, 2, 16, BT> : k_tri1<SMEM_BM, K4, 2, 8, BT>);
  }
}

template <bool SMEM_BM, int BT>
void allow_tri1() {
  for (int loads : {2, 4})
    for (int g : {8, 16, 32}) {
      allow_max_smem(tri1_fn<SMEM_BM, true, BT>(loads, g));
      allow_max_smem(tri1_fn<SMEM_BM, false, BT>(loads, g));
    }
}

// Block size of a class: the shared-memory-bitmap classes take 256 threads
// unless only one such block fits on an SM, then 1024 (more warps streaming
// out-lists per SM); the global-bitmap class always takes 1024.
static int tri1_threads(int dpmax, bool smem_bm, int hf) {
  if (!smem_bm) return TRI_T_BIG;
  allow_tri1<true, TRI_T>();
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tri1<true, true, 2, 32, TRI_T>, TRI_T,
                                                tri1_smem_impl(dpmax, true, hf));
  return per_sm <= 1 && tri1_smem_impl(dpmax, true, hf, TRI_T_BIG) <= tri_smem_limit() ? TRI_T_BIG : TRI_T;
}

static int tri1_grid(int dpmax, bool smem_bm, int hf) {
  const int bt = tri1_threads(dpmax, smem_bm, hf);
  const size_t smem = tri1_smem_impl(dpmax, smem_bm, hf, bt);
  if (smem_bm && bt == TRI_T) {
    allow_tri1<true, TRI_T>();
    return occupancy_grid((const void*)k_tri1<true, true, 2, 32, TRI_T>, smem);
  }
  if (smem_bm) {
    allow_tri1<true, TRI_T_BIG>();
    return occupancy_grid((const void*)k_tri1<true, true, 2, 32, TRI_T_BIG>, smem, TRI_T_BIG);
  }
  allow_tri1<false, TRI_T_BIG>();
  return occupancy_grid((const void*)k_tri1<false, true, 2, 32, TRI_T_BIG>, smem, TRI_T_BIG);
}

size_t tri1_gbm_bytes(int dpmax, int hf) {
  if (dpmax < 2 || tri1_bitmap_fits_smem(dpmax, hf)) return 0;
  const size_t W = (size_t)(dpmax + 31) / 32;
  const size_t per_block = (size_t)dpmax * (W + 1);  // bitmap rows at an odd stride of at most W + 1 words
  return (size_t)tri1_grid(dpmax, false, hf) * per_block * 4;
}

cudaError_t launch_tri1(const int64_t* orp, const int32_t* ocol, const int32_t* work, const int32_t* nwork,
                        int* next, int dpmax, int32_t* C3o, u64* c3r, u64* k4r, uint32_t* gbm, u64* work_ctr,
                        int* err, cudaStream_t st, bool cliques, int loads, int hf, int group, long long wait_ns) {
  if (dpmax < 2) return cudaSuccess;
  const bool smem_bm = tri1_bitmap_fits_smem(dpmax, hf);
  const int bt = tri1_threads(dpmax, smem_bm, hf);
  const size_t smem = tri1_smem_impl(dpmax, smem_bm, hf, bt);
  const int grid = tri1_grid(dpmax, smem_bm, hf);
  const int hb = hash_bits_for(dpmax, hf);
  auto* fn = smem_bm ? (bt == TRI_T ? (cliques ? tri1_fn<true, true, TRI_T>(loads, group)
                                               : tri1_fn<true, false, TRI_T>(loads, group))
                                    : (cliques ? tri1_fn<true, true, TRI_T_BIG>(loads, group)
                                               : tri1_fn<true, false, TRI_T_BIG>(loads, group)))
                     : (cliques ? tri1_fn<false, true, TRI_T_BIG>(loads, group)
                                : tri1_fn<false, false, TRI_T_BIG>(loads, group));
  fn<<<grid, bt, smem, st>>>(orp, ocol, work, nwork, next, dpmax, hb, hf, C3o, c3r, k4r, smem_bm ? nullptr : gbm,
                             work_ctr, err, wait_ns > 0 ? (uint64_t)wait_ns : TC_WAIT_NS);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tri2(const int64_t* orp, const int32_t* ocol, const int64_t* irp, const int2* iin,
                        const int32_t* work, const int32_t* nwork, int* next, int dpmax, const int32_t* C3o, u64* r13r,
                        int* err, cudaStream_t st, int loads, int hf, int group, bool middle) {
  if (dpmax < 2) return cudaSuccess;
  const size_t smem = tri2_smem_bytes(dpmax, hf);
  if (smem > SMEM_LIMIT) return cudaErrorInvalidConfiguration;
  // the out-degree class beyond the shared-memory bitmap of pass 1 runs with
  // 1024-thread blocks (its tables allow one block per SM)
  const bool big = !tri1_bitmap_fits_smem(dpmax, hf);
  const int threads = big ? TRI_T_BIG : TRI_T;
  const int hb = hash_bits_for(dpmax, hf);
  auto pick = [&](auto f8, auto f16, auto f32) { return group >= 32 ? f32 : (group >= 16 ? f16 : f8); };
  if (middle) {  // the scanned tails are short: 8 lanes per in-entry, except for the largest out-degrees
    auto* fn = big ? (loads >= 4 ? pick(k_tri2<4, TRI_T_BIG, 8>, k_tri2<4, TRI_T_BIG, 16>, k_tri2<4, TRI_T_BIG, 32>)
                                 : pick(k_tri2<2, TRI_T_BIG, 8>, k_tri2<2, TRI_T_BIG, 16>, k_tri2<2, TRI_T_BIG, 32>))
                   : (loads >= 4 ? k_tri2<4, TRI_T, 8> : k_tri2<2, TRI_T, 8>);
    allow_max_smem(fn);
    const int grid = occupancy_grid((const void*)fn, smem, threads);
    fn<<<grid, threads, smem, st>>>(orp, ocol, irp, iin, work, nwork, next, dpmax, hb, hf, C3o, r13r, err);
  } else {
    auto* fn =
        big ? (loads >= 4 ? pick(k_tri2_low<4, TRI_T_BIG, 8>, k_tri2_low<4, TRI_T_BIG, 16>, k_tri2_low<4, TRI_T_BIG, 32>)
                          : pick(k_tri2_low<2, TRI_T_BIG, 8>, k_tri2_low<2, TRI_T_BIG, 16>, k_tri2_low<2, TRI_T_BIG, 32>))
            : (loads >= 4 ? pick(k_tri2_low<4, TRI_T, 8>, k_tri2_low<4, TRI_T, 16>, k_tri2_low<4, TRI_T, 32>)
                          : pick(k_tri2_low<2, TRI_T, 8>, k_tri2_low<2, TRI_T, 16>, k_tri2_low<2, TRI_T, 32>));
    allow_max_smem(fn);
    const int grid = occupancy_grid((const void*)fn, smem, threads);
    fn<<<grid, threads, smem, st>>>(orp, ocol, work, nwork, next, dpmax, hb, hf, C3o, r13r, err);
  }
  note_launch();
  return cudaGetLastError();
}

int tri_warp_max() { return TW_MAX; }

cudaError_t launch_tri1_warp(const int64_t* orp, const int32_t* ocol, const int32_t* work, const int32_t* nwork,
                             int* next, int32_t* C3o, u64* c3r, u64* k4r, u64* work_ctr, int* err, cudaStream_t st,
                             bool cliques, int loads) {
  auto* fn = loads >= 4 ? (cliques ? k_tri1_warp<4, true> : k_tri1_warp<4, false>)
                        : (cliques ? k_tri1_warp<2, true> : k_tri1_warp<2, false>);
  const int grid = occupancy_grid((const void*)fn, 0, TW_T);
  fn<<<grid, TW_T, 0, st>>>(orp, ocol, work, nwork, next, C3o, c3r, k4r, work_ctr, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tri2_warp(const int64_t* orp, const int32_t* ocol, const int64_t* irp, const int2* iin,
                             const int32_t* work, const int32_t* nwork, int* next, const int32_t* C3o, u64* r13r,
                             int* err, cudaStream_t st, int loads, bool middle) {
  if (middle) {
    auto* fn = loads >= 4 ? k_tri2_warp<4> : k_tri2_warp<2>;
    const int grid = occupancy_grid((const void*)fn, 0, TW_T);
    fn<<<grid, TW_T, 0, st>>>(orp, ocol, irp, iin, work, nwork, next, C3o, r13r, err);
  } else {
    auto* fn = loads >= 4 ? k_tri2_warp_low<4> : k_tri2_warp_low<2>;
    const int grid = occupancy_grid((const void*)fn, 0, TW_T);
    fn<<<grid, TW_T, 0, st>>>(orp, ocol, work, nwork, next, C3o, r13r, err);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace fglt
