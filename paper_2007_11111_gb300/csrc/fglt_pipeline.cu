// The stage sequence of one transform (every entry point runs it).
//
//   degree            p1 = A e                                   (Sec. 3.1)
//   spmv1             p2 = A p1 - p1, d^7 = A((p1-1)o(p1-2))/2   (Sec. 3.1, 4.2)
//   rank, orient      degree order; oriented out-lists N+ sorted by rank
//   sort              (the cost model of Appendix A)
//   tri1              C3 = A o A^2 per edge, c3, 4-cliques T     (Lemma 2, Sec. 4.3)
//   c3_edges          d^10 = C3 (p1 - 2), d^14 = D4,3 e / 2      (Sec. 4.2, 4.3)
//   spmv2             p3 = A p2 - p1 o (p1-1) - 2 c3, d^9        (Sec. 4.1, 4.2)
//   wedges            in-lists, wedge counts of the 4-cycle stage
//   tri2              d^13 = D4,c e / 2                          (Sec. 4.3)
//   cyc               c4 = C4,2 e / 2                            (Lemma on c4)
//   epilogue          Table I, then f = U16^{-1} f^              (Table II)
#include "fglt_pipeline.h"

#include <algorithm>
#include <cstring>
#include <initializer_list>

#include <nvtx3/nvToolsExt.h>

#include "fglt_device.cuh"

namespace fglt {

const char* const STAGE_NAMES[NUM_STAGES] = {"degree", "spmv1", "rank", "orient", "sort", "tri1", "c3_edges",
                                             "spmv2", "wedges", "tri2", "cyc", "epilogue"};
const char* const SUB_NAMES[NUM_SUB] = {"cyc.warp",   "cyc.hash11", "cyc.hash12", "cyc.hash13", "cyc.dense",
                                        "cyc.dense_spill", "cyc.global", "tri1.w", "tri1.c0",  "tri1.c1",
                                        "tri1.c2",    "tri1.c3",    "tri2.w",     "tri2.c0",    "tri2.c1",
                                        "tri2.c2",    "tri2.c3"};

namespace {

constexpr int64_t MAX_DEGREE_EXACT = 2097151;  // binom(d,3) products stay inside int64
constexpr int TRI2_WARP_IN = 256;  // pass 2 from the middle vertex: in-entries one warp takes at most

// Small device counters, one int slot each.
enum CounterId {
  C_DMAX, C_NHEAVY, C_DPMAX, C_NTRI0, C_NEXT1_0 = C_NTRI0 + TRI_CLASSES, C_NEXT2_0 = C_NEXT1_0 + TRI_CLASSES,
  C_NCYC0 = C_NEXT2_0 + TRI_CLASSES, C_NEXTC0 = C_NCYC0 + CYC_CLASSES, C_ERR = C_NEXTC0 + CYC_CLASSES, C_NUM
};
// 64-bit work counters: triangle-pass scanned entries, triangles, 4-cliques,
// max and total wedges of the 4-cycle stage, largest global table need.
enum Counter64Id { W_PROBES, W_TRIANGLES, W_K4, W_WMAX, W_WSUM, W_GCAP, W_CLS, W_NUM = W_CLS + CYC_CLASSES };

// One NVTX range per stage of a transform (named as in fglt_stage_times),
// for timeline tools; at most one is open, and the last closes on return.
struct StageRange {
  bool open = false;
  void to(int i) {
    if (open) nvtxRangePop();
    open = i < NUM_STAGES;
    if (open) nvtxRangePushA(STAGE_NAMES[i]);
  }
  ~StageRange() {
    if (open) nvtxRangePop();
  }
};

int bits_for(int64_t cap) {
  int hb = 5;
  while ((1LL << hb) < 2 * cap) ++hb;
  return hb;
}

bool pow2_threads(int t) { return t == 128 || t == 256 || t == 512 || t == 1024; }

}  // namespace

int err_word_index() { return C_ERR; }

// Table II: U16 maps net to raw frequencies, U16 f = f^; row k = raw
// frequency of sigma_k, column l = net frequency of sigma_l.
static const int8_t U16_TABLE[16][16] = {
    {1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 1, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 1, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, 0, 0, 0, 2, 1, 0, 2, 4, 2, 6},
    {0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 1, 2, 2, 2, 4, 6},
    {0, 0, 0, 0, 0, 0, 0, 1, 0, 1, 1, 0, 0, 2, 1, 3},
    {0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 1, 1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 2, 0, 3},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 2, 2, 6},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 2, 3},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 3},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 3},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 3},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1},
};

int dict_columns(uint32_t mask) {
  if (mask == 0) return 16;
  int k = 0;
  for (int i = 0; i < 16; ++i) k += (mask >> i) & 1u;
  return k;
}

fglt_status make_subdict(uint32_t mask, SubDict* sd) {
  if (mask == 0) mask = 0xFFFFu;
  if ((mask & 3u) != 3u || (mask >> 16) != 0) return FGLT_ERR_INVALID_ARG;
  SubDict x{};
  for (int i = 0; i < 16; ++i)
    if ((mask >> i) & 1u) x.col[x.k++] = i;
  // U(s,s) is unit upper triangular; its inverse X solves U X = I by back
  // substitution, column by column, in exact integers.
  for (int c = 0; c < x.k; ++c)
    for (int r = c; r >= 0; --r) {
      long long v = (r == c) ? 1 : 0;
      for (int t = r + 1; t <= c; ++t) v -= (long long)U16_TABLE[x.col[r]][x.col[t]] * x.uinv[t][c];
      x.uinv[r][c] = v;
    }
  *sd = x;
  return FGLT_OK;
}

fglt_status tuning_from_options(const fglt_options& o, Tuning* t) {
  Tuning x;
  if (o.cyc_hub_span < 0 || o.cyc_hub_span > cyc_dense_span_max() || o.tri_class_bounds[0] < 0 ||
      o.tri_class_bounds[1] < 0 || o.cyc_warp_bits < 0 || o.cyc_heavy_threads < 0)
    return FGLT_ERR_INVALID_ARG;
  x.cyc_hub_span = o.cyc_hub_span;
  if (o.tri_class_bounds[0]) x.tri_t0 = o.tri_class_bounds[0];
  if (o.tri_class_bounds[1]) x.tri_t1 = o.tri_class_bounds[1];
  if (x.tri_t0 < 2 || x.tri_t1 <= x.tri_t0) return FGLT_ERR_INVALID_ARG;
  if (o.tri_probe_loads) x.tri_loads = o.tri_probe_loads;
  if (x.tri_loads != 2 && x.tri_loads != 4) return FGLT_ERR_INVALID_ARG;
  if (o.tri_hash_factor) x.tri_hash_factor = o.tri_hash_factor;
  if (x.tri_hash_factor != 2 && x.tri_hash_factor != 4) return FGLT_ERR_INVALID_ARG;
  if (o.tri_warp_max < -1 || o.tri_warp_max > tri_warp_max()) return FGLT_ERR_INVALID_ARG;
  if (o.tri_warp_max) x.tri_warp = o.tri_warp_max < 0 ? 0 : o.tri_warp_max;
  if (o.tri_group_lanes) x.tri_group = o.tri_group_lanes;
  if (x.tri_group != 8 && x.tri_group != 16 && x.tri_group != 32) return FGLT_ERR_INVALID_ARG;
  if (o.cyc_warp_bits) x.cyc_warp_bits = o.cyc_warp_bits;
  if (x.cyc_warp_bits < 6 || x.cyc_warp_bits > cyc_warp_bits_max()) return FGLT_ERR_INVALID_ARG;
  for (int c = 0; c < 3; ++c) {
    if (o.cyc_mid_threads[c]) x.cyc_mid_threads[c] = o.cyc_mid_threads[c];
    if (!pow2_threads(x.cyc_mid_threads[c])) return FGLT_ERR_INVALID_ARG;
  }
  if (o.cyc_spill_bits) x.cyc_spill_bits = o.cyc_spill_bits;
  if (x.cyc_spill_bits < 11 || x.cyc_spill_bits > 13) return FGLT_ERR_INVALID_ARG;
  if (o.cyc_long_segment) x.cyc_long_segment = o.cyc_long_segment;
  if (x.cyc_long_segment < 2 || x.cyc_long_segment > 512) return FGLT_ERR_INVALID_ARG;
  if (o.cyc_dense_min) x.cyc_dense_min = o.cyc_dense_min;
  if (x.cyc_dense_min < 0 || x.cyc_dense_min > 4096) return FGLT_ERR_INVALID_ARG;
  if (o.cyc_heavy_threads) x.cyc_heavy_threads = o.cyc_heavy_threads;
  if (!pow2_threads(x.cyc_heavy_threads)) return FGLT_ERR_INVALID_ARG;
  if (o.tri_pass2_from < 0 || o.tri_pass2_from > 2) return FGLT_ERR_INVALID_ARG;
  x.tri_pass2 = o.tri_pass2_from;
  *t = x;
  return FGLT_OK;
}

void tuning_to_options(const Tuning& t, fglt_options* o) {
  o->cyc_hub_span = t.cyc_hub_span;
  o->tri_class_bounds[0] = t.tri_t0;
  o->tri_class_bounds[1] = t.tri_t1;
  o->tri_probe_loads = t.tri_loads;
  o->tri_hash_factor = t.tri_hash_factor;
  o->tri_group_lanes = t.tri_group;
  o->tri_warp_max = t.tri_warp ? t.tri_warp : -1;
  o->cyc_warp_bits = t.cyc_warp_bits;
  for (int c = 0; c < 3; ++c) o->cyc_mid_threads[c] = t.cyc_mid_threads[c];
  o->cyc_heavy_threads = t.cyc_heavy_threads;
  o->cyc_dense_min = t.cyc_dense_min;
  o->cyc_long_segment = t.cyc_long_segment;
  o->cyc_spill_bits = t.cyc_spill_bits;
  o->tri_pass2_from = t.tri_pass2;
}

fglt_status run_pipeline(Workspace& ws, const Csr& in, int64_t* out_raw, int64_t* out_net, cudaStream_t st,
                         const RunOptions& ro) {
  const Bounds* b = ro.bounds;
  const bool capturing = ro.capturing;
  const Tuning& tu = ro.tuning;
  // Stages each Table I row needs (a sub-dictionary skips the others).
  SubDict sd;
  {
    fglt_status s = make_subdict(ro.dict_mask, &sd);
    if (s != FGLT_OK) return s;
  }
  const uint32_t mask = ro.dict_mask ? ro.dict_mask : 0xFFFFu;
  auto any = [&](std::initializer_list<int> ks) {
    for (int k : ks)
      if ((mask >> k) & 1u) return true;
    return false;
  };
  const bool full = mask == 0xFFFFu;
  const bool need_k4 = any({15});
  const bool need_edge_c3 = any({10, 13, 14});
  const bool need_tri1 = need_k4 || need_edge_c3 || any({4, 5, 6, 9, 11});
  const bool need_edges = any({10, 14});
  const bool need_spmv2 = any({5, 9});
  const bool need_tri2 = any({13});
  const bool need_cyc = any({12});
  Csr g = in;
  const int64_t n = g.n;
  const int64_t launches0 = g_launches;
  StageRange range;
  auto mark = [&](int i) {
    if (ro.stage_events && !capturing) cudaEventRecord(ro.stage_events[i], st);
    range.to(i);
  };
  auto sub = [&](int i, int edge) {  // sub-stage i: edge 0 = start, 1 = stop
    if (!ro.sub_events || capturing) return;
    cudaEventRecord(ro.sub_events[2 * i + edge], st);
    if (edge) ro.sub_recorded[i] = true;
  };
  if (ro.sub_recorded)
    for (int i = 0; i < NUM_SUB; ++i) ro.sub_recorded[i] = false;
#define CK(call)                            \
  do {                                      \
    cudaError_t e__ = (call);               \
    if (e__ != cudaSuccess) {               \
      ws.cuda_error(e__);                   \
      return e__ == cudaErrorMemoryAllocation ? FGLT_ERR_OOM : FGLT_ERR_CUDA; \
    }                                       \
  } while (0)
#define NEED(id, count, ptr)                                                                    \
  do {                                                                                          \
    void* p__ = nullptr;                                                                        \
    fglt_status s__ = ws.get(id, (size_t)std::max<int64_t>((count), 1) * sizeof(*(ptr)), &p__); \
    if (s__ != FGLT_OK) return s__;                                                             \
    ptr = static_cast<decltype(ptr)>(p__);                                                      \
  } while (0)
#define READ(dev, host)                                               \
  do {                                                                \
    fglt_status s__ = ws.read((host), (dev), sizeof(*(host)), st);    \
    if (s__ != FGLT_OK) return s__;                                   \
  } while (0)

  // Number of stored entries.
  if (b) {
    g.nnz = b->nnz;
  } else if (g.nnz < 0) {
    if (g.rp64) {
      READ(static_cast<const int64_t*>(g.rowptr) + n, &g.nnz);
    } else {
      int32_t v = 0;
      READ(static_cast<const int32_t*>(g.rowptr) + n, &v);
      g.nnz = v;
    }
    if (g.nnz < 0) return FGLT_ERR_INVALID_GRAPH;
  }
  if (g.nnz > 0 && !g.colidx) return FGLT_ERR_INVALID_ARG;
  const int64_t heavy_cap = g.nnz / HEAVY_DEGREE + 1;

  int32_t *d, *heavy, *cnt;
  u64* ctr;
  NEED(B_D, n, d);
  NEED(B_HEAVY, heavy_cap, heavy);
  NEED(B_CNT, C_NUM, cnt);
  NEED(B_CTR64, W_NUM, ctr);
  CK(cudaMemsetAsync(cnt, 0, C_NUM * sizeof(int32_t), st));
  CK(cudaMemsetAsync(ctr, 0, W_NUM * sizeof(u64), st));
  int* err = cnt + C_ERR;

  mark(0);
  CK(launch_degree(g, d, cnt + C_DMAX, heavy, cnt + C_NHEAVY, err, st, b ? b->dmax : 0x7fffffff));
  int32_t dmax = 0;
  if (b) {
    dmax = b->dmax;
  } else {
    int32_t c[C_ERR + 1];
    {
      fglt_status s = ws.read(c, cnt, sizeof c, st);
      if (s != FGLT_OK) return s;
    }
    if (c[C_ERR] & ERR_BAD_ROWPTR) return FGLT_ERR_INVALID_GRAPH;
    dmax = c[C_DMAX];
  }
  if (dmax > MAX_DEGREE_EXACT) return FGLT_ERR_OVERFLOW;
  if (ro.validate && !capturing) {
    CK(launch_validate(g, heavy, cnt + C_NHEAVY, heavy_cap, err, st));
    if (b && b->off) CK(launch_validate_batch(g, b->off, b->num_graphs, err, st));
    int e = 0;
    READ(err, &e);
    if (e & ERR_BAD_GRAPH) return FGLT_ERR_INVALID_GRAPH;
  }

  // SpMV chain 1: p2, d^7.
  mark(1);
  int64_t *p2, *r7;
  NEED(B_P2, n, p2);
  NEED(B_R7, n, r7);
  CK(launch_spmv1(g, d, heavy, cnt + C_NHEAVY, heavy_cap, p2, r7, err, st));

  // Degree ordering.
  mark(2);
  int32_t *hist, *cursor, *rank, *perm, *dr;
  int64_t* base;
  unsigned char* scan_tmp;
  NEED(B_HIST, (int64_t)dmax + 1, hist);
  NEED(B_BASE, (int64_t)dmax + 2, base);
  NEED(B_CURSOR, (int64_t)dmax + 1, cursor);
  NEED(B_RANK, n, rank);
  NEED(B_PERM, n, perm);
  NEED(B_DR, n, dr);
  NEED(B_SCAN, (int64_t)scan_temp_bytes(std::max<int64_t>(n, (int64_t)dmax + 1) + 1), scan_tmp);
  CK(cudaMemsetAsync(hist, 0, ((size_t)dmax + 1) * sizeof(int32_t), st));
  CK(cudaMemsetAsync(cursor, 0, ((size_t)dmax + 1) * sizeof(int32_t), st));
  CK(launch_degree_hist(d, n, hist, st));
  CK(launch_scan_i32_to_i64(hist, (int64_t)dmax + 1, base, scan_tmp, st));
  CK(launch_rank_assign(d, n, base, cursor, rank, perm, dr, st));

  // Oriented graph: out-degrees, row pointers, targets.
  mark(3);
  int32_t *opc, *ocol, *ocur;
  int64_t* orp;
  NEED(B_OPC, n, opc);
  NEED(B_ORP, n + 1, orp);
  CK(launch_orient_count(g, rank, heavy, cnt + C_NHEAVY, heavy_cap, opc, cnt + C_DPMAX, st));
  CK(launch_scan_i32_to_i64(opc, n, orp, scan_tmp, st));
  int64_t m_or = 0;
  int32_t dpmax = 0;
  if (b) {
    m_or = g.nnz;  // upper bound; the kernels read the exact row pointers
    dpmax = dmax;
  } else {
    READ(orp + n, &m_or);
    READ(cnt + C_DPMAX, &dpmax);
  }
  NEED(B_OCOL, m_or, ocol);
  NEED(B_OCUR, n, ocur);
  CK(cudaMemsetAsync(ocur, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(int32_t), st));
  CK(launch_orient_fill(g, rank, orp, heavy, cnt + C_NHEAVY, heavy_cap, ocur, ocol, st));

  mark(4);
  int32_t* sort_scratch = nullptr;
  const int64_t sort_ints = sort_rows_scratch_ints(m_or, dpmax);
  if (sort_ints > 0) NEED(B_SORT, sort_ints, sort_scratch);
  CK(launch_sort_rows(orp, n, dpmax, m_or, ocol, sort_scratch, st));
  // Triangle-pass work lists by out-degree; each class is launched with shared
  // memory sized for its largest out-degree.
  const int T0 = tu.tri_t0, T1 = tu.tri_t1;
  // The last class holds the vertices whose adjacency bitmap of the first
  // pass only fits in global memory.
  const int HF = tu.tri_hash_factor;
  // (at most 1024: above it the probe tables of the classes double in size)
  const int T2 = std::max(T1, std::min(1024, tri1_smem_bitmap_max(HF)));
  // The first class (out-degree up to TW) runs one warp per vertex.
  const int TW = std::min(tu.tri_warp, tri_warp_max());
  int32_t* twork;
  NEED(B_TWORK, (int64_t)TRI_CLASSES * n, twork);
  // Out-degree 1 is kept: pass 2 lists a triangle from its middle vertex,
  // which needs one out-neighbour only.
  CK(launch_worklist_outdeg5(opc, n, 1, TW, T0, T1, T2, twork, n, cnt + C_NTRI0, st));
  const int tri_cap[TRI_CLASSES] = {std::min(dpmax, TW), std::min(dpmax, T0), std::min(dpmax, T1),
                                    std::min(dpmax, T2), dpmax};
  const bool tri_on[TRI_CLASSES] = {TW >= 1 && dpmax >= 1, dpmax > TW && T0 > TW, dpmax > T0, dpmax > T1,
                                    dpmax > T2};

  // Triangle pass 1: C3, c3, 4-cliques.
  mark(5);
  int32_t* C3o;
  u64 *c3r, *k4r;
  NEED(B_C3O, m_or, C3o);
  NEED(B_C3R, n, c3r);
  NEED(B_K4R, n, k4r);
  CK(cudaMemsetAsync(C3o, 0, (size_t)std::max<int64_t>(m_or, 1) * sizeof(int32_t), st));
  CK(cudaMemsetAsync(c3r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  CK(cudaMemsetAsync(k4r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  // Hash-table slots per element, per class: the tuned value where both
  // passes' shared memory fits, else 2; a class that fits with neither is
  // outside what this build supports.
  int tri_hf[TRI_CLASSES];
  for (int c = 0; c < TRI_CLASSES; ++c) {
    tri_hf[c] = HF;
    if (!tri_on[c] || c == 0) continue;  // the warp class has fixed per-warp tables
    auto fits = [&](int hf) {
      return tri1_smem_bytes(tri_cap[c], tri1_bitmap_fits_smem(tri_cap[c], hf), hf) <= tri_smem_limit() &&
             tri2_smem_bytes(tri_cap[c], hf) <= tri_smem_limit();
    };
    if (!fits(tri_hf[c])) tri_hf[c] = 2;
    if (!fits(tri_hf[c])) return FGLT_ERR_UNSUPPORTED;
  }
  uint32_t* gbm = nullptr;
  size_t gbm_need = 0;  // classes whose bitmap does not fit in shared memory share one buffer
  for (int c = 1; c < TRI_CLASSES; ++c)
    if (tri_on[c]) gbm_need = std::max(gbm_need, tri1_gbm_bytes(tri_cap[c], tri_hf[c]));
  if (size_t gb = gbm_need) {
    unsigned char* p = nullptr;
    NEED(B_GBM, (int64_t)gb, p);
    gbm = reinterpret_cast<uint32_t*>(p);
  }
  for (int c = 0; c < TRI_CLASSES; ++c)
    if (tri_on[c] && need_tri1) {
      sub(CYC_CLASSES + c, 0);
      if (c == 0)
        CK(launch_tri1_warp(orp, ocol, twork, cnt + C_NTRI0, cnt + C_NEXT1_0, C3o, c3r, k4r, ctr + W_PROBES, err, st,
                            need_k4, tu.tri_loads));
      else
        CK(launch_tri1(orp, ocol, twork + c * n, cnt + C_NTRI0 + c, cnt + C_NEXT1_0 + c, tri_cap[c], C3o, c3r, k4r,
                       tri1_gbm_bytes(tri_cap[c], tri_hf[c]) ? gbm : nullptr, ctr + W_PROBES, err, st, need_k4,
                       tu.tri_loads, tri_hf[c], tu.tri_group, ro.wait_ns));
      sub(CYC_CLASSES + c, 1);
    }

  // Edge terms of the final C3, then SpMV chain 2.
  mark(6);
  u64 *r10r, *r14r;
  int64_t* c3oo;
  NEED(B_R10R, n, r10r);
  NEED(B_R14R, n, r14r);
  NEED(B_C3OO, n, c3oo);
  CK(cudaMemsetAsync(r10r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  CK(cudaMemsetAsync(r14r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  if (need_edges) CK(launch_c3_edge_terms(orp, ocol, C3o, dr, n, r10r, r14r, st));
  mark(7);
  int64_t *p3, *r9;
  NEED(B_P3, n, p3);
  NEED(B_R9, n, r9);
  if (need_spmv2) {
    CK(launch_unrank_u64(c3r, perm, n, c3oo, st));
    CK(launch_spmv2(g, d, p2, c3oo, heavy, cnt + C_NHEAVY, heavy_cap, p3, r9, st));
  } else {
    CK(cudaMemsetAsync(p3, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(int64_t), st));
    CK(cudaMemsetAsync(r9, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(int64_t), st));
  }

  // In-lists of the oriented graph: pass 2 lists each triangle from its
  // middle vertex, and the 4-cycle stage walks the middles of each vertex.
  // The same pass counts the 4-cycle stage's wedges.
  mark(8);
  // Dense window of top ranks: 32768 by default, 65536 for graphs above
  // 2^21 vertices (their wedge tops spread over more hubs).
  const int64_t span = tu.cyc_hub_span > 0 ? tu.cyc_hub_span : (n > (1 << 22) ? 65536 : 32768);
  const int32_t hub_lo = (int32_t)std::max<int64_t>(0, n - span);
  int64_t *wc = nullptr, *wcn = nullptr, *irp = nullptr;
  int32_t *hc = nullptr, *indeg = nullptr, *icur = nullptr;
  int2* iin = nullptr;
  // Pass 2 from the middle vertex unless the lowest is requested.
  const bool tri2_mid = tu.tri_pass2 != 1;
  if ((need_tri2 && tri2_mid) || need_cyc) {
    NEED(B_WC, n, wc);
    NEED(B_WCN, n, wcn);
    NEED(B_HC, n, hc);
    NEED(B_INDEG, n, indeg);
    NEED(B_IRP, n + 1, irp);
    NEED(B_ICUR, n, icur);
    NEED(B_IIN, m_or, iin);
    CK(cudaMemsetAsync(wc, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(int64_t), st));
    CK(cudaMemsetAsync(wcn, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(int64_t), st));
    CK(cudaMemsetAsync(icur, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(int32_t), st));
    CK(cudaMemsetAsync(iin, 0xFF, (size_t)std::max<int64_t>(m_or, 1) * sizeof(int2), st));
    CK(launch_in_lists(orp, ocol, dr, opc, n, hub_lo, hc, indeg, irp, scan_tmp, icur, iin, wc, wcn, st));
  }

  // Triangle pass 2: diamonds at the off-cord vertices.
  mark(9);
  u64* r13r;
  NEED(B_R13R, n, r13r);
  CK(cudaMemsetAsync(r13r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  if (need_tri2 && tri2_mid) {
    // Listed from the middle vertex, a vertex's work grows with its
    // in-degree: the out-degree classes are rebuilt (pass 1 is done with
    // them) with every vertex of more than TRI2_WARP_IN in-entries moved from
    // the warp class to the first block class.
    // (only where the first block class can hold a warp-class vertex)
    CK(cudaMemsetAsync(cnt + C_NTRI0, 0, TRI_CLASSES * sizeof(int32_t), st));
    CK(launch_worklist_outdeg5(opc, n, 1, TW, T0, T1, T2, twork, n, cnt + C_NTRI0, st, indeg,
                               T0 >= TW ? TRI2_WARP_IN : 0x7fffffff));
  }
  bool tri2_on[TRI_CLASSES];
  for (int c = 0; c < TRI_CLASSES; ++c) tri2_on[c] = tri_on[c];
  if (tri2_mid && T0 >= TW && TW >= 1 && dpmax >= 1) tri2_on[1] = true;  // may hold promoted vertices
  for (int c = 0; c < TRI_CLASSES; ++c)
    if (tri2_on[c] && need_tri2) {
      sub(CYC_CLASSES + TRI_CLASSES + c, 0);
      if (c == 0)
        CK(launch_tri2_warp(orp, ocol, irp, iin, twork, cnt + C_NTRI0, cnt + C_NEXT2_0, C3o, r13r, err, st,
                            tu.tri_loads, tri2_mid));
      else
        CK(launch_tri2(orp, ocol, irp, iin, twork + c * n, cnt + C_NTRI0 + c, cnt + C_NEXT2_0 + c, tri_cap[c], C3o,
                       r13r, err, st, tu.tri_loads, tri_hf[c], tu.tri_group, tri2_mid));
      sub(CYC_CLASSES + TRI_CLASSES + c, 1);
    }

  // 4-cycles: vertex classes, then the class kernels.
  mark(10);
  u64* r12r;
  NEED(B_R12R, n, r12r);
  CK(cudaMemsetAsync(r12r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  if (need_cyc) {
    const int spill_bits = cyc_fit_spill_bits((int)std::min<int64_t>(span, n), tu.cyc_spill_bits, tu.cyc_heavy_threads);
    int32_t* lists;
    NEED(B_LS, (int64_t)CYC_CLASSES * n, lists);
    const int64_t cap_bound = b ? std::min<int64_t>(b->cap, n) : n;
    CK(launch_cyc_worklists(wc, wcn, dr, n, lists, n, cnt + C_NCYC0, ctr + W_GCAP, ctr + W_WMAX, ctr + W_WSUM,
                            ctr + W_CLS, hub_lo < n, cap_bound, tu.cyc_warp_bits, tu.cyc_dense_min, spill_bits, st));
    int32_t n_gmem = 0;
    u64 gcap = 0;
    if (b) {
      if (cap_bound > cyc_block_cap()) {  // the global class may be needed: size it for the bound
        n_gmem = 1;
        gcap = (u64)cap_bound;
      }
    } else {
      int32_t ng[2];
      {
        fglt_status s2 = ws.read(ng, cnt + C_NCYC0 + (CYC_CLASSES - 2), sizeof ng, st);
        if (s2 != FGLT_OK) return s2;
      }
      n_gmem = ng[0] + ng[1];
      READ(ctr + W_GCAP, &gcap);
    }
    {
      CycArgs ca{};
      ca.n = n;
      ca.orp = orp;
      ca.ocol = ocol;
      ca.irp = irp;
      ca.iin = iin;
      ca.wc = wc;
      ca.wcn = wcn;
      ca.lists = lists;
      ca.list_stride = n;
      ca.counts = cnt + C_NCYC0;
      ca.next = cnt + C_NEXTC0;
      ca.hub_lo = hub_lo;
      ca.wbits = tu.cyc_warp_bits;
      for (int c = 0; c < 3; ++c) ca.mid_threads[c] = tu.cyc_mid_threads[c];
      ca.heavy_threads = tu.cyc_heavy_threads;
      ca.long_seg = tu.cyc_long_segment;
      ca.spill_bits = spill_bits;
      ca.r12r = r12r;
      ca.err = err;
      ca.cap_bound = cap_bound;
      ca.ev = capturing ? nullptr : ro.sub_events;
      ca.ev_rec = ro.sub_recorded;
      if (n_gmem > 0) {
        ca.gbits = bits_for((int64_t)gcap);
        const int64_t slots = (int64_t)cyc_gmem_blocks() << ca.gbits;
        NEED(B_GKEYS, 2 * slots, ca.gkeys);  // (key, count) per slot
        NEED(B_GTOUCH, slots / 2, ca.gtouch);
      }
      CK(launch_cyc(ca, st));
    }
  }

  // Table I + U16^{-1}.
  mark(11);
  EpilogueIn ein{d, rank, p2, p3, r7, r9, c3r, r10r, r12r, r13r, r14r, k4r};
  if (full) CK(launch_epilogue(ein, n, out_raw, out_net, st));
  else CK(launch_epilogue_sub(ein, sd, n, out_raw, out_net, st));
  mark(12);
  if (capturing) return FGLT_OK;

  int e = 0;
  READ(err, &e);
  if (e & (ERR_BAD_GRAPH | ERR_BAD_ROWPTR)) return FGLT_ERR_INVALID_GRAPH;
  if (e & ERR_TIMEOUT) return FGLT_ERR_TIMEOUT;
  if (e) return FGLT_ERR_INTERNAL;
  if (ro.work) {
    u64 w[W_NUM];
    fglt_status s = ws.read(w, ctr, sizeof w, st);
    if (s != FGLT_OK) return s;
    int64_t* o = ro.work;
    o[O_N] = n;
    o[O_NNZ] = g.nnz;
    o[O_M] = m_or;
    o[O_DMAX] = dmax;
    o[O_DPMAX] = dpmax;
    o[O_PROBES] = (int64_t)w[W_PROBES];
    o[O_TRIANGLES] = (int64_t)w[W_TRIANGLES];
    o[O_K4] = (int64_t)w[W_K4];
    o[O_WEDGES] = (int64_t)w[W_WSUM];
    o[O_WMAX] = (int64_t)w[W_WMAX];
    o[O_LAUNCHES] = g_launches - launches0;
    int32_t cls_n[CYC_CLASSES] = {};
    if (need_cyc) {
      fglt_status s2 = ws.read(cls_n, cnt + C_NCYC0, sizeof cls_n, st);
      if (s2 != FGLT_OK) return s2;
    }
    for (int c = 0; c < CYC_CLASSES; ++c) {
      o[O_CLS_VERTICES + c] = cls_n[c];
      o[O_CLS_WEDGES + c] = (int64_t)w[W_CLS + c];
    }
  }
  return FGLT_OK;
#undef CK
#undef NEED
#undef READ
}

}  // namespace fglt
