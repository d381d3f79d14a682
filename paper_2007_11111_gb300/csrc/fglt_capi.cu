// C ABI of the FGLT library: handle, workspace, and the stage sequence of one
// transform. See include/fglt.h for the contract of every entry point.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fglt.h"
#include "fglt_device.cuh"
#include "fglt_kernels.h"
#include "fglt_serve.h"

using namespace fglt;

namespace {

constexpr int64_t MAX_DEGREE_EXACT = 2097151;  // binom(d,3) products stay inside int64

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

enum BufId {
  B_D, B_HEAVY, B_CNT, B_HIST, B_BASE, B_CURSOR, B_RANK, B_PERM, B_DR, B_OPC, B_ORP, B_SCAN, B_OCOL, B_OCUR,
  B_SORT, B_TWORK, B_C3O, B_C3R, B_K4R, B_R10R, B_R14R, B_R13R, B_R12R, B_C3OO, B_P2, B_P3, B_R7, B_R9, B_WC,
  B_LS, B_WCN, B_GBM, B_GKEYS, B_GCNT,
  B_H_ROWPTR, B_H_COLIDX, B_H_RAW, B_H_NET, B_BATCH_OFF, B_CTR64,
  B_COUNT
};

// Small device counters, one int slot each.
enum CounterId {
  C_DMAX, C_NHEAVY, C_DPMAX, C_NTRI0, C_NTRI1, C_NTRI2, C_NEXT1_0, C_NEXT1_1, C_NEXT1_2, C_NEXT2_0,
  C_NEXT2_1, C_NEXT2_2, C_NCYC0, C_NCYC1, C_NCYC2, C_NCYC3, C_NEXTC0, C_NEXTC1, C_NEXTC2, C_NEXTC3, C_ERR,
  C_NUM
};
// 64-bit work counters: triangle-pass scanned entries, triangles, 4-cliques,
// max and total wedges of the 4-cycle stage.
enum Counter64Id { W_PROBES, W_TRIANGLES, W_K4, W_WMAX, W_WSUM, W_GCAP, W_NUM };

// Host copy of the last transform's work counters (fglt_work_counters order).
enum WorkOut { O_N, O_NNZ, O_M, O_DMAX, O_DPMAX, O_PROBES, O_TRIANGLES, O_K4, O_WEDGES, O_WMAX, O_LAUNCHES, O_NUM };

const char* const STAGE_NAMES[] = {"degree", "spmv1", "rank", "orient", "sort", "tri1", "c3_edges",
                                   "spmv2", "tri2", "wedges", "cyc", "epilogue"};
constexpr int NUM_STAGES = sizeof(STAGE_NAMES) / sizeof(STAGE_NAMES[0]);

}  // namespace

struct fglt_handle {
  int device = 0;
  fglt_options opt{};
  cudaStream_t stream = nullptr;
  cudaStream_t cur = nullptr;  // stream of the transform in progress
  Buf bufs[B_COUNT];
  int64_t* pinned = nullptr;  // small host staging for read-backs
  std::string cuda_err;
  cudaEvent_t ev[NUM_STAGES + 1] = {};
  float stage_ms[NUM_STAGES] = {};
  bool stages_valid = false;
  int64_t work[O_NUM] = {};
  bool work_valid = false;
  serve::Server* server = nullptr;
  std::mutex server_mu;  // guards creation of the server
  std::mutex mu;  // serialises transforms issued by the serving thread and the caller
  // Batched calls: the stage sequence captured as a CUDA graph for one batch
  // shape and buffer set, replayed while they stay the same.
  struct {
    bool valid = false;
    const void* rowptr = nullptr;
    const void* colidx = nullptr;
    int64_t* raw = nullptr;
    int64_t* net = nullptr;
    int rp64 = 0;
    int64_t n = 0, nnz = 0, maxg = 0;
    cudaGraphExec_t exec = nullptr;
  } batch;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int64_t batch_replays = 0;
};

namespace {

fglt_status cuda_fail(fglt_t h, cudaError_t e) {
  if (h) h->cuda_err = cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? FGLT_ERR_OOM : FGLT_ERR_CUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e__ = (call);                      \
    if (e__ != cudaSuccess) return cuda_fail(h, e__); \
  } while (0)

// Returns a device buffer of at least `bytes` (grows by reallocating; the
// caller guarantees no queued work still uses the old one).
fglt_status need(fglt_t h, BufId id, size_t bytes, void** out) {
  Buf& b = h->bufs[id];
  if (bytes == 0) bytes = 16;
  if (b.bytes < bytes) {
    if (b.p) {
      cudaError_t e = cudaStreamSynchronize(h->cur ? h->cur : h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e);
      cudaFree(b.p);
      b.p = nullptr;
      b.bytes = 0;
    }
    size_t want = bytes + bytes / 8;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
      b.p = nullptr;
      return cuda_fail(h, e);
    }
    b.bytes = want;
  }
  *out = b.p;
  return FGLT_OK;
}

template <typename T>
fglt_status needT(fglt_t h, BufId id, int64_t count, T** out) {
  void* p = nullptr;
  fglt_status s = need(h, id, (size_t)std::max<int64_t>(count, 1) * sizeof(T), &p);
  *out = static_cast<T*>(p);
  return s;
}

#define NEED(id, count, ptr)                         \
  do {                                               \
    fglt_status s__ = needT(h, id, (count), &(ptr)); \
    if (s__ != FGLT_OK) return s__;                  \
  } while (0)

// Blocking read of one device scalar via the pinned staging word.
template <typename T>
fglt_status read_scalar(fglt_t h, cudaStream_t st, const T* dev, T* out) {
  CK(cudaMemcpyAsync(h->pinned, dev, sizeof(T), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::memcpy(out, h->pinned, sizeof(T));
  return FGLT_OK;
}

int bits_for(int64_t cap) {
  int hb = 5;
  while ((1LL << hb) < 2 * cap) ++hb;
  return hb;
}

}  // namespace

namespace {

// The whole transform on stream st. Inputs and outputs are device pointers.
// With b, every read-back is replaced by b's bounds; with capturing, nothing
// that synchronises or allocates is issued (buffers were sized by an earlier
// run with the same bounds).
fglt_status run_pipeline(fglt_t h, const Csr& in, int64_t* out_raw, int64_t* out_net, cudaStream_t st,
                         const Bounds* b = nullptr, bool capturing = false) {
  Csr g = in;
  const int64_t n = g.n;
  const bool prof = h->opt.profile_stages != 0 && !capturing;
  h->stages_valid = false;
  h->cur = st;
  const int64_t launches0 = g_launches;
  auto mark = [&](int i) {
    if (prof) cudaEventRecord(h->ev[i], st);
  };

  // Number of stored entries.
  if (b) {
    g.nnz = b->nnz;
  } else {
    const size_t elt = g.rp64 ? 8 : 4;
    CK(cudaMemcpyAsync(h->pinned, static_cast<const char*>(g.rowptr) + (size_t)n * elt, elt,
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    g.nnz = g.rp64 ? h->pinned[0] : (int64_t) * reinterpret_cast<int32_t*>(h->pinned);
    if (g.nnz < 0) return FGLT_ERR_INVALID_GRAPH;
    if (g.nnz > 0 && !g.colidx) return FGLT_ERR_INVALID_ARG;
  }
  const int64_t heavy_cap = g.nnz / HEAVY_DEGREE + 1;

  int32_t *d, *heavy, *cnt;
  u64* ctr;
  NEED(B_D, n, d);
  NEED(B_HEAVY, heavy_cap, heavy);
  NEED(B_CNT, C_NUM, cnt);
  NEED(B_CTR64, W_NUM, ctr);
  CK(cudaMemsetAsync(cnt, 0, C_NUM * sizeof(int32_t), st));
  CK(cudaMemsetAsync(ctr, 0, W_NUM * sizeof(u64), st));
  h->work_valid = false;
  int* err = cnt + C_ERR;

  mark(0);
  CK(launch_degree(g, d, cnt + C_DMAX, heavy, cnt + C_NHEAVY, err, st, b ? b->dmax : 0x7fffffff));
  int32_t dmax = 0;
  if (b) {
    dmax = b->dmax;
  } else {
    int32_t c[C_NUM];
    CK(cudaMemcpyAsync(h->pinned, cnt, sizeof c, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::memcpy(c, h->pinned, sizeof c);
    if (c[C_ERR] & ERR_BAD_ROWPTR) return FGLT_ERR_INVALID_GRAPH;
    dmax = c[C_DMAX];
  }
  if (dmax > MAX_DEGREE_EXACT) return FGLT_ERR_OVERFLOW;
  if (h->opt.validate && !capturing) {
    CK(launch_validate(g, heavy, cnt + C_NHEAVY, heavy_cap, err, st));
    if (b && b->off) CK(launch_validate_batch(g, b->off, b->num_graphs, err, st));
    int e = 0;
    fglt_status s = read_scalar(h, st, err, &e);
    if (s != FGLT_OK) return s;
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
  void* scan_tmp;
  NEED(B_HIST, (int64_t)dmax + 1, hist);
  NEED(B_BASE, (int64_t)dmax + 2, base);
  NEED(B_CURSOR, (int64_t)dmax + 1, cursor);
  NEED(B_RANK, n, rank);
  NEED(B_PERM, n, perm);
  NEED(B_DR, n, dr);
  {
    fglt_status s = need(h, B_SCAN, scan_temp_bytes(std::max<int64_t>(n, (int64_t)dmax + 1) + 1), &scan_tmp);
    if (s != FGLT_OK) return s;
  }
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
    fglt_status s = read_scalar(h, st, orp + n, &m_or);
    if (s == FGLT_OK) s = read_scalar(h, st, cnt + C_DPMAX, &dpmax);
    if (s != FGLT_OK) return s;
  }
  NEED(B_OCOL, m_or, ocol);
  NEED(B_OCUR, n, ocur);
  CK(cudaMemsetAsync(ocur, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(int32_t), st));
  CK(launch_orient_fill(g, rank, orp, heavy, cnt + C_NHEAVY, heavy_cap, ocur, ocol, st));

  mark(4);
  int32_t* sort_scratch = nullptr;
  if (dpmax > 16384) {
    int64_t P = 16384;
    while (P < dpmax) P <<= 1;
    NEED(B_SORT, P, sort_scratch);
  }
  CK(launch_sort_rows(orp, n, dpmax, ocol, sort_scratch, st));
  // Triangle-pass work lists by out-degree; each class is launched with shared
  // memory sized for its largest out-degree.
  constexpr int TRI_T0 = 64, TRI_T1 = 256;
  int32_t* twork;
  NEED(B_TWORK, 3 * n, twork);
  CK(launch_worklist_outdeg3(opc, n, 2, TRI_T0, TRI_T1, twork, n, cnt + C_NTRI0, st));
  const int tri_cap[3] = {std::min(dpmax, TRI_T0), std::min(dpmax, TRI_T1), dpmax};
  const bool tri_on[3] = {dpmax >= 2, dpmax > TRI_T0, dpmax > TRI_T1};

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
  uint32_t* gbm = nullptr;
  if (size_t gb = tri1_gbm_bytes(dpmax)) {
    void* p = nullptr;
    fglt_status s = need(h, B_GBM, gb, &p);
    if (s != FGLT_OK) return s;
    gbm = static_cast<uint32_t*>(p);
  }
  if (dpmax >= 2 && tri2_smem_bytes(dpmax) > 227 * 1024) return FGLT_ERR_UNSUPPORTED;
  for (int c = 0; c < 3; ++c)
    if (tri_on[c])
      CK(launch_tri1(orp, ocol, twork + c * n, cnt + C_NTRI0 + c, cnt + C_NEXT1_0 + c, tri_cap[c], C3o, c3r, k4r,
                     c == 2 ? gbm : nullptr, ctr + W_PROBES, err, st));

  // Edge terms of the final C3, then SpMV chain 2.
  mark(6);
  u64 *r10r, *r14r;
  int64_t* c3oo;
  NEED(B_R10R, n, r10r);
  NEED(B_R14R, n, r14r);
  NEED(B_C3OO, n, c3oo);
  CK(cudaMemsetAsync(r10r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  CK(cudaMemsetAsync(r14r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  CK(launch_c3_edge_terms(orp, ocol, C3o, dr, n, r10r, r14r, st));
  CK(launch_unrank_u64(c3r, perm, n, c3oo, st));
  mark(7);
  int64_t *p3, *r9;
  NEED(B_P3, n, p3);
  NEED(B_R9, n, r9);
  CK(launch_spmv2(g, d, p2, c3oo, heavy, cnt + C_NHEAVY, heavy_cap, p3, r9, st));

  // Triangle pass 2: diamonds at the off-cord vertices.
  mark(8);
  u64* r13r;
  NEED(B_R13R, n, r13r);
  CK(cudaMemsetAsync(r13r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  for (int c = 0; c < 3; ++c)
    if (tri_on[c])
      CK(launch_tri2(orp, ocol, twork + c * n, cnt + C_NTRI0 + c, cnt + C_NEXT2_0 + c, tri_cap[c], C3o, r13r, err,
                     st));

  // 4-cycles.
  mark(9);
  int64_t *wc, *wcn;
  NEED(B_WC, n, wc);
  NEED(B_WCN, n, wcn);
  const bool c16 = dmax < 65536;
  int64_t span = cyc_dense_span(c16);
  if (h->opt.cyc_hub_span > 0) span = std::min<int64_t>(span, h->opt.cyc_hub_span);
  const int32_t hub_lo = (int32_t)std::max<int64_t>(0, n - span);
  CK(launch_wedge_count(g, rank, orp, ocol, heavy, cnt + C_NHEAVY, heavy_cap, hub_lo, wc, wcn, ctr + W_WMAX,
                        ctr + W_WSUM, st));
  int32_t* lists;
  NEED(B_LS, 4 * n, lists);
  const int64_t cap_bound = b ? std::min<int64_t>(b->cap, n) : n;
  CK(launch_cyc_worklists(wc, wcn, n, lists, n, cnt + C_NCYC0, ctr + W_GCAP, hub_lo < n, st, cap_bound));
  int32_t n_gmem = 0;
  u64 gcap = 0;
  if (b) {
    if (cap_bound > cyc_block_cap()) {  // the global class may be needed: size it for the bound
      n_gmem = 1;
      gcap = (u64)cap_bound;
    }
  } else {
    fglt_status s = read_scalar(h, st, cnt + C_NCYC3, &n_gmem);
    if (s == FGLT_OK) s = read_scalar(h, st, ctr + W_GCAP, &gcap);
    if (s != FGLT_OK) return s;
  }
  mark(10);
  u64* r12r;
  NEED(B_R12R, n, r12r);
  CK(cudaMemsetAsync(r12r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  {
    CycArgs ca{};
    ca.rank = rank;
    ca.perm = perm;
    ca.orp = orp;
    ca.ocol = ocol;
    ca.wc = wc;
    ca.lists = lists;
    ca.list_stride = n;
    ca.counts = cnt + C_NCYC0;
    ca.next = cnt + C_NEXTC0;
    ca.c16 = c16;
    ca.hub_lo = hub_lo;
    ca.r12r = r12r;
    ca.err = err;
    ca.cap_bound = cap_bound;
    if (n_gmem > 0) {
      ca.gbits = bits_for((int64_t)gcap);
      const size_t slots = (size_t)cyc_gmem_blocks() << ca.gbits;
      NEED(B_GKEYS, (int64_t)slots, ca.gkeys);
      NEED(B_GCNT, (int64_t)slots, ca.gcnt);
    }
    CK(launch_cyc(g, ca, st));
  }

  // Table I + U16^{-1}.
  mark(11);
  EpilogueIn ein{d, rank, p2, p3, r7, r9, c3r, r10r, r12r, r13r, r14r, k4r};
  CK(launch_epilogue(ein, n, out_raw, out_net, st));
  mark(12);
  if (capturing) return FGLT_OK;

  int e = 0;
  {
    fglt_status s = read_scalar(h, st, err, &e);
    if (s != FGLT_OK) return s;
  }
  if (e & (ERR_BAD_GRAPH | ERR_BAD_ROWPTR)) return FGLT_ERR_INVALID_GRAPH;
  if (e) return FGLT_ERR_INTERNAL;
  {
    u64 w[W_NUM];
    CK(cudaMemcpy(w, ctr, sizeof w, cudaMemcpyDeviceToHost));
    h->work[O_N] = n;
    h->work[O_NNZ] = g.nnz;
    h->work[O_M] = m_or;
    h->work[O_DMAX] = dmax;
    h->work[O_DPMAX] = dpmax;
    h->work[O_PROBES] = (int64_t)w[W_PROBES];
    h->work[O_TRIANGLES] = (int64_t)w[W_TRIANGLES];
    h->work[O_K4] = (int64_t)w[W_K4];
    h->work[O_WEDGES] = (int64_t)w[W_WSUM];
    h->work[O_WMAX] = (int64_t)w[W_WMAX];
    h->work[O_LAUNCHES] = g_launches - launches0;
    h->work_valid = true;
  }
  if (prof) {
    for (int i = 0; i < NUM_STAGES; ++i) cudaEventElapsedTime(&h->stage_ms[i], h->ev[i], h->ev[i + 1]);
    h->stages_valid = true;
  }
  return FGLT_OK;
}

fglt_status check_common(fglt_t h, const void* rowptr, int rp64, int64_t n, const int64_t* raw,
                         const int64_t* net) {
  if (!h) return FGLT_ERR_INVALID_ARG;
  if (n < 0 || (rp64 != 0 && rp64 != 1)) return FGLT_ERR_INVALID_ARG;
  if (!rp64 && n > 0x7ffffffeLL) return FGLT_ERR_INVALID_ARG;
  if (n > 0x7ffffffeLL) return FGLT_ERR_UNSUPPORTED;
  if (n > 0 && (!rowptr || (!raw && !net))) return FGLT_ERR_INVALID_ARG;
  return FGLT_OK;
}

}  // namespace

// ===========================================================================
// Entry points
// ===========================================================================
extern "C" {

fglt_status fglt_options_default(fglt_options* opt) {
  if (!opt) return FGLT_ERR_INVALID_ARG;
  std::memset(opt, 0, sizeof(*opt));
  return FGLT_OK;
}

const char* fglt_status_string(fglt_status s) {
  switch (s) {
    case FGLT_OK: return "ok";
    case FGLT_ERR_INVALID_ARG: return "invalid argument";
    case FGLT_ERR_INVALID_GRAPH: return "input is not a simple symmetric CSR graph";
    case FGLT_ERR_OOM: return "out of memory";
    case FGLT_ERR_OVERFLOW: return "maximum degree too large for exact int64 counts";
    case FGLT_ERR_CUDA: return "CUDA runtime error";
    case FGLT_ERR_TIMEOUT: return "timed out";
    case FGLT_ERR_PENDING: return "request pending";
    case FGLT_ERR_NOT_FOUND: return "unknown request";
    case FGLT_ERR_INTERNAL: return "internal consistency check failed";
    case FGLT_ERR_UNSUPPORTED: return "input size not supported by this build";
    case FGLT_ERR_BUSY: return "busy";
    case FGLT_ERR_CANCELLED: return "cancelled";
    default: return "unknown status";
  }
}

fglt_status fglt_create(fglt_t* out, const fglt_options* opt, int device) {
  if (!out) return FGLT_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FGLT_ERR_INVALID_ARG;
  fglt_t h = new (std::nothrow) fglt_handle();
  if (!h) return FGLT_ERR_OOM;
  h->device = device;
  if (opt) h->opt = *opt;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost(&h->pinned, 256);
  for (int i = 0; e == cudaSuccess && i <= NUM_STAGES; ++i) e = cudaEventCreate(&h->ev[i]);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    fglt_status s = cuda_fail(h, e);
    fglt_destroy(h);
    return s;
  }
  *out = h;
  return FGLT_OK;
}

fglt_status fglt_destroy(fglt_t h) {
  if (!h) return FGLT_OK;
  cudaSetDevice(h->device);
  if (h->server) {
    serve::destroy(h->server);
    h->server = nullptr;
  }
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->batch.exec) cudaGraphExecDestroy(h->batch.exec);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  for (auto& b : h->bufs)
    if (b.p) cudaFree(b.p);
  for (int i = 0; i <= NUM_STAGES; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  if (h->pinned) cudaFreeHost(h->pinned);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return FGLT_OK;
}

const char* fglt_last_cuda_error(fglt_t h) { return h ? h->cuda_err.c_str() : ""; }

fglt_status fglt_transform(fglt_t h, const void* rowptr, int rowptr_is_64bit, const int32_t* colidx, int64_t n,
                           int64_t* out_raw, int64_t* out_net, void* stream) {
  fglt_status s = check_common(h, rowptr, rowptr_is_64bit, n, out_raw, out_net);
  if (s != FGLT_OK || n == 0) return s;
  std::lock_guard<std::mutex> lock(h->mu);
  if (cudaSetDevice(h->device) != cudaSuccess) return FGLT_ERR_CUDA;
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
  Csr g{rowptr, rowptr_is_64bit != 0, colidx, n, 0};
  return run_pipeline(h, g, out_raw, out_net, st);
}

fglt_status fglt_transform_host(fglt_t h, const void* rowptr, int rowptr_is_64bit, const int32_t* colidx,
                                int64_t n, int64_t* out_raw, int64_t* out_net) {
  fglt_status s = check_common(h, rowptr, rowptr_is_64bit, n, out_raw, out_net);
  if (s != FGLT_OK || n == 0) return s;
  std::lock_guard<std::mutex> lock(h->mu);
  if (cudaSetDevice(h->device) != cudaSuccess) return FGLT_ERR_CUDA;
  const size_t elt = rowptr_is_64bit ? 8 : 4;
  const int64_t nnz = rowptr_is_64bit ? static_cast<const int64_t*>(rowptr)[n]
                                      : (int64_t) static_cast<const int32_t*>(rowptr)[n];
  if (nnz < 0) return FGLT_ERR_INVALID_GRAPH;
  if (nnz > 0 && !colidx) return FGLT_ERR_INVALID_ARG;
  void *drp, *dci, *draw = nullptr, *dnet = nullptr;
  if ((s = need(h, B_H_ROWPTR, (size_t)(n + 1) * elt, &drp)) != FGLT_OK) return s;
  if ((s = need(h, B_H_COLIDX, (size_t)std::max<int64_t>(nnz, 1) * 4, &dci)) != FGLT_OK) return s;
  if (out_raw && (s = need(h, B_H_RAW, (size_t)n * 16 * 8, &draw)) != FGLT_OK) return s;
  if (out_net && (s = need(h, B_H_NET, (size_t)n * 16 * 8, &dnet)) != FGLT_OK) return s;
  cudaStream_t st = h->stream;
  CK(cudaMemcpyAsync(drp, rowptr, (size_t)(n + 1) * elt, cudaMemcpyHostToDevice, st));
  if (nnz > 0) CK(cudaMemcpyAsync(dci, colidx, (size_t)nnz * 4, cudaMemcpyHostToDevice, st));
  Csr g{drp, rowptr_is_64bit != 0, static_cast<const int32_t*>(dci), n, 0};
  s = run_pipeline(h, g, static_cast<int64_t*>(draw), static_cast<int64_t*>(dnet), st);
  if (s != FGLT_OK) return s;
  if (out_raw) CK(cudaMemcpyAsync(out_raw, draw, (size_t)n * 16 * 8, cudaMemcpyDeviceToHost, st));
  if (out_net) CK(cudaMemcpyAsync(out_net, dnet, (size_t)n * 16 * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return FGLT_OK;
}

fglt_status fglt_transform_batched(fglt_t h, const void* rowptr, int rowptr_is_64bit, const int32_t* colidx,
                                   const int64_t* graph_offsets, int64_t num_graphs, int64_t* out_raw,
                                   int64_t* out_net, void* stream) {
  if (!h || !graph_offsets || num_graphs < 0) return FGLT_ERR_INVALID_ARG;
  if (graph_offsets[0] != 0) return FGLT_ERR_INVALID_ARG;
  int64_t maxg = 0;
  for (int64_t i = 0; i < num_graphs; ++i) {
    if (graph_offsets[i + 1] < graph_offsets[i]) return FGLT_ERR_INVALID_ARG;
    maxg = std::max(maxg, graph_offsets[i + 1] - graph_offsets[i]);
  }
  const int64_t n = graph_offsets[num_graphs];
  fglt_status s = check_common(h, rowptr, rowptr_is_64bit, n, out_raw, out_net);
  if (s != FGLT_OK || n == 0) return s;
  if (maxg - 1 > MAX_DEGREE_EXACT) return FGLT_ERR_OVERFLOW;
  std::lock_guard<std::mutex> lock(h->mu);
  if (cudaSetDevice(h->device) != cudaSuccess) return FGLT_ERR_CUDA;
  // The union of vertex-disjoint graphs is one graph whose transform is the
  // concatenation of theirs (every graphlet is connected). It runs on the
  // handle's stream, ordered after and before the caller's stream.
  cudaStream_t us = stream ? static_cast<cudaStream_t>(stream) : h->stream;
  cudaStream_t cs = h->stream;
  if (us != cs) {
    CK(cudaEventRecord(h->ev_in, us));
    CK(cudaStreamWaitEvent(cs, h->ev_in, 0));
  }
  auto finish = [&](fglt_status st) -> fglt_status {
    if (us != cs) {
      if (cudaEventRecord(h->ev_out, cs) != cudaSuccess) return FGLT_ERR_CUDA;
      if (cudaStreamWaitEvent(us, h->ev_out, 0) != cudaSuccess) return FGLT_ERR_CUDA;
    }
    return st;
  };
  const size_t elt = rowptr_is_64bit ? 8 : 4;
  CK(cudaMemcpyAsync(h->pinned, static_cast<const char*>(rowptr) + (size_t)n * elt, elt, cudaMemcpyDeviceToHost,
                     cs));
  CK(cudaStreamSynchronize(cs));
  const int64_t nnz = rowptr_is_64bit ? h->pinned[0] : (int64_t) * reinterpret_cast<int32_t*>(h->pinned);
  if (nnz < 0) return finish(FGLT_ERR_INVALID_GRAPH);
  if (nnz > 0 && !colidx) return finish(FGLT_ERR_INVALID_ARG);
  const int64_t* off_dev = nullptr;
  if (h->opt.validate) {
    void* p = nullptr;
    if ((s = need(h, B_BATCH_OFF, (size_t)(num_graphs + 1) * 8, &p)) != FGLT_OK) return finish(s);
    CK(cudaMemcpyAsync(p, graph_offsets, (size_t)(num_graphs + 1) * 8, cudaMemcpyHostToDevice, cs));
    off_dev = static_cast<const int64_t*>(p);
  }
  Bounds b{nnz, (int32_t)std::max<int64_t>(maxg - 1, 0), std::max<int64_t>(maxg - 1, 1), off_dev, num_graphs};
  Csr g{rowptr, rowptr_is_64bit != 0, colidx, n, nnz};
  auto& bc = h->batch;
  const bool same = bc.valid && bc.rowptr == rowptr && bc.colidx == colidx && bc.raw == out_raw &&
                    bc.net == out_net && bc.rp64 == rowptr_is_64bit && bc.n == n && bc.nnz == nnz &&
                    bc.maxg == maxg;
  if (same && !h->opt.validate && !h->opt.profile_stages) {
    // Replay: the graph re-zeroes its counters and accumulators itself.
    CK(cudaGraphLaunch(bc.exec, cs));
    ++h->batch_replays;
    int e = 0;
    s = read_scalar(h, cs, h->bufs[B_CNT].p ? static_cast<int*>(h->bufs[B_CNT].p) + C_ERR : nullptr, &e);
    if (s != FGLT_OK) return finish(s);
    h->work_valid = false;
    h->stages_valid = false;
    if (e & (ERR_BAD_GRAPH | ERR_BAD_ROWPTR)) return finish(FGLT_ERR_INVALID_GRAPH);
    return finish(e ? FGLT_ERR_INTERNAL : FGLT_OK);
  }
  s = run_pipeline(h, g, out_raw, out_net, cs, &b, false);
  if (s != FGLT_OK || h->opt.validate || h->opt.profile_stages) return finish(s);
  // Capture the same sequence (its buffers are sized now) for later calls.
  if (bc.exec) {
    cudaGraphExecDestroy(bc.exec);
    bc.exec = nullptr;
  }
  bc.valid = false;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const fglt_status cap = run_pipeline(h, g, out_raw, out_net, cs, &b, true);
    const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if (cap == FGLT_OK && ee == cudaSuccess && graph &&
        cudaGraphInstantiate(&bc.exec, graph, 0) == cudaSuccess) {
      bc.valid = true;
      bc.rowptr = rowptr;
      bc.colidx = colidx;
      bc.raw = out_raw;
      bc.net = out_net;
      bc.rp64 = rowptr_is_64bit;
      bc.n = n;
      bc.nnz = nnz;
      bc.maxg = maxg;
    }
    if (graph) cudaGraphDestroy(graph);
  }
  cudaGetLastError();  // a failed capture only disables replay
  return finish(FGLT_OK);
}

fglt_status fglt_work_counters(fglt_t h, int64_t* counters, int max_counters, int* count) {
  if (!h || !count || max_counters < 0 || (max_counters > 0 && !counters)) return FGLT_ERR_INVALID_ARG;
  if (!h->work_valid) {
    *count = 0;
    return FGLT_ERR_NOT_FOUND;
  }
  for (int i = 0; i < std::min<int>(max_counters, O_NUM); ++i) counters[i] = h->work[i];
  *count = O_NUM;
  return FGLT_OK;
}

fglt_status fglt_stage_times(fglt_t h, const char** names, float* ms, int max_stages, int* count) {
  if (!h || !count || max_stages < 0) return FGLT_ERR_INVALID_ARG;
  if (!h->stages_valid) {
    *count = 0;
    return FGLT_ERR_NOT_FOUND;
  }
  const int k = std::min(max_stages, NUM_STAGES);
  for (int i = 0; i < k; ++i) {
    if (names) names[i] = STAGE_NAMES[i];
    if (ms) ms[i] = h->stage_ms[i];
  }
  *count = NUM_STAGES;
  return FGLT_OK;
}

}  // extern "C"

// Used by the serving runtime: one transform on the handle's workspace.
namespace fglt {
namespace serve {
fglt_status transform_locked(fglt_t h, const Csr& g, int64_t* raw, int64_t* net, cudaStream_t st,
                             const Bounds* b) {
  std::lock_guard<std::mutex> lock(h->mu);
  if (cudaSetDevice(h->device) != cudaSuccess) return FGLT_ERR_CUDA;
  return run_pipeline(h, g, raw, net, st, b, false);
}
cudaStream_t handle_stream(fglt_t h) { return h->stream; }
const fglt_options* options_of(fglt_t h) { return &h->opt; }
int device_of(fglt_t h) { return h->device; }
Server* server_of(fglt_t h) {
  std::lock_guard<std::mutex> lock(h->server_mu);
  return h->server;
}
fglt_status ensure_server(fglt_t h, Server** out, fglt_status (*factory)(fglt_t, Server**)) {
  std::lock_guard<std::mutex> lock(h->server_mu);
  if (!h->server) {
    fglt_status s = factory(h, &h->server);
    if (s != FGLT_OK) {
      h->server = nullptr;
      return s;
    }
  }
  *out = h->server;
  return FGLT_OK;
}
}  // namespace serve
}  // namespace fglt
