// fglt_transform_noalloc: the single-graph transform for callers that cannot
// allocate device memory at call time.
//
// Who needs it: a process whose device memory is already owned by another
// allocator (for example a framework's caching pool that reserved most of the
// GPU), where a cudaMalloc could fail at an arbitrary point; a latency-bound
// loop in which the device-wide synchronisation that cudaMalloc/cudaFree may
// perform is not acceptable; code that must fix its device memory use when
// the library is loaded. fglt_transform grows a per-handle workspace with
// cudaMalloc; this entry point instead carves every buffer of the stage
// sequence from one file-scope device array, g_noalloc_scratch, of fixed size.
//
// Limits (checked before any device work; larger inputs return
// FGLT_ERR_UNSUPPORTED): n <= FGLT_NOALLOC_MAX_VERTICES, rowptr[n] <=
// FGLT_NOALLOC_MAX_ENTRIES, and a largest out-degree (in the degree order)
// small enough for the shared-memory adjacency bitmap of the triangle pass.
// Every device that loads the library holds the array until the process
// exits.
//
// The array is shared by every call in the process. A call clears what must
// start at zero and leaves its results in the array until the next call, so
// two calls whose device work overlaps (different streams, or different host
// threads on the same device) race on it; serialise them.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (once per device, with that device current). Make that
// first call before any stream capture.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "fglt.h"
#include "fglt_device.cuh"
#include "fglt_kernels.h"

using namespace fglt;

namespace {

constexpr size_t SCRATCH_BYTES = (size_t)16 << 20;
static_assert(FGLT_NOALLOC_SCRATCH_BYTES == SCRATCH_BYTES, "header and array size agree");

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_ptr[MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on the current device (set-up on first use).
cudaError_t scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    g_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_ptr[dev]);
  return cudaSuccess;
}

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Carver {
  unsigned char* base;
  size_t off = 0;
  bool ok = true;
  template <typename T>
  T* take(int64_t count) {
    const size_t bytes = ((size_t)std::max<int64_t>(count, 1) * sizeof(T) + 255) & ~(size_t)255;
    if (off + bytes > SCRATCH_BYTES) {
      ok = false;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

enum { K_DMAX, K_NHEAVY, K_DPMAX, K_NTRI0, K_NTRI1, K_NTRI2, K_NEXT1_0, K_NEXT1_1, K_NEXT1_2, K_NEXT2_0,
       K_NEXT2_1, K_NEXT2_2, K_NCYC0, K_NCYC1, K_NCYC2, K_NCYC3, K_NEXTC0, K_NEXTC1, K_NEXTC2, K_NEXTC3, K_ERR,
       K_NUM };
enum { W_PROBES, W_TRIANGLES, W_K4, W_WMAX, W_WSUM, W_GCAP, W_NUM };

#define CK(call)                                     \
  do {                                               \
    if ((call) != cudaSuccess) return FGLT_ERR_CUDA; \
  } while (0)

template <typename T>
fglt_status read_back(cudaStream_t st, const T* dev, T* host) {
  CK(cudaMemcpyAsync(host, dev, sizeof(T), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return FGLT_OK;
}

#define RB(dev, host)                               \
  do {                                              \
    fglt_status s__ = read_back(st, (dev), (host)); \
    if (s__ != FGLT_OK) return s__;                 \
  } while (0)

#define TAKE(T, ptr, count)           \
  T* ptr = C.take<T>(count);          \
  if (!C.ok) return FGLT_ERR_UNSUPPORTED

fglt_status run(const Csr& g0, int64_t* out_raw, int64_t* out_net, cudaStream_t st, unsigned char* scratch) {
  Csr g = g0;
  const int64_t n = g.n;
  Carver C{scratch};
  TAKE(int32_t, cnt, K_NUM);
  TAKE(u64, ctr, W_NUM);
  const int64_t heavy_cap = g.nnz / HEAVY_DEGREE + 1;
  TAKE(int32_t, d, n);
  TAKE(int32_t, heavy, heavy_cap);
  CK(cudaMemsetAsync(cnt, 0, K_NUM * sizeof(int32_t), st));
  CK(cudaMemsetAsync(ctr, 0, W_NUM * sizeof(u64), st));
  int* err = cnt + K_ERR;

  CK(launch_degree(g, d, cnt + K_DMAX, heavy, cnt + K_NHEAVY, err, st));
  int32_t dmax = 0, e0 = 0;
  RB(cnt + K_DMAX, &dmax);
  RB(err, &e0);
  if (e0 & ERR_BAD_ROWPTR) return FGLT_ERR_INVALID_GRAPH;

  TAKE(int64_t, p2, n);
  TAKE(int64_t, r7, n);
  CK(launch_spmv1(g, d, heavy, cnt + K_NHEAVY, heavy_cap, p2, r7, err, st));

  TAKE(int32_t, hist, (int64_t)dmax + 1);
  TAKE(int64_t, base, (int64_t)dmax + 2);
  TAKE(int32_t, cursor, (int64_t)dmax + 1);
  TAKE(int32_t, rank, n);
  TAKE(int32_t, perm, n);
  TAKE(int32_t, dr, n);
  unsigned char* scan_tmp = C.take<unsigned char>((int64_t)scan_temp_bytes(std::max<int64_t>(n, dmax + 1) + 1));
  if (!C.ok) return FGLT_ERR_UNSUPPORTED;
  CK(cudaMemsetAsync(hist, 0, ((size_t)dmax + 1) * sizeof(int32_t), st));
  CK(cudaMemsetAsync(cursor, 0, ((size_t)dmax + 1) * sizeof(int32_t), st));
  CK(launch_degree_hist(d, n, hist, st));
  CK(launch_scan_i32_to_i64(hist, (int64_t)dmax + 1, base, scan_tmp, st));
  CK(launch_rank_assign(d, n, base, cursor, rank, perm, dr, st));

  TAKE(int32_t, opc, n);
  TAKE(int64_t, orp, n + 1);
  CK(launch_orient_count(g, rank, heavy, cnt + K_NHEAVY, heavy_cap, opc, cnt + K_DPMAX, st));
  CK(launch_scan_i32_to_i64(opc, n, orp, scan_tmp, st));
  int64_t m_or = 0;
  int32_t dpmax = 0;
  RB(orp + n, &m_or);
  RB(cnt + K_DPMAX, &dpmax);
  if (dpmax > 16384 || (dpmax >= 2 && !tri1_bitmap_fits_smem(dpmax))) return FGLT_ERR_UNSUPPORTED;
  TAKE(int32_t, ocol, m_or);
  TAKE(int32_t, ocur, n);
  CK(cudaMemsetAsync(ocur, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(int32_t), st));
  CK(launch_orient_fill(g, rank, orp, heavy, cnt + K_NHEAVY, heavy_cap, ocur, ocol, st));
  CK(launch_sort_rows(orp, n, dpmax, ocol, nullptr, st));

  constexpr int T0 = 64, T1 = 256;
  TAKE(int32_t, twork, 3 * n);
  CK(launch_worklist_outdeg3(opc, n, 2, T0, T1, twork, n, cnt + K_NTRI0, st));
  const int cap[3] = {std::min(dpmax, T0), std::min(dpmax, T1), dpmax};
  const bool on[3] = {dpmax >= 2, dpmax > T0, dpmax > T1};

  TAKE(int32_t, C3o, m_or);
  TAKE(u64, c3r, n);
  TAKE(u64, k4r, n);
  CK(cudaMemsetAsync(C3o, 0, (size_t)std::max<int64_t>(m_or, 1) * sizeof(int32_t), st));
  CK(cudaMemsetAsync(c3r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  CK(cudaMemsetAsync(k4r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  for (int c = 0; c < 3; ++c)
    if (on[c])
      CK(launch_tri1(orp, ocol, twork + c * n, cnt + K_NTRI0 + c, cnt + K_NEXT1_0 + c, cap[c], C3o, c3r, k4r,
                     nullptr, ctr + W_PROBES, err, st));

  TAKE(u64, r10r, n);
  TAKE(u64, r14r, n);
  TAKE(int64_t, c3oo, n);
  CK(cudaMemsetAsync(r10r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  CK(cudaMemsetAsync(r14r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  CK(launch_c3_edge_terms(orp, ocol, C3o, dr, n, r10r, r14r, st));
  CK(launch_unrank_u64(c3r, perm, n, c3oo, st));
  TAKE(int64_t, p3, n);
  TAKE(int64_t, r9, n);
  CK(launch_spmv2(g, d, p2, c3oo, heavy, cnt + K_NHEAVY, heavy_cap, p3, r9, st));

  TAKE(u64, r13r, n);
  CK(cudaMemsetAsync(r13r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  for (int c = 0; c < 3; ++c)
    if (on[c])
      CK(launch_tri2(orp, ocol, twork + c * n, cnt + K_NTRI0 + c, cnt + K_NEXT2_0 + c, cap[c], C3o, r13r, err,
                     st));

  // 4-cycles: with n within the dense hub span every top vertex has a dense
  // counter, so no vertex needs the global-memory hash tables.
  TAKE(int64_t, wc, n);
  TAKE(int64_t, wcn, n);
  const bool c16 = dmax < 65536;
  if (n > cyc_dense_span(c16)) return FGLT_ERR_UNSUPPORTED;
  const int32_t hub_lo = 0;
  CK(launch_wedge_count(g, rank, orp, ocol, heavy, cnt + K_NHEAVY, heavy_cap, hub_lo, wc, wcn, ctr + W_WMAX,
                        ctr + W_WSUM, st));
  TAKE(int32_t, lists, 4 * n);
  CK(launch_cyc_worklists(wc, wcn, n, lists, n, cnt + K_NCYC0, ctr + W_GCAP, true, st, n));
  int32_t n_gmem = 0;
  RB(cnt + K_NCYC3, &n_gmem);
  if (n_gmem != 0) return FGLT_ERR_INTERNAL;
  TAKE(u64, r12r, n);
  CK(cudaMemsetAsync(r12r, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(u64), st));
  CycArgs ca{};
  ca.rank = rank;
  ca.perm = perm;
  ca.orp = orp;
  ca.ocol = ocol;
  ca.wc = wc;
  ca.lists = lists;
  ca.list_stride = n;
  ca.counts = cnt + K_NCYC0;
  ca.next = cnt + K_NEXTC0;
  ca.c16 = c16;
  ca.hub_lo = hub_lo;
  ca.r12r = r12r;
  ca.err = err;
  ca.cap_bound = n;
  CK(launch_cyc(g, ca, st));

  EpilogueIn ein{d, rank, p2, p3, r7, r9, c3r, r10r, r12r, r13r, r14r, k4r};
  CK(launch_epilogue(ein, n, out_raw, out_net, st));
  int32_t e = 0;
  RB(err, &e);
  if (e & (ERR_BAD_GRAPH | ERR_BAD_ROWPTR)) return FGLT_ERR_INVALID_GRAPH;
  if (e) return FGLT_ERR_INTERNAL;
  return FGLT_OK;
}

}  // namespace

extern "C" fglt_status fglt_transform_noalloc(const void* rowptr, int rowptr_is_64bit, const int32_t* colidx,
                                              int64_t n, int64_t* out_raw, int64_t* out_net, void* stream) {
  if (n < 0 || (rowptr_is_64bit != 0 && rowptr_is_64bit != 1)) return FGLT_ERR_INVALID_ARG;
  if (n > FGLT_NOALLOC_MAX_VERTICES) return FGLT_ERR_UNSUPPORTED;
  if (n == 0) return FGLT_OK;
  if (!rowptr || (!out_raw && !out_net)) return FGLT_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FGLT_ERR_CUDA;
  unsigned char* scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) return FGLT_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Number of stored entries, read into host stack memory.
  int64_t nnz = 0;
  if (rowptr_is_64bit) {
    CK(cudaMemcpyAsync(&nnz, static_cast<const int64_t*>(rowptr) + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                       st));
  } else {
    int32_t v = 0;
    CK(cudaMemcpyAsync(&v, static_cast<const int32_t*>(rowptr) + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    nnz = v;
  }
  CK(cudaStreamSynchronize(st));
  if (nnz < 0) return FGLT_ERR_INVALID_GRAPH;
  if (nnz > FGLT_NOALLOC_MAX_ENTRIES) return FGLT_ERR_UNSUPPORTED;
  if (nnz > 0 && !colidx) return FGLT_ERR_INVALID_ARG;
  Csr g{rowptr, rowptr_is_64bit != 0, colidx, n, nnz};
  return run(g, out_raw, out_net, st, scratch);
}
