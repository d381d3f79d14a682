// Host-side launchers of the FGLT kernels. Every launcher enqueues work on
// `st` and returns the launch status; none synchronises.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fglt {

typedef unsigned long long u64;

// Kernel launches issued by the calling host thread (the pipeline reports the
// count per transform).
extern thread_local int64_t g_launches;
inline void note_launch(int k = 1) { g_launches += k; }

// Input CSR as given by the caller (device pointers).
struct Csr {
  const void* rowptr;
  bool rp64;
  const int32_t* colidx;
  int64_t n;
  int64_t nnz;
};

// Degree threshold above which a vertex of the input CSR is handled by a
// whole thread block instead of an 8-lane group.
constexpr int HEAVY_DEGREE = 512;

// --- input CSR passes ------------------------------------------------------
// Degrees, max degree, heavy-row list; flags malformed row pointers in *err.
// Degrees above dcap (a caller-supplied bound) are flagged and clamped.
cudaError_t launch_degree(const Csr& g, int32_t* d, int32_t* dmax, int32_t* heavy, int32_t* nheavy, int* err,
                          cudaStream_t st, int32_t dcap = 0x7fffffff);
// Batched inputs: flags an edge that joins two graphs (graph offsets on the device).
cudaError_t launch_validate_batch(const Csr& g, const int64_t* off, int64_t num_graphs, int* err, cudaStream_t st);
cudaError_t launch_validate(const Csr& g, const int32_t* heavy, const int32_t* nheavy, int64_t heavy_cap,
                            int* err, cudaStream_t st);
// p2 = A p1 - p1 and d^7 = A((p1-1)o(p1-2))/2 (SpMV chain 1)
// (also flags column indices outside [0, n) in *err; later passes skip them)
cudaError_t launch_spmv1(const Csr& g, const int32_t* d, const int32_t* heavy, const int32_t* nheavy,
                         int64_t heavy_cap, int64_t* p2, int64_t* r7, int* err, cudaStream_t st);
// p3 = A p2 - p1 o (p1-1) - 2 c3 and d^9 = A c3 - 2 c3 (SpMV chain 2)
cudaError_t launch_spmv2(const Csr& g, const int32_t* d, const int64_t* p2, const int64_t* c3o,
                         const int32_t* heavy, const int32_t* nheavy, int64_t heavy_cap,
                         int64_t* p3, int64_t* r9, cudaStream_t st);

// --- degree ordering and the oriented graph ---------------------------------
cudaError_t launch_degree_hist(const int32_t* d, int64_t n, int32_t* hist, cudaStream_t st);
cudaError_t launch_rank_assign(const int32_t* d, int64_t n, const int64_t* base, int32_t* cursor,
                               int32_t* rank, int32_t* perm, int32_t* dr, cudaStream_t st);
cudaError_t launch_orient_count(const Csr& g, const int32_t* rank, const int32_t* heavy,
                                const int32_t* nheavy, int64_t heavy_cap, int32_t* opc, int32_t* dpmax,
                                cudaStream_t st);
cudaError_t launch_orient_fill(const Csr& g, const int32_t* rank, const int64_t* orp, const int32_t* heavy,
                               const int32_t* nheavy, int64_t heavy_cap, int32_t* cursor, int32_t* ocol,
                               cudaStream_t st);
// Sorts every row of a CSR ascending (entries = total row length, dpmax = the
// longest row). Rows longer than 16384 are sorted one block per row in
// gscratch, which must hold sort_rows_scratch_ints(entries, dpmax) int32
// (none needed when dpmax <= 16384).
int64_t sort_rows_scratch_ints(int64_t entries, int32_t dpmax);
cudaError_t launch_sort_rows(const int64_t* orp, int64_t n, int32_t dpmax, int64_t entries, int32_t* ocol,
                             int32_t* gscratch, cudaStream_t st);
// Vertices (rank labels) with at least `min_out` out-neighbours.
cudaError_t launch_worklist_outdeg(const int32_t* opc, int64_t n, int min_out, int32_t* list,
                                   int32_t* count, cudaStream_t st);
// The same split into five lists by out-degree: [min_out, tw], (tw, t0],
// (t0, t1], (t1, t2], (t2, ...) at lists + c * stride, sizes in counts[0..4]
// (zeroed beforehand). With indeg, a vertex of the first list whose
// in-degree is above promote goes to the second.
cudaError_t launch_worklist_outdeg5(const int32_t* opc, int64_t n, int min_out, int tw, int t0, int t1, int t2,
                                    int32_t* lists, int64_t stride, int32_t* counts, cudaStream_t st,
                                    const int32_t* indeg = nullptr, int promote = 0);

// --- scans -----------------------------------------------------------------
// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.
size_t scan_temp_bytes(int64_t n);
cudaError_t launch_scan_i32_to_i64(const int32_t* in, int64_t n, int64_t* out, void* temp, cudaStream_t st);

// --- triangle passes (oriented, rank space) ---------------------------------
// Per-block shared memory the triangle kernels need for a max out-degree (hf:
// hash-table slots per element of N+(a), 2 or 4).
size_t tri1_smem_bytes(int dpmax, bool bitmap_in_smem, int hf = 2);
size_t tri2_smem_bytes(int dpmax, int hf = 2);
bool tri1_bitmap_fits_smem(int dpmax, int hf = 2);
// Dynamic shared memory a triangle-pass block may ask for.
size_t tri_smem_limit();
// Largest out-degree whose adjacency bitmap fits in shared memory.
int tri1_smem_bitmap_max(int hf = 2);
int tri_grid_blocks();
// C3 per oriented edge, c3 per vertex, 4-clique count per vertex (only with
// cliques = true). loads: list entries each lane has in flight per scan step
// (2 or 4); group: lanes that scan one out-list N+(b) together (8, 16, 32).
// work_ctr[0..2] += (scanned out-list entries, triangles, 4-cliques).
cudaError_t launch_tri1(const int64_t* orp, const int32_t* ocol, const int32_t* work, const int32_t* nwork,
                        int* next, int dpmax, int32_t* C3o, u64* c3r, u64* k4r, uint32_t* gbm,
                        u64* work_ctr, int* err, cudaStream_t st, bool cliques = true, int loads = 2, int hf = 2,
                        int group = 32, long long wait_ns = 0);
size_t tri1_gbm_bytes(int dpmax, int hf = 2);
// The same two passes for vertices of out-degree at most tri_warp_max(): one
// warp per vertex, everything in shared memory.
int tri_warp_max();
cudaError_t launch_tri1_warp(const int64_t* orp, const int32_t* ocol, const int32_t* work, const int32_t* nwork,
                             int* next, int32_t* C3o, u64* c3r, u64* k4r, u64* work_ctr, int* err, cudaStream_t st,
                             bool cliques, int loads);
cudaError_t launch_tri2_warp(const int64_t* orp, const int32_t* ocol, const int64_t* irp, const int2* iin,
                             const int32_t* work, const int32_t* nwork, int* next, const int32_t* C3o, u64* r13r,
                             int* err, cudaStream_t st, int loads, bool middle);
// d^13 (diamond, off-cord) per vertex from the final C3, listing each
// triangle from its middle vertex b (middle = true; work = the b of one
// out-degree class; irp/iin = in-lists, see launch_in_lists) or from its
// lowest vertex a like pass 1 (middle = false; irp/iin unused).
cudaError_t launch_tri2(const int64_t* orp, const int32_t* ocol, const int64_t* irp, const int2* iin,
                        const int32_t* work, const int32_t* nwork, int* next, int dpmax, const int32_t* C3o,
                        u64* r13r, int* err, cudaStream_t st, int loads, int hf, int group, bool middle);
// d^10 = C3 (p1 - 2) and d^14 = D4,3 e / 2 from the final C3 (rank space).
cudaError_t launch_c3_edge_terms(const int64_t* orp, const int32_t* ocol, const int32_t* C3o,
                                 const int32_t* dr, int64_t n, u64* r10r, u64* r14r, cudaStream_t st);
// c3o[perm[r]] = c3r[r]
cudaError_t launch_unrank_u64(const u64* src_r, const int32_t* perm, int64_t n, int64_t* dst_o,
                              cudaStream_t st);

// --- 4-cycles (rank space) ---------------------------------------------------
constexpr int CYC_CLASSES = 7;
constexpr int TRI_CLASSES = 5;  // out-degree classes of the triangle passes (the first: one warp per vertex)
// Largest window of top ranks the dense class can hold (16-bit counters in
// shared memory).
int cyc_dense_span_max();
// Largest spill-table size (at most spill_bits, at least 11) whose dense-class
// block fits in shared memory next to a window of span tops.
int cyc_fit_spill_bits(int span, int spill_bits, int threads);
// Largest per-vertex table need served by shared-memory tables; vertices above
// it may need the global-memory class.
int cyc_block_cap();
int cyc_gmem_blocks();
int cyc_warp_bits_max();
// In-lists of the oriented graph and the stage's wedge counts. For each rank w:
// iin[irp[w] .. irp[w+1]) = (v, j) with w = N+(v)[j] (any order; capacity
// dr[w] - opc[w]); wc[w] = wedges w - v - u with u in N+(v) above w; wcn[w] =
// those with u < hub_lo. hc, indeg: n int32 scratch; irp: n+1; icur: n int32
// zeroed; iin: m entries set to -1 bytes beforehand; wc, wcn zeroed.
cudaError_t launch_in_lists(const int64_t* orp, const int32_t* ocol, const int32_t* dr, const int32_t* opc,
                            int64_t n, int32_t hub_lo, int32_t* hc, int32_t* indeg, int64_t* irp, void* scan_tmp,
                            int32_t* icur, int2* iin, int64_t* wc, int64_t* wcn, cudaStream_t st);
// Splits the vertices with at least two wedges into CYC_CLASSES classes (lists
// at lists + c * list_stride, counts[c]): warp table (wc <= 2^(wbits-1)),
// three block hash-table sizes, dense hub counters with a shared spill table
// of 2^spill_bits slots (at most 2^(spill_bits-1) wedges outside the window)
// and with a global spill table (only if dense_ok, for vertices of degree
// dr < 65536), global hash table; *gcap_max = largest global table need;
// *wmax, *wsum = largest and total wedge count; cls_wedges[c] += wedges of the
// vertices in class c. cap_bound caps the distinct tops of one vertex (e.g.
// the largest graph of a block-diagonal batch minus one); pass n when unknown.
// Vertices with more than dense_min possible tops go to the dense class when
// they qualify for it, before the hash-table classes are considered.
cudaError_t launch_cyc_worklists(const int64_t* wc, const int64_t* wcn, const int32_t* dr, int64_t n, int32_t* lists,
                                 int64_t list_stride, int32_t* counts, u64* gcap_max, u64* wmax, u64* wsum,
                                 u64* cls_wedges, bool dense_ok, int64_t cap_bound, int wbits, int64_t dense_min,
                                 int spill_bits, cudaStream_t st);
struct CycArgs {
  int64_t n;
  const int64_t* orp;
  const int32_t* ocol;
  const int64_t* irp;
  const int2* iin;
  const int64_t* wc;
  const int64_t* wcn;
  const int32_t* lists;
  int64_t list_stride;
  const int32_t* counts;  // CYC_CLASSES class sizes
  int* next;              // CYC_CLASSES scheduling counters (zeroed)
  int32_t hub_lo;
  int wbits;              // warp-class table slots (log2, at most cyc_warp_bits_max())
  int mid_threads[3];     // block sizes of the three hash-table classes (128 .. 1024)
  int heavy_threads;      // block size of the dense and global classes
  int long_seg;           // block classes: segments at least this long are cut into warp-walked pieces
  int spill_bits;         // dense class: shared spill table of 2^spill_bits slots
  int gbits;              // global tables: cyc_gmem_blocks() << gbits slots each
  uint32_t* gkeys;        // 2 words (key, count) per slot; NULL when both global-table classes are empty
  uint32_t* gtouch;       // cyc_gmem_blocks() << (gbits - 1) claimed-slot lists
  u64* r12r;
  int* err;
  int64_t cap_bound;      // bound on distinct tops of one vertex (n when unknown)
  cudaEvent_t* ev;        // 2 * CYC_CLASSES events (start, stop of each class launch), or NULL
  bool* ev_rec;           // CYC_CLASSES flags: the class's pair was recorded
};
cudaError_t launch_cyc(const CycArgs& a, cudaStream_t st);

// --- edge-list ingest (k_ingest.cu) ---------------------------------------------
// deg0[v] += entries of v (both directions, self-loops skipped; zeroed
// beforehand); *dmax = max deg0 (zeroed); ids outside [0, n) flag ERR_BAD_GRAPH.
cudaError_t launch_edge_count(const int32_t* src, const int32_t* dst, int64_t E, int64_t n, int32_t* deg0,
                              int32_t* dmax, int* err, cudaStream_t st);
// tmp[rp0[v] + k] = the other end of v's k-th entry (cursor zeroed).
cudaError_t launch_edge_fill(const int32_t* src, const int32_t* dst, int64_t E, int64_t n, const int64_t* rp0,
                             int32_t* cursor, int32_t* tmp, cudaStream_t st);
// Rows of tmp sorted: colidx == NULL counts the distinct entries of each row
// into deg; otherwise writes them to colidx at rowptr.
cudaError_t launch_row_unique(const int64_t* rp0, const int32_t* tmp, int64_t n, int32_t* deg, const int64_t* rowptr,
                              int32_t* colidx, cudaStream_t st);
// Degree relabelling: d[v] from the row pointers and *dmax = max d (dmax
// zeroed by the caller); ids from the degree ranks (perm[v] = rank or n - 1 -
// rank, inv = perm^-1, ndeg[perm[v]] = d[v]); rows of the relabelled CSR,
// unsorted (ERR_BAD_GRAPH in *err for a column outside [0, n)).
cudaError_t launch_row_degree(const void* rowptr, bool rp64, int64_t n, int32_t* d, int32_t* dmax, cudaStream_t st);
cudaError_t launch_relabel_ids(const int32_t* rank, const int32_t* d, int64_t n, bool descending, int32_t* perm,
                               int32_t* inv, int32_t* ndeg, cudaStream_t st);
cudaError_t launch_relabel_fill(const void* rowptr, bool rp64, const int32_t* colidx, const int32_t* perm,
                                const int32_t* inv, int64_t n, const int64_t* out_rowptr, int32_t* out_colidx,
                                int* err, cudaStream_t st);

// --- batched small graphs (k_small.cu) ------------------------------------------
// Largest graph (vertices) of the fused small-graph launch.
constexpr int SMALL_N_MAX = 512;
struct SubDict;
// One block per graph of a block-diagonal batch (graph g owns vertices
// [off[g], off[g+1]), at most SMALL_N_MAX of them; blocks take the graphs in
// the given order): the whole transform in shared memory, Table I and
// U16^{-1} (or the sub-dictionary sd when !full) into raw / net. *next (zeroed)
// is the work queue; structural violations set ERR_BAD_GRAPH in *err.
cudaError_t launch_small_fglt(const Csr& g, const int64_t* off, const int32_t* order, int64_t num_graphs, int* next,
                              int64_t* raw, int64_t* net, const SubDict& sd, bool full, int* err, cudaStream_t st);

// --- epilogue ------------------------------------------------------------------
struct EpilogueIn {
  const int32_t* d;
  const int32_t* rank;
  const int64_t* p2;
  const int64_t* p3;
  const int64_t* r7;
  const int64_t* r9;
  const u64* c3r;
  const u64* r10r;
  const u64* r12r;
  const u64* r13r;
  const u64* r14r;
  const u64* r15r;
};
// Table I assembly and the exact int64 U16^{-1} product.
cudaError_t launch_epilogue(const EpilogueIn& in, int64_t n, int64_t* raw, int64_t* net, cudaStream_t st);

// Sub-dictionary s (Table II caption): the k columns col[0..k) of Table I
// (increasing sigma index) and the inverse of U16(s,s), row-major k x k.
struct SubDict {
  int k;
  int col[16];
  long long uinv[16][16];
};
cudaError_t launch_epilogue_sub(const EpilogueIn& in, const SubDict& sd, int64_t n, int64_t* raw, int64_t* net,
                                cudaStream_t st);

}  // namespace fglt
