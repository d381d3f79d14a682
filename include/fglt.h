/*
 * fglt.h — C ABI of the GB300 (sm_103a) Fast Graphlet Transform library.
 *
 * The graphlet transform (Floros, Pitsianis, Sun, "Fast Graphlet Transform of
 * Sparse Graphs", Sec. 2, eq. graphlet-transform) maps a simple undirected
 * graph G = (V, E) to one frequency vector per vertex over the dictionary
 * Sigma16 of Fig. 1 (all connected graphlets on up to 4 nodes, sigma_0 ..
 * sigma_15). This library computes both
 *   - the raw frequencies f^(v) = [d^_0(v) .. d^_15(v)] of Table I (subgraphs,
 *     induced or not, Sec. 4), and
 *   - the net frequencies f(v) = U16^{-1} f^(v) of Table II (Sec. 5), which for
 *     Sigma16 are the induced-subgraph orbit counts.
 * All counts are exact integers (int64).
 *
 * Conventions shared by every entry point:
 *  - Graph input is a symmetric CSR: row pointers (int32 or int64, n+1 entries,
 *    rowptr[0] = 0) and int32 column indices (rowptr[n] entries). Vertex ids are
 *    0-based (the paper numbers vertices from 1). The graph must be simple
 *    and undirected, as Sec. 1 assumes: no self-loops, every row strictly
 *    increasing (so no repeated neighbour), and j in N(i) iff i in N(j). With
 *    fglt_options.validate = 1 these preconditions are checked on the device
 *    and a violation returns FGLT_ERR_INVALID_GRAPH; otherwise a violating
 *    input gives unspecified counts (never a fault).
 *  - Output is row-major int64 [n][C]: row v, column k = frequency of sigma_k
 *    at vertex v (the orientation of the tables of Fig. 2); C = 16 for
 *    Sigma16, or the size of the handle's sub-dictionary (see
 *    fglt_options.dictionary_mask). Either output pointer may be NULL to skip
 *    it (not both).
 *  - Ownership: the caller owns every buffer it passes; the library never frees
 *    them and keeps no pointer to them after the call returns. The handle owns
 *    its device workspace, its stream and its serving slots.
 *  - Errors are returned as fglt_status, never thrown, printed or exited.
 *    A call that fails leaves the outputs unspecified.
 *  - Threading: a handle may be used by one host thread at a time, except the
 *    fglt_stream_* entries, which are safe to call from any thread.
 */
#ifndef FGLT_H
#define FGLT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FGLT_NUM_GRAPHLETS 16

typedef int fglt_status;

enum {
    FGLT_OK = 0,
    FGLT_ERR_INVALID_ARG = 1,   /* null pointer, negative size, bad flag */
    FGLT_ERR_INVALID_GRAPH = 2, /* validate = 1 and the CSR is not a simple symmetric graph */
    FGLT_ERR_OOM = 3,           /* device or host allocation failed */
    FGLT_ERR_OVERFLOW = 4,      /* max degree > 2,097,151: binom(d, 3) may leave int64 */
    FGLT_ERR_CUDA = 5,          /* a CUDA runtime call failed (see fglt_last_cuda_error) */
    FGLT_ERR_TIMEOUT = 6,       /* a bounded wait ran out (serving poll, device spin limit) */
    FGLT_ERR_PENDING = 7,       /* serving: the request has not finished yet */
    FGLT_ERR_NOT_FOUND = 8,     /* serving: unknown or already collected request id */
    FGLT_ERR_INTERNAL = 9,      /* a device-side consistency check failed */
    FGLT_ERR_UNSUPPORTED = 10,  /* input outside the sizes this build supports */
    FGLT_ERR_BUSY = 11,         /* serving: queue full or budget cannot ever fit the request */
    FGLT_ERR_CANCELLED = 12     /* serving: the request was cancelled */
};

typedef struct fglt_handle* fglt_t;

typedef struct {
    /* 1: check the CSR preconditions on the device before the transform. */
    int validate;
    /* Serving: bytes of device memory the resident request slots may use.
     * 0 selects half of the device memory free at fglt_create. */
    size_t serve_memory_budget;
    /* Serving: most requests packed into one launch (0 selects 256). */
    int serve_max_batch;
    /* Serving: most requests queued but not yet admitted (0 selects 65536). */
    int serve_max_queue;
    /* 1: record CUDA events around every stage of each transform so that
     * fglt_stage_times can report per-stage device time. */
    int profile_stages;
    /* Tuning (fglt_autotune picks these; the counts never depend on them; 0
     * selects the default):
     * cyc_hub_span: number of top-ranked (highest-degree) vertices that get
     *   dense 16-bit shared-memory counters in the 4-cycle stage (at most
     *   90112). 0 selects 32768, or 65536 for graphs above 2^22 vertices.
     *   Smaller values move work to the hash-table paths and raise occupancy. */
    int cyc_hub_span;
    /* tri_class_bounds: the triangle passes split the vertices by out-degree
     *   d+ in the degree order into (2, t0], (t0, t1], (t1, ...), each launched
     *   with shared memory sized for its largest d+ (default 128, 512;
     *   2 <= t0 < t1). */
    int tri_class_bounds[2];
    /* tri_probe_loads: list entries each lane of the triangle passes keeps in
     *   flight per scan step, 2 or 4 (default 4): more hides more memory
     *   latency, at the cost of scanning up to 32 * loads entries past the end
     *   of a scan. */
    int tri_probe_loads;
    /* tri_hash_factor: slots per element of the shared-memory hash table of
     *   N+(a) in the triangle passes, 2 or 4 (default 4): 4 shortens the probe
     *   runs that every lane of a warp waits for, at twice the table memory. */
    int tri_hash_factor;
    /* tri_group_lanes: lanes that scan one out-list N+(b) together in the
     *   triangle passes, 8, 16 or 32 (default 32): short out-lists leave most
     *   lanes of a 32-lane group idle. */
    int tri_group_lanes;
    /* tri_warp_max: vertices whose out-degree in the degree order is at most
     *   this run the triangle passes one warp per vertex instead of one block
     *   (at most 32; 0 selects the default 32; -1 turns the warp class off). */
    int tri_warp_max;
    /* cyc_warp_bits: log2 of the per-warp hash-table slots of the 4-cycle
     *   stage's warp class, which takes vertices with at most 2^(bits-1)
     *   wedges (6..10, default 10). */
    int cyc_warp_bits;
    /* cyc_mid_threads: thread-block size (128, 256, 512 or 1024; default 256) of
     *   the three block hash-table classes of the 4-cycle stage (tables of
     *   2^11, 2^12, 2^13 slots). */
    int cyc_mid_threads[3];
    /* cyc_heavy_threads: block size of the dense-counter and global-table
     *   classes of the 4-cycle stage (128, 256, 512 or 1024; default 1024). */
    int cyc_heavy_threads;
    /* cyc_dense_min: vertices with more possible 4-cycle tops than this
     *   (and few tops outside the dense window) use the dense-window class
     *   instead of a hash-table class (1 .. 4096; default 2048). */
    int cyc_dense_min;
    /* cyc_long_segment: in the block classes of the 4-cycle stage, a
     *   middle's segment of tops at least this long is cut into pieces, each
     *   walked by one warp (coalesced); shorter ones are walked by groups of 8
     *   lanes (2 .. 512; default 32). */
    int cyc_long_segment;
    /* cyc_spill_bits: the dense-window class keeps the tops outside its window
     *   in a shared-memory table of 2^bits slots and takes vertices with at
     *   most 2^(bits-1) wedges there; the others use a global-memory table
     *   (11 .. 13; default 11). */
    int cyc_spill_bits;
    /* Sub-dictionary s of Sigma16 (Table II caption): bit k set = sigma_k in
     * s; 0 (or 0xFFFF) selects Sigma16. Bits 0 and 1 must be set and no bit
     * above 15. Outputs then hold C = popcount(s) columns, sigma indices in
     * increasing order: raw = the Table I rows in s, net = U16(s,s)^{-1} raw.
     * Stages that no row in s needs are skipped; e.g. Sigma5 = 0x1F (the
     * graphlets on up to 3 nodes, the Sigma5 theorem of Sec. 3) needs only
     * degrees, p2 and the triangle counts c3. Applies to every entry point of
     * the handle (fglt_transform_noalloc always computes Sigma16). */
    unsigned int dictionary_mask;
    /* batch_small_max: fglt_transform_batched computes a batch whose graphs
     *   all have at most this many vertices with one fused launch, one thread
     *   block per graph, the graph's adjacency bitmap in shared memory (at
     *   most 512; 0 selects 512; -1 always runs the stage sequence). Batches
     *   with a larger graph run the stage sequence. */
    int batch_small_max;
    /* tri_pass2_from: the vertex from which the second triangle pass lists each
     *   triangle: 1 = its lowest vertex in the degree order (like the first
     *   pass: N+(b) scanned for every b in N+(a)), 2 = its middle vertex (the
     *   tail of N+(a) after b scanned for every in-entry a of b: at most
     *   sum_a binom(d+(a), 2) entries), 0 = the default, 2. */
    int tri_pass2_from;
    /* device_wait_limit_ns: limit of each bounded wait of a kernel on the
     *   completion of its tensor-core work (0 selects 2 s; 1 gives up after
     *   the first unsuccessful test, which exercises the error path). A wait
     *   that runs out ends the kernel's work cleanly, and the call returns
     *   FGLT_ERR_TIMEOUT; its outputs are then unspecified. */
    long long device_wait_limit_ns;
} fglt_options;

/* dictionary_mask of Sigma5 = {sigma_0 .. sigma_4}. */
#define FGLT_DICT_SIGMA5 0x1Fu

/* Fills *opt with the defaults (all fields 0 = automatic). */
fglt_status fglt_options_default(fglt_options* opt);

/* Creates a handle bound to CUDA device `device`. opt may be NULL (defaults).
 * Allocates the handle's stream; device workspace grows on demand. */
fglt_status fglt_create(fglt_t* handle, const fglt_options* opt, int device);

/* Destroys the handle: waits for its work, frees its workspace and stream.
 * Pending serving requests are cancelled. NULL is accepted. */
fglt_status fglt_destroy(fglt_t handle);

/* Static description of a status code. */
const char* fglt_status_string(fglt_status status);

/* Text of the last CUDA error seen by this handle ("" if none). */
const char* fglt_last_cuda_error(fglt_t handle);

/*
 * Single-graph transform, device buffers.
 *   rowptr          device pointer, n+1 entries, int64 if rowptr_is_64bit else int32
 *   colidx          device pointer, rowptr[n] int32 entries (NULL allowed if no edges)
 *   n               number of vertices (0 allowed: nothing is written)
 *   out_raw/out_net device pointers to n*C int64 (C = 16 for Sigma16), or NULL to skip one
 *   stream          cudaStream_t to order the work on (cudaStreamLegacy for the legacy
 *                   default stream), or NULL for the handle's stream, which is a
 *                   non-blocking stream: work the caller queued elsewhere is not
 *                   ordered before it
 * Computes Table I (raw) and Table II's inverse (net) for every vertex:
 * degrees and the SpMV chains of Sec. 3-4 (p1, p2, p3, d^7, d^9, d^10),
 * per-edge triangle counts C3 = A o A^2 (Lemma 2), the 4-cycle term c4 (Lemma
 * on c4), the diamond terms D4,c and D4,3 and the 4-clique term T (Sec. 4.3).
 * Returns after the work has completed on `stream` (it synchronises it).
 */
fglt_status fglt_transform(fglt_t handle, const void* rowptr, int rowptr_is_64bit,
                           const int32_t* colidx, int64_t n,
                           int64_t* out_raw, int64_t* out_net, void* stream);

/*
 * Single-graph transform, host buffers: copies the CSR to the device, runs
 * fglt_transform on the handle's stream and copies the outputs back. Same
 * arguments as fglt_transform, with every pointer a host pointer.
 */
fglt_status fglt_transform_host(fglt_t handle, const void* rowptr, int rowptr_is_64bit,
                                const int32_t* colidx, int64_t n,
                                int64_t* out_raw, int64_t* out_net);

/*
 * Batched transform of many independent graphs packed block-diagonally.
 *   rowptr, colidx    device CSR of the union (global vertex ids; no edge may
 *                     join two graphs)
 *   graph_offsets     HOST array, num_graphs+1 entries: graph g owns vertices
 *                     [graph_offsets[g], graph_offsets[g+1]); graph_offsets[0] = 0
 *   out_raw, out_net  device n*C int64 (n = graph_offsets[num_graphs])
 * The transform of a disjoint union is the concatenation of the transforms
 * (every graphlet is connected, Fig. 1), so the whole batch runs as one
 * sequence of launches captured once as a CUDA graph and replayed for batches
 * of the same shape.
 */
fglt_status fglt_transform_batched(fglt_t handle, const void* rowptr, int rowptr_is_64bit,
                                   const int32_t* colidx, const int64_t* graph_offsets,
                                   int64_t num_graphs, int64_t* out_raw, int64_t* out_net,
                                   void* stream);

/*
 * Autotuner: times the transform of the given graph (device buffers, as for
 * fglt_transform) under candidate settings of the tuning fields of
 * fglt_options (degree-class bounds of the triangle passes, hash-table sizes
 * and thread-block shapes of the 4-cycle classes, dense hub span and dense
 * threshold, the last two as pairs), one parameter at a time from the
 * current settings, keeps every change that lowers the device time of the
 * stage it affects, and installs the result on the handle for its later
 * single-graph, host and batched calls (serving lanes take the handle's
 * settings when the first request is submitted). The counts never depend on
 * these settings. Runs about 30 + 2 * reps transforms on `stream`; reps >= 1 timings per candidate (minimum
 * taken). chosen (nullable) receives the full option set in use afterwards.
 * tuned_ms / default_ms (nullable) receive the device time of one transform
 * with the chosen and with the starting settings.
 */
fglt_status fglt_autotune(fglt_t handle, const void* rowptr, int rowptr_is_64bit, const int32_t* colidx,
                          int64_t n, int reps, void* stream, fglt_options* chosen, float* tuned_ms,
                          float* default_ms);

/*
 * Builds the CSR input of the transform from an undirected edge list (device
 * buffers). The paper assumes a simple undirected graph (Sec. 1); this entry
 * makes one from any list of vertex pairs: vertex set {0 .. n-1}, an edge
 * {src[e], dst[e]} for every e, pairs in any order, in either or both
 * directions, repeated or not; self-loops are dropped and repeats merged.
 *   src, dst     device int32[num_edges], ids in [0, n)
 *   out_rowptr   device int64[n+1]
 *   out_colidx   device int32 with room for 2 * num_edges entries (the most
 *                the graph can have)
 *   out_nnz      host; receives rowptr[n] (twice the number of edges)
 * Rows come out sorted, symmetric and duplicate-free, ready for
 * fglt_transform. FGLT_ERR_INVALID_GRAPH if an id is outside [0, n) (the
 * outputs are then unspecified). Uses the handle's workspace; returns after
 * the work completed on stream (NULL = the handle's stream).
 */
fglt_status fglt_csr_from_edges(fglt_t handle, const int32_t* src, const int32_t* dst, int64_t num_edges,
                                int64_t n, int64_t* out_rowptr, int32_t* out_colidx, int64_t* out_nnz,
                                void* stream);

/*
 * Degree-ordered relabelling of a CSR graph (device buffers), for locality:
 * vertex v gets the new id perm[v] = its position in non-increasing degree
 * order (descending = 1) or non-decreasing degree order (descending = 0);
 * vertices of equal degree take their positions in an unspecified order. The
 * transform of the relabelled graph is the transform of the input with its
 * rows permuted by perm (Sec. 2: the transform is invariant under graph
 * isomorphism, vertex by vertex).
 *   rowptr, colidx  the input CSR (int64 or int32 row pointers, int32
 *                   columns in [0, n)); it is not modified
 *   out_rowptr      device int64[n+1], the relabelled row pointers
 *   out_colidx      device int32[rowptr[n]], the relabelled columns, each
 *                   row sorted ascending (may be NULL when rowptr[n] = 0)
 *   out_perm        device int32[n], perm[old id] = new id
 * FGLT_ERR_INVALID_GRAPH if a column is outside [0, n) (the outputs are then
 * unspecified); FGLT_ERR_UNSUPPORTED above 2^31 - 2 vertices. The outputs
 * must not overlap the inputs. Uses the handle's workspace; returns after
 * the work completed on stream (NULL = the handle's stream).
 */
fglt_status fglt_csr_relabel_by_degree(fglt_t handle, const void* rowptr, int rowptr_is_64bit,
                                       const int32_t* colidx, int64_t n, int descending,
                                       int64_t* out_rowptr, int32_t* out_colidx, int32_t* out_perm,
                                       void* stream);

/* Per-stage device times (ms) of the last transform on this handle; requires
 * fglt_options.profile_stages = 1. names[i] points to static strings.
 * *count receives the number of entries (at most max_stages are written):
 * the stages in order (degree, spmv1, rank, orient, sort, tri1, c3_edges,
 * spmv2, tri2, wedges, cyc, epilogue), then their parts: the seven 4-cycle
 * vertex classes inside "cyc" (cyc.warp, cyc.hash11, cyc.hash12, cyc.hash13,
 * cyc.dense, cyc.dense_spill, cyc.global) and the five out-degree classes of
 * each triangle pass (tri1.w, tri1.c0 .. tri1.c3, tri2.w, tri2.c0 ..
 * tri2.c3; ".w" is the warp-per-vertex class); a part that did not run reads
 * 0. */
fglt_status fglt_stage_times(fglt_t handle, const char** names, float* ms,
                             int max_stages, int* count);

/* Work counters of the last successful transform on this handle, for
 * roofline accounting. counters[i] (at most max_counters written; *count
 * receives the number available):
 *   0 n                 vertices
 *   1 nnz               stored CSR entries (2m for a valid graph)
 *   2 m                 edges of the degree-ordered orientation (= undirected edges)
 *   3 max degree
 *   4 max out-degree in the degree orientation
 *   5 out-list entries scanned by the first triangle pass (sum over a -> b of
 *     the part of N+(b) not above max N+(a))
 *   6 triangles (each once; e^T C3 e / 6, Lemma 3)
 *   7 4-cliques (each once)
 *   8 wedges enumerated by the 4-cycle stage
 *   9 largest wedge count of one vertex
 *  10 kernel launches the transform issued (memsets not included)
 *  11..17 vertices in each 4-cycle vertex class (the order of the cyc.*
 *         entries of fglt_stage_times)
 *  18..24 wedges of the vertices in each class
 * FGLT_ERR_NOT_FOUND if no transform has completed on the handle. */
fglt_status fglt_work_counters(fglt_t handle, int64_t* counters, int max_counters, int* count);

/*
 * Single-graph transform that allocates nothing (no cudaMalloc, cudaFree or
 * other allocating call) — for callers that cannot allocate device memory at
 * call time: a process whose device memory is already owned by another
 * allocator (so cudaMalloc could fail at any point), a latency-bound loop that
 * cannot afford the device-wide synchronisation allocation may cause, or code
 * that must fix its memory use when the library loads. The paper has no
 * counterpart; this is a library facility.
 *   Same arguments and results as fglt_transform, without a handle; stream may
 *   be NULL (the legacy default stream). Returns after the work completed.
 *   Scratch: one file-scope device array of FGLT_NOALLOC_SCRATCH_BYTES held by
 *   every device that loads the library until exit. Limits: n <=
 *   FGLT_NOALLOC_MAX_VERTICES and rowptr[n] <= FGLT_NOALLOC_MAX_ENTRIES;
 *   larger inputs return FGLT_ERR_UNSUPPORTED before any device work. Every
 *   buffer of an input within both limits fits the array (the out-degree
 *   classes that would need more, above 1024, need more entries than the
 *   limit); each piece is still checked, and one that did not fit would
 *   also return FGLT_ERR_UNSUPPORTED. An error return has waited for the
 *   call's queued work.
 *   The first call on each device looks up the array's address; make it before
 *   any stream capture. All calls share the array and each leaves its data
 *   there: calls whose device work overlaps race — serialise them.
 */
#define FGLT_NOALLOC_SCRATCH_BYTES (16u << 20)
#define FGLT_NOALLOC_MAX_VERTICES 32768
#define FGLT_NOALLOC_MAX_ENTRIES 1048576
fglt_status fglt_transform_noalloc(const void* rowptr, int rowptr_is_64bit, const int32_t* colidx,
                                   int64_t n, int64_t* out_raw, int64_t* out_net, void* stream);

/* ---------------------------------------------------------------------------
 * Serving: requests arrive one by one from host memory; the library admits
 * them into resident device slots within fglt_options.serve_memory_budget,
 * packs admitted requests into shared launches (continuous batching) and
 * copies the results back to the caller's host buffers.
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t n;              /* vertices */
    const int64_t* rowptr;  /* host, n+1 entries */
    const int32_t* colidx;  /* host, rowptr[n] entries */
    int64_t* out_raw;       /* host, n*C (C as for fglt_transform), or NULL */
    int64_t* out_net;       /* host, n*C, or NULL */
} fglt_graph_host;

/* Queues a request. The CSR is copied into a staging buffer before the call
 * returns; the output buffers must stay valid until the request is collected
 * by fglt_stream_poll or fglt_stream_cancel. */
fglt_status fglt_stream_submit(fglt_t handle, const fglt_graph_host* graph, uint64_t* request_id);

/* Waits up to timeout_ms (0 = do not wait, -1 = forever) for a request.
 * FGLT_OK: results are in the request's output buffers and the id is retired.
 * FGLT_ERR_PENDING (timeout 0) / FGLT_ERR_TIMEOUT: not finished yet.
 * latency_us (nullable) receives submit-to-results-on-host time. */
fglt_status fglt_stream_poll(fglt_t handle, uint64_t request_id, int timeout_ms, double* latency_us);

/* Cancels a request that has not been admitted yet (FGLT_ERR_BUSY if it is
 * already on the device, in which case poll it as usual). */
fglt_status fglt_stream_cancel(fglt_t handle, uint64_t request_id);

#ifdef __cplusplus
}
#endif

#endif /* FGLT_H */
