// The stage sequence of one transform, shared by every entry point. Where its
// buffers come from (a handle's grow-only workspace, or a fixed scratch array)
// and how it reads device scalars back are supplied by a Workspace.
#pragma once

#include "fglt.h"
#include "fglt_kernels.h"

// Host-side bounds that replace the pipeline's read-backs (block-diagonal
// batches: every degree, out-degree and per-vertex count of distinct 4-cycle
// tops is below the largest graph's vertex count). With them the stage
// sequence has no host synchronisation and can be captured as a CUDA graph.
struct Bounds {
  int64_t nnz;         // exact stored entries
  int32_t dmax;        // bound on every degree
  int64_t cap;         // bound on distinct tops per vertex
  const int64_t* off;  // device graph offsets for validation (or NULL)
  int64_t num_graphs;
};

namespace fglt {

// Buffers of the stage sequence (one slot each in a workspace).
enum BufId {
  B_D, B_HEAVY, B_CNT, B_HIST, B_BASE, B_CURSOR, B_RANK, B_PERM, B_DR, B_OPC, B_ORP, B_SCAN, B_OCOL, B_OCUR,
  B_SORT, B_TWORK, B_C3O, B_C3R, B_K4R, B_R10R, B_R14R, B_R13R, B_R12R, B_C3OO, B_P2, B_P3, B_R7, B_R9, B_WC,
  B_LS, B_WCN, B_GBM, B_GKEYS, B_GTOUCH, B_HC, B_INDEG, B_IRP, B_ICUR, B_IIN, B_CTR64,
  B_PIPELINE_COUNT
};

// Order of the work counters (fglt_work_counters).
enum WorkOut {
  O_N, O_NNZ, O_M, O_DMAX, O_DPMAX, O_PROBES, O_TRIANGLES, O_K4, O_WEDGES, O_WMAX, O_LAUNCHES,
  O_CLS_VERTICES, O_CLS_WEDGES = O_CLS_VERTICES + CYC_CLASSES, O_NUM = O_CLS_WEDGES + CYC_CLASSES
};

constexpr int NUM_STAGES = 12;
extern const char* const STAGE_NAMES[NUM_STAGES];
// Sub-stages: the 4-cycle vertex classes inside "cyc", then the out-degree
// classes of "tri1" and of "tri2".
constexpr int NUM_SUB = CYC_CLASSES + 2 * TRI_CLASSES;
extern const char* const SUB_NAMES[NUM_SUB];

// Tunables; the counts never depend on them (fglt_options documents each).
struct Tuning {
  int tri_t0 = 128, tri_t1 = 512;
  int tri_loads = 4;
  int tri_hash_factor = 4;
  int tri_group = 32;
  int tri_warp = 32;  // out-degrees up to this run one warp per vertex (0: off)
  int cyc_warp_bits = 10;
  int cyc_mid_threads[3] = {256, 256, 256};
  int cyc_heavy_threads = 1024;
  int cyc_hub_span = 0;
  int cyc_dense_min = 2048;
  int cyc_long_segment = 32;
  int cyc_spill_bits = 11;
  int tri_pass2 = 0;  // 0 automatic, 1 lowest vertex, 2 middle vertex
};

// Fills t from the options (0 fields keep the defaults) and checks ranges.
fglt_status tuning_from_options(const fglt_options& o, Tuning* t);
void tuning_to_options(const Tuning& t, fglt_options* o);

class Workspace {
 public:
  virtual ~Workspace() = default;
  // A device buffer of at least `bytes` for slot id, valid until the next
  // get of the same slot. FGLT_ERR_OOM / FGLT_ERR_UNSUPPORTED if unavailable.
  virtual fglt_status get(BufId id, size_t bytes, void** out) = 0;
  // Copies bytes from device memory to host memory after the work queued on
  // st, and waits for it.
  virtual fglt_status read(void* host, const void* dev, size_t bytes, cudaStream_t st) = 0;
  // Text of the last CUDA error (for the handle's diagnostics).
  virtual void cuda_error(cudaError_t) {}
};

// Sub-dictionary s of Sigma16 as a bit mask (bit k = sigma_k); 0 and 0xFFFF
// both select Sigma16. FGLT_ERR_INVALID_ARG unless bits 0 and 1 are set and
// no bit above 15 is (Table II caption: {0,1} is a subset of s).
fglt_status make_subdict(uint32_t mask, SubDict* sd);
// Output columns of a dictionary mask (16 for Sigma16).
int dict_columns(uint32_t mask);

struct RunOptions {
  Tuning tuning;
  uint32_t dict_mask = 0;           // sub-dictionary (0 = Sigma16)
  bool validate = false;
  const Bounds* bounds = nullptr;   // replaces every read-back (see Bounds)
  bool capturing = false;           // stream capture in progress: no read-back, no allocation
  cudaEvent_t* stage_events = nullptr;  // NUM_STAGES + 1 events, or NULL
  cudaEvent_t* sub_events = nullptr;    // 2 * NUM_SUB events (start, stop per sub-stage), or NULL
  bool* sub_recorded = nullptr;         // NUM_SUB flags set for the sub-stages that ran
  int64_t* work = nullptr;              // O_NUM counters out, or NULL
  long long wait_ns = 0;                // limit of a bounded device wait (0 = the kernels' default)
};

// Index of the device error word in the B_CNT buffer (any set bit is a
// failure; see the ERR_ bits).
int err_word_index();

// The whole transform on stream st. g.nnz < 0 means "read rowptr[n]".
fglt_status run_pipeline(Workspace& ws, const Csr& g, int64_t* out_raw, int64_t* out_net, cudaStream_t st,
                         const RunOptions& ro);

}  // namespace fglt
