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
#include "fglt_pipeline.h"
#include "fglt_serve.h"

using namespace fglt;

namespace {

// Handle-owned buffers beyond the stage sequence's own.
enum HandleBufId {
  X_H_ROWPTR = B_PIPELINE_COUNT, X_H_COLIDX, X_H_RAW, X_H_NET, X_BATCH_OFF,
  X_IN_DEG0, X_IN_RP0, X_IN_CUR, X_IN_TMP, X_IN_DEG, X_IN_SCAN, X_IN_CNT, X_IN_SORT,
  X_RL_D, X_RL_HIST, X_RL_BASE, X_RL_CURSOR, X_RL_RANK, X_RL_INV, X_RL_NDEG, X_SMALL_ORDER, X_SMALL_CNT,
  X_COUNT
};

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct fglt_handle {
  int device = 0;
  fglt_options opt{};
  cudaStream_t stream = nullptr;
  Buf bufs[X_COUNT];
  Tuning tuning;  // from the options, or installed by fglt_autotune
  int cols = 16;  // output columns (sub-dictionary size)
  int64_t* pinned = nullptr;  // small host staging for read-backs
  std::string cuda_err;
  cudaEvent_t ev[NUM_STAGES + 1] = {};
  cudaEvent_t sub_ev[2 * NUM_SUB] = {};
  bool sub_rec[NUM_SUB] = {};
  float stage_ms[NUM_STAGES + NUM_SUB] = {};
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
    bool small = false;     // the fused small-graph launch (else the stage sequence)
    uint64_t off_hash = 0;  // fused launch: hash of the graph offsets it was set up for
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

// Returns a device buffer of at least `bytes` (grows by reallocating after
// the work queued on st and on the handle's stream, which may still use the
// old one, has finished).
fglt_status need(fglt_t h, int id, size_t bytes, void** out, cudaStream_t st) {
  Buf& b = h->bufs[id];
  if (bytes == 0) bytes = 16;
  if (b.bytes < bytes) {
    if (b.p) {
      cudaError_t e = cudaStreamSynchronize(st);
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

// The handle's grow-only workspace; scalars come back through its pinned word.
struct HandleWs final : Workspace {
  fglt_t h;
  cudaStream_t st;
  HandleWs(fglt_t hh, cudaStream_t s) : h(hh), st(s) {}
  fglt_status get(BufId id, size_t bytes, void** out) override { return need(h, id, bytes, out, st); }
  fglt_status read(void* host, const void* dev, size_t bytes, cudaStream_t s) override {
    if (bytes > 256) {
      CK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      return FGLT_OK;
    }
    CK(cudaMemcpyAsync(h->pinned, dev, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::memcpy(host, h->pinned, bytes);
    return FGLT_OK;
  }
  void cuda_error(cudaError_t e) override { h->cuda_err = cudaGetErrorString(e); }
};

// One transform on the handle's workspace (b: optional bounds, see Bounds).
fglt_status run_on_handle(fglt_t h, const Csr& g, int64_t* out_raw, int64_t* out_net, cudaStream_t st,
                          const Bounds* b = nullptr, bool capturing = false, const Tuning* tuning = nullptr,
                          bool force_profile = false) {
  HandleWs ws(h, st);
  RunOptions ro;
  ro.tuning = tuning ? *tuning : h->tuning;
  ro.validate = h->opt.validate != 0;
  ro.dict_mask = h->opt.dictionary_mask;
  ro.wait_ns = h->opt.device_wait_limit_ns;
  ro.bounds = b;
  ro.capturing = capturing;
  const bool prof = (h->opt.profile_stages != 0 || force_profile) && !capturing;
  ro.stage_events = prof ? h->ev : nullptr;
  ro.sub_events = prof ? h->sub_ev : nullptr;
  ro.sub_recorded = prof ? h->sub_rec : nullptr;
  int64_t work[O_NUM];
  ro.work = capturing ? nullptr : work;
  h->stages_valid = false;
  h->work_valid = false;
  fglt_status s = run_pipeline(ws, g, out_raw, out_net, st, ro);
  if (s != FGLT_OK || capturing) return s;
  std::memcpy(h->work, work, sizeof work);
  h->work_valid = true;
  if (prof) {
    for (int i = 0; i < NUM_STAGES; ++i) cudaEventElapsedTime(&h->stage_ms[i], h->ev[i], h->ev[i + 1]);
    for (int c = 0; c < NUM_SUB; ++c) {  // sub-stages that did not run read 0
      float t = 0;
      if (h->sub_rec[c] && cudaEventElapsedTime(&t, h->sub_ev[2 * c], h->sub_ev[2 * c + 1]) != cudaSuccess) t = 0;
      h->stage_ms[NUM_STAGES + c] = t;
    }
    cudaGetLastError();
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
// ---------------------------------------------------------------------------
// Autotuner: coordinate search over the tuning fields. The triangle-pass
// bounds only change the tri1/tri2 stages and the 4-cycle settings only the
// wedges/cyc stages, so one timed transform scores one candidate of each
// group at once (per-stage CUDA events).
// ---------------------------------------------------------------------------
namespace {

struct TuneScore {
  float tri = 0, cyc = 0, total = 0;
};

fglt_status time_once(fglt_t h, const Csr& g, cudaStream_t st, const Tuning& t, int reps, TuneScore* out) {
  TuneScore best{1e30f, 1e30f, 1e30f};
  for (int r = 0; r < reps; ++r) {
    fglt_status s = run_on_handle(h, g, nullptr, nullptr, st, nullptr, false, &t, true);
    if (s != FGLT_OK) return s;
    float tri = h->stage_ms[5] + h->stage_ms[9];
    float cyc = h->stage_ms[8] + h->stage_ms[10];
    float tot = 0;
    for (int i = 0; i < NUM_STAGES; ++i) tot += h->stage_ms[i];
    best.tri = std::min(best.tri, tri);
    best.cyc = std::min(best.cyc, cyc);
    best.total = std::min(best.total, tot);
  }
  *out = best;
  return FGLT_OK;
}

// The triangle-pass settings of a tuning (class bounds, loads in flight, hash
// slots per element, lanes per scanned list, warp-per-vertex bound).
void copy_tri(Tuning& dst, const Tuning& src) {
  dst.tri_t0 = src.tri_t0;
  dst.tri_t1 = src.tri_t1;
  dst.tri_loads = src.tri_loads;
  dst.tri_hash_factor = src.tri_hash_factor;
  dst.tri_group = src.tri_group;
  dst.tri_warp = src.tri_warp;
  dst.tri_pass2 = src.tri_pass2;
}

bool same_tri(const Tuning& a, const Tuning& b) {
  return a.tri_t0 == b.tri_t0 && a.tri_t1 == b.tri_t1 && a.tri_loads == b.tri_loads &&
         a.tri_hash_factor == b.tri_hash_factor && a.tri_group == b.tri_group && a.tri_warp == b.tri_warp &&
         a.tri_pass2 == b.tri_pass2;
}

}  // namespace

extern "C" fglt_status fglt_autotune(fglt_t h, const void* rowptr, int rowptr_is_64bit, const int32_t* colidx,
                                     int64_t n, int reps, void* stream, fglt_options* chosen, float* tuned_ms,
                                     float* default_ms) {
  if (!h || reps < 0) return FGLT_ERR_INVALID_ARG;
  if (n < 0 || (rowptr_is_64bit != 0 && rowptr_is_64bit != 1) || (n > 0 && !rowptr)) return FGLT_ERR_INVALID_ARG;
  if (reps == 0) reps = 1;
  std::lock_guard<std::mutex> lock(h->mu);
  if (cudaSetDevice(h->device) != cudaSuccess) return FGLT_ERR_CUDA;
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
  Csr g{rowptr, rowptr_is_64bit != 0, colidx, n, -1};
  const Tuning start = h->tuning;
  Tuning best = start;
  TuneScore base{};
  fglt_status s = FGLT_OK;
  if (n > 0) {
    if ((s = time_once(h, g, st, start, 1, &base)) != FGLT_OK) return s;  // warm-up (sizes the workspace)
    if ((s = time_once(h, g, st, start, reps, &base)) != FGLT_OK) return s;
    // Candidate values per parameter, tried one parameter at a time.
    // triangle candidates: class bounds t0, t1, loads in flight, hash slots per element, group lanes,
    // warp-per-vertex bound, vertex pass 2 lists from (0 automatic, 1 lowest, 2 middle)
    const int t_bounds[][7] = {{128, 512, 4, 4, 32, 32, 0}, {128, 512, 4, 4, 32, 16, 0}, {128, 512, 4, 4, 8, 32, 0},
                               {64, 256, 4, 4, 32, 32, 0},  {256, 768, 4, 4, 32, 32, 0}, {128, 512, 2, 4, 32, 32, 0},
                               {128, 512, 4, 4, 16, -1, 0}, {64, 256, 4, 4, 32, -1, 0},  {128, 384, 4, 2, 32, 32, 0},
                               {128, 512, 4, 4, 32, 32, 1}, {128, 512, 4, 4, 32, 32, 2}, {128, 384, 4, 2, 32, 32, 1},
                               {128, 384, 4, 2, 32, 32, 2}};
    const int wbits[] = {8, 9, 10};
    const int spans[] = {0, 16384, 32768, 65536, 90112};
    const int threads[] = {128, 256, 512, 1024};
    std::vector<Tuning> tri_c;
    for (auto& tb : t_bounds) {
      Tuning t = best;
      t.tri_t0 = tb[0];
      t.tri_t1 = tb[1];
      t.tri_loads = tb[2];
      t.tri_hash_factor = tb[3];
      t.tri_group = tb[4];
      t.tri_warp = tb[5] < 0 ? 0 : tb[5];
      t.tri_pass2 = tb[6];
      if (!same_tri(t, start)) tri_c.push_back(t);
    }
    TuneScore cur = base;
    // The 4-cycle parameters interact through the class split: search them in
    // sequence, each from the best found so far.
    auto try_cyc = [&](auto mutate, const int* vals, int nv) -> fglt_status {
      for (int i = 0; i < nv; ++i) {
        Tuning t = best;
        if (!mutate(t, vals[i])) continue;
        // pair this 4-cycle candidate with the next triangle candidate, if any
        Tuning run = t;
        const bool with_tri = !tri_c.empty();
        if (with_tri) copy_tri(run, tri_c.back());
        TuneScore sc;
        fglt_status e = time_once(h, g, st, run, reps, &sc);
        if (e != FGLT_OK) return e;
        if (with_tri) {
          if (sc.tri < cur.tri) {
            copy_tri(best, run);
            cur.tri = sc.tri;
          }
          tri_c.pop_back();
        }
        if (sc.cyc < cur.cyc) {  // keep the best triangle settings found so far
          Tuning next = t;
          copy_tri(next, best);
          best = next;
          cur.cyc = sc.cyc;
        }
      }
      return FGLT_OK;
    };
    // a candidate that sets one integer field (none if it already has that value)
    auto field = [](int Tuning::*f) {
      return [f](Tuning& t, int v) {
        if (t.*f == v) return false;
        t.*f = v;
        return true;
      };
    };
    if ((s = try_cyc(field(&Tuning::cyc_warp_bits), wbits, 3)) != FGLT_OK) return s;
    for (int c = 0; c < 3; ++c)
      if ((s = try_cyc([c](Tuning& t, int v) {
             if (t.cyc_mid_threads[c] == v) return false;
             t.cyc_mid_threads[c] = v;
             return true;
           }, threads, 4)) != FGLT_OK) return s;
    if ((s = try_cyc(field(&Tuning::cyc_heavy_threads), threads + 2, 2)) != FGLT_OK) return s;
    // The dense window and the dense-class threshold decide together which
    // vertices go dense, spill or hash: try them as pairs.
    const int dmins[] = {1024, 2048, 4096};
    int pairs[5 * 3];
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 3; ++b) pairs[a * 3 + b] = a * 3 + b;
    if ((s = try_cyc([&](Tuning& t, int v) {
           const int sp = spans[v / 3], dm = dmins[v % 3];
           if (t.cyc_hub_span == sp && t.cyc_dense_min == dm) return false;
           if (sp == 90112 && dm != 4096) return false;  // the widest window only pays for the heaviest vertices
           t.cyc_hub_span = sp;
           t.cyc_dense_min = dm;
           return true;
         }, pairs, 15)) != FGLT_OK) return s;
    const int sbits[] = {12, 13, 11};
    if ((s = try_cyc(field(&Tuning::cyc_spill_bits), sbits, 3)) != FGLT_OK) return s;
    const int lsegs[] = {12, 20, 32};
    if ((s = try_cyc(field(&Tuning::cyc_long_segment), lsegs, 3)) != FGLT_OK) return s;
    // triangle candidates left over
    while (!tri_c.empty()) {
      Tuning run = best;
      copy_tri(run, tri_c.back());
      tri_c.pop_back();
      TuneScore sc;
      if ((s = time_once(h, g, st, run, reps, &sc)) != FGLT_OK) return s;
      if (sc.tri < cur.tri) {
        copy_tri(best, run);
        cur.tri = sc.tri;
      }
    }
    // Confirm against the starting point on the whole transform.
    TuneScore fin;
    if ((s = time_once(h, g, st, best, reps + 1, &fin)) != FGLT_OK) return s;
    TuneScore again;
    if ((s = time_once(h, g, st, start, reps + 1, &again)) != FGLT_OK) return s;
    if (again.total < fin.total) {
      best = start;
      fin = again;
    }
    if (tuned_ms) *tuned_ms = fin.total;
    if (default_ms) *default_ms = again.total;
  } else {
    if (tuned_ms) *tuned_ms = 0;
    if (default_ms) *default_ms = 0;
  }
  h->tuning = best;
  tuning_to_options(best, &h->opt);
  if (chosen) *chosen = h->opt;
  h->batch.valid = false;  // a captured batch sequence used the old settings
  return FGLT_OK;
}

// Batched transform of graphs of at most SMALL_N_MAX vertices: one fused
// launch (k_small_fglt), captured as a CUDA graph and replayed while the
// buffers and the graph offsets stay the same. The device copies of the
// offsets and of the work order (largest graphs first) are made when they
// change. Called with h->mu held; runs on cs.
fglt_status batched_small(fglt_t h, const void* rowptr, int rp64, const int32_t* colidx, const int64_t* off,
                          int64_t num_graphs, int64_t* out_raw, int64_t* out_net, cudaStream_t cs) {
  const int64_t n = off[num_graphs];
  SubDict sd;
  fglt_status s = make_subdict(h->opt.dictionary_mask, &sd);
  if (s != FGLT_OK) return s;
  int64_t nnz = 0;
  {
    HandleWs ws(h, cs);
    int32_t v32 = 0;
    s = rp64 ? ws.read(&nnz, static_cast<const int64_t*>(rowptr) + n, 8, cs)
             : ws.read(&v32, static_cast<const int32_t*>(rowptr) + n, 4, cs);
    if (s != FGLT_OK) return s;
    if (!rp64) nnz = v32;
  }
  if (nnz < 0) return FGLT_ERR_INVALID_GRAPH;
  if (nnz > 0 && !colidx) return FGLT_ERR_INVALID_ARG;
  const bool full = sd.k == 16;
  uint64_t hash = 1469598103934665603ull;  // FNV-1a over the offsets
  for (int64_t i = 0; i <= num_graphs; ++i) hash = (hash ^ (uint64_t)off[i]) * 1099511628211ull;
  auto& bc = h->batch;
  void *doff = nullptr, *dorder = nullptr, *dcnt = nullptr;
  if ((s = need(h, X_BATCH_OFF, (size_t)(num_graphs + 1) * 8, &doff, cs)) != FGLT_OK) return s;
  if ((s = need(h, X_SMALL_ORDER, (size_t)std::max<int64_t>(num_graphs, 1) * 4, &dorder, cs)) != FGLT_OK) return s;
  if ((s = need(h, X_SMALL_CNT, 16, &dcnt, cs)) != FGLT_OK) return s;
  int* cnt = static_cast<int*>(dcnt);  // [0] work queue, [1] error word
  const bool same = bc.valid && bc.small && bc.rowptr == rowptr && bc.colidx == colidx && bc.raw == out_raw &&
                    bc.net == out_net && bc.rp64 == rp64 && bc.n == n && bc.nnz == nnz && bc.maxg == num_graphs &&
                    bc.off_hash == hash;
  if (!same) {
    std::vector<int32_t> order((size_t)num_graphs);
    for (int64_t i = 0; i < num_graphs; ++i) order[(size_t)i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return off[a + 1] - off[a] > off[b + 1] - off[b];
    });
    CK(cudaMemcpyAsync(doff, off, (size_t)(num_graphs + 1) * 8, cudaMemcpyHostToDevice, cs));
    CK(cudaMemcpyAsync(dorder, order.data(), (size_t)num_graphs * 4, cudaMemcpyHostToDevice, cs));
    CK(cudaStreamSynchronize(cs));  // the host order vector goes out of scope
    if (bc.exec) {
      cudaGraphExecDestroy(bc.exec);
      bc.exec = nullptr;
    }
    bc.valid = false;
    Csr g{rowptr, rp64 != 0, colidx, n, nnz};
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t e = cudaMemsetAsync(cnt, 0, 16, cs);
      if (e == cudaSuccess)
        e = launch_small_fglt(g, static_cast<const int64_t*>(doff), static_cast<const int32_t*>(dorder),
                              num_graphs, cnt, out_raw, out_net, sd, full, cnt + 1, cs);
      const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess && ee == cudaSuccess && graph && cudaGraphInstantiate(&bc.exec, graph, 0) == cudaSuccess) {
        bc.valid = true;
        bc.small = true;
        bc.rowptr = rowptr;
        bc.colidx = colidx;
        bc.raw = out_raw;
        bc.net = out_net;
        bc.rp64 = rp64;
        bc.n = n;
        bc.nnz = nnz;
        bc.maxg = num_graphs;
        bc.off_hash = hash;
      }
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
    if (!bc.valid) {  // capture unavailable: launch directly
      Csr g2{rowptr, rp64 != 0, colidx, n, nnz};
      CK(cudaMemsetAsync(cnt, 0, 16, cs));
      CK(launch_small_fglt(g2, static_cast<const int64_t*>(doff), static_cast<const int32_t*>(dorder), num_graphs,
                           cnt, out_raw, out_net, sd, full, cnt + 1, cs));
    }
  }
  if (bc.valid) {
    CK(cudaGraphLaunch(bc.exec, cs));
    ++h->batch_replays;
  }
  int e = 0;
  {
    HandleWs ws(h, cs);
    s = ws.read(&e, cnt + 1, sizeof e, cs);
  }
  if (s != FGLT_OK) return s;
  h->work_valid = false;
  h->stages_valid = false;
  if (e & (ERR_BAD_GRAPH | ERR_BAD_ROWPTR)) return FGLT_ERR_INVALID_GRAPH;
  if (e & ERR_TIMEOUT) return FGLT_ERR_TIMEOUT;
  return e ? FGLT_ERR_INTERNAL : FGLT_OK;
}

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
  Tuning tu;
  if (opt && opt->device_wait_limit_ns < 0) return FGLT_ERR_INVALID_ARG;
  if (opt) {
    fglt_status ts = tuning_from_options(*opt, &tu);
    if (ts != FGLT_OK) return ts;
    SubDict sd;
    if ((ts = make_subdict(opt->dictionary_mask, &sd)) != FGLT_OK) return ts;
  }
  fglt_t h = new (std::nothrow) fglt_handle();
  if (!h) return FGLT_ERR_OOM;
  h->device = device;
  if (opt) h->opt = *opt;
  h->tuning = tu;
  h->cols = dict_columns(h->opt.dictionary_mask);
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost(&h->pinned, 256);
  for (int i = 0; e == cudaSuccess && i <= NUM_STAGES; ++i) e = cudaEventCreate(&h->ev[i]);
  for (int i = 0; e == cudaSuccess && i < 2 * NUM_SUB; ++i) e = cudaEventCreate(&h->sub_ev[i]);
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
  for (int i = 0; i < 2 * NUM_SUB; ++i)
    if (h->sub_ev[i]) cudaEventDestroy(h->sub_ev[i]);
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
  Csr g{rowptr, rowptr_is_64bit != 0, colidx, n, -1};
  return run_on_handle(h, g, out_raw, out_net, st);
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
  if ((s = need(h, X_H_ROWPTR, (size_t)(n + 1) * elt, &drp, h->stream)) != FGLT_OK) return s;
  if ((s = need(h, X_H_COLIDX, (size_t)std::max<int64_t>(nnz, 1) * 4, &dci, h->stream)) != FGLT_OK) return s;
  const size_t out_bytes = (size_t)n * h->cols * 8;
  if (out_raw && (s = need(h, X_H_RAW, out_bytes, &draw, h->stream)) != FGLT_OK) return s;
  if (out_net && (s = need(h, X_H_NET, out_bytes, &dnet, h->stream)) != FGLT_OK) return s;
  cudaStream_t st = h->stream;
  CK(cudaMemcpyAsync(drp, rowptr, (size_t)(n + 1) * elt, cudaMemcpyHostToDevice, st));
  if (nnz > 0) CK(cudaMemcpyAsync(dci, colidx, (size_t)nnz * 4, cudaMemcpyHostToDevice, st));
  Csr g{drp, rowptr_is_64bit != 0, static_cast<const int32_t*>(dci), n, nnz};
  s = run_on_handle(h, g, static_cast<int64_t*>(draw), static_cast<int64_t*>(dnet), st);
  if (s != FGLT_OK) return s;
  if (out_raw) CK(cudaMemcpyAsync(out_raw, draw, out_bytes, cudaMemcpyDeviceToHost, st));
  if (out_net) CK(cudaMemcpyAsync(out_net, dnet, out_bytes, cudaMemcpyDeviceToHost, st));
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
  if (maxg - 1 > 2097151) return FGLT_ERR_OVERFLOW;  // binom(d,3) products must stay inside int64
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
  const int small_max = h->opt.batch_small_max == 0 ? SMALL_N_MAX : std::min(h->opt.batch_small_max, SMALL_N_MAX);
  if (small_max > 0 && maxg <= small_max)
    return finish(batched_small(h, rowptr, rowptr_is_64bit, colidx, graph_offsets, num_graphs, out_raw, out_net, cs));
  int64_t nnz = 0;
  {
    HandleWs ws(h, cs);
    int32_t v32 = 0;
    s = rowptr_is_64bit ? ws.read(&nnz, static_cast<const int64_t*>(rowptr) + n, 8, cs)
                        : ws.read(&v32, static_cast<const int32_t*>(rowptr) + n, 4, cs);
    if (s != FGLT_OK) return finish(s);
    if (!rowptr_is_64bit) nnz = v32;
  }
  if (nnz < 0) return finish(FGLT_ERR_INVALID_GRAPH);
  if (nnz > 0 && !colidx) return finish(FGLT_ERR_INVALID_ARG);
  const int64_t* off_dev = nullptr;
  if (h->opt.validate) {
    void* p = nullptr;
    if ((s = need(h, X_BATCH_OFF, (size_t)(num_graphs + 1) * 8, &p, cs)) != FGLT_OK) return finish(s);
    CK(cudaMemcpyAsync(p, graph_offsets, (size_t)(num_graphs + 1) * 8, cudaMemcpyHostToDevice, cs));
    off_dev = static_cast<const int64_t*>(p);
  }
  Bounds b{nnz, (int32_t)std::max<int64_t>(maxg - 1, 0), std::max<int64_t>(maxg - 1, 1), off_dev, num_graphs};
  Csr g{rowptr, rowptr_is_64bit != 0, colidx, n, nnz};
  auto& bc = h->batch;
  const bool same = bc.valid && !bc.small && bc.rowptr == rowptr && bc.colidx == colidx && bc.raw == out_raw &&
                    bc.net == out_net && bc.rp64 == rowptr_is_64bit && bc.n == n && bc.nnz == nnz &&
                    bc.maxg == maxg;
  if (same && !h->opt.validate && !h->opt.profile_stages) {
    // Replay: the graph re-zeroes its counters and accumulators itself.
    CK(cudaGraphLaunch(bc.exec, cs));
    ++h->batch_replays;
    int e = 0;
    {
      HandleWs ws(h, cs);
      s = ws.read(&e, static_cast<int*>(h->bufs[B_CNT].p) + err_word_index(), sizeof e, cs);
    }
    if (s != FGLT_OK) return finish(s);
    h->work_valid = false;
    h->stages_valid = false;
    if (e & (ERR_BAD_GRAPH | ERR_BAD_ROWPTR)) return finish(FGLT_ERR_INVALID_GRAPH);
    if (e & ERR_TIMEOUT) return finish(FGLT_ERR_TIMEOUT);
    return finish(e ? FGLT_ERR_INTERNAL : FGLT_OK);
  }
  s = run_on_handle(h, g, out_raw, out_net, cs, &b, false);
  if (s != FGLT_OK || h->opt.validate || h->opt.profile_stages) return finish(s);
  // Capture the same sequence (its buffers are sized now) for later calls.
  if (bc.exec) {
    cudaGraphExecDestroy(bc.exec);
    bc.exec = nullptr;
  }
  bc.valid = false;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const fglt_status cap = run_on_handle(h, g, out_raw, out_net, cs, &b, true);
    const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if (cap == FGLT_OK && ee == cudaSuccess && graph &&
        cudaGraphInstantiate(&bc.exec, graph, 0) == cudaSuccess) {
      bc.valid = true;
      bc.small = false;
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

fglt_status fglt_csr_from_edges(fglt_t h, const int32_t* src, const int32_t* dst, int64_t num_edges, int64_t n,
                                int64_t* out_rowptr, int32_t* out_colidx, int64_t* out_nnz, void* stream) {
  if (!h || n < 0 || num_edges < 0 || !out_rowptr || !out_nnz || (num_edges > 0 && (!src || !dst || !out_colidx)))
    return FGLT_ERR_INVALID_ARG;
  if (n > 0x7ffffffeLL || num_edges > (1LL << 30)) return FGLT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(h->mu);
  if (cudaSetDevice(h->device) != cudaSuccess) return FGLT_ERR_CUDA;
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
  HandleWs ws(h, st);
  fglt_status s;
  void *deg0, *rp0, *cur, *tmp, *deg, *scan, *cnt;
  const int64_t cap = 2 * num_edges;
  if ((s = need(h, X_IN_DEG0, (size_t)std::max<int64_t>(n, 1) * 4, &deg0, st)) != FGLT_OK) return s;
  if ((s = need(h, X_IN_RP0, (size_t)(n + 1) * 8, &rp0, st)) != FGLT_OK) return s;
  if ((s = need(h, X_IN_CUR, (size_t)std::max<int64_t>(n, 1) * 4, &cur, st)) != FGLT_OK) return s;
  if ((s = need(h, X_IN_TMP, (size_t)std::max<int64_t>(cap, 1) * 4, &tmp, st)) != FGLT_OK) return s;
  if ((s = need(h, X_IN_DEG, (size_t)std::max<int64_t>(n, 1) * 4, &deg, st)) != FGLT_OK) return s;
  if ((s = need(h, X_IN_SCAN, scan_temp_bytes(n + 1), &scan, st)) != FGLT_OK) return s;
  if ((s = need(h, X_IN_CNT, 16, &cnt, st)) != FGLT_OK) return s;
  int32_t* c = static_cast<int32_t*>(cnt);  // [0] max degree, [1] error bits
  CK(cudaMemsetAsync(cnt, 0, 16, st));
  if (n == 0) {
    CK(cudaMemsetAsync(out_rowptr, 0, 8, st));
    CK(cudaStreamSynchronize(st));
    *out_nnz = 0;
    return FGLT_OK;
  }
  CK(cudaMemsetAsync(deg0, 0, (size_t)n * 4, st));
  CK(cudaMemsetAsync(cur, 0, (size_t)n * 4, st));
  CK(launch_edge_count(src, dst, num_edges, n, static_cast<int32_t*>(deg0), c, c + 1, st));
  int32_t hc[2];
  if ((s = ws.read(hc, cnt, sizeof hc, st)) != FGLT_OK) return s;
  if (hc[1] & ERR_BAD_GRAPH) return FGLT_ERR_INVALID_GRAPH;
  int64_t* rp0p = static_cast<int64_t*>(rp0);
  CK(launch_scan_i32_to_i64(static_cast<int32_t*>(deg0), n, rp0p, scan, st));
  CK(launch_edge_fill(src, dst, num_edges, n, rp0p, static_cast<int32_t*>(cur), static_cast<int32_t*>(tmp), st));
  int32_t* sort_scratch = nullptr;
  if (const int64_t sort_ints = sort_rows_scratch_ints(cap, hc[0])) {
    void* p = nullptr;
    if ((s = need(h, X_IN_SORT, (size_t)sort_ints * 4, &p, st)) != FGLT_OK) return s;
    sort_scratch = static_cast<int32_t*>(p);
  }
  CK(launch_sort_rows(rp0p, n, hc[0], cap, static_cast<int32_t*>(tmp), sort_scratch, st));
  CK(launch_row_unique(rp0p, static_cast<int32_t*>(tmp), n, static_cast<int32_t*>(deg), nullptr, nullptr, st));
  CK(launch_scan_i32_to_i64(static_cast<int32_t*>(deg), n, out_rowptr, scan, st));
  CK(launch_row_unique(rp0p, static_cast<int32_t*>(tmp), n, nullptr, out_rowptr, out_colidx, st));
  return ws.read(out_nnz, out_rowptr + n, 8, st);
}

fglt_status fglt_csr_relabel_by_degree(fglt_t h, const void* rowptr, int rowptr_is_64bit, const int32_t* colidx,
                                       int64_t n, int descending, int64_t* out_rowptr, int32_t* out_colidx,
                                       int32_t* out_perm, void* stream) {
  if (!h || n < 0 || (rowptr_is_64bit != 0 && rowptr_is_64bit != 1) || (descending != 0 && descending != 1) ||
      !out_rowptr || (n > 0 && (!rowptr || !out_perm)))
    return FGLT_ERR_INVALID_ARG;
  if (n > 0x7ffffffeLL) return FGLT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(h->mu);
  if (cudaSetDevice(h->device) != cudaSuccess) return FGLT_ERR_CUDA;
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
  HandleWs ws(h, st);
  fglt_status s;
  if (n == 0) {
    CK(cudaMemsetAsync(out_rowptr, 0, 8, st));
    CK(cudaStreamSynchronize(st));
    return FGLT_OK;
  }
  const bool rp64 = rowptr_is_64bit != 0;
  int64_t nnz = 0;
  if (rp64) {
    if ((s = ws.read(&nnz, static_cast<const int64_t*>(rowptr) + n, 8, st)) != FGLT_OK) return s;
  } else {
    int32_t nnz32 = 0;
    if ((s = ws.read(&nnz32, static_cast<const int32_t*>(rowptr) + n, 4, st)) != FGLT_OK) return s;
    nnz = nnz32;
  }
  if (nnz < 0) return FGLT_ERR_INVALID_GRAPH;
  if (nnz > 0 && (!colidx || !out_colidx)) return FGLT_ERR_INVALID_ARG;
  void *d, *cnt, *rank, *inv, *ndeg;
  if ((s = need(h, X_RL_D, (size_t)n * 4, &d, st)) != FGLT_OK) return s;
  if ((s = need(h, X_IN_CNT, 16, &cnt, st)) != FGLT_OK) return s;
  if ((s = need(h, X_RL_RANK, (size_t)n * 4, &rank, st)) != FGLT_OK) return s;
  if ((s = need(h, X_RL_INV, (size_t)n * 4, &inv, st)) != FGLT_OK) return s;
  if ((s = need(h, X_RL_NDEG, (size_t)n * 4, &ndeg, st)) != FGLT_OK) return s;
  int32_t* c = static_cast<int32_t*>(cnt);  // [0] max degree, [1] error bits
  CK(cudaMemsetAsync(cnt, 0, 16, st));
  CK(launch_row_degree(rowptr, rp64, n, static_cast<int32_t*>(d), c, st));
  int32_t dmax = 0;
  if ((s = ws.read(&dmax, c, 4, st)) != FGLT_OK) return s;
  // counting sort by degree, as for the transform's degree order
  void *hist, *base, *cursor, *scan;
  if ((s = need(h, X_RL_HIST, ((size_t)dmax + 1) * 4, &hist, st)) != FGLT_OK) return s;
  if ((s = need(h, X_RL_BASE, ((size_t)dmax + 2) * 8, &base, st)) != FGLT_OK) return s;
  if ((s = need(h, X_RL_CURSOR, ((size_t)dmax + 1) * 4, &cursor, st)) != FGLT_OK) return s;
  if ((s = need(h, X_IN_SCAN, scan_temp_bytes(std::max<int64_t>(n, (int64_t)dmax + 1) + 1), &scan, st)) != FGLT_OK)
    return s;
  CK(cudaMemsetAsync(hist, 0, ((size_t)dmax + 1) * 4, st));
  CK(cudaMemsetAsync(cursor, 0, ((size_t)dmax + 1) * 4, st));
  CK(launch_degree_hist(static_cast<int32_t*>(d), n, static_cast<int32_t*>(hist), st));
  CK(launch_scan_i32_to_i64(static_cast<int32_t*>(hist), (int64_t)dmax + 1, static_cast<int64_t*>(base), scan, st));
  CK(launch_rank_assign(static_cast<int32_t*>(d), n, static_cast<int64_t*>(base), static_cast<int32_t*>(cursor),
                        static_cast<int32_t*>(rank), static_cast<int32_t*>(inv), static_cast<int32_t*>(ndeg), st));
  // inv and ndeg are rewritten for the requested direction
  CK(launch_relabel_ids(static_cast<int32_t*>(rank), static_cast<int32_t*>(d), n, descending != 0, out_perm,
                        static_cast<int32_t*>(inv), static_cast<int32_t*>(ndeg), st));
  CK(launch_scan_i32_to_i64(static_cast<int32_t*>(ndeg), n, out_rowptr, scan, st));
  CK(launch_relabel_fill(rowptr, rp64, colidx, out_perm, static_cast<int32_t*>(inv), n, out_rowptr, out_colidx,
                         c + 1, st));
  int32_t* sort_scratch = nullptr;
  if (const int64_t sort_ints = sort_rows_scratch_ints(nnz, dmax)) {
    void* p = nullptr;
    if ((s = need(h, X_IN_SORT, (size_t)sort_ints * 4, &p, st)) != FGLT_OK) return s;
    sort_scratch = static_cast<int32_t*>(p);
  }
  CK(launch_sort_rows(out_rowptr, n, dmax, nnz, out_colidx, sort_scratch, st));
  int32_t errw = 0;
  if ((s = ws.read(&errw, c + 1, 4, st)) != FGLT_OK) return s;
  return (errw & ERR_BAD_GRAPH) ? FGLT_ERR_INVALID_GRAPH : FGLT_OK;
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
  const int total = NUM_STAGES + NUM_SUB;
  const int k = std::min(max_stages, total);
  for (int i = 0; i < k; ++i) {
    if (names) names[i] = i < NUM_STAGES ? STAGE_NAMES[i] : SUB_NAMES[i - NUM_STAGES];
    if (ms) ms[i] = h->stage_ms[i];
  }
  *count = total;
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
  return run_on_handle(h, g, raw, net, st, b, false);
}
cudaStream_t handle_stream(fglt_t h) { return h->stream; }
int columns_of(fglt_t h) { return h->cols; }
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
