// Serving runtime: continuous batching of host-submitted graphs.
//
// Requests are staged in host memory at submit time and queued. Worker lanes
// (each with its own device workspace, stream and pinned staging buffers) take
// queued requests as device memory allows (fglt_options.serve_memory_budget,
// split evenly over the lanes), pack them block-diagonally into one CSR — the
// transform of a disjoint union is the concatenation of the transforms, since
// every graphlet is connected (Fig. 1) — run one transform for the pack, and
// copy each request's rows back to its output buffers. While one lane's pack is
// on the device, the next lane admits and launches whatever arrived in the
// meantime, so the work of different packs overlaps on the GPU. A pack that
// fails is retried request by request so that one bad input does not fail the
// others.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fglt_serve.h"

namespace fglt {
namespace serve {

namespace {

using clk = std::chrono::steady_clock;

enum State { QUEUED, RUNNING, DONE, FAILED };

struct Request {
  uint64_t id = 0;
  int64_t n = 0, nnz = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colidx;
  int64_t* out_raw = nullptr;
  int64_t* out_net = nullptr;
  size_t est = 0;
  clk::time_point t_submit;
  double latency_us = 0;
  State state = QUEUED;
  fglt_status status = FGLT_OK;
  int passed = 0;  // times a later request was admitted ahead of this one
};

// Device bytes a request occupies while on the device: the packed input and
// output, and the transform's workspace (per-vertex arrays, the oriented graph
// and its per-edge counts).
size_t estimate_bytes(int64_t n, int64_t nnz) {
  return (size_t)n * 512 + (size_t)nnz * 24 + ((size_t)4 << 20);
}

template <typename T>
struct HostBuf {  // pinned, grow-only
  T* p = nullptr;
  size_t cap = 0;
  bool reserve(size_t count) {
    if (count <= cap) return true;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    const size_t want = count + count / 4 + 1024;
    if (cudaMallocHost(&p, want * sizeof(T)) != cudaSuccess) {
      p = nullptr;
      return false;
    }
    cap = want;
    return true;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
  }
};

template <typename T>
struct DevBuf {  // device, grow-only
  T* p = nullptr;
  size_t cap = 0;
  bool reserve(size_t count, cudaStream_t st) {
    if (count <= cap) return true;
    cudaStreamSynchronize(st);
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = count + count / 4 + 1024;
    if (cudaMalloc(&p, want * sizeof(T)) != cudaSuccess) {
      p = nullptr;
      return false;
    }
    cap = want;
    return true;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

}  // namespace

struct Lane {
  fglt_t h = nullptr;  // private handle: workspace
  // Packs holding a large request run on the high-priority stream, so that
  // packs of small requests on the other lanes fill the SMs it leaves idle
  // rather than slow it down; the others run on the low-priority one.
  cudaStream_t hi = nullptr, lo = nullptr;
  std::thread th;
  HostBuf<int64_t> h_rowptr, h_raw, h_net;
  HostBuf<int32_t> h_colidx;
  DevBuf<int64_t> d_rowptr, d_raw, d_net, d_parts;
  DevBuf<int32_t> d_colidx;
  HostBuf<int64_t> h_parts;
};

struct Server {
  fglt_t owner = nullptr;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> all;
  uint64_t next_id = 1;
  size_t budget = 0, lane_cap = 0, reserved = 0;
  int max_batch = 256, max_queue = 65536;
  bool stop = false;
  std::vector<Lane*> lanes;
};

namespace {

constexpr int64_t BOUNDED_MAX_GRAPH = 4096;      // packs whose graphs are all this small skip read-backs
constexpr int64_t PACK_MAX_ENTRIES = 1LL << 22;  // a pack stops growing past this many CSR entries
constexpr int ADMIT_LOOKAHEAD = 64;  // queued requests scanned per admission
constexpr int64_t LARGE_REQUEST_ENTRIES = 1LL << 20;  // packs with a request this large take the high-priority stream
constexpr int MAX_PASSED = 8;        // a request overtaken this often stops later ones from passing it

// Block-diagonal packing on the device: the parts' rows and columns were
// copied with their own (local) ids; part p = (vertex offset, entry offset,
// n, nnz) at parts[4p..4p+3]. Adds the vertex offset to its columns and the
// entry offset to its row pointers rowptr[vo+1 .. vo+n].
__global__ void k_rebase_pack(int64_t* __restrict__ rowptr, int32_t* __restrict__ colidx,
                              const int64_t* __restrict__ parts, int np) {
  const int p = blockIdx.y;
  if (p >= np) return;
  const int64_t vo = parts[4 * p], eo = parts[4 * p + 1], n = parts[4 * p + 2], nnz = parts[4 * p + 3];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride)
    colidx[eo + k] += (int32_t)vo;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) rowptr[vo + 1 + v] += eo;
}

// Runs one pack on a lane. Returns the status of the whole pack.
fglt_status run_pack(Lane* L, const std::vector<Request*>& pack) {
  int64_t n = 0, nnz = 0;
  for (Request* r : pack) {
    n += r->n;
    nnz += r->nnz;
  }
  if (!L->h_rowptr.reserve(n + 1) || !L->h_colidx.reserve(std::max<int64_t>(nnz, 1)) ||
      !L->h_raw.reserve(n * columns_of(L->h)) || !L->h_net.reserve(n * columns_of(L->h)))
    return FGLT_ERR_OOM;
  // Block-diagonal packing: each part is copied as it is (local ids) and the
  // device adds its offsets (k_rebase_pack).
  const int np = (int)pack.size();
  if (!L->h_parts.reserve(4 * (size_t)np)) return FGLT_ERR_OOM;
  int64_t vo = 0, eo = 0;
  L->h_rowptr.p[0] = 0;
  for (int p = 0; p < np; ++p) {
    const Request* r = pack[p];
    std::memcpy(L->h_rowptr.p + vo + 1, r->rowptr.data() + 1, (size_t)r->n * 8);
    if (r->nnz) std::memcpy(L->h_colidx.p + eo, r->colidx.data(), (size_t)r->nnz * 4);
    int64_t* q = L->h_parts.p + 4 * p;
    q[0] = vo;
    q[1] = eo;
    q[2] = r->n;
    q[3] = r->nnz;
    vo += r->n;
    eo += r->nnz;
  }
  int64_t biggest = 0;
  for (Request* r : pack) biggest = std::max(biggest, r->nnz);
  cudaStream_t st = biggest >= LARGE_REQUEST_ENTRIES ? L->hi : L->lo;
  if (!L->d_rowptr.reserve(n + 1, st) || !L->d_colidx.reserve(std::max<int64_t>(nnz, 1), st) ||
      !L->d_raw.reserve(n * columns_of(L->h), st) || !L->d_net.reserve(n * columns_of(L->h), st) ||
      !L->d_parts.reserve(4 * (size_t)np, st))
    return FGLT_ERR_OOM;
  if (cudaMemcpyAsync(L->d_rowptr.p, L->h_rowptr.p, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FGLT_ERR_CUDA;
  if (nnz > 0 &&
      cudaMemcpyAsync(L->d_colidx.p, L->h_colidx.p, (size_t)nnz * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FGLT_ERR_CUDA;
  if (np > 1) {
    if (cudaMemcpyAsync(L->d_parts.p, L->h_parts.p, (size_t)np * 32, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return FGLT_ERR_CUDA;
    const unsigned gx = (unsigned)std::min<int64_t>(std::max<int64_t>((biggest + 255) / 256, 1), 1024);
    k_rebase_pack<<<dim3(gx, (unsigned)np), 256, 0, st>>>(L->d_rowptr.p, L->d_colidx.p, L->d_parts.p, np);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return FGLT_ERR_CUDA;
  }
  Csr g{L->d_rowptr.p, true, L->d_colidx.p, n, nnz};
  // Packs of small graphs run the stage sequence without host read-backs:
  // the largest request bounds every degree and every per-vertex table.
  int64_t maxg = 0;
  for (Request* r : pack) maxg = std::max(maxg, r->n);
  fglt_status s;
  if (maxg <= BOUNDED_MAX_GRAPH) {
    Bounds b{nnz, (int32_t)std::max<int64_t>(maxg - 1, 0), std::max<int64_t>(maxg - 1, 1), nullptr, 0};
    s = transform_locked(L->h, g, L->d_raw.p, L->d_net.p, st, &b);
  } else {
    s = transform_locked(L->h, g, L->d_raw.p, L->d_net.p, st);
  }
  if (s != FGLT_OK) return s;
  const int64_t C = columns_of(L->h);
  if (cudaMemcpyAsync(L->h_raw.p, L->d_raw.p, (size_t)n * C * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(L->h_net.p, L->d_net.p, (size_t)n * C * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FGLT_ERR_CUDA;
  vo = 0;
  for (Request* r : pack) {
    if (r->out_raw) std::memcpy(r->out_raw, L->h_raw.p + vo * C, (size_t)r->n * C * 8);
    if (r->out_net) std::memcpy(r->out_net, L->h_net.p + vo * C, (size_t)r->n * C * 8);
    vo += r->n;
  }
  return FGLT_OK;
}

void lane_loop(Server* S, Lane* L) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<Request*> pack;
    size_t pack_est = 0;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      for (;;) {
        if (S->stop && S->queue.empty()) return;
        if (!S->queue.empty()) {
          // Admit in arrival order while the pack fits this lane's share of
          // the budget. A request that does not fit (memory, or a pack already
          // near its size limit) may be overtaken by later ones within the
          // first ADMIT_LOOKAHEAD of the queue, until it has been passed
          // MAX_PASSED times; then nothing passes it.
          int64_t pack_nnz = 0;
          size_t i = 0;
          while (i < S->queue.size() && i < (size_t)ADMIT_LOOKAHEAD && (int)pack.size() < S->max_batch) {
            Request* r = S->queue[i];
            const bool fits = pack_est + r->est <= S->lane_cap && S->reserved + r->est <= S->budget &&
                              (pack.empty() || pack_nnz + r->nnz <= PACK_MAX_ENTRIES);
            if (!fits) {
              if (r->passed >= MAX_PASSED) break;
              ++i;
              continue;
            }
            for (size_t k = 0; k < i; ++k) ++S->queue[k]->passed;
            pack_nnz += r->nnz;
            S->queue.erase(S->queue.begin() + (std::ptrdiff_t)i);
            r->state = RUNNING;
            pack.push_back(r);
            pack_est += r->est;
            S->reserved += r->est;
          }
          if (!pack.empty()) break;
        }
        S->cv_work.wait(lock);
      }
    }
    fglt_status s = run_pack(L, pack);
    std::vector<fglt_status> each(pack.size(), s);
    if (s != FGLT_OK && pack.size() > 1) {
      for (size_t i = 0; i < pack.size(); ++i) each[i] = run_pack(L, std::vector<Request*>{pack[i]});
    }
    const auto now = clk::now();
    {
      std::lock_guard<std::mutex> lock(S->mu);
      for (size_t i = 0; i < pack.size(); ++i) {
        Request* r = pack[i];
        r->status = each[i];
        r->state = each[i] == FGLT_OK ? DONE : FAILED;
        r->latency_us = std::chrono::duration<double, std::micro>(now - r->t_submit).count();
        r->rowptr.clear();
        r->rowptr.shrink_to_fit();
        r->colidx.clear();
        r->colidx.shrink_to_fit();
      }
      S->reserved -= pack_est;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

constexpr int NUM_LANES = 3;

fglt_status start(fglt_t owner, Server** out) {
  const fglt_options* o = options_of(owner);
  Server* S = new (std::nothrow) Server();
  if (!S) return FGLT_ERR_OOM;
  S->owner = owner;
  S->device = device_of(owner);
  if (cudaSetDevice(S->device) != cudaSuccess) {
    delete S;
    return FGLT_ERR_CUDA;
  }
  size_t budget = o->serve_memory_budget;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete S;
      return FGLT_ERR_CUDA;
    }
    budget = fr / 2;
  }
  S->budget = budget;
  S->lane_cap = budget / NUM_LANES;
  S->max_batch = o->serve_max_batch > 0 ? o->serve_max_batch : 256;
  S->max_queue = o->serve_max_queue > 0 ? o->serve_max_queue : 65536;
  fglt_options lo = *o;
  lo.profile_stages = 0;
  for (int i = 0; i < NUM_LANES; ++i) {
    Lane* L = new (std::nothrow) Lane();
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (!L || fglt_create(&L->h, &lo, S->device) != FGLT_OK ||
        cudaStreamCreateWithPriority(&L->hi, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&L->lo, cudaStreamNonBlocking, prio_lo) != cudaSuccess) {
      if (L && L->h) fglt_destroy(L->h);
      if (L && L->hi) cudaStreamDestroy(L->hi);
      if (L && L->lo) cudaStreamDestroy(L->lo);
      delete L;
      destroy(S);
      return FGLT_ERR_CUDA;
    }
    S->lanes.push_back(L);
  }
  for (Lane* L : S->lanes) L->th = std::thread(lane_loop, S, L);
  *out = S;
  return FGLT_OK;
}

}  // namespace

void destroy(Server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    // Requests not yet admitted are dropped; admitted ones finish.
    for (Request* r : S->queue) {
      S->all.erase(r->id);
      delete r;
    }
    S->queue.clear();
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (Lane* L : S->lanes) {
    if (L->th.joinable()) L->th.join();
    L->h_rowptr.release();
    L->h_colidx.release();
    L->h_raw.release();
    L->h_net.release();
    L->d_rowptr.release();
    L->d_colidx.release();
    L->d_raw.release();
    L->d_net.release();
    L->d_parts.release();
    L->h_parts.release();
    if (L->h) fglt_destroy(L->h);
    if (L->hi) cudaStreamDestroy(L->hi);
    if (L->lo) cudaStreamDestroy(L->lo);
    delete L;
  }
  for (auto& kv : S->all) delete kv.second;
  delete S;
}

}  // namespace serve
}  // namespace fglt

using namespace fglt::serve;

extern "C" {

fglt_status fglt_stream_submit(fglt_t h, const fglt_graph_host* g, uint64_t* id) {
  if (!h || !g || !id) return FGLT_ERR_INVALID_ARG;
  if (g->n < 0 || (g->n > 0 && !g->rowptr) || (!g->out_raw && !g->out_net && g->n > 0)) return FGLT_ERR_INVALID_ARG;
  if (g->n > 0x7ffffffeLL) return FGLT_ERR_UNSUPPORTED;
  const int64_t n = g->n;
  const int64_t nnz = n > 0 ? g->rowptr[n] : 0;
  if (n > 0 && g->rowptr[0] != 0) return FGLT_ERR_INVALID_GRAPH;
  if (nnz < 0) return FGLT_ERR_INVALID_GRAPH;
  if (nnz > 0 && !g->colidx) return FGLT_ERR_INVALID_ARG;
  Server* S = nullptr;
  {
    fglt_status s = ensure_server(h, &S, [](fglt_t owner, Server** out) { return start(owner, out); });
    if (s != FGLT_OK) return s;
  }
  const size_t est = estimate_bytes(n, nnz);
  Request* r = new (std::nothrow) Request();
  if (!r) return FGLT_ERR_OOM;
  r->n = n;
  r->nnz = nnz;
  r->out_raw = g->out_raw;
  r->out_net = g->out_net;
  r->est = est;
  try {
    r->rowptr.assign(g->rowptr, g->rowptr + n + 1);
    r->colidx.assign(g->colidx, g->colidx + nnz);
  } catch (...) {
    delete r;
    return FGLT_ERR_OOM;
  }
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (est > S->lane_cap) {
      delete r;
      return FGLT_ERR_BUSY;  // can never fit the budget
    }
    if ((int)S->queue.size() >= S->max_queue) {
      delete r;
      return FGLT_ERR_BUSY;
    }
    r->id = S->next_id++;
    r->t_submit = clk::now();
    if (n == 0) {
      r->state = DONE;
    } else {
      S->queue.push_back(r);
    }
    S->all[r->id] = r;
    *id = r->id;
  }
  S->cv_work.notify_one();
  if (n == 0) S->cv_done.notify_all();
  return FGLT_OK;
}

fglt_status fglt_stream_poll(fglt_t h, uint64_t request_id, int timeout_ms, double* latency_us) {
  if (!h) return FGLT_ERR_INVALID_ARG;
  Server* S = server_of(h);
  if (!S) return FGLT_ERR_NOT_FOUND;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->all.find(request_id);
  if (it == S->all.end()) return FGLT_ERR_NOT_FOUND;
  Request* r = it->second;
  auto finished = [&] { return r->state == DONE || r->state == FAILED; };
  if (!finished()) {
    if (timeout_ms == 0) return FGLT_ERR_PENDING;
    if (timeout_ms < 0) {
      S->cv_done.wait(lock, finished);
    } else if (!S->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), finished)) {
      return FGLT_ERR_TIMEOUT;
    }
  }
  if (latency_us) *latency_us = r->latency_us;
  const fglt_status s = r->status;
  S->all.erase(it);
  delete r;
  return s;
}

fglt_status fglt_stream_cancel(fglt_t h, uint64_t request_id) {
  if (!h) return FGLT_ERR_INVALID_ARG;
  Server* S = server_of(h);
  if (!S) return FGLT_ERR_NOT_FOUND;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->all.find(request_id);
  if (it == S->all.end()) return FGLT_ERR_NOT_FOUND;
  Request* r = it->second;
  if (r->state != QUEUED) return FGLT_ERR_BUSY;
  S->queue.erase(std::find(S->queue.begin(), S->queue.end(), r));
  S->all.erase(it);
  delete r;
  return FGLT_OK;
}

}  // extern "C"
