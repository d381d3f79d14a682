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
// Limits (larger inputs return FGLT_ERR_UNSUPPORTED): n <=
// FGLT_NOALLOC_MAX_VERTICES and rowptr[n] <= FGLT_NOALLOC_MAX_ENTRIES, checked
// before any device work; every buffer of the stage sequence must fit in the
// array, checked as the sequence carves them (a largest out-degree in the
// degree order above about 1000 needs a global-memory bitmap that does not).
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
#include "fglt_pipeline.h"

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

// Bump allocator over the scratch array (256-byte aligned pieces); a piece
// that does not fit makes the transform return FGLT_ERR_UNSUPPORTED.
struct CarverWs final : Workspace {
  unsigned char* base;
  size_t off = 0;
  explicit CarverWs(unsigned char* b) : base(b) {}
  fglt_status get(BufId, size_t bytes, void** out) override {
    const size_t need = (bytes + 255) & ~(size_t)255;
    if (need > SCRATCH_BYTES - off) return FGLT_ERR_UNSUPPORTED;
    *out = base + off;
    off += need;
    return FGLT_OK;
  }
  // Scalars are read into the caller's (pageable) host memory.
  fglt_status read(void* host, const void* dev, size_t bytes, cudaStream_t st) override {
    if (cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return FGLT_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FGLT_ERR_CUDA;
    return FGLT_OK;
  }
};

#define CK(call)                                     \
  do {                                               \
    if ((call) != cudaSuccess) return FGLT_ERR_CUDA; \
  } while (0)

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
  if (rowptr_is_64bit) CK(cudaStreamSynchronize(st));
  if (nnz < 0) return FGLT_ERR_INVALID_GRAPH;
  if (nnz > FGLT_NOALLOC_MAX_ENTRIES) return FGLT_ERR_UNSUPPORTED;
  if (nnz > 0 && !colidx) return FGLT_ERR_INVALID_ARG;
  Csr g{rowptr, rowptr_is_64bit != 0, colidx, n, nnz};
  CarverWs ws(scratch);
  RunOptions ro;  // default tuning, no validation, no profiling
  const fglt_status s = run_pipeline(ws, g, out_raw, out_net, st, ro);
  // An error can leave work of this call queued on st (a buffer that did not
  // fit stops the sequence midway); wait for it, so that no later call, on
  // any stream, meets it still writing the shared array.
  if (s != FGLT_OK) cudaStreamSynchronize(st);
  return s;
}
