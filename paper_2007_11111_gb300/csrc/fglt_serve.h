// Serving runtime (continuous batching of host-submitted graphs).
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
namespace serve {

struct Server;

// One transform on the handle's workspace, serialised with the caller's calls
// (b: optional bounds, see Bounds).
fglt_status transform_locked(fglt_t h, const Csr& g, int64_t* raw, int64_t* net, cudaStream_t st,
                             const Bounds* b = nullptr);

// Accessors of the opaque handle used by the serving runtime.
cudaStream_t handle_stream(fglt_t h);
const fglt_options* options_of(fglt_t h);
int device_of(fglt_t h);
Server* server_of(fglt_t h);
// Returns the handle's server, creating it with factory on first use.
fglt_status ensure_server(fglt_t h, Server** out, fglt_status (*factory)(fglt_t, Server**));

void destroy(Server* s);

}  // namespace serve
}  // namespace fglt
