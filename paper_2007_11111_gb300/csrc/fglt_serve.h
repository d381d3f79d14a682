// Serving runtime (continuous batching of host-submitted graphs).
#pragma once

#include "fglt.h"
#include "fglt_kernels.h"
#include "fglt_pipeline.h"

namespace fglt {
namespace serve {

struct Server;

// One transform on the handle's workspace, serialised with the caller's calls
// (b: optional bounds, see Bounds).
fglt_status transform_locked(fglt_t h, const Csr& g, int64_t* raw, int64_t* net, cudaStream_t st,
                             const Bounds* b = nullptr);

// Accessors of the opaque handle used by the serving runtime.
cudaStream_t handle_stream(fglt_t h);
int columns_of(fglt_t h);  // output columns per vertex
const fglt_options* options_of(fglt_t h);
int device_of(fglt_t h);
Server* server_of(fglt_t h);
// Returns the handle's server, creating it with factory on first use.
fglt_status ensure_server(fglt_t h, Server** out, fglt_status (*factory)(fglt_t, Server**));

void destroy(Server* s);

}  // namespace serve
}  // namespace fglt
