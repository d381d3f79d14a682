// Serving runtime (continuous batching of host-submitted graphs).
#pragma once

#include "fglt.h"
#include "fglt_kernels.h"

namespace fglt {
namespace serve {

struct Server;

// One transform on the handle's workspace, serialised with the caller's calls.
fglt_status transform_locked(fglt_t h, const Csr& g, int64_t* raw, int64_t* net, cudaStream_t st);

void destroy(Server* s);

}  // namespace serve
}  // namespace fglt
