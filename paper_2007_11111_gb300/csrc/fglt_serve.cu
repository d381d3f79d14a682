// Serving entry points.
#include "fglt_serve.h"

namespace fglt {
namespace serve {

struct Server {};

void destroy(Server* s) { delete s; }

}  // namespace serve
}  // namespace fglt

extern "C" {

fglt_status fglt_stream_submit(fglt_t h, const fglt_graph_host* g, uint64_t* id) {
  if (!h || !g || !id) return FGLT_ERR_INVALID_ARG;
  return FGLT_ERR_UNSUPPORTED;
}

fglt_status fglt_stream_poll(fglt_t h, uint64_t, int, double*) {
  if (!h) return FGLT_ERR_INVALID_ARG;
  return FGLT_ERR_NOT_FOUND;
}

fglt_status fglt_stream_cancel(fglt_t h, uint64_t) {
  if (!h) return FGLT_ERR_INVALID_ARG;
  return FGLT_ERR_NOT_FOUND;
}

}  // extern "C"
