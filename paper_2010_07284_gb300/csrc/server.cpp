// Serving loop (continuous batching) -- see vl.h.
#include "runtime.h"

using namespace vl;

namespace vl {
void server_destroy(vl_server*) {}
}  // namespace vl

extern "C" {
VL_API vl_status vl_server_create(vl_context*, const vl_server_config*, vl_server**) { return VL_ERR_ARG; }
VL_API vl_status vl_server_submit(vl_server*, const vl_formula*, vl_image* const*, int32_t, int64_t*) { return VL_ERR_ARG; }
VL_API vl_status vl_server_wait(vl_server*, int64_t, int64_t, vl_result**) { return VL_ERR_ARG; }
VL_API vl_status vl_server_cancel(vl_server*, int64_t) { return VL_ERR_ARG; }
VL_API vl_status vl_server_stats_get(vl_server*, vl_server_stats*) { return VL_ERR_ARG; }
}
