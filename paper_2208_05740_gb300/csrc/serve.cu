// Serving loop (continuous batching of verification requests).
#include "gcp_ctx.h"

namespace gcp {
void serve_shutdown(Ctx&) {}
}  // namespace gcp

extern "C" {
gcp_status gcp_serve_start(gcp_ctx*, int32_t) { return GCP_EINVAL; }
gcp_status gcp_serve_submit(gcp_ctx*, const gcp_request*, uint64_t*) { return GCP_EINVAL; }
gcp_status gcp_serve_poll(gcp_ctx*, uint64_t, gcp_result*) { return GCP_EINVAL; }
gcp_status gcp_serve_wait(gcp_ctx*, uint64_t, int32_t, gcp_result*) { return GCP_EINVAL; }
gcp_status gcp_serve_stop(gcp_ctx*) { return GCP_EINVAL; }
}
