// Continuous-batching serving engine: placeholder.
#include "internal.h"
using namespace tang;
extern "C" {
int tang_serve_start(tang_ctx *ctx, const tang_serve_cfg *cfg) { return TANG_EUNSUPPORTED; }
int tang_serve_submit(tang_ctx *ctx, uint32_t rs, const tang_header *h, uint32_t n, uint32_t *ids, uint64_t *req) { return TANG_EUNSUPPORTED; }
int tang_serve_poll(tang_ctx *ctx, uint64_t req, int wait_ms, tang_req_stats *s) { return TANG_EUNSUPPORTED; }
int tang_serve_stop(tang_ctx *ctx) { return TANG_OK; }
int tang_autotune(tang_ctx *ctx, uint32_t rs, const tang_header *h, uint32_t n, uint32_t flags) { return TANG_EUNSUPPORTED; }
}
