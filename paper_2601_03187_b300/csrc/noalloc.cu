// Staged classification that allocates nothing at call time.
//
// The staged path runs the tensor-core network kernel, which writes one predicted tuple per
// packet, and then the search kernel, which reads it. tang_classify keeps those predictions in
// the context's scratch buffer and grows it with cudaMalloc when a batch needs more. Some
// callers cannot let a call allocate: code running inside a custom allocator or an allocation
// hook, a process whose device memory is fixed up front, or a latency-bound loop that cannot
// accept cudaMalloc's implicit device synchronisation. tang_classify_noalloc serves them by
// passing the predictions through the file-scope device array below instead.
#include "internal.h"

namespace tang {

// One int32 predicted tuple per packet of the largest allowed batch (4 MiB). It is part of this
// library's device module: a GPU holds it from the moment the module is loaded on it (at the
// latest when a context is created there, see noalloc_prepare) until the process exits. All
// calls and contexts on a device share it.
static __device__ __align__(256) int32_t g_noalloc_tuples[TANG_NOALLOC_MAX_PACKETS];

// Called by tang_create with the context's device current: looks up the array's device address
// once per context, so that the entry point itself never loads a module or allocates. In host
// code the symbol's name is only a host-side stand-in, never a device address.
int noalloc_prepare(tang_ctx *ctx) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_tuples);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return set_err(ctx, TANG_EDEVICE, "cudaGetSymbolAddress(no-alloc scratch): %s", cudaGetErrorString(e));
    }
    ctx->noalloc_tuples = static_cast<int32_t *>(p);
    return TANG_OK;
}

}  // namespace tang

using namespace tang;

extern "C" int tang_classify_noalloc(tang_ctx *ctx, uint32_t rsh, const tang_header *d_headers, uint32_t n,
                                     uint32_t *d_ids, void *stream) {
    if (!ctx) return TANG_EINVAL;
    auto it = ctx->rulesets.find(rsh);
    if (it == ctx->rulesets.end()) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    Ruleset &rs = *it->second;
    if (n > TANG_NOALLOC_MAX_PACKETS)
        return set_err(ctx, TANG_EINVAL, "tang_classify_noalloc: n = %u exceeds the static scratch of %u packets", n,
                       TANG_NOALLOC_MAX_PACKETS);
    if (n == 0) return TANG_OK;
    if (!d_headers || !d_ids || (reinterpret_cast<uintptr_t>(d_headers) & 15) || (reinterpret_cast<uintptr_t>(d_ids) & 3))
        return set_err(ctx, TANG_EINVAL, "headers must be 16-byte aligned device memory and ids 4-byte aligned");
    if (!rs.model) return set_err(ctx, TANG_EINVAL, "ruleset %u has no model", rsh);
    if (!rs.model->d_wbf16)
        return set_err(ctx, TANG_EUNSUPPORTED, "tensor-core path needs N == 256 or 512 and 1 <= blocks <= 31");
    if (!ctx->noalloc_tuples) return set_err(ctx, TANG_EDEVICE, "no-alloc scratch address unknown");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "cudaSetDevice failed");
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    if (rs.has_update && cudaStreamWaitEvent(st, rs.last_update, 0) != cudaSuccess)
        return set_err(ctx, TANG_EDEVICE, "cudaStreamWaitEvent failed");
    // every entry below n is written by the network kernel before the search kernel reads it,
    // so the array needs no clearing between calls
    int rc = tc_launch(ctx, rs, d_headers, n, nullptr, nullptr, ctx->noalloc_tuples, TANG_BF16, false, nullptr, st,
                       nullptr, 0);
    if (rc) return rc;
    cudaError_t e = launch_search(rs.d_desc, uint32_t(rs.host.tuples.size()), rs.host.cw, d_headers,
                                  ctx->noalloc_tuples, n, d_ids, nullptr, nullptr, st);
    if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "search: %s", cudaGetErrorString(e));
    note_classify(rs, st);
    return checked_sync(ctx, st);
}
