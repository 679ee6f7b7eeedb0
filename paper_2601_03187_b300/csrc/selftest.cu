// Failure-path self-test of the bounded device waits. Every persistent kernel of this library
// waits on mbarriers with a limit in %globaltimer time; when a wait runs out, the waiting thread
// records an error bit in the context's device error word and raises its block's abort flag, the
// block's other waits give up on seeing the flag, and the host reports TANG_ETIMEOUT at its next
// synchronising call. This kernel exercises exactly that path with barriers nothing completes,
// so a test can check it without faulting, trapping or hanging the GPU.
#include <chrono>

#include "internal.h"
#include "tc_ptx.cuh"

namespace tang {

__global__ void __launch_bounds__(64) k_wait_selftest(int *err, uint64_t limit_ns) {
    __shared__ uint64_t bar[2];
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar[0], 1);
        ptx::mbar_init(&bar[1], 1);
        abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();
    volatile int *abort_v = &abort_flag;
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        if (warp == 0) {
            // nothing ever arrives on bar[0]: the wait runs out after limit_ns
            if (!ptx::mbar_wait(&bar[0], 0, abort_v, limit_ns)) {
                atomicOr(err, 1);
                *abort_v = 1;
            }
        } else {
            // nor on bar[1], with a 10 s limit: this wait ends on the abort flag instead
            if (!ptx::mbar_wait(&bar[1], 0, abort_v, 10000000000ull)) atomicOr(err, 2);
        }
    }
}

}  // namespace tang

using namespace tang;

extern "C" int tang_selftest_wait_timeout(tang_ctx *ctx, uint32_t limit_ms, float *elapsed_ms) {
    if (!ctx) return TANG_EINVAL;
    if (limit_ms < 1 || limit_ms > 2000) return set_err(ctx, TANG_EINVAL, "limit_ms must be in [1, 2000]");
    cudaSetDevice(ctx->device);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "selftest: stream sync failed");
    int rc = check_device_error(ctx);  // start from a clear error word
    if (rc != TANG_OK && rc != TANG_ETIMEOUT) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, ctx->stream);
    k_wait_selftest<<<1, 64, 0, ctx->stream>>>(ctx->d_err, uint64_t(limit_ms) * 1000000ull);
    cudaEventRecord(e1, ctx->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "selftest kernel failed");
    if (elapsed_ms) *elapsed_ms = ms;
    return check_device_error(ctx);
}
