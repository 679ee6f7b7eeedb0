// FP32 CUDA-core kernels: the §6.2 feature encoder, a tiled SGEMM with a fused epilogue (the
// plain one-kernel-per-stage network path and the trainer's forward/backward), argmax,
// column sums, softmax cross-entropy and Adam.
#include <algorithm>

#include "internal.h"

namespace tang {

// §6.2: SIP hi/lo, DIP hi/lo, SP, DP, PRO as floats (exact), times `scale`; column 7 = 0.
__global__ void k_encode(const tang_header *__restrict__ h, uint32_t n, float *__restrict__ X, uint32_t ldx,
                         float scale) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint4 v = __ldg(reinterpret_cast<const uint4 *>(h + i));
        float f[8] = {float(v.x >> 16), float(v.x & 0xFFFFu), float(v.y >> 16), float(v.y & 0xFFFFu),
                      float(v.z & 0xFFFFu), float(v.z >> 16), float(v.w & 0xFFu), 0.f};
        float *row = X + size_t(i) * ldx;
        if (ldx == 8) {
            reinterpret_cast<float4 *>(row)[0] = make_float4(f[0] * scale, f[1] * scale, f[2] * scale, f[3] * scale);
            reinterpret_cast<float4 *>(row)[1] = make_float4(f[4] * scale, f[5] * scale, f[6] * scale, 0.f);
        } else {
            for (uint32_t j = 0; j < 7 && j < ldx; ++j) row[j] = f[j] * scale;
        }
    }
}

cudaError_t launch_encode(const tang_header *h, uint32_t n, float *X, uint32_t ldx, float scale, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    uint32_t blocks = std::min<uint32_t>((n + 255) / 256, 148 * 16);
    k_encode<<<blocks, 256, 0, st>>>(h, n, X, ldx, scale);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// SGEMM: C[M,N] = epi( op(A)[M,K] . op(B)[K,N] )
//   op(A)(m,k) = TA ? A[k*lda + m] : A[m*lda + k]
//   op(B)(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n]
//   epi(v) = v + bias[n] + resid[m,n] + beta*C[m,n]; ReLU if relu; 0 where mask[m,n] <= 0
// 128x128 block tile, K step 8, 256 threads, 8x8 outputs per thread (two 4x4 quadrants at a
// 64-element offset so shared-memory reads are conflict-free float4s), register-staged double
// buffering of the shared tiles.
// ---------------------------------------------------------------------------------------
struct Epi {
    const float *bias;
    const float *resid;
    int ldr;
    const float *mask;
    int ldm;
    int relu;
    float beta;
};

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float *__restrict__ A, int lda,
                                               const float *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                                               Epi epi) {
    __shared__ __align__(16) float As[2][8][128];
    __shared__ __align__(16) float Bs[2][8][128];
    const int tid = threadIdx.x;
    const int bm = blockIdx.y * 128, bn = blockIdx.x * 128;
    const int tx = tid & 15, ty = tid >> 4;

    // global -> register staging: 4 elements of A and 4 of B per thread per K step
    float ra[4], rb[4];
    auto load_a = [&](int k0) {
        if (!TA) {  // A row-major: thread loads row m = tid/2, k = k0 + (tid&1)*4 .. +3
            const int m = bm + (tid >> 1), k = k0 + (tid & 1) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) ra[q] = (m < M && k + q < K) ? __ldg(A + size_t(m) * lda + k + q) : 0.f;
        } else {  // A stored k-major: k = k0 + tid/32, m = bm + (tid&31)*4 .. +3
            const int k = k0 + (tid >> 5), m = bm + (tid & 31) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) ra[q] = (k < K && m + q < M) ? __ldg(A + size_t(k) * lda + m + q) : 0.f;
        }
    };
    auto load_b = [&](int k0) {
        if (!TB) {  // B row-major (k, n): k = k0 + tid/32, n = bn + (tid&31)*4 .. +3
            const int k = k0 + (tid >> 5), n = bn + (tid & 31) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) rb[q] = (k < K && n + q < N) ? __ldg(B + size_t(k) * ldb + n + q) : 0.f;
        } else {  // B stored (n, k): n = bn + tid/2, k = k0 + (tid&1)*4 .. +3
            const int n = bn + (tid >> 1), k = k0 + (tid & 1) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) rb[q] = (n < N && k + q < K) ? __ldg(B + size_t(n) * ldb + k + q) : 0.f;
        }
    };
    auto store_ab = [&](int buf) {
        if (!TA) {
            const int m = tid >> 1, k = (tid & 1) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) As[buf][k + q][m] = ra[q];
        } else {
            const int k = tid >> 5, m = (tid & 31) * 4;
            *reinterpret_cast<float4 *>(&As[buf][k][m]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
        }
        if (!TB) {
            const int k = tid >> 5, n = (tid & 31) * 4;
            *reinterpret_cast<float4 *>(&Bs[buf][k][n]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
        } else {
            const int n = tid >> 1, k = (tid & 1) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) Bs[buf][k + q][n] = rb[q];
        }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    load_a(0);
    load_b(0);
    store_ab(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += 8) {
        const bool more = k0 + 8 < K;
        if (more) {
            load_a(k0 + 8);
            load_b(k0 + 8);
        }
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            float a[8], b[8];
            float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
            float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
            float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
            float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            store_ab(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }

#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = bm + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = bn + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (n >= N) continue;
            float v = acc[i][j];
            if (epi.bias) v += __ldg(epi.bias + n);
            if (epi.resid) v += epi.resid[size_t(m) * epi.ldr + n];
            if (epi.beta != 0.f) v += epi.beta * C[size_t(m) * ldc + n];
            if (epi.relu) v = fmaxf(v, 0.f);
            if (epi.mask && !(epi.mask[size_t(m) * epi.ldm + n] > 0.f)) v = 0.f;
            C[size_t(m) * ldc + n] = v;
        }
    }
}

cudaError_t launch_sgemm(int ta, int tb, int M, int N, int K, const float *A, int lda, const float *B, int ldb,
                         float *C, int ldc, const float *bias, const float *resid, int ldr, const float *mask, int ldm,
                         int relu, float beta, cudaStream_t st) {
    if (M == 0 || N == 0) return cudaSuccess;
    dim3 grid((N + 127) / 128, (M + 127) / 128);
    Epi e{bias, resid, ldr, mask, ldm, relu, beta};
    if (!ta && !tb)
        k_sgemm<false, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, e);
    else if (!ta && tb)
        k_sgemm<false, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, e);
    else if (ta && !tb)
        k_sgemm<true, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, e);
    else
        k_sgemm<true, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, e);
    return cudaGetLastError();
}

// Argmax over each row of logits; the lowest index wins ties (like the float64 reference).
__global__ void k_argmax(const float *__restrict__ Z, int ldz, int n, int C, int32_t *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float *z = Z + size_t(i) * ldz;
        float best = z[0];
        int arg = 0;
        for (int c = 1; c < C; ++c) {
            float v = z[c];
            if (v > best) {
                best = v;
                arg = c;
            }
        }
        out[i] = arg;
    }
}

cudaError_t launch_argmax(const float *Z, int ldz, int n, int C, int32_t *out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int blocks = std::min((n + 255) / 256, 148 * 16);
    k_argmax<<<blocks, 256, 0, st>>>(Z, ldz, n, C, out);
    return cudaGetLastError();
}

// Plain FP32 network forward, one kernel per layer, in chunks that fit the scratch buffer.
int mlp_fp32_forward(tang_ctx *ctx, const DeviceModel &m, const tang_header *h, uint32_t n, float *logits,
                     int32_t *tuple, cudaStream_t st) {
    const uint32_t N = m.N, C = m.C;
    const uint32_t ldz = C;
    uint32_t chunk = std::min<uint32_t>(n, 262144);
    chunk = (chunk + 127) / 128 * 128;
    size_t need = size_t(chunk) * (8 + 2 * N + ldz) * sizeof(float);
    int rc = ensure_scratch(ctx, need);
    if (rc) return rc;
    float *X = reinterpret_cast<float *>(ctx->scratch);
    float *H = X + size_t(chunk) * 8;
    float *U = H + size_t(chunk) * N;
    float *Z = U + size_t(chunk) * N;
    for (uint32_t c0 = 0; c0 < n; c0 += chunk) {
        const int rows = int(std::min(chunk, n - c0));
        cudaError_t e = launch_encode(h + c0, rows, X, 8, 1.0f, st);
        if (e == cudaSuccess) e = launch_sgemm(0, 0, rows, N, m.S, X, 8, m.W0, N, H, N, m.b0, nullptr, 0, nullptr, 0, 1, 0.f, st);
        for (uint32_t b = 0; b < m.blocks && e == cudaSuccess; ++b) {
            e = launch_sgemm(0, 0, rows, N, N, H, N, m.W1[b], N, U, N, m.b1[b], nullptr, 0, nullptr, 0, 1, 0.f, st);
            if (e == cudaSuccess)
                e = launch_sgemm(0, 0, rows, N, N, U, N, m.W2[b], N, H, N, m.b2[b], H, N, nullptr, 0, 1, 0.f, st);
        }
        float *zout = logits ? logits + size_t(c0) * C : Z;
        if (e == cudaSuccess) e = launch_sgemm(0, 0, rows, C, N, H, N, m.Wc, C, zout, C, m.bc, nullptr, 0, nullptr, 0, 0, 0.f, st);
        if (e == cudaSuccess && tuple) e = launch_argmax(zout, C, rows, C, tuple + c0, st);
        if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "fp32 forward: %s", cudaGetErrorString(e));
    }
    return TANG_OK;
}

// ---------------------------------------------------------------------------------------
// Trainer helpers
// ---------------------------------------------------------------------------------------

// Partial column sums: block (bx, by) sums 32 columns over rows [by*rows_per, ...).
__global__ void k_colsum_partial(const float *__restrict__ G, int M, int N, int ldg, int rows_per,
                                 float *__restrict__ part) {
    __shared__ float red[8][33];
    const int n = blockIdx.x * 32 + (threadIdx.x & 31);
    const int r0 = blockIdx.y * rows_per;
    const int r1 = min(M, r0 + rows_per);
    float s = 0.f;
    if (n < N)
        for (int m = r0 + (threadIdx.x >> 5); m < r1; m += 8) s += G[size_t(m) * ldg + n];
    red[threadIdx.x >> 5][threadIdx.x & 31] = s;
    __syncthreads();
    if (threadIdx.x < 32 && n < N) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
        part[size_t(blockIdx.y) * N + n] = t;
    }
}

__global__ void k_colsum_final(const float *__restrict__ part, int parts, int N, float *__restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int p = 0; p < parts; ++p) s += part[size_t(p) * N + n];
    out[n] = s;
}

// out[n] = sum_m G[m, n]; `part` needs 64 * N floats.
cudaError_t launch_colsum(const float *G, int M, int N, int ldg, float *out, float *part, cudaStream_t st) {
    const int parts = 64;
    const int rows_per = (M + parts - 1) / parts;
    dim3 grid((N + 31) / 32, parts);
    k_colsum_partial<<<grid, 256, 0, st>>>(G, M, N, ldg, rows_per, part);
    k_colsum_final<<<(N + 255) / 256, 256, 0, st>>>(part, parts, N, out);
    return cudaGetLastError();
}

// Softmax cross-entropy of a batch: dz = (softmax(z) - onehot(y)) / B, per-row loss and
// correctness (argmax == y, lowest index on ties).
__global__ void k_softmax_ce(const float *__restrict__ Z, int ldz, int B, int C, const int32_t *__restrict__ y,
                             float *__restrict__ dz, float *__restrict__ row_loss, int32_t *__restrict__ row_ok) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
        const float *z = Z + size_t(i) * ldz;
        float mx = z[0];
        int arg = 0;
        for (int c = 1; c < C; ++c)
            if (z[c] > mx) {
                mx = z[c];
                arg = c;
            }
        float s = 0.f;
        for (int c = 0; c < C; ++c) s += expf(z[c] - mx);
        const float lse = mx + logf(s);
        const int yi = y[i];
        row_loss[i] = lse - z[yi];
        row_ok[i] = arg == yi;
        float *d = dz + size_t(i) * ldz;
        const float inv = 1.0f / float(B);
        for (int c = 0; c < C; ++c) d[c] = (expf(z[c] - lse) - (c == yi ? 1.f : 0.f)) * inv;
    }
}

cudaError_t launch_softmax_ce(const float *Z, int ldz, int B, int C, const int32_t *y, float *dz, float *row_loss,
                              int32_t *row_ok, cudaStream_t st) {
    int blocks = std::min((B + 255) / 256, 1184);
    k_softmax_ce<<<blocks, 256, 0, st>>>(Z, ldz, B, C, y, dz, row_loss, row_ok);
    return cudaGetLastError();
}

// Adam (Kingma & Ba) with bias correction; c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, size_t count, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += size_t(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, size_t count, int t, float lr, float b1,
                        float b2, float eps, cudaStream_t st) {
    const float c1 = float(1.0 - pow(double(b1), double(t)));
    const float c2 = float(1.0 - pow(double(b2), double(t)));
    size_t blocks = std::min<size_t>((count + 255) / 256, 148 * 8);
    if (blocks == 0) blocks = 1;
    k_adam<<<unsigned(blocks), 256, 0, st>>>(p, g, m, v, count, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

// Row-wise max |x| over a matrix (for FP8 activation calibration): out = max(out, max|x|).
__global__ void k_absmax(const float *__restrict__ X, size_t count, unsigned int *__restrict__ out_bits) {
    float mx = 0.f;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += size_t(gridDim.x) * blockDim.x)
        mx = fmaxf(mx, fabsf(X[i]));
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(mx));  // non-negative floats order as uints
}

cudaError_t launch_absmax(const float *X, size_t count, unsigned int *out_bits, cudaStream_t st) {
    size_t blocks = std::min<size_t>((count + 255) / 256, 148 * 8);
    if (blocks == 0) return cudaSuccess;
    k_absmax<<<unsigned(blocks), 256, 0, st>>>(X, count, out_bits);
    return cudaGetLastError();
}

}  // namespace tang
