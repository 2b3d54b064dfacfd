// Small device helpers used by the host runtime.
#include "gsw_impl.cuh"

namespace gsw {
namespace {

__global__ void k_max_lengths(const int32_t *q_len, const int32_t *t_len, int32_t n, int32_t *out2) {
    int mq = 0, mt = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        mq = max(mq, q_len[i]);
        mt = max(mt, t_len[i]);
    }
    mq = __reduce_max_sync(0xFFFFFFFFu, mq);
    mt = __reduce_max_sync(0xFFFFFFFFu, mt);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out2[0], mq);
        atomicMax(&out2[1], mt);
    }
}

__global__ void k_fill_const(int32_t *dst, int32_t v, int32_t n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = v;
}
__global__ void k_fill_const64(int64_t *dst, int64_t v, int32_t n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = v;
}

// one warp per pair: every letter code of both sequences must be < A
__global__ void k_validate(BatchView b, int32_t A, int32_t *bad) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int found = 0;
    for (int p = w; p < b.npairs; p += nw) {
        const uint8_t *q = b.q + b.q_off[p];
        const uint8_t *t = b.t + b.t_off[p];
        const int m = b.q_len[p], n = b.t_len[p];
        for (int i = lane; i < m; i += 32) found |= q[i] >= A;
        for (int j = lane; j < n; j += 32) found |= t[j] >= A;
    }
    if (__any_sync(0xFFFFFFFFu, found) && lane == 0) atomicOr(bad, 1);
}

}  // namespace

cudaError_t launch_validate(const BatchView &b, const Scoring &sc, int32_t *bad, cudaStream_t st) {
    cudaMemsetAsync(bad, 0, sizeof(int32_t), st);
    if (b.npairs > 0) {
        int blocks = (b.npairs * 32 + 255) / 256;
        blocks = blocks > 4096 ? 4096 : blocks;
        k_validate<<<blocks, 256, 0, st>>>(b, sc.A, bad);
    }
    return cudaGetLastError();
}

cudaError_t launch_max_lengths(const int32_t *q_len, const int32_t *t_len, int32_t n, int32_t *out2,
                               cudaStream_t st) {
    cudaMemsetAsync(out2, 0, 2 * sizeof(int32_t), st);
    if (n > 0) {
        int blocks = (n + 255) / 256;
        blocks = blocks > 1024 ? 1024 : blocks;
        k_max_lengths<<<blocks, 256, 0, st>>>(q_len, t_len, n, out2);
    }
    return cudaGetLastError();
}

cudaError_t launch_fill_const(int32_t *dst, int32_t v, int32_t n, cudaStream_t st) {
    if (n > 0) k_fill_const<<<(n + 255) / 256 > 1024 ? 1024 : (n + 255) / 256, 256, 0, st>>>(dst, v, n);
    return cudaGetLastError();
}
cudaError_t launch_fill_const64(int64_t *dst, int64_t v, int32_t n, cudaStream_t st) {
    if (n > 0) k_fill_const64<<<(n + 255) / 256 > 1024 ? 1024 : (n + 255) / 256, 256, 0, st>>>(dst, v, n);
    return cudaGetLastError();
}

}  // namespace gsw
