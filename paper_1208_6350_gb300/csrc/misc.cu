// Small device helpers used by the host runtime.
#include "gsw_impl.cuh"

namespace gsw {
namespace {

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

// Checks and sizes of a batch in one pass: [0] largest query length, [1]
// largest target length, [2] query arena extent, [3] target arena extent
// (offset + length, letters), [4] nonzero if a length is outside [0, 2^24)
// or an offset is negative.
__global__ void k_batch_stats(const int64_t *q_off, const int32_t *q_len, const int64_t *t_off,
                              const int32_t *t_len, int32_t n, unsigned long long *out5) {
    unsigned long long mq = 0, mt = 0, eq = 0, et = 0, bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t ql = q_len[i], tl = t_len[i];
        const int64_t qo = q_off[i], to = t_off[i];
        bad |= ((uint32_t)ql >= (1u << 24)) | ((uint32_t)tl >= (1u << 24)) | (qo < 0) | (to < 0);
        mq = max(mq, (unsigned long long)(uint32_t)ql);
        mt = max(mt, (unsigned long long)(uint32_t)tl);
        eq = max(eq, (unsigned long long)(qo + ql));
        et = max(et, (unsigned long long)(to + tl));
    }
    mq = __reduce_max_sync(0xFFFFFFFFu, (unsigned)min(mq, 0xFFFFFFFFull));
    mt = __reduce_max_sync(0xFFFFFFFFu, (unsigned)min(mt, 0xFFFFFFFFull));
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        eq = max(eq, __shfl_xor_sync(0xFFFFFFFFu, eq, d));
        et = max(et, __shfl_xor_sync(0xFFFFFFFFu, et, d));
    }
    bad = __reduce_or_sync(0xFFFFFFFFu, (unsigned)bad);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out5[0], mq);
        atomicMax(&out5[1], mt);
        atomicMax(&out5[2], eq);
        atomicMax(&out5[3], et);
        if (bad) atomicOr(&out5[4], 1ull);
    }
}

// number of records whose flags have `flag` set
__global__ void k_count_flag(const gsw_result *res, int32_t n, int32_t flag, unsigned long long *count) {
    unsigned c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        c += (res[i].flags & flag) ? 1u : 0u;
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

__global__ void k_unpack2(const uint8_t *in, uint8_t *out, long long nletters) {
    const long long groups = (nletters + 15) / 16;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < groups;
         g += (long long)gridDim.x * blockDim.x) {
        const long long nbytes = (nletters + 3) / 4;
        uint32_t w = 0;
        for (int b = 0; b < 4; b++) {
            const long long at = g * 4 + b;
            if (at < nbytes) w |= (uint32_t)in[at] << (8 * b);
        }
        uint32_t o[4];
        for (int k = 0; k < 4; k++) {
            uint32_t v = 0;
            for (int x = 0; x < 4; x++) v |= ((w >> (2 * (4 * k + x))) & 3u) << (8 * x);
            o[k] = v;
        }
        if ((g + 1) * 16 <= nletters) {
            *reinterpret_cast<uint4 *>(out + g * 16) = make_uint4(o[0], o[1], o[2], o[3]);
        } else {
            for (long long x = g * 16; x < nletters; x++) out[x] = (uint8_t)((o[(x - g * 16) / 4] >> (8 * ((x - g * 16) % 4))) & 3u);
        }
    }
}

}  // namespace

cudaError_t launch_unpack2(const uint8_t *in, uint8_t *out, long long nletters, cudaStream_t st) {
    if (nletters > 0) {
        long long blocks = ((nletters + 15) / 16 + 255) / 256;
        k_unpack2<<<(int)(blocks > 8192 ? 8192 : blocks), 256, 0, st>>>(in, out, nletters);
    }
    return cudaGetLastError();
}

cudaError_t launch_validate(const BatchView &b, const Scoring &sc, int32_t *bad, cudaStream_t st) {
    cudaMemsetAsync(bad, 0, sizeof(int32_t), st);
    if (b.npairs > 0) {
        int blocks = (b.npairs * 32 + 255) / 256;
        blocks = blocks > 4096 ? 4096 : blocks;
        k_validate<<<blocks, 256, 0, st>>>(b, sc.A, bad);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_stats(const int64_t *q_off, const int32_t *q_len, const int64_t *t_off,
                               const int32_t *t_len, int32_t n, unsigned long long *out5, cudaStream_t st) {
    cudaMemsetAsync(out5, 0, 5 * sizeof(unsigned long long), st);
    if (n > 0) {
        int blocks = (n + 255) / 256;
        blocks = blocks > 1024 ? 1024 : blocks;
        k_batch_stats<<<blocks, 256, 0, st>>>(q_off, q_len, t_off, t_len, n, out5);
    }
    return cudaGetLastError();
}

cudaError_t launch_count_flag(const gsw_result *res, int32_t n, int32_t flag, unsigned long long *count,
                              cudaStream_t st) {
    if (n > 0) {
        int blocks = (n + 255) / 256;
        blocks = blocks > 1024 ? 1024 : blocks;
        k_count_flag<<<blocks, 256, 0, st>>>(res, n, flag, count);
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
