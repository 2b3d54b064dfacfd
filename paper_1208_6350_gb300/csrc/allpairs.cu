// All-vs-all alignment of a read set (gsw_align_all_pairs, include/gsw.h):
// the paper's read-overlap use (Applications: a read-overlap graph built from
// all pairwise local alignments of a read set).
//
// Pair k of the triangle is (i, j), i < j, in row-major order: row i holds
// n - 1 - i pairs and starts at k = i*n - i*(i+1)/2.  The pairs are generated
// on the device chunk by chunk (each thread finds its row by binary search
// over the row starts) and every chunk runs through the batched path against
// the caller's sequence arena; CIGAR offsets are moved to the chunk's place in
// the caller's buffer.
#include "gsw_impl.cuh"

#include <algorithm>
#include <vector>

namespace gsw {
namespace {

__host__ __device__ inline long long row_start(long long i, long long n) { return i * n - i * (i + 1) / 2; }

__global__ void k_triangle_pairs(int n, long long k0, long long count, const int64_t *off, const int32_t *len,
                                 int64_t *qo, int32_t *ql, int64_t *to, int32_t *tl) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < count;
         x += (long long)gridDim.x * blockDim.x) {
        const long long k = k0 + x;
        int lo = 0, hi = n - 2;  // largest i with row_start(i) <= k
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_start(mid, n) <= k) lo = mid;
            else hi = mid - 1;
        }
        const int i = lo;
        const int j = (int)(k - row_start(i, n)) + i + 1;
        qo[x] = off[i];
        ql[x] = len[i];
        to[x] = off[j];
        tl[x] = len[j];
    }
}

__global__ void k_shift_cigar(gsw_result *res, long long count, long long base) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < count;
         x += (long long)gridDim.x * blockDim.x)
        if (res[x].cigar_len > 0) res[x].cigar_off += base;
}

int grid_for(long long n) { return (int)std::max(1LL, std::min(8192LL, (n + 255) / 256)); }

}  // namespace
}  // namespace gsw

extern "C" int gsw_align_all_pairs(gsw_ctx *ctx, int32_t n, const uint8_t *seq, const int64_t *off,
                                   const int32_t *len, const int8_t *matrix, int32_t alphabet, int32_t gap_open,
                                   int32_t gap_extend, uint32_t flags, int32_t mask_len, int64_t chunk,
                                   gsw_result *results, uint32_t *cigar, int64_t cigar_capacity, void *stream) {
    using namespace gsw;
    if (!ctx || n < 0 || chunk < 0 || n > 65536) return set_err(GSW_EINVAL, "context, n (<= 65,536) or chunk");
    if (flags & ~(GSW_BEGIN | GSW_CIGAR | GSW_HOST_IO | GSW_PACKED2)) return set_err(GSW_EINVAL, "unknown flag bits 0x%x", flags);
    const long long total = (long long)n * (n - 1) / 2;
    if (total == 0) return GSW_OK;
    if (!seq || !off || !len || !results) return set_err(GSW_EINVAL, "NULL input or result pointer");
    if ((flags & GSW_CIGAR) && !cigar && cigar_capacity > 0) return set_err(GSW_EINVAL, "cigar is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaSetDevice(context_device(ctx)) != cudaSuccess) return set_err(GSW_ECUDA, "cudaSetDevice");
    const bool hio = (flags & GSW_HOST_IO) != 0;
    const long long C = chunk > 0 ? std::min<long long>(chunk, 1LL << 30) : (1LL << 22);
    const uint32_t f = flags & (GSW_BEGIN | GSW_CIGAR | GSW_PACKED2);
    int rc = GSW_OK;
    uint8_t *dseq = nullptr;
    int64_t *doff = nullptr, *qo = nullptr, *to = nullptr;
    int32_t *dlen = nullptr, *ql = nullptr, *tl = nullptr;
    gsw_result *dres = nullptr;
    uint32_t *dcig = nullptr;
    auto alloc = [&](void **p, size_t bytes) {
        if (rc == GSW_OK && cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) rc = GSW_ENOMEM;
    };
    const uint8_t *S = seq;
    const int64_t *OFF = off;
    const int32_t *LEN = len;
    if (hio) {
        // the sequences once on the device; the chunks' results go back to the host
        int64_t ext = 0;
        for (int r = 0; r < n; r++) {
            if (len[r] < 0 || off[r] < 0) return set_err(GSW_EINVAL, "sequence %d: negative length or offset", r);
            ext = std::max<int64_t>(ext, off[r] + len[r]);
        }
        const size_t bytes = (f & GSW_PACKED2) ? (size_t)(ext + 3) / 4 : (size_t)ext;
        alloc((void **)&dseq, bytes);
        alloc((void **)&doff, 8 * (size_t)n);
        alloc((void **)&dlen, 4 * (size_t)n);
        alloc((void **)&dres, sizeof(gsw_result) * (size_t)std::min(C, total));
        if (f & GSW_CIGAR) alloc((void **)&dcig, 4 * (size_t)std::max<int64_t>(cigar_capacity, 1));
        if (rc == GSW_OK) {
            bool ok = cudaMemcpyAsync(dseq, seq, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                      cudaMemcpyAsync(doff, off, 8 * (size_t)n, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                      cudaMemcpyAsync(dlen, len, 4 * (size_t)n, cudaMemcpyHostToDevice, st) == cudaSuccess;
            if (!ok) rc = GSW_ECUDA;
        }
        S = dseq;
        OFF = doff;
        LEN = dlen;
    }
    const long long cmax = std::min(C, total);
    alloc((void **)&qo, 8 * (size_t)cmax);
    alloc((void **)&to, 8 * (size_t)cmax);
    alloc((void **)&ql, 4 * (size_t)cmax);
    alloc((void **)&tl, 4 * (size_t)cmax);
    long long cig_used = 0;
    int rc_cigar = GSW_OK;
    for (long long k0 = 0; k0 < total && rc == GSW_OK; k0 += C) {
        const long long cnt = std::min(C, total - k0);
        k_triangle_pairs<<<grid_for(cnt), 256, 0, st>>>(n, k0, cnt, OFF, LEN, qo, ql, to, tl);
        gsw_result *R = hio ? dres : results + k0;
        uint32_t *G = (f & GSW_CIGAR) ? (hio ? dcig : cigar) + cig_used : nullptr;
        const int64_t gcap = (f & GSW_CIGAR) ? std::max<int64_t>(cigar_capacity - cig_used, 0) : 0;
        int r = gsw_align_batch(ctx, (int32_t)cnt, S, qo, ql, S, to, tl, matrix, alphabet, gap_open, gap_extend, f,
                                mask_len, R, G, gcap, nullptr, nullptr, stream);
        if (r == GSW_ECIGAR_SPACE || r == GSW_EINTERNAL) {  // records complete: carry on
            if (rc_cigar != GSW_EINTERNAL) rc_cigar = r;
            r = GSW_OK;
        }
        if (r != GSW_OK) {
            rc = r;
            break;
        }
        gsw_stats sts;
        gsw_last_stats(ctx, &sts);
        if ((f & GSW_CIGAR) && cig_used > 0) k_shift_cigar<<<grid_for(cnt), 256, 0, st>>>(R, cnt, cig_used);
        if (f & GSW_CIGAR) cig_used += std::min<long long>(sts.cigar_words, gcap);
        if (hio && cudaMemcpyAsync(results + k0, dres, sizeof(gsw_result) * (size_t)cnt, cudaMemcpyDeviceToHost,
                                   st) != cudaSuccess)
            rc = GSW_ECUDA;
    }
    if (rc == GSW_OK && hio && (f & GSW_CIGAR) && cig_used > 0 &&
        cudaMemcpyAsync(cigar, dcig, 4 * (size_t)cig_used, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = GSW_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == GSW_OK) rc = GSW_ECUDA;
    void *bufs[] = {dseq, doff, dlen, dres, dcig, qo, to, ql, tl};
    for (void *b : bufs)
        if (b) cudaFree(b);
    return rc != GSW_OK ? rc : rc_cigar;
}
