// Autotuner of the fill class per query length (gsw_autotune, include/gsw.h).
//
// The classes trade differently against each other with the query length: a
// 16-lane group with fewer row words per lane wastes no rows on a short query
// but spends more of each step on the wavefront's fixed costs (shuffles,
// letter loads, trackers); a taller strip amortises those over more rows; the
// CTA kernel runs a query's strips concurrently at the price of a barrier per
// 64 steps.  Which wins depends on the device, the alphabet and the target
// length, so it is measured: for every bucket of 32 query lengths, seeded
// random pairs of the bucket's longest query against targets of the given
// length are filled (score only, ~2 G cells, best of 3 runs) with each
// candidate class installed for that bucket, and the fastest is kept.  The
// classes are interchangeable: each gives the same results.
#include "gsw_impl.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

namespace gsw {
namespace {

// the plan's default rule (plan.cu pick_class16 without a table)
int default_class(int rows, bool dna) {
    if (long_pair(rows, false, dna)) return 8;
    for (int v = 0; v <= kVarMaxS16; v++)
        if (variant_rows(v) >= rows) return v;
    return kVarMaxS16;
}

struct Rng {  // 64-bit LCG (Knuth's MMIX constants), top bits
    uint64_t s;
    uint32_t next() {
        s = s * 6364136223846793005ULL + 1442695040888963407ULL;
        return (uint32_t)(s >> 33);
    }
};

struct DevBatch {
    uint8_t *q = nullptr, *t = nullptr;
    int64_t *qo = nullptr, *to = nullptr;
    int32_t *ql = nullptr, *tl = nullptr;
    gsw_result *res = nullptr;
    void free_all() {
        cudaFree(q); cudaFree(t); cudaFree(qo); cudaFree(to); cudaFree(ql); cudaFree(tl); cudaFree(res);
        *this = DevBatch();
    }
};

}  // namespace
}  // namespace gsw

extern "C" int gsw_autotune(gsw_ctx *ctx, const int8_t *matrix, int32_t alphabet, int32_t gap_open,
                            int32_t gap_extend, int32_t target_len, gsw_tune *out) {
    using namespace gsw;
    if (!ctx || !matrix || alphabet < 1 || alphabet > kMaxAlpha || target_len < 1 || target_len > (1 << 20))
        return GSW_EINVAL;
    if (cudaSetDevice(context_device(ctx)) != cudaSuccess) return GSW_ECUDA;
    gsw_tune tune;
    std::memset(tune.fill_class, -1, sizeof(tune.fill_class));
    std::memset(tune.gcups, 0, sizeof(tune.gcups));
    std::memset(tune.gcups_default, 0, sizeof(tune.gcups_default));
    const bool dna = alphabet == 4;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return GSW_ECUDA;
    int rc = GSW_OK;
    DevBatch d;
    Rng rng{0x5353575475ULL};
    for (int b = 0; b < GSW_TUNE_BUCKETS && rc == GSW_OK; b++) {
        const int rows = GSW_TUNE_ROWS * (b + 1);
        const long long cells_target = 2000000000LL;
        const int np = (int)std::max(256LL, std::min(200000LL, cells_target / ((long long)rows * target_len)));
        // seeded random letters, packed pair after pair
        std::vector<uint8_t> hq((size_t)np * rows), ht((size_t)np * target_len);
        for (auto &x : hq) x = (uint8_t)(rng.next() % (uint32_t)alphabet);
        for (auto &x : ht) x = (uint8_t)(rng.next() % (uint32_t)alphabet);
        std::vector<int64_t> hqo(np), hto(np);
        std::vector<int32_t> hql(np, rows), htl(np, target_len);
        for (int p = 0; p < np; p++) {
            hqo[p] = (int64_t)p * rows;
            hto[p] = (int64_t)p * target_len;
        }
        d.free_all();
        bool ok = cudaMalloc(&d.q, hq.size()) == cudaSuccess && cudaMalloc(&d.t, ht.size()) == cudaSuccess &&
                  cudaMalloc(&d.qo, 8 * (size_t)np) == cudaSuccess && cudaMalloc(&d.to, 8 * (size_t)np) == cudaSuccess &&
                  cudaMalloc(&d.ql, 4 * (size_t)np) == cudaSuccess && cudaMalloc(&d.tl, 4 * (size_t)np) == cudaSuccess &&
                  cudaMalloc(&d.res, sizeof(gsw_result) * (size_t)np) == cudaSuccess;
        if (!ok) {
            rc = GSW_ENOMEM;
            break;
        }
        ok = cudaMemcpy(d.q, hq.data(), hq.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(d.t, ht.data(), ht.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(d.qo, hqo.data(), 8 * (size_t)np, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(d.to, hto.data(), 8 * (size_t)np, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(d.ql, hql.data(), 4 * (size_t)np, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(d.tl, htl.data(), 4 * (size_t)np, cudaMemcpyHostToDevice) == cudaSuccess;
        if (!ok) {
            rc = GSW_ECUDA;
            break;
        }
        const int def = default_class(rows, dna);
        std::vector<int> cand;  // public codes (include/gsw.h)
        if (rows <= variant_rows(kVarMaxS16)) {
            cand = {def, std::min(def + 1, (int)kVarMaxS16), kVarMaxS16, 8};
            // 8-lane variants: the smallest holding the query in one strip, and the next
            for (int i = 0, got = 0; i <= kNumVariants - 1 - kVarP8First && got < 2; i++)
                if (variant_rows(kVarP8First + i) >= rows) {
                    cand.push_back(9 + i);
                    got++;
                }
        } else {
            cand = {4, 5, kVarMaxS16, 8, 9 + (kNumVariants - 1 - kVarP8First)};  // several strips, or the CTA kernel
            cand.push_back(def);
        }
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        const double cells = (double)np * rows * target_len;
        float best_rate = -1.f, def_rate = 0.f;
        int best = def;
        for (int c : cand) {
            gsw_tune one;
            std::memset(one.fill_class, -1, sizeof(one.fill_class));
            one.fill_class[b] = (int8_t)c;
            if ((rc = gsw_context_set_tune(ctx, &one)) != GSW_OK) break;
            float ms_best = 1e30f;
            for (int rep = 0; rep < 4 && rc == GSW_OK; rep++) {  // 1 warm-up + best of 3
                rc = gsw_align_batch(ctx, np, d.q, d.qo, d.ql, d.t, d.to, d.tl, matrix, alphabet, gap_open,
                                     gap_extend, GSW_TIMING, -1, d.res, nullptr, 0, nullptr, nullptr, st);
                if (rc != GSW_OK) break;
                if (cudaStreamSynchronize(st) != cudaSuccess) {
                    rc = GSW_ECUDA;
                    break;
                }
                gsw_stats stt;
                if (gsw_last_stats(ctx, &stt) == GSW_OK && stt.timed && rep > 0)
                    ms_best = std::min(ms_best, stt.stage_ms[1]);
            }
            if (rc != GSW_OK) break;
            const float rate = (float)(cells / (ms_best * 1e-3) / 1e9);
            if (c == def) def_rate = rate;
            if (rate > best_rate) {
                best_rate = rate;
                best = c;
            }
        }
        tune.fill_class[b] = (int8_t)best;
        tune.gcups[b] = best_rate;
        tune.gcups_default[b] = def_rate;
    }
    d.free_all();
    cudaStreamDestroy(st);
    if (rc != GSW_OK) {
        gsw_context_set_tune(ctx, nullptr);
        return rc;
    }
    rc = gsw_context_set_tune(ctx, &tune);
    if (out) *out = tune;
    return rc;
}
