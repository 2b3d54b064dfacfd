// Library-owned results (gsw_align_batch_results, gsw_results_get,
// gsw_results_free in include/gsw.h): the same pipeline as gsw_align_batch,
// with the records, CIGAR words and max arrays copied into a handle the
// library allocates, so a caller sizes no buffer of its own.
#include "gsw_impl.cuh"

#include <algorithm>
#include <cstring>
#include <memory>
#include <new>

using namespace gsw;

namespace {

// CIGAR words reserved for the whole batch: a sixteenth of each pair's
// shorter sequence plus 4 (short reads need 1-5 runs).  Pairs that need more
// are marked by the pipeline (GSW_RES_CIGAR_SPACE, cigar_len = -needed) and
// aligned once more on their own with the exact room.
int64_t first_capacity(const std::vector<int32_t> &ql, const std::vector<int32_t> &tl) {
    int64_t cap = 1024;
    for (size_t p = 0; p < ql.size(); p++) cap += std::max(0, std::min(ql[p], tl[p])) / 16 + 4;
    return cap;
}

// One run of gsw_align_batch into host buffers: with GSW_HOST_IO straight
// from the caller's host inputs, else from device inputs into device outputs
// of this call, then copied to the host.
int run_once(gsw_ctx *ctx, int32_t npairs, const uint8_t *q, const int64_t *q_off, const int32_t *q_len,
             const uint8_t *t, const int64_t *t_off, const int32_t *t_len, const int8_t *matrix, int32_t alphabet,
             int32_t O, int32_t X, uint32_t flags, int32_t mask_len, cudaStream_t st, gsw_result *res,
             uint32_t *cig, int64_t cap, int32_t *cm, const int64_t *cmoff, int64_t cm_total) {
    if (flags & GSW_HOST_IO)
        return gsw_align_batch(ctx, npairs, q, q_off, q_len, t, t_off, t_len, matrix, alphabet, O, X, flags,
                               mask_len, res, cig, cap, cm, cmoff, st);
    gsw_result *dres = nullptr;
    uint32_t *dcig = nullptr;
    int32_t *dcm = nullptr;
    int64_t *dcmo = nullptr;
    int rc = GSW_OK;
    cudaError_t e = cudaMallocAsync((void **)&dres, sizeof(gsw_result) * (size_t)std::max(npairs, 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dcig, 4 * (size_t)std::max<int64_t>(cap, 1), st);
    if (e == cudaSuccess && cm) {
        e = cudaMallocAsync((void **)&dcm, 4 * (size_t)std::max<int64_t>(cm_total, 1), st);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&dcmo, 8 * (size_t)std::max(npairs, 1), st);
        if (e == cudaSuccess && npairs > 0)
            e = cudaMemcpyAsync(dcmo, cmoff, 8 * (size_t)npairs, cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) {
        rc = set_err(GSW_ENOMEM, "result buffers: %s", cudaGetErrorString(e));
    } else {
        rc = gsw_align_batch(ctx, npairs, q, q_off, q_len, t, t_off, t_len, matrix, alphabet, O, X, flags, mask_len,
                             dres, dcig, cap, dcm, dcmo, st);
        if (rc == GSW_OK || rc == GSW_ECIGAR_SPACE || rc == GSW_EINTERNAL) {
            e = cudaMemcpyAsync(res, dres, sizeof(gsw_result) * (size_t)npairs, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && cap > 0)
                e = cudaMemcpyAsync(cig, dcig, 4 * (size_t)cap, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && cm && cm_total > 0)
                e = cudaMemcpyAsync(cm, dcm, 4 * (size_t)cm_total, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) rc = set_err(GSW_ECUDA, "result readback: %s", cudaGetErrorString(e));
        }
    }
    for (void *b : {(void *)dres, (void *)dcig, (void *)dcm, (void *)dcmo})
        if (b) cudaFreeAsync(b, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == GSW_OK) rc = set_err(GSW_ECUDA, "synchronize");
    return rc;
}

}  // namespace

extern "C" {

int gsw_align_batch_results(gsw_ctx *ctx, int32_t npairs, const uint8_t *q, const int64_t *q_off,
                            const int32_t *q_len, const uint8_t *t, const int64_t *t_off, const int32_t *t_len,
                            const int8_t *matrix, int32_t alphabet, int32_t gap_open, int32_t gap_extend,
                            uint32_t flags, int32_t mask_len, void *stream, gsw_results **out) {
    if (!out) return set_err(GSW_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctx || npairs < 0) return set_err(GSW_EINVAL, "context is NULL or npairs < 0");
    if (npairs > 0 && (!q_off || !q_len || !t_off || !t_len)) return set_err(GSW_EINVAL, "NULL offsets or lengths");
    std::unique_ptr<gsw_results> r(new (std::nothrow) gsw_results());
    if (!r) return set_err(GSW_ENOMEM, "host allocation");
    const bool hio = (flags & GSW_HOST_IO) != 0;
    cudaStream_t st = (cudaStream_t)stream;
    // host copies of the lengths (sizes) and offsets (the second pass)
    std::vector<int32_t> ql((size_t)npairs), tl((size_t)npairs);
    std::vector<int64_t> qo((size_t)npairs), to((size_t)npairs);
    if (npairs > 0) {
        if (hio) {
            std::copy(q_len, q_len + npairs, ql.begin());
            std::copy(t_len, t_len + npairs, tl.begin());
            std::copy(q_off, q_off + npairs, qo.begin());
            std::copy(t_off, t_off + npairs, to.begin());
        } else if (cudaSetDevice(context_device(ctx)) != cudaSuccess ||
                   cudaMemcpyAsync(ql.data(), q_len, 4 * (size_t)npairs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                   cudaMemcpyAsync(tl.data(), t_len, 4 * (size_t)npairs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                   cudaMemcpyAsync(qo.data(), q_off, 8 * (size_t)npairs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                   cudaMemcpyAsync(to.data(), t_off, 8 * (size_t)npairs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                   cudaStreamSynchronize(st) != cudaSuccess) {
            return set_err(GSW_ECUDA, "length and offset readback");
        }
    }
    r->res.resize((size_t)npairs);
    r->t_len = tl;
    int64_t cm_total = 0;
    if (flags & GSW_COLMAX) {
        r->colmax_off.resize((size_t)npairs);
        for (int32_t p = 0; p < npairs; p++) {
            r->colmax_off[p] = cm_total;
            cm_total += std::max(tl[p], 0);
        }
        r->colmax.assign((size_t)std::max<int64_t>(cm_total, 1), 0);
    }
    const bool cig = (flags & GSW_CIGAR) != 0;
    const int64_t cap = cig ? first_capacity(ql, tl) : 0;
    r->cigar.assign((size_t)std::max<int64_t>(cap, 1), 0u);
    int rc = run_once(ctx, npairs, q, q_off, q_len, t, t_off, t_len, matrix, alphabet, gap_open, gap_extend, flags,
                      mask_len, st, r->res.data(), r->cigar.data(), cap,
                      (flags & GSW_COLMAX) ? r->colmax.data() : nullptr, r->colmax_off.data(), cm_total);
    bool internal = rc == GSW_EINTERNAL;
    if (rc != GSW_OK && rc != GSW_ECIGAR_SPACE && rc != GSW_EINTERNAL) return rc;
    // keep the words the placed records index
    int64_t used = 0;
    for (const gsw_result &x : r->res)
        if (x.cigar_len > 0) used = std::max<int64_t>(used, x.cigar_off + x.cigar_len);
    r->cigar.resize((size_t)used);
    if (cig) {
        // second pass: the pairs whose CIGAR did not fit, on their own, with
        // exactly the room they reported (their other fields are already set)
        std::vector<int32_t> idx;
        int64_t need = 0;
        for (int32_t p = 0; p < npairs; p++)
            if (r->res[p].flags & GSW_RES_CIGAR_SPACE) {
                idx.push_back(p);
                need += -(int64_t)r->res[p].cigar_len;
            }
        if (!idx.empty()) {
            const int32_t n2 = (int32_t)idx.size();
            std::vector<int64_t> qo2(n2), to2(n2);
            std::vector<int32_t> ql2(n2), tl2(n2);
            for (int32_t k = 0; k < n2; k++) {
                qo2[k] = qo[idx[k]];
                to2[k] = to[idx[k]];
                ql2[k] = ql[idx[k]];
                tl2[k] = tl[idx[k]];
            }
            std::vector<gsw_result> res2(n2);
            std::vector<uint32_t> cig2((size_t)std::max<int64_t>(need, 1));
            const uint32_t f2 = flags & ~(uint32_t)GSW_COLMAX;
            int rc2;
            if (hio) {
                rc2 = run_once(ctx, n2, q, qo2.data(), ql2.data(), t, to2.data(), tl2.data(), matrix, alphabet,
                               gap_open, gap_extend, f2, mask_len, st, res2.data(), cig2.data(), need, nullptr,
                               nullptr, 0);
            } else {
                // the subset's offsets and lengths on the device
                int64_t *d64 = nullptr;
                int32_t *d32 = nullptr;
                cudaError_t e = cudaMallocAsync((void **)&d64, 16 * (size_t)n2, st);
                if (e == cudaSuccess) e = cudaMallocAsync((void **)&d32, 8 * (size_t)n2, st);
                if (e == cudaSuccess) e = cudaMemcpyAsync(d64, qo2.data(), 8 * (size_t)n2, cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(d64 + n2, to2.data(), 8 * (size_t)n2, cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess) e = cudaMemcpyAsync(d32, ql2.data(), 4 * (size_t)n2, cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(d32 + n2, tl2.data(), 4 * (size_t)n2, cudaMemcpyHostToDevice, st);
                rc2 = e != cudaSuccess ? set_err(GSW_ENOMEM, "second-pass inputs: %s", cudaGetErrorString(e))
                                       : run_once(ctx, n2, q, d64, d32, t, d64 + n2, d32 + n2, matrix, alphabet,
                                                  gap_open, gap_extend, f2, mask_len, st, res2.data(), cig2.data(),
                                                  need, nullptr, nullptr, 0);
                for (void *b : {(void *)d64, (void *)d32})
                    if (b) cudaFreeAsync(b, st);
                cudaStreamSynchronize(st);
            }
            if (rc2 == GSW_EINTERNAL) internal = true;
            else if (rc2 != GSW_OK) return rc2;  // GSW_ECIGAR_SPACE cannot repeat with the exact room
            const int64_t base = (int64_t)r->cigar.size();
            int64_t used2 = 0;
            for (const gsw_result &x : res2)
                if (x.cigar_len > 0) used2 = std::max<int64_t>(used2, x.cigar_off + x.cigar_len);
            r->cigar.insert(r->cigar.end(), cig2.begin(), cig2.begin() + used2);
            for (int32_t k = 0; k < n2; k++) {
                gsw_result &x = r->res[idx[k]];
                const gsw_result &y = res2[k];
                x.cigar_len = y.cigar_len;
                x.cigar_off = y.cigar_len > 0 ? base + y.cigar_off : -1;
                x.flags = (x.flags & ~(int32_t)GSW_RES_CIGAR_SPACE) | (y.flags & (int32_t)GSW_RES_INTERNAL);
            }
        }
    }
    *out = r.release();
    return internal ? set_err(GSW_EINTERNAL, "pairs failed a consistency check (GSW_RES_INTERNAL)") : GSW_OK;
}

int32_t gsw_results_count(const gsw_results *r) { return r ? (int32_t)r->res.size() : 0; }

int gsw_results_get(const gsw_results *r, int32_t i, gsw_record *rec) {
    if (!r || !rec) return set_err(GSW_EINVAL, "NULL argument");
    if (i < 0 || (size_t)i >= r->res.size()) return set_err(GSW_EINVAL, "record %d of %zu", i, r->res.size());
    const gsw_result &x = r->res[(size_t)i];
    std::memset(rec, 0, sizeof(*rec));
    rec->score1 = x.score1;
    rec->score2 = x.score2;
    rec->ref_begin1 = x.ref_begin1;
    rec->ref_end1 = x.ref_end1;
    rec->read_begin1 = x.read_begin1;
    rec->read_end1 = x.read_end1;
    rec->ref_end2 = x.ref_end2;
    rec->lane_bits_used = (x.flags & GSW_RES_S32) ? 32 : 16;
    rec->flags = x.flags;
    if (x.cigar_len > 0 && x.cigar_off >= 0 && (size_t)(x.cigar_off + x.cigar_len) <= r->cigar.size()) {
        rec->cigar = r->cigar.data() + x.cigar_off;
        rec->cigar_len = x.cigar_len;
    }
    rec->n = r->t_len.empty() ? 0 : r->t_len[(size_t)i];
    rec->colmax = r->colmax_off.empty() ? nullptr : r->colmax.data() + r->colmax_off[(size_t)i];
    return GSW_OK;
}

void gsw_results_free(gsw_results *r) { delete r; }

}  // extern "C"
