// Serving loop behind gsw_serve_* (include/gsw.h): continuous batching of
// alignment requests over several batch slots ("workers").  Requests of many
// cells (long reads) queue apart from the others and go to the heavy workers,
// whose persistent launches leave a few SMs free, so the light requests'
// batches start at once beside them instead of waiting behind seconds of
// long-read work.
//
// Each worker owns a context (its own scratch, a share of the memory budget),
// a stream and pinned host / device staging sized for one batch.  Submitted
// requests are copied into a FIFO.  A free worker takes as many whole requests
// from the head of the queue as fit one batch, packs them into its staging,
// copies them to the device, runs the whole hot path (gsw_align_batch on
// device buffers, its own stream) and hands every request its own records and
// CIGAR words.  With several workers, the batch being formed, the batches on
// the GPU and the results being copied back overlap, and a request that
// arrives while others are aligned joins the next batch a worker forms.
#include "gsw_impl.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t id = 0;
    int32_t npairs = 0;
    std::vector<uint8_t> q, t;
    std::vector<int64_t> qoff, toff;
    std::vector<int32_t> qlen, tlen;
    int64_t letters = 0;
    int64_t cells = 0;
    std::vector<gsw_result> res;
    std::vector<uint32_t> cigar;
    int status = GSW_OK;
    bool done = false;
    bool heavy = false;
    double t_submit = 0, t_start = 0, t_done = 0;  // server clock, seconds
};

struct Worker {
    bool heavy = false;  // takes heavy requests first (light ones when none is queued)
    gsw_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    int32_t cap_pairs = 0;
    int64_t cap_letters = 0, cap_cigar = 0;
    uint8_t *h_q = nullptr, *h_t = nullptr, *d_q = nullptr, *d_t = nullptr;
    int64_t *h_qoff = nullptr, *h_toff = nullptr, *d_qoff = nullptr, *d_toff = nullptr;
    int32_t *h_qlen = nullptr, *h_tlen = nullptr, *d_qlen = nullptr, *d_tlen = nullptr;
    gsw_result *h_res = nullptr, *d_res = nullptr;
    uint32_t *h_cig = nullptr, *d_cig = nullptr;
    bool graphs = false;  // light worker replaying captured pipelines (padded batches)
    double eager_until = 0;  // server clock: no graph replay before (set by a backlog)
    std::atomic<uint64_t> graph_batches{0};  // written by the worker, read by get_stats
    std::thread th;
};

}  // namespace

struct gsw_server {
    gsw_serve_config cfg;
    std::vector<int8_t> matrix;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue, heavy_queue;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::vector<std::unique_ptr<Worker>> workers;
    gsw_serve_stats stats;
    Clock::time_point t0 = Clock::now();
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void free_worker(Worker *w) {
    if (!w) return;
    cudaFreeHost(w->h_q); cudaFreeHost(w->h_t); cudaFreeHost(w->h_qoff); cudaFreeHost(w->h_toff);
    cudaFreeHost(w->h_qlen); cudaFreeHost(w->h_tlen); cudaFreeHost(w->h_res); cudaFreeHost(w->h_cig);
    cudaFree(w->d_q); cudaFree(w->d_t); cudaFree(w->d_qoff); cudaFree(w->d_toff);
    cudaFree(w->d_qlen); cudaFree(w->d_tlen); cudaFree(w->d_res); cudaFree(w->d_cig);
    if (w->st) cudaStreamDestroy(w->st);
    if (w->ctx) gsw_context_destroy(w->ctx);
}

int alloc_worker(Worker *w, const gsw_serve_config &c, size_t budget) {
    w->cap_pairs = c.max_batch_pairs;
    w->cap_letters = c.max_batch_letters;
    w->cap_cigar = c.max_batch_letters + 2LL * c.max_batch_pairs;  // a pair has at most m + n runs
    const size_t P = (size_t)w->cap_pairs, L = (size_t)w->cap_letters, G = (size_t)w->cap_cigar;
    bool ok = cudaMallocHost(&w->h_q, L) == cudaSuccess && cudaMallocHost(&w->h_t, L) == cudaSuccess &&
              cudaMallocHost(&w->h_qoff, P * 8) == cudaSuccess && cudaMallocHost(&w->h_toff, P * 8) == cudaSuccess &&
              cudaMallocHost(&w->h_qlen, P * 4) == cudaSuccess && cudaMallocHost(&w->h_tlen, P * 4) == cudaSuccess &&
              cudaMallocHost(&w->h_res, P * sizeof(gsw_result)) == cudaSuccess &&
              cudaMallocHost(&w->h_cig, G * 4) == cudaSuccess && cudaMalloc(&w->d_q, L) == cudaSuccess &&
              cudaMalloc(&w->d_t, L) == cudaSuccess && cudaMalloc(&w->d_qoff, P * 8) == cudaSuccess &&
              cudaMalloc(&w->d_toff, P * 8) == cudaSuccess && cudaMalloc(&w->d_qlen, P * 4) == cudaSuccess &&
              cudaMalloc(&w->d_tlen, P * 4) == cudaSuccess &&
              cudaMalloc(&w->d_res, P * sizeof(gsw_result)) == cudaSuccess && cudaMalloc(&w->d_cig, G * 4) == cudaSuccess &&
              cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) return GSW_ENOMEM;
    const size_t staging = 2 * L + P * (16 + 8 + sizeof(gsw_result)) + G * 4;
    if (budget <= staging) return GSW_ENOMEM;
    const int rc = gsw_context_create(c.device, budget - staging, &w->ctx);
    if (rc == GSW_OK && !w->heavy && c.light_graphs >= 0) {
        w->graphs = true;
        gsw::context_set_graph_buckets(w->ctx, true);
    }
    return rc;
}

// Light batches of at most this many pairs replay captured graphs: there the
// launch sequence costs as much as the work; larger batches (a queue that
// built up) launch eagerly, since each new shape would pay a capture.
constexpr int32_t kGraphMaxPairs = 1024;
// ... whose sequences are short reads: a light request may hold a few reads
// of several kb, whose rounded-up scratch would be large for a replay to pay
constexpr int32_t kGraphMaxLen = 1024;
constexpr double kGraphHoldSeconds = 1.0;

// Pair count a light batch is padded to: the next power of four from 64
// (64, 256, 1024) for batches that replay graphs, else the batch's own count.
int32_t padded_pairs(const Worker *w, int32_t np) {
    int64_t b = 64;
    while (b < np) b <<= 2;
    return (int32_t)std::min<int64_t>(b, w->cap_pairs);
}

// One batch: pack, copy in, align, copy out, scatter to the requests.
int run_batch(gsw_server *srv, Worker *w, std::vector<Req *> &batch, bool backlog) {
    int32_t np = 0;
    int64_t ql = 0, tl = 0;
    for (Req *r : batch) {
        for (int32_t p = 0; p < r->npairs; p++) {
            w->h_qoff[np] = ql + r->qoff[p];
            w->h_toff[np] = tl + r->toff[p];
            w->h_qlen[np] = r->qlen[p];
            w->h_tlen[np] = r->tlen[p];
            np++;
        }
        std::memcpy(w->h_q + ql, r->q.data(), r->q.size());
        std::memcpy(w->h_t + tl, r->t.data(), r->t.size());
        ql += (int64_t)r->q.size();
        tl += (int64_t)r->t.size();
    }
    // padding to the batch's bucket: empty pairs (records ignored)
    // a light batch replays a captured graph when the queue is keeping up
    // (nothing left behind it) and the batch is small; under a backlog the
    // batches grow and vary, and launching them eagerly costs no captures
    const int32_t nreal = np;
    int32_t maxq = 0, maxt = 0;
    for (int32_t p = 0; p < np; p++) {
        maxq = std::max(maxq, w->h_qlen[p]);
        maxt = std::max(maxt, w->h_tlen[p]);
    }
    // a backlog keeps the worker eager for a while (an overloaded queue comes
    // and goes between batches; captures there only add to the wait)
    const double tnow = srv->now();
    if (backlog) w->eager_until = tnow + kGraphHoldSeconds;
    const bool graph = w->graphs && !backlog && tnow >= w->eager_until && np <= kGraphMaxPairs &&
                       maxq <= kGraphMaxLen && maxt <= kGraphMaxLen;
    if (w->graphs) gsw::context_set_graph_buckets(w->ctx, graph);
    for (const int32_t npad = graph ? padded_pairs(w, np) : np; np < npad; np++) {
        w->h_qoff[np] = 0;
        w->h_toff[np] = 0;
        w->h_qlen[np] = 0;
        w->h_tlen[np] = 0;
    }
    cudaStream_t st = w->st;
    // on an error, copies from this worker's pinned staging may still be
    // queued: wait for them before the next batch refills it
    auto fail = [st](int rc) {
        cudaStreamSynchronize(st);
        return rc;
    };
    cudaError_t e = cudaSuccess;
    if (ql) e = cudaMemcpyAsync(w->d_q, w->h_q, ql, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && tl) e = cudaMemcpyAsync(w->d_t, w->h_t, tl, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w->d_qoff, w->h_qoff, 8 * (size_t)np, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w->d_toff, w->h_toff, 8 * (size_t)np, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w->d_qlen, w->h_qlen, 4 * (size_t)np, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w->d_tlen, w->h_tlen, 4 * (size_t)np, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(GSW_ECUDA);
    const gsw_serve_config &c = srv->cfg;
    int rc = gsw_align_batch(w->ctx, np, w->d_q, w->d_qoff, w->d_qlen, w->d_t, w->d_toff, w->d_tlen,
                             srv->matrix.data(), c.alphabet, c.gap_open, c.gap_extend, c.flags, c.mask_len,
                             w->d_res, (c.flags & GSW_CIGAR) ? w->d_cig : nullptr,
                             (c.flags & GSW_CIGAR) ? w->cap_cigar : 0, nullptr, nullptr, st);
    // GSW_EINTERNAL: every record is complete, the flagged pairs' requests
    // report it (the worker sets each request's status from its records)
    if (rc != GSW_OK && rc != GSW_EINTERNAL) return fail(rc);
    {
        gsw_stats sts;
        if (gsw_last_stats(w->ctx, &sts) == GSW_OK && sts.graph_segments > 0) w->graph_batches++;
    }
    np = nreal;
    e = cudaMemcpyAsync(w->h_res, w->d_res, sizeof(gsw_result) * (size_t)np, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(GSW_ECUDA);
    int64_t cig_words = 0;
    if (c.flags & GSW_CIGAR) {
        for (int32_t p = 0; p < np; p++)
            if (w->h_res[p].cigar_len > 0) cig_words = std::max(cig_words, w->h_res[p].cigar_off + w->h_res[p].cigar_len);
        if (cig_words) {
            e = cudaMemcpyAsync(w->h_cig, w->d_cig, 4 * (size_t)cig_words, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return fail(GSW_ECUDA);
        }
    }
    int32_t at = 0;
    for (Req *r : batch) {
        r->res.assign(w->h_res + at, w->h_res + at + r->npairs);
        r->cigar.clear();
        for (gsw_result &x : r->res) {
            if (x.cigar_len > 0) {
                const int64_t off = (int64_t)r->cigar.size();
                r->cigar.insert(r->cigar.end(), w->h_cig + x.cigar_off, w->h_cig + x.cigar_off + x.cigar_len);
                x.cigar_off = off;
            }
        }
        at += r->npairs;
    }
    return rc;
}

// Takes as many whole requests from the head of `q` as fit one batch.
void take(std::deque<Req *> &q, const Worker *w, std::vector<Req *> &batch) {
    int32_t pairs = 0;
    int64_t letters = 0;
    while (!q.empty()) {
        Req *r = q.front();
        if (!batch.empty() && (pairs + r->npairs > w->cap_pairs || letters + r->letters > w->cap_letters)) break;
        q.pop_front();
        batch.push_back(r);
        pairs += r->npairs;
        letters += r->letters;
    }
}

void worker_loop(gsw_server *srv, Worker *w) {
    cudaSetDevice(srv->cfg.device);
    for (;;) {
        std::vector<Req *> batch;
        bool backlog = false;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            // a heavy worker takes heavy requests, else light ones; a light
            // worker only light ones
            auto has_work = [&] { return !srv->queue.empty() || (w->heavy && !srv->heavy_queue.empty()); };
            srv->cv_work.wait(lk, [&] { return srv->stop || has_work(); });
            if (!has_work()) return;  // stopping and drained
            if (w->heavy && !srv->heavy_queue.empty()) take(srv->heavy_queue, w, batch);
            else take(srv->queue, w, batch);
            backlog = !srv->queue.empty();
            srv->stats.queued = (int32_t)(srv->queue.size() + srv->heavy_queue.size());
            srv->stats.running++;
            const double ts = srv->now();
            for (Req *r : batch) r->t_start = ts;
        }
        const auto t0 = Clock::now();
        const int rc = run_batch(srv, w, batch, backlog);
        const double secs = std::chrono::duration<double>(Clock::now() - t0).count();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            const double td = srv->now();
            for (Req *r : batch) {
                r->status = rc;
                if (rc == GSW_EINTERNAL) {
                    r->status = GSW_OK;
                    for (const gsw_result &x : r->res)
                        if (x.flags & GSW_RES_INTERNAL) r->status = GSW_EINTERNAL;
                }
                r->done = true;
                r->t_done = td;
                srv->stats.completed++;
                srv->stats.pairs += r->npairs;
                srv->stats.cells += r->cells;
            }
            srv->stats.batches++;
            srv->stats.busy_seconds += secs;
            srv->stats.running--;
        }
        srv->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

int gsw_serve_create(const gsw_serve_config *cfg_in, gsw_server **out) {
    if (!cfg_in || !out) return gsw::set_err(GSW_EINVAL, "NULL argument");
    *out = nullptr;
    gsw_serve_config c = *cfg_in;
    if (c.workers <= 0) c.workers = 4;
    if (c.max_batch_pairs <= 0) c.max_batch_pairs = 8192;
    if (c.max_batch_letters <= 0) c.max_batch_letters = 16 << 20;
    if (c.mem_budget_bytes == 0) c.mem_budget_bytes = (size_t)8 << 30;
    if (c.max_queue_requests <= 0) c.max_queue_requests = 1 << 20;
    if (c.heavy_workers == 0) c.heavy_workers = c.workers / 2;
    if (c.heavy_workers < 0) c.heavy_workers = 0;
    if (c.heavy_workers > c.workers) c.heavy_workers = c.workers;
    if (c.heavy_cells <= 0) c.heavy_cells = (int64_t)1 << 25;
    if (c.flags & ~(uint32_t)(GSW_BEGIN | GSW_CIGAR)) return gsw::set_err(GSW_EINVAL, "flags other than GSW_BEGIN | GSW_CIGAR");
    if (c.workers > 64) return gsw::set_err(GSW_EINVAL, "more than 64 workers");
    {
        gsw::Scoring chk;
        const int e = gsw::make_scoring(c.matrix, c.alphabet, c.gap_open, c.gap_extend, &chk);
        if (e != GSW_OK) return e;
    }
    if (cudaSetDevice(c.device) != cudaSuccess) return gsw::set_err(GSW_ECUDA, "device %d", c.device);
    std::unique_ptr<gsw_server> srv(new (std::nothrow) gsw_server());
    if (!srv) return GSW_ENOMEM;
    srv->matrix.assign(c.matrix, c.matrix + c.alphabet * c.alphabet);
    c.matrix = srv->matrix.data();
    srv->cfg = c;
    std::memset(&srv->stats, 0, sizeof(srv->stats));
    const size_t share = c.mem_budget_bytes / (size_t)c.workers;
    for (int k = 0; k < c.workers; k++) {
        std::unique_ptr<Worker> w(new Worker());
        w->heavy = k < c.heavy_workers;
        int rc = alloc_worker(w.get(), c, share);
        if (rc == GSW_OK && w->heavy && c.heavy_sm_limit >= 0) {
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device);
            rc = gsw_context_set_sm_limit(w->ctx, c.heavy_sm_limit > 0 ? c.heavy_sm_limit : std::max(1, sms * 7 / 8));
        }
        if (rc != GSW_OK) {
            free_worker(w.get());
            for (auto &x : srv->workers) free_worker(x.get());
            srv->workers.clear();
            return rc;
        }
        srv->workers.push_back(std::move(w));
    }
    for (auto &w : srv->workers) w->th = std::thread(worker_loop, srv.get(), w.get());
    *out = srv.release();
    return GSW_OK;
}

int gsw_serve_destroy(gsw_server *srv) {
    if (!srv) return GSW_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto &w : srv->workers)
        if (w->th.joinable()) w->th.join();
    cudaSetDevice(srv->cfg.device);
    for (auto &w : srv->workers) free_worker(w.get());
    delete srv;
    return GSW_OK;
}

int gsw_serve_submit(gsw_server *srv, int32_t npairs, const uint8_t *q, const int64_t *q_off, const int32_t *q_len,
                     const uint8_t *t, const int64_t *t_off, const int32_t *t_len, uint64_t *req_id) {
    if (!srv || !req_id || npairs < 1 || !q_off || !q_len || !t_off || !t_len)
        return gsw::set_err(GSW_EINVAL, "NULL argument or npairs < 1");
    if (npairs > srv->cfg.max_batch_pairs) return gsw::set_err(GSW_EINVAL, "request larger than max_batch_pairs");
    std::unique_ptr<Req> r(new (std::nothrow) Req());
    if (!r) return GSW_ENOMEM;
    r->npairs = npairs;
    int64_t qn = 0, tn = 0;
    for (int32_t p = 0; p < npairs; p++) {
        if (q_len[p] < 0 || t_len[p] < 0 || q_len[p] >= (1 << 24) || t_len[p] >= (1 << 24) || q_off[p] < 0 ||
            t_off[p] < 0)
            return gsw::set_err(GSW_EINVAL, "pair %d: length out of [0, 2^24) or negative offset", p);
        qn += q_len[p];
        tn += t_len[p];
    }
    if (qn + tn > srv->cfg.max_batch_letters || (qn && !q) || (tn && !t))
        return gsw::set_err(GSW_EINVAL, "request larger than max_batch_letters, or NULL sequences");
    r->q.resize((size_t)qn);
    r->t.resize((size_t)tn);
    r->qoff.resize(npairs);
    r->toff.resize(npairs);
    r->qlen.assign(q_len, q_len + npairs);
    r->tlen.assign(t_len, t_len + npairs);
    int64_t qa = 0, ta = 0;
    const int A = srv->cfg.alphabet;
    for (int32_t p = 0; p < npairs; p++) {
        std::memcpy(r->q.data() + qa, q + q_off[p], (size_t)q_len[p]);
        std::memcpy(r->t.data() + ta, t + t_off[p], (size_t)t_len[p]);
        r->qoff[p] = qa;
        r->toff[p] = ta;
        qa += q_len[p];
        ta += t_len[p];
        r->cells += (int64_t)q_len[p] * t_len[p];
    }
    for (uint8_t x : r->q)
        if (x >= A) return gsw::set_err(GSW_EINVAL, "a query letter code is >= the alphabet size (%d)", A);
    for (uint8_t x : r->t)
        if (x >= A) return gsw::set_err(GSW_EINVAL, "a target letter code is >= the alphabet size (%d)", A);
    r->letters = qn + tn;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if ((int32_t)(srv->queue.size() + srv->heavy_queue.size()) >= srv->cfg.max_queue_requests)
            return gsw::set_err(GSW_ENOMEM, "queue full (%d requests)", srv->cfg.max_queue_requests);
        r->id = srv->next_id++;
        r->t_submit = srv->now();
        *req_id = r->id;
        // with no heavy worker every request is light
        r->heavy = srv->cfg.heavy_workers > 0 && r->cells >= srv->cfg.heavy_cells;
        (r->heavy ? srv->heavy_queue : srv->queue).push_back(r.get());
        srv->stats.submitted++;
        srv->stats.queued = (int32_t)(srv->queue.size() + srv->heavy_queue.size());
        srv->reqs.emplace(r->id, std::move(r));
    }
    srv->cv_work.notify_all();  // the request may need a worker of its kind
    return GSW_OK;
}

int gsw_serve_poll_timed(gsw_server *srv, uint64_t req_id, int32_t timeout_us, gsw_result *results, uint32_t *cigar,
                         int64_t cigar_capacity, int64_t *cigar_words, gsw_serve_times *times) {
    if (!srv || !results) return GSW_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) return GSW_ENOTFOUND;
    Req *r = it->second.get();
    auto ready = [&] { return r->done; };
    if (timeout_us < 0) srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) return GSW_ETIMEDOUT;
    if ((int64_t)r->cigar.size() > cigar_capacity || (!r->cigar.empty() && !cigar)) {
        if (cigar_words) *cigar_words = (int64_t)r->cigar.size();
        return GSW_ECIGAR_SPACE;
    }
    const int status = r->status;
    if (times) {
        times->submitted = r->t_submit;
        times->started = r->t_start;
        times->done = r->t_done;
    }
    if (status == GSW_OK || status == GSW_EINTERNAL) {  // records complete (flagged ones included)
        std::memcpy(results, r->res.data(), sizeof(gsw_result) * (size_t)r->npairs);
        if (!r->cigar.empty()) std::memcpy(cigar, r->cigar.data(), 4 * r->cigar.size());
    }
    if (cigar_words) *cigar_words = (int64_t)r->cigar.size();
    srv->reqs.erase(it);
    return status;
}

int gsw_serve_poll(gsw_server *srv, uint64_t req_id, int32_t timeout_us, gsw_result *results, uint32_t *cigar,
                   int64_t cigar_capacity, int64_t *cigar_words) {
    return gsw_serve_poll_timed(srv, req_id, timeout_us, results, cigar, cigar_capacity, cigar_words, nullptr);
}

int gsw_serve_poll_results(gsw_server *srv, uint64_t req_id, int32_t timeout_us, gsw_results **out) {
    if (!srv || !out) return gsw::set_err(GSW_EINVAL, "NULL argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) return gsw::set_err(GSW_ENOTFOUND, "request %llu", (unsigned long long)req_id);
    Req *r = it->second.get();
    auto ready = [&] { return r->done; };
    if (timeout_us < 0) srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) return GSW_ETIMEDOUT;
    const int status = r->status;
    if (status == GSW_OK || status == GSW_EINTERNAL) {
        gsw_results *h = new (std::nothrow) gsw_results();
        if (!h) return gsw::set_err(GSW_ENOMEM, "host allocation");  // the request is kept
        h->res.swap(r->res);
        h->cigar.swap(r->cigar);
        h->t_len = r->tlen;
        *out = h;
    }
    srv->reqs.erase(it);
    return status;
}

double gsw_serve_now(gsw_server *srv) { return srv ? srv->now() : -1.0; }

int gsw_serve_get_stats(gsw_server *srv, gsw_serve_stats *out) {
    if (!srv || !out) return GSW_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    out->queued = (int32_t)(srv->queue.size() + srv->heavy_queue.size());
    out->graph_batches = 0;
    for (const auto &w : srv->workers) out->graph_batches += w->graph_batches.load();
    return GSW_OK;
}

}  // extern "C"
