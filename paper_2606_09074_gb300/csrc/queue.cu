// Request queue (refine_queue_*): a serving loop that admits pruning
// requests by HBM footprint and scores the requests admitted together with
// one batched launch, while earlier rounds are still on the GPU.
//
// Threads and streams:
//   dispatcher   admits (FIFO, budget, slots) and issues each admitted
//                request at once: a pool allocation and the host->device
//                copies on the queue's one input-copy stream, then the
//                preparation on the request's slot stream.
//   scorer       continuous batching: as soon as the previous batched launch
//                has ended, takes every request whose preparation has ended
//                and scores them with ONE k_score_batch launch on the score
//                stream (its round); per request on its slot stream again the
//                selection and the compaction, the copies back on the queue's
//                one output-copy stream (asynchronous when the host buffers
//                are page-locked) and a completion event.
// The copies of all requests go through one stream per direction, in
// admission order: each request's copy then ends as early as the link
// allows and its kernels overlap the next request's copy.  (Copies issued
// on the slot streams shared the link and ended together, so the kernels
// of a whole group of requests waited for all of their copies.)
//   completion   polls the completion events of the requests in flight,
//                finishes copies into pageable buffers, reads the request's
//                status and threshold, frees its block and its slot.
// Device status words are per request: the batched launch reports an error
// on the status word of the request whose scene it concerns, so an error is
// reported on the request that caused it, and no request reads a word that
// belongs to its round (the round ring is reused while earlier requests may
// still be finishing).
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "api_internal.h"

using namespace refine;
using namespace refine_api;

namespace {

constexpr int kQueueMaxSlots = 64;

// Rows of the device copy start on 16-byte boundaries.
inline int64_t dev_stride(int64_t n) { return (n + 7) & ~int64_t(7); }

inline int64_t keep_count(int64_t n, double ratio) { return n - (int64_t)floor(ratio * (double)n); }

struct SlotHost {  // page-locked read-back of one slot
    unsigned int kstar;
    int status;
    int pad[2];
};

struct QJob {
    uint64_t ticket = 0;
    refine_request req{};
    refine_params params{};
    int64_t n_keep = 0;
    uint64_t footprint = 0;
    bool compact = false, pinned_out = false;
    double t_submit = 0, t_admit = 0;
    int slot = -1;
    int round_size = 0;
    void *block = nullptr;
    refine_scene scene{};
    refine_camera *cams = nullptr;
    float *scores = nullptr;
    uint32_t *mask = nullptr;
    float *out_pos = nullptr;
    void *out_attr = nullptr;
    int32_t *idx = nullptr;
    int *status = nullptr;
    ScenePlan plan;
    SceneScratch sx{};
    void *sel_scr = nullptr, *cmp_scr = nullptr;
    unsigned int *kstar = nullptr;
    long long *total = nullptr;
    refine_status host_status = REFINE_OK;
    bool issued = false;  // GPU work enqueued (its completion event is recorded)
    bool copied = false, prepped = false, finishing = false;  // timeline events recorded for this request
};

struct RoundRes {  // one entry of the round ring
    ScoreLaunch *h_launch = nullptr;  // page-locked [slots]
    long long *h_tb = nullptr;        // page-locked [slots + 1]
    ScoreLaunch *d_launch = nullptr;
    long long *d_tb = nullptr;
    unsigned long long *d_counter = nullptr;
    int *d_status = nullptr;
    cudaEvent_t scored = nullptr;
};

double now_ms(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

bool is_pinned(const void *p)
{
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// Bytes of the 56 attribute rows per primitive (per element of the stride).
size_t elem_size(int dtype) { return attr_col_bytes(dtype); }

}  // namespace

struct refine_queue {
    refine_ctx pc;  // private context of the dispatcher (error text, device, SM count)
    refine_ctx sc;  // private context of the scorer (error text)
    refine_params params{};
    ScoreShape shape;  // the creating context's tuned shape
    uint64_t budget = 0;
    int slots = 0;
    std::chrono::steady_clock::time_point t0;
    cudaMemPool_t pool = nullptr;
    cudaStream_t score_stream = nullptr;
    cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;  // all copies, FIFO per direction
    std::vector<cudaStream_t> slot_stream;
    std::vector<cudaEvent_t> prepped, done;
    std::vector<cudaEvent_t> copied, computed, read_back;  // per slot: copy in done, kernels done, copy out done
    std::vector<cudaEvent_t> scored_at;                     // per slot: the round's batched score done
    cudaEvent_t ev_ref = nullptr;                           // device-time origin of the per-request timeline
    SlotHost *slot_host = nullptr;  // page-locked [slots]
    std::vector<RoundRes> ring;
    void *ring_dev = nullptr;
    void *ring_host = nullptr;
    int64_t round_seq = 0;

    std::mutex mu;
    std::condition_variable cv_dispatch, cv_score, cv_complete, cv_poll;
    std::deque<QJob *> pending;
    std::deque<QJob *> prepping;  // admitted and issued, waiting for a batched score launch
    std::list<QJob *> inflight;
    std::unordered_map<uint64_t, refine_result> results;
    std::unordered_set<uint64_t> live;  // submitted, not yet returned by refine_queue_poll
    std::vector<int> free_slots;
    uint64_t used = 0, peak = 0;
    uint64_t next_ticket = 1;
    bool stop = false, dispatcher_done = false, scorer_done = false;
    int64_t n_submitted = 0, n_admitted = 0, n_completed = 0, n_rounds = 0;
    int max_round = 0;
    double dispatch_ms = 0.0, retire_ms = 0.0;  // host time issuing rounds / retiring requests
    std::atomic<int64_t> launches{0};
    char err_copy[1024] = {0};
    char cerr[256] = {0};  // last failure seen by the completion thread
    std::thread dispatcher, scorer, completer;
};

namespace {

// V input cameras; pl the request's plan (views scored, camera block).
uint64_t footprint_of(int64_t n, int dtype, int V, const ScenePlan &pl, double ratio, bool compact)
{
    const size_t S = (size_t)dev_stride(n), es = elem_size(dtype);
    const int64_t nk = keep_count(n, ratio);
    const size_t parts = carve_size({3 * S * 4, S * es, sizeof(refine_camera) * (size_t)V, 4 * (size_t)n,
                                     4 * (size_t)((n + 31) / 32), compact ? 3 * (size_t)nk * 4 : 0,
                                     compact ? (size_t)nk * es : 0, compact ? 4 * (size_t)nk : 0, 256});
    return parts + scene_bytes(pl) + select_bytes(n) + compact_bytes(n) + 3 * 256;
}

// Carves the request's block (the order of footprint_of).
void carve_job(QJob *j)
{
    const int64_t n = j->req.n, S = dev_stride(n), nk = j->n_keep;
    const size_t es = elem_size(j->req.dtype);
    Carver cv(j->block);
    float *pos = cv.take<float>(3 * (size_t)S);
    char *attr = cv.take<char>((size_t)S * es);
    j->cams = cv.take<refine_camera>(j->req.n_views);
    j->scores = cv.take<float>(n);
    j->mask = cv.take<uint32_t>((n + 31) / 32);
    if (j->compact) {
        j->out_pos = cv.take<float>(3 * (size_t)nk);
        j->out_attr = cv.take<char>((size_t)nk * es);
        j->idx = cv.take<int32_t>(nk);
    } else {
        cv.take<char>(0);
        cv.take<char>(0);
        cv.take<char>(0);
    }
    j->status = cv.take<int>(64);
    j->scene.n = n;
    j->scene.dtype = j->req.dtype;
    j->scene.reserved = 0;
    j->scene.pos = pos;
    j->scene.attr = attr;
    j->scene.row_stride = S;
    j->sx = carve_scene(cv, j->plan);
    j->sel_scr = cv.take<char>(select_bytes(n));
    j->cmp_scr = cv.take<char>(compact_bytes(n));
}

template <typename F>
refine_status counted_run(refine_queue *q, refine_ctx *c, int cls, F &&f)
{
    const cudaError_t e = f();
    if (e != cudaSuccess) return cuda_fail(c, e, kClassName[cls]);
    q->launches.fetch_add(1, std::memory_order_relaxed);
    return REFINE_OK;
}

// Issues the preparation of one admitted request on its slot stream.
refine_status issue_prep(refine_queue *q, QJob *j)
{
    cudaStream_t s = q->slot_stream[j->slot], cs = q->h2d_stream;
    refine_ctx *c = &q->pc;
    cudaError_t e = cudaMallocFromPoolAsync(&j->block, j->footprint, q->pool, cs);
    if (e != cudaSuccess) {
        j->block = nullptr;
        return cuda_fail(c, e, "queue: device block");
    }
    carve_job(j);
    const int64_t n = j->req.n, S = dev_stride(n);
    e = cudaMemcpy2DAsync(const_cast<float *>(j->scene.pos), (size_t)S * 4, j->req.pos_host, (size_t)n * 4,
                          (size_t)n * 4, 3, cudaMemcpyHostToDevice, cs);
    // the attribute rows block by block (float32 rows, then bfloat16 rows),
    // from host rows of n elements to device rows of S
    const int nf = attr_f32_rows(j->req.dtype);
    char *dst = static_cast<char *>(const_cast<void *>(j->scene.attr));
    const char *src = static_cast<const char *>(j->req.attr_host);
    if (e == cudaSuccess && nf > 0)
        e = cudaMemcpy2DAsync(dst, (size_t)S * 4, src, (size_t)n * 4, (size_t)n * 4, nf, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && nf < 56)
        e = cudaMemcpy2DAsync(dst + (size_t)nf * 4 * S, (size_t)S * 2, src + (size_t)nf * 4 * n, (size_t)n * 2,
                              (size_t)n * 2, 56 - nf, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(j->cams, j->req.cams_host, sizeof(refine_camera) * j->req.n_views,
                            cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(q->copied[j->slot], cs);
    j->copied = e == cudaSuccess;
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, q->copied[j->slot], 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(j->status, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "queue: input copy");
    auto run = [q, c](int cls, auto &&f) { return counted_run(q, c, cls, f); };
    refine_status st = enqueue_prep(c, run, &j->scene, j->cams, j->plan, j->sx, j->params, false, j->status, s);
    if (st) return st;
    e = cudaEventRecord(q->prepped[j->slot], s);
    j->prepped = e == cudaSuccess;
    return e == cudaSuccess ? REFINE_OK : cuda_fail(c, e, "queue: event");
}

// Selection, compaction and read-back of one scored request.
refine_status issue_finish(refine_queue *q, QJob *j, const RoundRes &R)
{
    cudaStream_t s = q->slot_stream[j->slot];
    refine_ctx *c = &q->sc;
    cudaError_t e = cudaStreamWaitEvent(s, R.scored, 0);
    if (e == cudaSuccess) e = cudaEventRecord(q->scored_at[j->slot], s);
    if (e != cudaSuccess) return cuda_fail(c, e, "queue: wait");
    auto run = [q, c](int cls, auto &&f) { return counted_run(q, c, cls, f); };
    const int64_t n = j->req.n, nk = j->n_keep;
    refine_status st = enqueue_select(c, run, j->scores, n, nk, j->mask, j->sel_scr, &j->kstar, j->status, s);
    if (!st && j->compact)
        st = enqueue_compact(c, run, &j->scene, j->mask, j->out_pos, j->out_attr, nk, j->idx, j->cmp_scr, &j->total,
                             j->status, s);
    if (st) return st;
    // the copies back go through the output-copy stream, after the kernels
    e = cudaEventRecord(q->computed[j->slot], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q->d2h_stream, q->computed[j->slot], 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "queue: event");
    const cudaStream_t cs = q->d2h_stream;
    SlotHost *h = &q->slot_host[j->slot];
    h->kstar = 0u;
    if (j->kstar) e = cudaMemcpyAsync(&h->kstar, j->kstar, sizeof(unsigned), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h->status, j->status, sizeof(int), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess && j->pinned_out) {
        const size_t es = elem_size(j->req.dtype);
        if (j->req.keep_mask_host)
            e = cudaMemcpyAsync(j->req.keep_mask_host, j->mask, 4 * (size_t)((n + 31) / 32), cudaMemcpyDeviceToHost,
                                cs);
        if (e == cudaSuccess && j->req.scores_host)
            e = cudaMemcpyAsync(j->req.scores_host, j->scores, 4 * (size_t)n, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && j->compact) {
            e = cudaMemcpyAsync(j->req.out_pos_host, j->out_pos, 12 * (size_t)nk, cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(j->req.out_attr_host, j->out_attr, es * (size_t)nk, cudaMemcpyDeviceToHost,
                                    cs);
            if (e == cudaSuccess && j->req.kept_idx_host)
                e = cudaMemcpyAsync(j->req.kept_idx_host, j->idx, 4 * (size_t)nk, cudaMemcpyDeviceToHost, cs);
        }
    }
    // the slot stream (its completion event, its block's release) follows the copies back
    if (e == cudaSuccess) e = cudaEventRecord(q->read_back[j->slot], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, q->read_back[j->slot], 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "queue: read-back");
    j->finishing = true;
    return REFINE_OK;
}

// Scores `round` (requests whose preparation has ended, or whose issue
// failed) with one batched launch and issues their selection, compaction
// and copies back.  Returns the launch's completion event (NULL if nothing
// was launched).  Runs on the scorer thread.
cudaEvent_t issue_scoring(refine_queue *q, std::vector<QJob *> &round)
{
    const double t_issue = now_ms(q->t0);
    RoundRes &R = q->ring[(size_t)(q->round_seq++ % q->ring.size())];
    std::vector<QJob *> live;
    for (QJob *j : round) {
        j->round_size = (int)round.size();
        if (!j->host_status) live.push_back(j);
    }
    refine_status st = REFINE_OK;
    if (!live.empty()) {
        int max_v = 0;
        std::vector<int64_t> ns;
        for (size_t i = 0; i < live.size(); ++i) {
            QJob *j = live[i];
            R.h_launch[i] = make_score_launch(&j->scene, j->plan, j->sx, j->params, 0, j->scores, nullptr, false,
                                              j->status);
            max_v = std::max(max_v, R.h_launch[i].vcount);
            ns.push_back(j->req.n);
        }
        const int full_grid = score_batch_grid(q->pc.num_sms, max_v, q->shape);
        const int rounds = batch_rounds(q->shape, ns.data(), (int)ns.size(), full_grid);
        const long long tile = batch_tile(q->shape, rounds);
        R.h_tb[0] = 0;
        for (size_t i = 0; i < live.size(); ++i) R.h_tb[i + 1] = R.h_tb[i] + (ns[i] + tile - 1) / tile;
        const int k = (int)live.size();
        cudaStream_t m = q->score_stream;
        cudaError_t e = cudaMemcpyAsync(R.d_launch, R.h_launch, sizeof(ScoreLaunch) * k, cudaMemcpyHostToDevice, m);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(R.d_tb, R.h_tb, sizeof(long long) * (k + 1), cudaMemcpyHostToDevice, m);
        if (e == cudaSuccess) e = cudaMemsetAsync(R.d_counter, 0, sizeof(unsigned long long), m);
        if (e == cudaSuccess) e = cudaMemsetAsync(R.d_status, 0, sizeof(int), m);
        for (QJob *j : live)
            if (e == cudaSuccess) e = cudaStreamWaitEvent(m, q->prepped[j->slot], 0);
        if (e == cudaSuccess) {
            BatchLaunch bl;
            bl.scenes = R.d_launch;
            bl.tile_begin = R.d_tb;
            bl.n_scenes = k;
            bl.total_tiles = R.h_tb[k];
            bl.counter = R.d_counter;
            bl.status = R.d_status;
            bl.rounds = rounds;
            int grid = full_grid;
            if (grid > bl.total_tiles) grid = (int)bl.total_tiles;
            e = launch_score_batch(bl, max_v, grid, q->shape, m);
            if (e == cudaSuccess) q->launches.fetch_add(1, std::memory_order_relaxed);
        }
        // Further camera blocks of requests with more views than one block:
        // per-request launches of the plain score kernel, in block order,
        // after the batched launch (which scored every first block).
        for (QJob *j : live) {
            for (int v0 = j->plan.vpp; v0 < j->plan.V && e == cudaSuccess; v0 += j->plan.vpp) {
                ScoreLaunch a = make_score_launch(&j->scene, j->plan, j->sx, j->params, v0, j->scores, nullptr, false,
                                                  j->status);
                a.grid = score_grid(q->pc.num_sms, j->plan.n, a.vcount, q->shape);
                a.tiles_taken = j->sx.tiles;
                e = cudaMemsetAsync(j->sx.tiles, 0, sizeof(unsigned long long), m);
                if (e == cudaSuccess) e = launch_score(a, q->shape, m);
                if (e == cudaSuccess) q->launches.fetch_add(1, std::memory_order_relaxed);
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(R.scored, m);
        if (e != cudaSuccess) st = cuda_fail(&q->sc, e, "queue: batched score");
    }
    for (QJob *j : round) {
        if (!j->host_status) j->host_status = st ? st : issue_finish(q, j, R);
        // the completion event closes the slot stream's work in every case
        if (cudaEventRecord(q->done[j->slot], q->slot_stream[j->slot]) == cudaSuccess) j->issued = true;
        else cudaGetLastError();
    }
    {
        std::lock_guard<std::mutex> lk(q->mu);
        for (QJob *j : round) q->inflight.push_back(j);
        q->n_rounds++;
        q->max_round = std::max(q->max_round, (int)round.size());
        q->dispatch_ms += now_ms(q->t0) - t_issue;
    }
    q->cv_complete.notify_one();
    return (!live.empty() && !st) ? R.scored : nullptr;
}

bool admissible(const refine_queue *q, const QJob *j)
{
    return !q->free_slots.empty() && q->used + j->footprint <= q->budget;
}

void dispatcher_main(refine_queue *q)
{
    cudaSetDevice(q->pc.device);
    for (;;) {
        std::vector<QJob *> admitted;
        {
            std::unique_lock<std::mutex> lk(q->mu);
            q->cv_dispatch.wait(lk, [q] { return q->stop || (!q->pending.empty() && admissible(q, q->pending.front())); });
            if (q->stop) break;
            const double t = now_ms(q->t0);
            while (!q->pending.empty() && admissible(q, q->pending.front())) {
                QJob *j = q->pending.front();
                q->pending.pop_front();
                j->slot = q->free_slots.back();
                q->free_slots.pop_back();
                j->t_admit = t;
                q->used += j->footprint;
                q->n_admitted++;
                admitted.push_back(j);
            }
            q->peak = std::max(q->peak, q->used);
        }
        // copies and preparation of each request, at once, in admission order
        for (QJob *j : admitted) {
            const double t_issue = now_ms(q->t0);
            j->host_status = issue_prep(q, j);
            std::lock_guard<std::mutex> lk(q->mu);
            q->prepping.push_back(j);
            q->dispatch_ms += now_ms(q->t0) - t_issue;
            q->cv_score.notify_one();
        }
    }
    std::lock_guard<std::mutex> lk(q->mu);
    q->dispatcher_done = true;
    q->cv_score.notify_one();
}

// Continuous batching: each batched launch scores every request whose
// preparation has ended by the time the previous launch has ended.
void scorer_main(refine_queue *q)
{
    cudaSetDevice(q->pc.device);
    cudaEvent_t last = nullptr;  // the previous batched launch's completion
    for (;;) {
        QJob *head = nullptr;
        {
            std::unique_lock<std::mutex> lk(q->mu);
            q->cv_score.wait(lk, [q] { return !q->prepping.empty() || q->dispatcher_done; });
            if (q->prepping.empty()) break;  // the dispatcher has stopped and nothing is left
            head = q->prepping.front();
        }
        // outside the lock: the oldest waiting request's preparation, then the
        // previous launch (the requests prepared meanwhile join this one)
        if (head->prepped && !head->host_status) cudaEventSynchronize(q->prepped[head->slot]);
        if (last) cudaEventSynchronize(last);
        cudaGetLastError();
        std::vector<QJob *> ready;
        {
            std::lock_guard<std::mutex> lk(q->mu);
            for (auto it = q->prepping.begin(); it != q->prepping.end();) {
                QJob *j = *it;
                const bool done = j->host_status || !j->prepped ||
                                  cudaEventQuery(q->prepped[j->slot]) != cudaErrorNotReady;
                if (done) {
                    ready.push_back(j);
                    it = q->prepping.erase(it);
                } else {
                    ++it;
                }
            }
            cudaGetLastError();
        }
        if (!ready.empty()) last = issue_scoring(q, ready);
    }
    std::lock_guard<std::mutex> lk(q->mu);
    q->scorer_done = true;
    q->cv_complete.notify_one();
}

// Copies into pageable host buffers (synchronous), then frees the block.
refine_status finish_pageable(refine_queue *q, QJob *j)
{
    cudaStream_t s = q->slot_stream[j->slot];
    const int64_t n = j->req.n, nk = j->n_keep;
    const size_t es = elem_size(j->req.dtype);
    cudaError_t e = cudaSuccess;
    if (j->req.keep_mask_host)
        e = cudaMemcpyAsync(j->req.keep_mask_host, j->mask, 4 * (size_t)((n + 31) / 32), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && j->req.scores_host)
        e = cudaMemcpyAsync(j->req.scores_host, j->scores, 4 * (size_t)n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && j->compact) {
        e = cudaMemcpyAsync(j->req.out_pos_host, j->out_pos, 12 * (size_t)nk, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(j->req.out_attr_host, j->out_attr, es * (size_t)nk, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && j->req.kept_idx_host)
            e = cudaMemcpyAsync(j->req.kept_idx_host, j->idx, 4 * (size_t)nk, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(q->mu);
        snprintf(q->cerr, sizeof q->cerr, "queue: request %llu: copy back: %s", (unsigned long long)j->ticket,
                 cudaGetErrorString(e));
        return REFINE_ECUDA;
    }
    return REFINE_OK;
}

void retire(refine_queue *q, QJob *j)
{
    const double t_retire = now_ms(q->t0);
    refine_status st = j->host_status;
    const SlotHost &h = q->slot_host[j->slot];
    if (!st && j->issued) {
        if (h.status) st = (refine_status)h.status;
        if (!st && !j->pinned_out) st = finish_pageable(q, j);
    }
    refine_result r{};
    r.status = st;
    r.round_size = j->round_size;
    r.n_keep = j->n_keep;
    r.threshold = (!st && j->kstar) ? key_to_score(h.kstar) : -INFINITY;
    r.submit_ms = j->t_submit;
    r.admit_ms = j->t_admit;
    // device timeline: the slot's events still belong to this request
    double *tl[5] = {&r.copied_ms, &r.prepped_ms, &r.scored_ms, &r.computed_ms, &r.read_ms};
    cudaEvent_t ev[5] = {q->copied[j->slot], q->prepped[j->slot], q->scored_at[j->slot], q->computed[j->slot],
                         q->read_back[j->slot]};
    const bool reached[5] = {j->copied, j->prepped, j->finishing, j->finishing, j->finishing};
    for (int k = 0; k < 5; ++k) {
        float ms = -1.f;
        if (!(j->issued && reached[k] && !st && cudaEventElapsedTime(&ms, q->ev_ref, ev[k]) == cudaSuccess)) ms = -1.f;
        cudaGetLastError();
        *tl[k] = ms;
    }
    if (j->block) {
        cudaFreeAsync(j->block, q->slot_stream[j->slot]);
        cudaGetLastError();
    }
    r.done_ms = now_ms(q->t0);
    {
        std::lock_guard<std::mutex> lk(q->mu);
        q->used -= j->footprint;
        q->free_slots.push_back(j->slot);
        q->n_completed++;
        q->results[j->ticket] = r;
        q->retire_ms += now_ms(q->t0) - t_retire;
    }
    delete j;
    q->cv_dispatch.notify_one();
    q->cv_poll.notify_all();
}

void completer_main(refine_queue *q)
{
    cudaSetDevice(q->pc.device);
    for (;;) {
        std::vector<QJob *> ready;
        {
            std::unique_lock<std::mutex> lk(q->mu);
            q->cv_complete.wait(lk, [q] { return !q->inflight.empty() || q->scorer_done; });
            if (q->inflight.empty() && q->scorer_done) break;
            for (auto it = q->inflight.begin(); it != q->inflight.end();) {
                QJob *j = *it;
                bool fin = !j->issued;
                if (!fin) {
                    const cudaError_t e = cudaEventQuery(q->done[j->slot]);
                    fin = e != cudaErrorNotReady;
                    if (e != cudaSuccess && e != cudaErrorNotReady) {
                        cudaGetLastError();
                        snprintf(q->cerr, sizeof q->cerr, "queue: request %llu: %s", (unsigned long long)j->ticket,
                                 cudaGetErrorString(e));
                        if (!j->host_status) j->host_status = REFINE_ECUDA;
                    }
                }
                if (fin) {
                    ready.push_back(j);
                    it = q->inflight.erase(it);
                } else {
                    ++it;
                }
            }
        }
        for (QJob *j : ready) retire(q, j);
        if (ready.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

void queue_free(refine_queue *q)
{
    for (cudaStream_t s : q->slot_stream)
        if (s) cudaStreamDestroy(s);
    if (q->score_stream) cudaStreamDestroy(q->score_stream);
    if (q->h2d_stream) cudaStreamDestroy(q->h2d_stream);
    if (q->d2h_stream) cudaStreamDestroy(q->d2h_stream);
    for (auto *v : {&q->prepped, &q->copied, &q->computed, &q->read_back, &q->scored_at})
        for (cudaEvent_t e : *v)
            if (e) cudaEventDestroy(e);
    if (q->ev_ref) cudaEventDestroy(q->ev_ref);
    for (cudaEvent_t e : q->done)
        if (e) cudaEventDestroy(e);
    for (RoundRes &r : q->ring)
        if (r.scored) cudaEventDestroy(r.scored);
    if (q->ring_dev) cudaFree(q->ring_dev);
    if (q->ring_host) cudaFreeHost(q->ring_host);
    if (q->slot_host) cudaFreeHost(q->slot_host);
    if (q->pool) cudaMemPoolDestroy(q->pool);
    if (q->pc.d_status) cudaFree(q->pc.d_status);
    delete q;
}

}  // namespace

extern "C" {

uint64_t refine_queue_footprint(int64_t n, int32_t dtype, int32_t n_views, double ratio, int32_t compact)
{
    if (n < 1 || n > INT32_MAX || !valid_dtype(dtype) || n_views < 1 ||
        n_views > 65535 || !(ratio >= 0.0 && ratio < 1.0))
        return 0;
    // the smallest camera block: the running sums are included whenever a
    // scene could take more than one pass
    return footprint_of(n, dtype, n_views, plan_scene(n, n_views, 0, 32), ratio, compact != 0);
}

refine_status refine_queue_create(refine_ctx *c, uint64_t hbm_budget_bytes, int32_t max_slots,
                                  const refine_params *params, refine_queue **out)
{
    if (!c || !out) return REFINE_EINVAL;
    *out = nullptr;
    refine_status st = use_device(c);
    if (st) return st;
    if (max_slots < 1 || max_slots > kQueueMaxSlots)
        return fail(c, REFINE_EINVAL, "queue: max_slots must lie in [1, %d]", kQueueMaxSlots);
    if (hbm_budget_bytes == 0) return fail(c, REFINE_EINVAL, "queue: zero HBM budget");
    refine_params p;
    if (params) p = *params; else refine_params_default(&p);
    if ((st = check_params(c, &p))) return st;
    refine_queue *q = new refine_queue();
    q->pc.device = c->device;
    q->pc.num_sms = c->num_sms;
    q->sc.device = c->device;
    q->sc.num_sms = c->num_sms;
    q->shape = c->shape;
    q->params = p;
    q->budget = hbm_budget_bytes;
    q->slots = max_slots;
    q->t0 = std::chrono::steady_clock::now();
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c->device;
    cudaError_t e = cudaMemPoolCreate(&q->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = hbm_budget_bytes;  // keep freed blocks cached up to the budget
        e = cudaMemPoolSetAttribute(q->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->score_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->h2d_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->d2h_stream, cudaStreamNonBlocking);
    q->slot_stream.assign(max_slots, nullptr);
    for (auto *v : {&q->prepped, &q->done, &q->copied, &q->computed, &q->read_back, &q->scored_at})
        v->assign(max_slots, nullptr);
    for (int s = 0; s < max_slots && e == cudaSuccess; ++s) {
        e = cudaStreamCreateWithFlags(&q->slot_stream[s], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->done[s], cudaEventDisableTiming);
        // the timeline events keep timestamps (refine_result's device times)
        for (auto *v : {&q->prepped, &q->copied, &q->computed, &q->read_back, &q->scored_at})
            if (e == cudaSuccess) e = cudaEventCreate(&(*v)[s]);
    }
    if (e == cudaSuccess) e = cudaEventCreate(&q->ev_ref);
    if (e == cudaSuccess) e = cudaEventRecord(q->ev_ref, q->h2d_stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(q->ev_ref);
    if (e == cudaSuccess) e = cudaMallocHost(&q->slot_host, sizeof(SlotHost) * max_slots);
    const size_t per_dev = carve_size({sizeof(ScoreLaunch) * (size_t)max_slots, sizeof(long long) * (max_slots + 1),
                                       sizeof(unsigned long long), sizeof(int)});
    const size_t per_host = carve_size({sizeof(ScoreLaunch) * (size_t)max_slots, sizeof(long long) * (max_slots + 1)});
    if (e == cudaSuccess) e = cudaMalloc(&q->ring_dev, per_dev * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&q->ring_host, per_host * max_slots);
    q->ring.resize(max_slots);
    for (int r = 0; r < max_slots && e == cudaSuccess; ++r) {
        RoundRes &R = q->ring[r];
        Carver dv(static_cast<char *>(q->ring_dev) + per_dev * r);
        R.d_launch = dv.take<ScoreLaunch>(max_slots);
        R.d_tb = dv.take<long long>(max_slots + 1);
        R.d_counter = dv.take<unsigned long long>(1);
        R.d_status = dv.take<int>(1);
        Carver hv(static_cast<char *>(q->ring_host) + per_host * r);
        R.h_launch = hv.take<ScoreLaunch>(max_slots);
        R.h_tb = hv.take<long long>(max_slots + 1);
        e = cudaEventCreateWithFlags(&R.scored, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        st = cuda_fail(c, e, "queue: set-up");
        queue_free(q);
        return st;
    }
    for (int s = max_slots - 1; s >= 0; --s) q->free_slots.push_back(s);
    try {
        q->dispatcher = std::thread(dispatcher_main, q);
        q->scorer = std::thread(scorer_main, q);
        q->completer = std::thread(completer_main, q);
    } catch (...) {
        // stop what started, in pipeline order (nothing has been submitted)
        {
            std::lock_guard<std::mutex> lk(q->mu);
            q->stop = true;
        }
        q->cv_dispatch.notify_all();
        if (q->dispatcher.joinable()) q->dispatcher.join();
        {
            std::lock_guard<std::mutex> lk(q->mu);
            q->dispatcher_done = true;
        }
        q->cv_score.notify_all();
        if (q->scorer.joinable()) q->scorer.join();
        {
            std::lock_guard<std::mutex> lk(q->mu);
            q->scorer_done = true;
        }
        q->cv_complete.notify_all();
        if (q->completer.joinable()) q->completer.join();
        queue_free(q);
        return fail(c, REFINE_ENOMEM, "queue: cannot start threads");
    }
    *out = q;
    return REFINE_OK;
}

refine_status refine_queue_submit(refine_queue *q, const refine_request *req, uint64_t *ticket)
{
    if (!q || !req || !ticket) return REFINE_EINVAL;
    const refine_request &r = *req;
    if (r.n < 1 || r.n > INT32_MAX || !valid_dtype(r.dtype) || r.n_views < 1 ||
        r.n_views > 65535 || !(r.ratio >= 0.0 && r.ratio < 1.0) || !r.pos_host || !r.attr_host ||
        !r.cams_host || (r.out_pos_host && !r.out_attr_host) || (!r.out_pos_host && (r.out_attr_host || r.kept_idx_host)))
        return REFINE_EINVAL;
    QJob *j = new QJob();
    j->req = r;
    j->params = r.params ? *r.params : q->params;
    if (!(j->params.eta > 0.f) || !isfinite(j->params.eta) || j->params.e_ln_gem == 0.0 || j->params.e_col == 0.0 ||
        j->params.e_opa == 0.0 || j->params.max_views < 0) {
        delete j;
        return REFINE_EINVAL;
    }
    j->req.params = nullptr;
    j->n_keep = keep_count(r.n, r.ratio);
    j->compact = r.out_pos_host != nullptr;
    j->plan = plan_scene(r.n, r.n_views, j->params.max_views, q->shape.views_per_pass);
    j->footprint = footprint_of(r.n, r.dtype, r.n_views, j->plan, r.ratio, j->compact);
    j->pinned_out = is_pinned(r.keep_mask_host) && is_pinned(r.scores_host) && is_pinned(r.out_pos_host) &&
                    is_pinned(r.out_attr_host) && is_pinned(r.kept_idx_host);
    if (j->footprint > q->budget) {
        delete j;
        return REFINE_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(q->mu);
        if (q->stop) {
            delete j;
            return REFINE_ECANCELLED;
        }
        j->ticket = q->next_ticket++;
        j->t_submit = now_ms(q->t0);
        *ticket = j->ticket;
        q->live.insert(j->ticket);
        q->pending.push_back(j);
        q->n_submitted++;
    }
    q->cv_dispatch.notify_one();
    return REFINE_OK;
}

refine_status refine_queue_poll(refine_queue *q, uint64_t ticket, refine_result *out, int32_t timeout_ms)
{
    if (!q || !out) return REFINE_EINVAL;
    std::unique_lock<std::mutex> lk(q->mu);
    if (!q->live.count(ticket)) return REFINE_ENOTFOUND;
    auto ready = [&] { return q->results.count(ticket) != 0; };
    if (!ready()) {
        if (timeout_ms == 0) return REFINE_ETIMEOUT;
        if (timeout_ms < 0)
            q->cv_poll.wait(lk, ready);
        else if (!q->cv_poll.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
            return REFINE_ETIMEOUT;
    }
    auto it = q->results.find(ticket);
    *out = it->second;
    q->results.erase(it);
    q->live.erase(ticket);
    return REFINE_OK;
}

refine_status refine_queue_poll_any(refine_queue *q, uint64_t *ticket_out, refine_result *out, int32_t timeout_ms)
{
    if (!q || !ticket_out || !out) return REFINE_EINVAL;
    std::unique_lock<std::mutex> lk(q->mu);
    if (q->live.empty()) return REFINE_ENOTFOUND;
    auto ready = [&] { return !q->results.empty(); };
    if (!ready()) {
        if (timeout_ms == 0) return REFINE_ETIMEOUT;
        if (timeout_ms < 0)
            q->cv_poll.wait(lk, ready);
        else if (!q->cv_poll.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
            return REFINE_ETIMEOUT;
    }
    auto best = q->results.begin();
    for (auto it = q->results.begin(); it != q->results.end(); ++it)
        if (it->first < best->first) best = it;
    *ticket_out = best->first;
    *out = best->second;
    q->live.erase(best->first);
    q->results.erase(best);
    return REFINE_OK;
}

const char *refine_queue_last_error(refine_queue *q)
{
    if (!q) return "NULL queue";
    std::lock_guard<std::mutex> lk(q->mu);
    snprintf(q->err_copy, sizeof q->err_copy, "%s%s%s%s%s", q->pc.err, q->pc.err[0] && q->sc.err[0] ? "; " : "",
             q->sc.err, (q->pc.err[0] || q->sc.err[0]) && q->cerr[0] ? "; " : "", q->cerr);
    return q->err_copy;
}

refine_status refine_queue_stats_get(refine_queue *q, refine_queue_stats *out)
{
    if (!q || !out) return REFINE_EINVAL;
    std::lock_guard<std::mutex> lk(q->mu);
    out->submitted = q->n_submitted;
    out->admitted = q->n_admitted;
    out->completed = q->n_completed;
    out->rounds = q->n_rounds;
    out->pending = (int64_t)q->pending.size();
    out->in_flight = q->n_admitted - q->n_completed;
    out->bytes_in_use = q->used;
    out->peak_bytes = q->peak;
    out->budget_bytes = q->budget;
    out->max_round = q->max_round;
    out->slots = q->slots;
    out->kernel_launches = q->launches.load();
    out->dispatch_ms = q->dispatch_ms;
    out->retire_ms = q->retire_ms;
    return REFINE_OK;
}

void refine_queue_destroy(refine_queue *q)
{
    if (!q) return;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        q->stop = true;
        for (QJob *j : q->pending) {
            q->live.erase(j->ticket);
            delete j;
        }
        q->pending.clear();
    }
    q->cv_dispatch.notify_all();
    // the dispatcher stops admitting; the scorer then scores what was
    // admitted and stops; the completion thread retires it and stops
    if (q->dispatcher.joinable()) q->dispatcher.join();
    if (q->scorer.joinable()) q->scorer.join();
    if (q->completer.joinable()) q->completer.join();
    cudaSetDevice(q->pc.device);
    for (cudaStream_t s : q->slot_stream)
        if (s) cudaStreamSynchronize(s);
    for (cudaStream_t s : {q->h2d_stream, q->d2h_stream, q->score_stream})
        if (s) cudaStreamSynchronize(s);
    queue_free(q);
}

}  // extern "C"
