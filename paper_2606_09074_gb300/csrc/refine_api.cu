// C ABI of librefine: argument validation, context scratch, launches.
#include "api_internal.h"

using namespace refine;
using namespace refine_api;

// ====================================================================== ABI

extern "C" {

const char *refine_version(void) { return "librefine 0.1 (sm_103a)"; }

refine_status refine_params_default(refine_params *out)
{
    if (!out) return REFINE_EINVAL;
    memset(out, 0, sizeof *out);
    out->eta = (float)REFINE_DEFAULT_ETA;
    out->luma[0] = 0.299f;
    out->luma[1] = 0.587f;
    out->luma[2] = 0.114f;
    out->e_ln_gem = REFINE_DEFAULT_E_LN_GEM;
    out->e_col = REFINE_DEFAULT_E_COL;
    out->e_opa = REFINE_DEFAULT_E_OPA;
    out->flags = REFINE_FLAG_NORM_ATTR;
    return REFINE_OK;
}

refine_status refine_ctx_create(refine_ctx **out, int device)
{
    if (!out) return REFINE_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return REFINE_ECUDA;
    }
    if (device < 0 || device >= count) return REFINE_EINVAL;
    refine_ctx *c = new refine_ctx();
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&c->d_status, 256) != cudaSuccess || cudaMemset(c->d_status, 0, 256) != cudaSuccess ||
        cudaMallocHost(&c->h_small, 4096) != cudaSuccess) {
        cudaGetLastError();
        if (c->d_status) cudaFree(c->d_status);
        delete c;
        return REFINE_ECUDA;
    }
    *out = c;
    return REFINE_OK;
}

void refine_ctx_destroy(refine_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (Arena *a : {&c->score, &c->select, &c->compact, &c->host})
        if (a->p) cudaFree(a->p);
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    if (c->d_status) cudaFree(c->d_status);
    if (c->h_small) cudaFreeHost(c->h_small);
    delete c;
}

const char *refine_last_error(const refine_ctx *c) { return c ? c->err : "NULL context"; }

refine_status refine_score(refine_ctx *c, const refine_scene *scene, const refine_camera *cams_dev,
                           int32_t n_views, const refine_params *params, float *scores_dev,
                           refine_stream_t stream)
{
    return refine_score_ex(c, scene, cams_dev, n_views, params, scores_dev, nullptr, nullptr, stream);
}

refine_status refine_score_ex(refine_ctx *c, const refine_scene *scene, const refine_camera *cams_dev,
                              int32_t n_views, const refine_params *params, float *scores_dev,
                              float *view_sum_dev, refine_scene_stats *stats_out, refine_stream_t stream)
{
    if (!c) return REFINE_EINVAL;
    refine_status st = use_device(c);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    SceneStats *sd = nullptr;
    unsigned long long *nd = nullptr;
    if ((st = score_impl(c, scene, cams_dev, n_views, params, scores_dev, view_sum_dev, &sd,
                         stats_out ? &nd : nullptr, s)))
        return st;
    if (stats_out) {
        memset(stats_out, 0, sizeof *stats_out);
        if (scene->n == 0) {
            for (int k = 0; k < 3; ++k) stats_out->lambda[k] = 1.0 / 3.0;
            return REFINE_OK;
        }
        SceneStats *h = reinterpret_cast<SceneStats *>(static_cast<char *>(c->h_small) + 256);
        unsigned long long *hn = reinterpret_cast<unsigned long long *>(static_cast<char *>(c->h_small) + 1024);
        cudaError_t e = cudaMemcpyAsync(h, sd, sizeof(SceneStats), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hn, nd, kCountSlots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "stats read-back");
        if ((st = read_status(c, s))) return st;
        static_assert(offsetof(refine_scene_stats, pairs) == sizeof(SceneStats), "stats layout");
        memcpy(stats_out, h, sizeof(SceneStats));
        stats_out->pairs = scene->n * (int64_t)n_views;
        stats_out->tile_views = (int64_t)hn[kCntTiles];
        stats_out->in_pairs = (int64_t)hn[kCntInPairs];
        stats_out->out_pairs = (int64_t)hn[kCntOutPairs];
        stats_out->mixed_pairs = (int64_t)hn[kCntMixedPairs];
        stats_out->bound_pairs = (int64_t)hn[kCntBoundPairs];
        stats_out->footprint_pairs = (int64_t)hn[kCntExactPairs];
        stats_out->visible_mixed_pairs = (int64_t)hn[kCntVisMixed];
        stats_out->open_u_pairs = (int64_t)hn[kCntOpenX];
        stats_out->open_v_pairs = (int64_t)hn[kCntOpenY];
        stats_out->open_z_pairs = (int64_t)hn[kCntOpenZ];
        stats_out->bound_u_pairs = (int64_t)hn[kCntBoundX];
        stats_out->bound_v_pairs = (int64_t)hn[kCntBoundY];
        stats_out->exact_u_pairs = (int64_t)hn[kCntExactX];
        stats_out->exact_v_pairs = (int64_t)hn[kCntExactY];
        stats_out->exact_warp_axes = (int64_t)hn[kCntExactWarpAxes];
    }
    return REFINE_OK;
}

refine_status refine_select(refine_ctx *c, const float *scores_dev, int64_t n, double ratio,
                            uint32_t *keep_mask_dev, float *threshold_out, int64_t *n_keep_out,
                            refine_stream_t stream)
{
    if (!c) return REFINE_EINVAL;
    refine_status st = use_device(c);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned int *kd = nullptr;
    int64_t nk = 0;
    if ((st = select_impl(c, scores_dev, n, ratio, keep_mask_dev, &kd, &nk, s))) return st;
    if (n_keep_out) *n_keep_out = nk;
    if (threshold_out) return read_threshold(c, kd, threshold_out, s);
    return REFINE_OK;
}

refine_status refine_compact(refine_ctx *c, const refine_scene *in, const uint32_t *keep_mask_dev,
                             float *out_pos_dev, void *out_attr_dev, int64_t out_row_stride,
                             int32_t *kept_idx_dev, int64_t *n_keep_out, refine_stream_t stream)
{
    if (!c) return REFINE_EINVAL;
    refine_status st = use_device(c);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    long long *td = nullptr;
    if ((st = compact_impl(c, in, keep_mask_dev, out_pos_dev, out_attr_dev, out_row_stride, kept_idx_dev, &td,
                           s)))
        return st;
    if (n_keep_out) {
        if (!td) {
            *n_keep_out = 0;
            return REFINE_OK;
        }
        long long *h = reinterpret_cast<long long *>(static_cast<char *>(c->h_small) + 128);
        cudaError_t e = cudaMemcpyAsync(h, td, sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "count read-back");
        if ((st = read_status(c, s))) return st;
        *n_keep_out = *h;
    }
    return REFINE_OK;
}

refine_status refine_prune_host(refine_ctx *c, int64_t n, int32_t dtype, const float *pos_host,
                                const void *attr_host, const refine_camera *cams_host, int32_t n_views,
                                const refine_params *params, double ratio, float *out_pos_host,
                                void *out_attr_host, int32_t *out_idx_host, float *scores_host,
                                int64_t *n_keep_out, float *threshold_out, refine_stream_t stream)
{
    if (!c) return REFINE_EINVAL;
    refine_status st = use_device(c);
    if (st) return st;
    if (n < 0 || n > INT32_MAX) return fail(c, REFINE_EINVAL, "prune_host: n out of range");
    if (!valid_dtype(dtype)) return fail(c, REFINE_EINVAL, "prune_host: bad dtype");
    if (n_views < 1 || n_views > 65535 || !cams_host) return fail(c, REFINE_EINVAL, "prune_host: bad cameras");
    if (!(ratio >= 0.0 && ratio < 1.0)) return fail(c, REFINE_EINVAL, "prune_host: ratio must lie in [0, 1)");
    if (n > 0 && (!pos_host || !attr_host || !out_pos_host || !out_attr_host))
        return fail(c, REFINE_EINVAL, "prune_host: NULL host buffer");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t es = attr_col_bytes(dtype);  // bytes of the 56 attribute rows per primitive
    const int64_t n_keep = n - (int64_t)floor(ratio * (double)n);
    const int64_t words = (n + 31) / 32;
    const int64_t nk_alloc = n_keep > 0 ? n_keep : 1;
    if ((st = ensure(c, c->host,
                     carve_size({12 * (size_t)n, es * (size_t)n, sizeof(refine_camera) * (size_t)n_views,
                                 4 * (size_t)n, 4 * (size_t)words, 12 * (size_t)nk_alloc,
                                 es * (size_t)nk_alloc, 4 * (size_t)nk_alloc}))))
        return st;
    Carver cv(c->host.p);
    float *d_pos = cv.take<float>(3 * (size_t)n);
    char *d_attr = cv.take<char>(es * (size_t)n);
    refine_camera *d_cams = cv.take<refine_camera>(n_views);
    float *d_scores = cv.take<float>(n);
    uint32_t *d_mask = cv.take<uint32_t>(words);
    float *d_opos = cv.take<float>(3 * (size_t)nk_alloc);
    char *d_oattr = cv.take<char>(es * (size_t)nk_alloc);
    int32_t *d_idx = cv.take<int32_t>(nk_alloc);
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = cudaMemcpyAsync(d_pos, pos_host, 12 * (size_t)n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_attr, attr_host, es * (size_t)n, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_cams, cams_host, sizeof(refine_camera) * (size_t)n_views, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "prune_host: host-to-device copy");
    refine_scene sc;
    sc.n = n;
    sc.dtype = dtype;
    sc.reserved = 0;
    sc.pos = d_pos;
    sc.attr = d_attr;
    sc.row_stride = n;
    if ((st = score_impl(c, &sc, d_cams, n_views, params, d_scores, nullptr, nullptr, nullptr, s))) return st;
    unsigned int *kd = nullptr;
    int64_t nk = 0;
    if ((st = select_impl(c, d_scores, n, ratio, d_mask, &kd, &nk, s))) return st;
    long long *td = nullptr;
    if ((st = compact_impl(c, &sc, d_mask, d_opos, d_oattr, nk, d_idx, &td, s))) return st;
    if (n_keep > 0) {
        e = cudaMemcpyAsync(out_pos_host, d_opos, 12 * (size_t)n_keep, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out_attr_host, d_oattr, es * (size_t)n_keep, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && out_idx_host)
            e = cudaMemcpyAsync(out_idx_host, d_idx, 4 * (size_t)n_keep, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess && scores_host && n > 0)
        e = cudaMemcpyAsync(scores_host, d_scores, 4 * (size_t)n, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "prune_host: device-to-host copy");
    float thr = -INFINITY;
    if ((st = read_threshold(c, kd, &thr, s))) return st;  // synchronises
    if (n_keep_out) *n_keep_out = n_keep;
    if (threshold_out) *threshold_out = thr;
    return REFINE_OK;
}

refine_status refine_ctx_check(refine_ctx *c, refine_stream_t stream)
{
    if (!c) return REFINE_EINVAL;
    refine_status st = use_device(c);
    if (st) return st;
    return read_status(c, reinterpret_cast<cudaStream_t>(stream));
}

refine_status refine_ctx_set_timing(refine_ctx *c, int enable)
{
    if (!c) return REFINE_EINVAL;
    if (enable != 0 && enable != REFINE_TIMING_ALL && enable != REFINE_TIMING_SCORE)
        return fail(c, REFINE_EINVAL, "set_timing: 0, REFINE_TIMING_ALL or REFINE_TIMING_SCORE");
    c->timing = enable;
    return REFINE_OK;
}

refine_status refine_ctx_kernel_times(refine_ctx *c, const char **names, double *ms, int64_t *launches,
                                      int32_t cap, int32_t *count)
{
    if (!c || !count) return REFINE_EINVAL;
    refine_status st = use_device(c);
    if (st) return st;
    double acc[K_NCLASS] = {0};
    int64_t cnt[K_NCLASS] = {0};
    for (auto &p : c->pending) {
        float t = 0.f;
        cudaEventSynchronize(p.b);
        if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) acc[p.cls] += t;
        cnt[p.cls]++;
        c->pool.push_back(p.a);
        c->pool.push_back(p.b);
    }
    c->pending.clear();
    int32_t k = 0;
    for (int i = 0; i < K_NCLASS; ++i) {
        if (!cnt[i]) continue;
        if (k < cap) {
            if (names) names[k] = kClassName[i];
            if (ms) ms[k] = acc[i];
            if (launches) launches[k] = cnt[i];
        }
        ++k;
    }
    *count = k < cap ? k : cap;
    cudaGetLastError();
    return REFINE_OK;
}

int64_t refine_ctx_launch_count(const refine_ctx *c) { return c ? c->launch_count : -1; }

refine_status refine_selftest_wait(refine_ctx *c, uint32_t bytes, uint32_t missing_bytes, int64_t wait_cycles,
                                   refine_stream_t stream)
{
    if (!c) return REFINE_EINVAL;
    refine_status st = use_device(c);
    if (st) return st;
    if (bytes < 16 || bytes > kSelftestMaxBytes || bytes % 16 || missing_bytes > 65536 || wait_cycles < 1 ||
        wait_cycles > kWaitCycles)
        return fail(c, REFINE_EINVAL, "selftest_wait: bytes %u, missing %u or cycles %lld out of range", bytes,
                    missing_bytes, (long long)wait_cycles);
    if ((st = ensure(c, c->score, kSelftestMaxBytes))) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if ((st = launch(c, K_SELFTEST, s, [&] {
             return launch_wait_selftest(c->score.p, bytes, missing_bytes, (long long)wait_cycles, c->d_status, s);
         })))
        return st;
    return read_status(c, s);
}

refine_status refine_fma_rate(refine_ctx *c, int32_t iters, double *flops_per_s, double *ms_out,
                              refine_stream_t stream)
{
    if (!c || !flops_per_s) return REFINE_EINVAL;
    refine_status st = use_device(c);
    if (st) return st;
    if (iters < 1 || iters > kFmaProbeMaxIters)
        return fail(c, REFINE_EINVAL, "fma_rate: iters %d out of [1, %d]", (int)iters, kFmaProbeMaxIters);
    if ((st = ensure(c, c->score, 256))) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float *sink = static_cast<float *>(c->score.p);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e != cudaSuccess) {
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
        return cuda_fail(c, e, "cudaEventCreate");
    }
    // one untimed launch (clocks ramp, code loaded), then the timed one
    st = launch(c, K_FMA_PROBE, s, [&] { return launch_fma_probe(c->num_sms, iters, sink, s); });
    if (!st && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) st = cuda_fail(c, e, "cudaEventRecord");
    if (!st) st = launch(c, K_FMA_PROBE, s, [&] { return launch_fma_probe(c->num_sms, iters, sink, s); });
    if (!st && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) st = cuda_fail(c, e, "cudaEventRecord");
    if (!st && (e = cudaEventSynchronize(ev[1])) != cudaSuccess) st = cuda_fail(c, e, "cudaEventSynchronize");
    float ms = 0.f;
    if (!st && (e = cudaEventElapsedTime(&ms, ev[0], ev[1])) != cudaSuccess) st = cuda_fail(c, e, "cudaEventElapsedTime");
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st) return st;
    if (!(ms > 0.f)) return fail(c, REFINE_ECUDA, "fma_rate: no elapsed time");
    *flops_per_s = fma_probe_flops(c->num_sms, iters) / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return REFINE_OK;
}

}  // extern "C"

// ==================================================================== batch

struct refine_batch {
    refine_ctx *ctx = nullptr;
    std::vector<refine_job> jobs;
    refine_params params;
    std::vector<ScenePlan> plans;
    std::vector<SceneScratch> sx;
    std::vector<void *> sel_scr, cmp_scr;
    std::vector<int64_t> n_keep;
    std::vector<unsigned int *> kstar;
    std::vector<long long *> total;
    void *scratch = nullptr;
    void *h_res = nullptr;  // pinned read-back area
    // One batched score launch per pass level: level p scores views
    // [p vpp, (p + 1) vpp) of every scene with more than p passes, so a
    // scene's passes run in order, as refine_score runs them.
    struct Level {
        ScoreLaunch *d_launch = nullptr;       // [scenes] this pass of each scene taking part
        long long *d_tile_begin = nullptr;     // [scenes + 1]
        unsigned long long *d_counter = nullptr;
        std::vector<int> jobs;                 // the scenes taking part
        long long total_tiles = 0;
        int max_v = 0;                         // largest camera block of the level
        int grid = 1;
        int rounds = kBatchRounds;             // item size (batch_rounds)
    };
    std::vector<Level> levels;
    ScoreShape shape;
    cudaStream_t main = nullptr;
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> events;  // fork, join[lanes], fork2, join2[lanes]
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches_per_run = 0;
};

namespace refine_api {

refine_status batch_record(refine_batch *b)
{
    refine_ctx *c = b->ctx;
    const int S = (int)b->jobs.size(), L = (int)b->lanes.size();
    cudaStream_t m = b->main;
    int64_t launches = 0;
    auto counted = [&](cudaStream_t) {
        return [&launches, c](int, auto &&f) -> refine_status {
            const cudaError_t e = f();
            if (e != cudaSuccess) return cuda_fail(c, e, "batch launch");
            ++launches;
            return REFINE_OK;
        };
    };
    cudaError_t e = cudaStreamBeginCapture(m, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
    refine_status st = REFINE_OK;
    cudaEvent_t fork = b->events[0], fork2 = b->events[1 + L];
    e = cudaSuccess;
    for (const refine_batch::Level &lv : b->levels)
        if (e == cudaSuccess) e = cudaMemsetAsync(lv.d_counter, 0, sizeof(unsigned long long), m);
    if (e == cudaSuccess) e = cudaEventRecord(fork, m);
    for (int l = 0; l < L && e == cudaSuccess && !st; ++l) {
        cudaStream_t ls = b->lanes[l];
        e = cudaStreamWaitEvent(ls, fork, 0);
        for (int j = l; j < S && e == cudaSuccess && !st; j += L)
            st = enqueue_prep(c, counted(ls), &b->jobs[j].scene, b->jobs[j].cams_dev, b->plans[j], b->sx[j],
                              b->params, false, c->d_status, ls);
        if (e == cudaSuccess && !st) e = cudaEventRecord(b->events[1 + l], ls);
    }
    for (int l = 0; l < L && e == cudaSuccess && !st; ++l) e = cudaStreamWaitEvent(m, b->events[1 + l], 0);
    for (const refine_batch::Level &lv : b->levels) {
        if (e != cudaSuccess || st) break;
        BatchLaunch bl;
        bl.scenes = lv.d_launch;
        bl.tile_begin = lv.d_tile_begin;
        bl.n_scenes = (int)lv.jobs.size();
        bl.total_tiles = lv.total_tiles;
        bl.counter = lv.d_counter;
        bl.status = c->d_status;
        bl.rounds = lv.rounds;
        e = launch_score_batch(bl, lv.max_v, lv.grid, b->shape, m);
        if (e == cudaSuccess) ++launches;
    }
    if (e == cudaSuccess && !st) e = cudaEventRecord(fork2, m);
    for (int l = 0; l < L && e == cudaSuccess && !st; ++l) {
        cudaStream_t ls = b->lanes[l];
        e = cudaStreamWaitEvent(ls, fork2, 0);
        for (int j = l; j < S && e == cudaSuccess && !st; j += L) {
            const refine_job &jb = b->jobs[j];
            st = enqueue_select(c, counted(ls), jb.scores_dev, jb.scene.n, b->n_keep[j], jb.keep_mask_dev,
                                b->sel_scr[j], &b->kstar[j], c->d_status, ls);
            if (!st && jb.out_pos_dev)
                st = enqueue_compact(c, counted(ls), &jb.scene, jb.keep_mask_dev, jb.out_pos_dev, jb.out_attr_dev,
                                     jb.out_row_stride, jb.kept_idx_dev, b->cmp_scr[j], &b->total[j], c->d_status,
                                     ls);
        }
        if (e == cudaSuccess && !st) e = cudaEventRecord(b->events[2 + L + l], ls);
    }
    for (int l = 0; l < L && e == cudaSuccess && !st; ++l) e = cudaStreamWaitEvent(m, b->events[2 + L + l], 0);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(m, &g);
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e != cudaSuccess ? e : e2, "batch capture");
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    b->graph = g;
    b->launches_per_run = launches;
    return REFINE_OK;
}

// Tile prefix of a level for the work-item size of `sh`, copied to the
// device (on `s`, or synchronously when s is NULL), and its grid.
cudaError_t set_level_tiles(refine_batch *b, refine_batch::Level &lv, const ScoreShape &sh, cudaStream_t s)
{
    std::vector<int64_t> ns;
    for (int j : lv.jobs) ns.push_back(b->jobs[j].scene.n);
    const int full_grid = score_batch_grid(b->ctx->num_sms, lv.max_v, sh);
    lv.rounds = batch_rounds(sh, ns.data(), (int)ns.size(), full_grid);
    const long long tile = batch_tile(sh, lv.rounds);
    std::vector<long long> tb(lv.jobs.size() + 1, 0);
    for (size_t k = 0; k < lv.jobs.size(); ++k) tb[k + 1] = tb[k] + (ns[k] + tile - 1) / tile;
    lv.total_tiles = tb.back();
    lv.grid = full_grid;
    if (lv.grid > lv.total_tiles) lv.grid = (int)lv.total_tiles;
    if (lv.grid < 1) lv.grid = 1;
    const size_t bytes = sizeof(long long) * tb.size();
    return s ? cudaMemcpyAsync(lv.d_tile_begin, tb.data(), bytes, cudaMemcpyHostToDevice, s)
             : cudaMemcpy(lv.d_tile_begin, tb.data(), bytes, cudaMemcpyHostToDevice);
}

void batch_free(refine_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaStream_t s : b->lanes) cudaStreamDestroy(s);
    if (b->main) cudaStreamDestroy(b->main);
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    if (b->scratch) cudaFree(b->scratch);
    if (b->h_res) cudaFreeHost(b->h_res);
    delete b;
}

}  // namespace refine_api

extern "C" {

refine_status refine_batch_create(refine_ctx *c, const refine_job *jobs, int32_t n_jobs,
                                  const refine_params *params, refine_batch **out)
{
    if (!c || !out) return REFINE_EINVAL;
    *out = nullptr;
    refine_status st = use_device(c);
    if (st) return st;
    if (!jobs || n_jobs < 1 || n_jobs > 4096) return fail(c, REFINE_EINVAL, "batch: n_jobs must lie in [1, 4096]");
    refine_params p;
    if (params) p = *params; else refine_params_default(&p);
    if ((st = check_params(c, &p))) return st;
    const int S = n_jobs;
    refine_batch *b = new refine_batch();
    b->ctx = c;
    b->params = p;
    b->jobs.assign(jobs, jobs + S);
    b->shape = c->shape;
    size_t total = 0;
    int max_passes = 1;
    for (int j = 0; j < S; ++j) {
        const refine_job &jb = jobs[j];
        if ((st = check_score_args(c, &jb.scene, jb.cams_dev, jb.n_views, p, jb.scores_dev))) {
            delete b;
            return fail(c, st, "batch job %d: %s", j, std::string(c->err).c_str());
        }
        const ScenePlan jp = plan_scene(jb.scene.n, jb.n_views, p.max_views, b->shape.views_per_pass);
        if (jb.scene.n < 1 || !jb.keep_mask_dev || !(jb.ratio >= 0.0 && jb.ratio < 1.0)) {
            delete b;
            return fail(c, REFINE_EINVAL, "batch job %d: needs n >= 1, a keep mask and a ratio in [0, 1)", j);
        }
        const int64_t nk = jb.scene.n - (int64_t)floor(jb.ratio * (double)jb.scene.n);
        if (jb.out_pos_dev && (!jb.out_attr_dev || jb.out_row_stride < nk)) {
            delete b;
            return fail(c, REFINE_EINVAL, "batch job %d: compaction output missing or shorter than n_keep", j);
        }
        b->n_keep.push_back(nk);
        b->plans.push_back(jp);
        total += scene_bytes(b->plans.back()) + select_bytes(jb.scene.n) + compact_bytes(jb.scene.n) + 768;
        max_passes = std::max(max_passes, jp.passes);
    }
    for (int lv = 0; lv < max_passes; ++lv)
        total += carve_size({sizeof(ScoreLaunch) * (size_t)S, sizeof(long long) * (size_t)(S + 1),
                             sizeof(unsigned long long)});
    cudaError_t e = cudaMalloc(&b->scratch, total);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(c, e, "batch scratch");
    }
    if ((e = cudaMallocHost(&b->h_res, (size_t)S * 16 + 64)) != cudaSuccess) {
        batch_free(b);
        return cuda_fail(c, e, "batch pinned read-back");
    }
    Carver cv(b->scratch);
    b->levels.resize(max_passes);
    for (refine_batch::Level &lv : b->levels) {
        lv.d_launch = cv.take<ScoreLaunch>(S);
        lv.d_tile_begin = cv.take<long long>(S + 1);
        lv.d_counter = cv.take<unsigned long long>(1);
    }
    for (int j = 0; j < S; ++j) {
        b->sx.push_back(carve_scene(cv, b->plans[j]));
        b->sel_scr.push_back(cv.take<char>(select_bytes(jobs[j].scene.n)));
        b->cmp_scr.push_back(cv.take<char>(compact_bytes(jobs[j].scene.n)));
    }
    b->kstar.assign(S, nullptr);
    b->total.assign(S, nullptr);
    e = cudaSuccess;
    for (int l = 0; l < max_passes && e == cudaSuccess; ++l) {
        refine_batch::Level &lv = b->levels[l];
        std::vector<ScoreLaunch> hl;
        for (int j = 0; j < S; ++j) {
            if (b->plans[j].passes <= l) continue;
            const int v0 = l * b->plans[j].vpp;
            hl.push_back(make_score_launch(&jobs[j].scene, b->plans[j], b->sx[j], p, v0, jobs[j].scores_dev, nullptr,
                                           false, c->d_status));
            lv.jobs.push_back(j);
            lv.max_v = std::max(lv.max_v, hl.back().vcount);
        }
        e = cudaMemcpy(lv.d_launch, hl.data(), sizeof(ScoreLaunch) * hl.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = set_level_tiles(b, lv, b->shape, nullptr);
    }
    const int L = std::min(8, S);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking);
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        cudaStream_t ls = nullptr;
        e = cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->lanes.push_back(ls);
    }
    for (int k = 0; k < 2 * L + 2 && e == cudaSuccess; ++k) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->events.push_back(ev);
    }
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(c, e, "batch set-up");
    }
    *out = b;
    return REFINE_OK;
}

refine_status refine_batch_run(refine_batch *b, refine_stream_t stream)
{
    if (!b) return REFINE_EINVAL;
    refine_ctx *c = b->ctx;
    refine_status st = use_device(c);
    if (st) return st;
    if (!b->exec && (st = batch_record(b))) return st;
    const cudaError_t e = cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
    c->launch_count += b->launches_per_run;
    return REFINE_OK;
}

refine_status refine_batch_results(refine_batch *b, int64_t *n_keep_out, float *threshold_out,
                                   refine_stream_t stream)
{
    if (!b) return REFINE_EINVAL;
    refine_ctx *c = b->ctx;
    refine_status st = use_device(c);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int S = (int)b->jobs.size();
    unsigned int *hk = static_cast<unsigned int *>(b->h_res);
    cudaError_t e = cudaSuccess;
    if (threshold_out)
        for (int j = 0; j < S && e == cudaSuccess; ++j)
            if (b->kstar[j]) e = cudaMemcpyAsync(hk + j, b->kstar[j], sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "batch read-back");
    if ((st = read_status(c, s))) return st;  // synchronises
    for (int j = 0; j < S; ++j) {
        if (n_keep_out) n_keep_out[j] = b->n_keep[j];
        if (threshold_out) threshold_out[j] = b->kstar[j] ? key_to_score(hk[j]) : -INFINITY;
    }
    return REFINE_OK;
}

int64_t refine_batch_launches(const refine_batch *b) { return b ? b->launches_per_run : -1; }

void refine_batch_destroy(refine_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    batch_free(b);
}

}  // extern "C"

// ============================================================ autotuner
namespace refine_api {

refine_shape shape_to_abi(const ScoreShape &sh, double ms)
{
    refine_shape r{};
    r.tile = 32 * sh.gpt;
    r.cta_threads = sh.threads;
    r.ctas_per_sm = sh.ctas_per_sm;
    r.camera_block = sh.views_per_pass;
    r.ms = ms;
    return r;
}

bool shape_from_abi(const refine_shape &r, ScoreShape *sh)
{
    ScoreShape t;
    t.gpt = r.tile / 32;
    t.threads = r.cta_threads;
    t.ctas_per_sm = r.ctas_per_sm;
    t.views_per_pass = r.camera_block;
    if ((r.tile != 32 && r.tile != 64) || !shape_valid(t)) return false;
    *sh = t;
    return true;
}

}  // namespace refine_api

extern "C" {

refine_status refine_ctx_get_shape(const refine_ctx *c, refine_shape *out)
{
    if (!c || !out) return REFINE_EINVAL;
    *out = shape_to_abi(c->shape, 0.0);
    return REFINE_OK;
}

refine_status refine_ctx_set_shape(refine_ctx *c, const refine_shape *shape)
{
    if (!c || !shape) return REFINE_EINVAL;
    ScoreShape sh;
    if (!shape_from_abi(*shape, &sh))
        return fail(c, REFINE_EINVAL,
                    "shape: tile 32|64, cta_threads 128|256, ctas_per_sm >= 0, camera_block 32..512 in steps of 32");
    c->shape = sh;
    return REFINE_OK;
}

refine_status refine_autotune(refine_ctx *c, const refine_job *jobs, int32_t n_jobs, const refine_params *params,
                              int32_t reps, refine_shape *best_out, refine_shape *table_out, int32_t table_cap,
                              int32_t *table_count)
{
    if (!c) return REFINE_EINVAL;
    if (reps < 1) return fail(c, REFINE_EINVAL, "autotune: reps must be >= 1");
    if (!jobs || n_jobs < 1) return fail(c, REFINE_EINVAL, "autotune: no jobs");
    const ScoreShape keep = c->shape;
    std::vector<ScoreShape> cand;
    std::vector<double> ms;
    std::vector<std::vector<int>> seen;  // passes per scene of each camera block tried
    refine_status st = REFINE_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) st = cuda_fail(c, e, "autotune events");
    // Camera blocks (views per pass) that change how some scene is split.
    for (int vpp : {512, 256, 128}) {
        if (st) break;
        std::vector<int> passes;
        for (int j = 0; j < n_jobs; ++j) {
            const int mv = params ? params->max_views : 0;
            passes.push_back(plan_scene(jobs[j].scene.n, jobs[j].n_views, mv, vpp).passes);
        }
        if (std::find(seen.begin(), seen.end(), passes) != seen.end()) continue;
        seen.push_back(passes);
        c->shape.views_per_pass = vpp;
        refine_batch *b = nullptr;
        if ((st = refine_batch_create(c, jobs, n_jobs, params, &b))) break;
        cudaStream_t m = b->main;
        auto run = [c](int cls, auto &&f) -> refine_status {
            const cudaError_t err = f();
            return err == cudaSuccess ? REFINE_OK : cuda_fail(c, err, kClassName[cls]);
        };
        const int S = (int)b->jobs.size();
        for (int j = 0; j < S && !st; ++j)
            st = enqueue_prep(c, run, &b->jobs[j].scene, b->jobs[j].cams_dev, b->plans[j], b->sx[j], b->params, false,
                              c->d_status, m);
        for (int gpt : {2, 1})
            for (int threads : {256, 128})
                for (int cap : {0, threads == 256 ? 2 : 4}) {
                    if (st || e != cudaSuccess) break;
                    ScoreShape sh;
                    sh.gpt = gpt;
                    sh.threads = threads;
                    sh.ctas_per_sm = cap;
                    sh.views_per_pass = vpp;
                    for (refine_batch::Level &lv : b->levels)
                        if (e == cudaSuccess) e = set_level_tiles(b, lv, sh, m);
                    // one warm-up run, then `reps` timed runs of every level's launch
                    for (int r = -1; r < reps && e == cudaSuccess; ++r) {
                        if (r == 0) e = cudaEventRecord(e0, m);
                        for (const refine_batch::Level &lv : b->levels) {
                            if (e != cudaSuccess) break;
                            BatchLaunch bl;
                            bl.scenes = lv.d_launch;
                            bl.tile_begin = lv.d_tile_begin;
                            bl.n_scenes = (int)lv.jobs.size();
                            bl.total_tiles = lv.total_tiles;
                            bl.counter = lv.d_counter;
                            bl.status = c->d_status;
                            bl.rounds = lv.rounds;
                            e = cudaMemsetAsync(lv.d_counter, 0, sizeof(unsigned long long), m);
                            if (e == cudaSuccess) e = launch_score_batch(bl, lv.max_v, lv.grid, sh, m);
                        }
                    }
                    if (e == cudaSuccess) e = cudaEventRecord(e1, m);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float t = 0.f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                    cand.push_back(sh);
                    ms.push_back((double)t / reps);
                }
        if (e != cudaSuccess && !st) st = cuda_fail(c, e, "autotune");
        if (!st) st = read_status(c, m);
        refine_batch_destroy(b);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c->shape = keep;
    if (st) return st;
    size_t best = 0;
    for (size_t k = 1; k < cand.size(); ++k)
        if (ms[k] < ms[best]) best = k;
    c->shape = cand[best];
    if (best_out) *best_out = shape_to_abi(cand[best], ms[best]);
    if (table_out)
        for (size_t k = 0; k < cand.size() && (int)k < table_cap; ++k) table_out[k] = shape_to_abi(cand[k], ms[k]);
    if (table_count) *table_count = (int32_t)cand.size();
    return REFINE_OK;
}

}  // extern "C"
