// C ABI of librefine: argument validation, context scratch, launches.
#include <math.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

using namespace refine;

namespace {

enum KClass {
    K_CAM_PREP = 0,
    K_FEATURES,
    K_FEAT_FINAL,
    K_CELLS,
    K_CELL_SCAN,
    K_CELL_SCATTER,
    K_SCORE,
    K_SEL_PASS,
    K_SEL_TIES,
    K_SEL_MASK,
    K_MASK_FILL,
    K_CMP_COUNT,
    K_CMP_SCATTER,
    K_NCLASS
};
const char *const kClassName[K_NCLASS] = {"cam_prep",      "features",     "features_finalize",
                                          "cells",         "cell_scan",    "cell_scatter",
                                          "score",         "select_pass",  "select_ties",
                                          "select_mask",   "mask_fill",    "compact_count",
                                          "compact_scatter"};

struct Arena {
    void *p = nullptr;
    size_t cap = 0;
};

struct Pending {
    int cls;
    cudaEvent_t a, b;
};

// Bump allocator over an arena (256-byte aligned sub-blocks).
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *p) : base(static_cast<char *>(p)) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *r = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return r;
    }
};

size_t carve_size(std::initializer_list<size_t> parts)
{
    size_t off = 0;
    for (size_t p : parts) off = ((off + 255) & ~size_t(255)) + p;
    return off + 256;
}

}  // namespace

struct refine_ctx {
    int device = 0;
    int num_sms = 0;
    char err[512] = {0};
    int *d_status = nullptr;
    void *h_small = nullptr;  // pinned 4 KB for read-backs
    Arena score, select, compact, host;
    bool timing = false;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[K_NCLASS] = {0};
    int64_t launches[K_NCLASS] = {0};
    int64_t launch_count = 0;
};

namespace {

refine_status fail(refine_ctx *c, refine_status st, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

refine_status cuda_fail(refine_ctx *c, cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear non-sticky errors
    return fail(c, e == cudaErrorMemoryAllocation ? REFINE_ENOMEM : REFINE_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

refine_status use_device(refine_ctx *c)
{
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != c->device) {
        cudaError_t e = cudaSetDevice(c->device);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    }
    return REFINE_OK;
}

refine_status ensure(refine_ctx *c, Arena &a, size_t bytes)
{
    if (bytes <= a.cap) return REFINE_OK;
    size_t want = bytes + bytes / 4;
    want = (want + (size_t(2) << 20) - 1) & ~((size_t(2) << 20) - 1);
    if (a.p) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceSynchronize (scratch growth)");
        cudaFree(a.p);
        a.p = nullptr;
        a.cap = 0;
    }
    cudaError_t e = cudaMalloc(&a.p, want);
    if (e != cudaSuccess) {
        a.p = nullptr;
        return cuda_fail(c, e, "cudaMalloc (scratch)");
    }
    a.cap = want;
    return REFINE_OK;
}

cudaEvent_t take_event(refine_ctx *c)
{
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Runs one kernel launcher, bracketed by events when timing is enabled.
template <typename F>
refine_status launch(refine_ctx *c, int cls, cudaStream_t s, F &&f)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->timing) {
        a = take_event(c);
        cudaEventRecord(a, s);
    }
    cudaError_t e = f();
    if (e != cudaSuccess) return cuda_fail(c, e, kClassName[cls]);
    if (c->timing) {
        b = take_event(c);
        cudaEventRecord(b, s);
        c->pending.push_back({cls, a, b});
    }
    c->launch_count++;
    c->launches[cls]++;
    return REFINE_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

refine_status check_params(refine_ctx *c, const refine_params *p)
{
    if (!(p->eta > 0.f) || !isfinite(p->eta)) return fail(c, REFINE_EINVAL, "params: eta must be finite and > 0");
    for (int k = 0; k < 3; ++k)
        if (!isfinite(p->luma[k])) return fail(c, REFINE_EINVAL, "params: luma must be finite");
    if (!(isfinite(p->e_ln_gem) && p->e_ln_gem != 0.0 && isfinite(p->e_col) && p->e_col != 0.0 &&
          isfinite(p->e_opa) && p->e_opa != 0.0))
        return fail(c, REFINE_EINVAL, "params: calibration constants must be finite and nonzero");
    return REFINE_OK;
}

refine_status check_scene(refine_ctx *c, const refine_scene *s)
{
    if (!s) return fail(c, REFINE_EINVAL, "scene is NULL");
    if (s->n < 0 || s->n > INT32_MAX) return fail(c, REFINE_EINVAL, "scene: n=%lld out of [0, 2^31-1]", (long long)s->n);
    if (s->dtype != REFINE_F32 && s->dtype != REFINE_BF16) return fail(c, REFINE_EINVAL, "scene: unknown dtype %d", s->dtype);
    if (s->n == 0) return REFINE_OK;
    if (!s->pos || !s->attr) return fail(c, REFINE_EINVAL, "scene: NULL pos/attr");
    if (s->row_stride < s->n) return fail(c, REFINE_EINVAL, "scene: row_stride < n");
    if (!aligned16(s->pos) || !aligned16(s->attr)) return fail(c, REFINE_EINVAL, "scene: pos/attr must be 16-byte aligned");
    return REFINE_OK;
}

// Rows may be read with 16-byte vector loads.
// Reads back and clears the device status word (synchronises `s`).
refine_status read_status(refine_ctx *c, cudaStream_t s)
{
    int *h = static_cast<int *>(c->h_small);
    cudaError_t e = cudaMemcpyAsync(h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "status read-back");
    int st = h[0];
    if (st != 0) {
        cudaMemsetAsync(c->d_status, 0, sizeof(int), s);
        switch (st) {
        case kEnonfinite: return fail(c, REFINE_ENONFINITE, "device: non-finite input value");
        case kEtimeout: return fail(c, REFINE_ETIMEOUT, "device: a bounded wait ran out");
        default: return fail(c, REFINE_EINVAL, "device: invalid input (camera, quaternion or output size)");
        }
    }
    return REFINE_OK;
}

// ------------------------------------------------------------------ score
// Scratch layout of one scene's score pass.
struct ScenePlan {
    int64_t n = 0;
    int V = 0;
    bool multipass = false;
    int nb = 1;    // feature-pass blocks
    int bits = 4;  // processing-order grid resolution
};

struct SceneScratch {
    CamRec *cams;
    PrimRec *recs;
    double *partials;
    SceneConsts *consts;
    SceneStats *stats;
    uint32_t *cell;
    unsigned *counts;  // cell_count(bits) + 64 words; the last ones hold the scan's done counter
    unsigned *off_local;
    unsigned *bsum;
    uint32_t *perm;
    unsigned long long *need;
    float *running;
};

ScenePlan plan_scene(const refine_ctx *c, const refine_scene *sc, int V)
{
    ScenePlan pl;
    pl.n = sc->n;
    pl.V = V;
    pl.multipass = V > kViewsPerPass;
    pl.nb = feature_blocks(pl.n);
    pl.bits = cell_bits_for(pl.n);
    return pl;
}

size_t scene_bytes(const ScenePlan &pl)
{
    const size_t n = (size_t)pl.n, cells = (size_t)cell_count(pl.bits);
    return carve_size({sizeof(CamRec) * (size_t)pl.V, sizeof(PrimRec) * n, sizeof(double) * kFeatSums * 1024,
                       sizeof(SceneConsts), sizeof(SceneStats), sizeof(uint32_t) * n,
                       sizeof(unsigned) * (cells + 64), sizeof(unsigned) * cells,
                       sizeof(unsigned) * (cells / kScanThreads), sizeof(uint32_t) * n,
                       kCountSlots * sizeof(unsigned long long), pl.multipass ? sizeof(float) * n : 0});
}

SceneScratch carve_scene(Carver &cv, const ScenePlan &pl)
{
    const int64_t n = pl.n;
    const int cells = cell_count(pl.bits);
    SceneScratch x;
    x.cams = cv.take<CamRec>(pl.V);
    x.recs = cv.take<PrimRec>(n);
    x.partials = cv.take<double>(kFeatSums * 1024);
    x.consts = cv.take<SceneConsts>(1);
    x.stats = cv.take<SceneStats>(1);
    x.cell = cv.take<uint32_t>(n);
    x.counts = cv.take<unsigned>(cells + 64);
    x.off_local = cv.take<unsigned>(cells);
    x.bsum = cv.take<unsigned>(cells / kScanThreads);
    x.perm = cv.take<uint32_t>(n);
    x.need = cv.take<unsigned long long>(kCountSlots);
    x.running = pl.multipass ? cv.take<float>(n) : nullptr;
    return x;
}

// Camera records, content features and lambda, processing order.
template <typename L>
refine_status enqueue_prep(refine_ctx *c, L &&run, const refine_scene *sc, const refine_camera *cams,
                           const ScenePlan &pl, const SceneScratch &x, const refine_params &p, bool count,
                           int *status, cudaStream_t s)
{
    const int64_t n = pl.n;
    const int cells = cell_count(pl.bits);
    cudaError_t e = cudaMemsetAsync(x.counts, 0, sizeof(unsigned) * (cells + 64), s);
    if (e == cudaSuccess && count) e = cudaMemsetAsync(x.need, 0, kCountSlots * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
    refine_status st;
    if ((st = run(K_CAM_PREP, [&] { return launch_cam_prep(cams, pl.V, x.cams, status, s); }))) return st;
    if ((st = run(K_FEATURES, [&] {
             return launch_features(sc->pos, sc->attr, sc->dtype, sc->row_stride, n, p.eta, p.luma, x.recs,
                                    x.partials, status, s);
         })))
        return st;
    if ((st = run(K_FEAT_FINAL,
                  [&] { return launch_features_finalize(x.partials, pl.nb, n, &p, pl.bits, x.consts, x.stats, s); })))
        return st;
    if ((st = run(K_CELLS, [&] {
             return launch_cells(sc->pos, sc->row_stride, n, pl.bits, x.consts, x.cell, x.counts, c->num_sms, s);
         })))
        return st;
    if ((st = run(K_CELL_SCAN,
                  [&] { return launch_cell_scan(x.counts, x.off_local, x.bsum, x.counts + cells, pl.bits, s); })))
        return st;
    return run(K_CELL_SCATTER,
               [&] { return launch_cell_scatter(x.cell, n, x.counts, x.off_local, x.bsum, x.perm, c->num_sms, s); });
}

ScoreLaunch make_score_launch(const refine_scene *sc, const ScenePlan &pl, const SceneScratch &x,
                              const refine_params &p, int v0, float *scores, float *view_sum, bool count, int *status)
{
    ScoreLaunch a;
    a.recs = x.recs;
    a.perm = x.perm;
    a.n = pl.n;
    a.cams = x.cams + v0;
    a.vcount = pl.V - v0 < kViewsPerPass ? pl.V - v0 : kViewsPerPass;
    a.first = v0 == 0;
    a.last = v0 + a.vcount >= pl.V;
    a.eta = p.eta;
    a.inv_views = 1.0f / (float)pl.V;
    a.flags = p.flags;
    a.consts = x.consts;
    a.running = x.running;
    a.scores = scores;
    a.view_sum = view_sum;
    a.need = count ? x.need : nullptr;
    a.status = status;
    a.grid = 0;
    return a;
}

refine_status check_score_args(refine_ctx *c, const refine_scene *sc, const refine_camera *cams, int V,
                               const refine_params &p, const float *scores)
{
    refine_status st = check_scene(c, sc);
    if (st) return st;
    if (V < 1 || V > 65535) return fail(c, REFINE_EINVAL, "n_views=%d out of [1, 65535]", V);
    if (!cams) return fail(c, REFINE_EINVAL, "cams_dev is NULL");
    if ((st = check_params(c, &p))) return st;
    if (sc->n > 0 && !scores) return fail(c, REFINE_EINVAL, "scores_dev is NULL");
    return REFINE_OK;
}

refine_status score_impl(refine_ctx *c, const refine_scene *sc, const refine_camera *cams, int V,
                         const refine_params *pin, float *scores, float *view_sum, SceneStats **stats_dev,
                         unsigned long long **need_dev, cudaStream_t s)
{
    refine_params p;
    if (pin) p = *pin; else refine_params_default(&p);
    refine_status st = check_score_args(c, sc, cams, V, p, scores);
    if (st || sc->n == 0) return st;
    const ScenePlan pl = plan_scene(c, sc, V);
    if ((st = ensure(c, c->score, scene_bytes(pl)))) return st;
    Carver cv(c->score.p);
    const SceneScratch x = carve_scene(cv, pl);
    if (stats_dev) *stats_dev = x.stats;
    if (need_dev) *need_dev = x.need;
    auto run = [&](int cls, auto &&f) { return launch(c, cls, s, f); };
    if ((st = enqueue_prep(c, run, sc, cams, pl, x, p, need_dev != nullptr, c->d_status, s))) return st;
    for (int v0 = 0; v0 < V; v0 += kViewsPerPass) {
        ScoreLaunch a = make_score_launch(sc, pl, x, p, v0, scores, view_sum, need_dev != nullptr, c->d_status);
        a.grid = score_grid(c->num_sms, pl.n, a.vcount);
        if ((st = launch(c, K_SCORE, s, [&] { return launch_score(a, s); }))) return st;
    }
    return REFINE_OK;
}

// ----------------------------------------------------------------- select
size_t select_bytes(int64_t n)
{
    return carve_size({sizeof(SelState), sizeof(unsigned) * (size_t)((n + kTieSeg - 1) / kTieSeg)});
}

// Radix select into the given state; *kstar_dev is NULL when nothing is pruned.
template <typename L>
refine_status enqueue_select(refine_ctx *c, L &&run, const float *scores, int64_t n, int64_t n_keep,
                             uint32_t *mask, void *scratch, unsigned int **kstar_dev, int *status, cudaStream_t s)
{
    *kstar_dev = nullptr;
    if (n == 0) return REFINE_OK;
    if (n_keep == n) return run(K_MASK_FILL, [&] { return launch_mask_fill(mask, n, s); });
    Carver cv(scratch);
    SelState *ss = cv.take<SelState>(1);
    unsigned *seg = cv.take<unsigned>((n + kTieSeg - 1) / kTieSeg);
    cudaError_t e = cudaMemsetAsync(ss, 0, sizeof(SelState), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
    const bool vec = aligned16(scores);
    const int grid = select_grid(c->num_sms, n);
    refine_status st;
    for (int pass = 0; pass < 3; ++pass)
        if ((st = run(K_SEL_PASS, [&] {
                 return launch_select_pass(pass, scores, n, (uint32_t)n_keep, ss, vec, grid, status, s);
             })))
            return st;
    if ((st = run(K_SEL_TIES, [&] { return launch_select_ties(scores, n, ss, seg, grid, s); }))) return st;
    if ((st = run(K_SEL_MASK, [&] { return launch_select_mask(scores, n, ss, mask, grid, s); }))) return st;
    *kstar_dev = &ss->kstar;
    return REFINE_OK;
}

refine_status select_impl(refine_ctx *c, const float *scores, int64_t n, double ratio, uint32_t *mask,
                          unsigned int **kstar_dev, int64_t *n_keep, cudaStream_t s)
{
    *kstar_dev = nullptr;
    if (n < 0 || n > INT32_MAX) return fail(c, REFINE_EINVAL, "select: n=%lld out of range", (long long)n);
    if (!(ratio >= 0.0 && ratio < 1.0)) return fail(c, REFINE_EINVAL, "select: ratio must lie in [0, 1)");
    *n_keep = n - (int64_t)floor(ratio * (double)n);
    if (n == 0) return REFINE_OK;
    if (!scores || !mask) return fail(c, REFINE_EINVAL, "select: NULL scores or mask");
    refine_status st;
    if ((st = ensure(c, c->select, select_bytes(n)))) return st;
    auto run = [&](int cls, auto &&f) { return launch(c, cls, s, f); };
    return enqueue_select(c, run, scores, n, *n_keep, mask, c->select.p, kstar_dev, c->d_status, s);
}

refine_status read_threshold(refine_ctx *c, unsigned int *kstar_dev, float *thr, cudaStream_t s)
{
    if (!kstar_dev) {
        *thr = -INFINITY;
        return read_status(c, s);
    }
    unsigned int *h = reinterpret_cast<unsigned int *>(static_cast<char *>(c->h_small) + 64);
    cudaError_t e = cudaMemcpyAsync(h, kstar_dev, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "threshold read-back");
    refine_status st = read_status(c, s);  // synchronises
    if (st) return st;
    *thr = key_to_score(*h);
    return REFINE_OK;
}

// ---------------------------------------------------------------- compact
size_t compact_bytes(int64_t n)
{
    const size_t nseg = (size_t)((n + kCmpSeg - 1) / kCmpSeg);
    return carve_size({sizeof(CmpState), sizeof(unsigned) * nseg, sizeof(unsigned long long) * nseg});
}

template <typename L>
refine_status enqueue_compact(refine_ctx *c, L &&run, const refine_scene *in, const uint32_t *mask, float *out_pos,
                              void *out_attr, int64_t out_stride, int32_t *idx, void *scratch, long long **total_dev,
                              int *status, cudaStream_t s)
{
    const int64_t n = in->n;
    const int64_t nseg = (n + kCmpSeg - 1) / kCmpSeg;
    Carver cv(scratch);
    CmpState *cs = cv.take<CmpState>(1);
    unsigned *seg_cnt = cv.take<unsigned>(nseg);
    unsigned long long *seg_off = cv.take<unsigned long long>(nseg);
    cudaError_t e = cudaMemsetAsync(cs, 0, sizeof(CmpState), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
    int64_t cgrid = (nseg + 1023) / 1024;
    if (cgrid > c->num_sms) cgrid = c->num_sms;
    if (cgrid < 1) cgrid = 1;
    refine_status st;
    if ((st = run(K_CMP_COUNT, [&] {
             return launch_compact_count(mask, n, seg_cnt, seg_off, cs, out_stride, (int)cgrid, status, s);
         })))
        return st;
    const int sgrid = compact_grid(c->num_sms, n);
    if ((st = run(K_CMP_SCATTER, [&] {
             return launch_compact_scatter(*in, mask, seg_off, cs, out_pos, out_attr, out_stride, idx, sgrid, s);
         })))
        return st;
    *total_dev = &cs->total;
    return REFINE_OK;
}

refine_status compact_impl(refine_ctx *c, const refine_scene *in, const uint32_t *mask, float *out_pos,
                           void *out_attr, int64_t out_stride, int32_t *idx, long long **total_dev,
                           cudaStream_t s)
{
    refine_status st = check_scene(c, in);
    if (st) return st;
    *total_dev = nullptr;
    if (in->n == 0) return REFINE_OK;
    if (!mask || !out_pos || !out_attr) return fail(c, REFINE_EINVAL, "compact: NULL mask or output");
    if (out_stride < 0) return fail(c, REFINE_EINVAL, "compact: negative out_row_stride");
    if ((st = ensure(c, c->compact, compact_bytes(in->n)))) return st;
    auto run = [&](int cls, auto &&f) { return launch(c, cls, s, f); };
    return enqueue_compact(c, run, in, mask, out_pos, out_attr, out_stride, idx, c->compact.p, total_dev,
                           c->d_status, s);
}

}  // namespace

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
    if (dtype != REFINE_F32 && dtype != REFINE_BF16) return fail(c, REFINE_EINVAL, "prune_host: bad dtype");
    if (n_views < 1 || n_views > 65535 || !cams_host) return fail(c, REFINE_EINVAL, "prune_host: bad cameras");
    if (!(ratio >= 0.0 && ratio < 1.0)) return fail(c, REFINE_EINVAL, "prune_host: ratio must lie in [0, 1)");
    if (n > 0 && (!pos_host || !attr_host || !out_pos_host || !out_attr_host))
        return fail(c, REFINE_EINVAL, "prune_host: NULL host buffer");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t es = dtype == REFINE_BF16 ? 2 : 4;
    const int64_t n_keep = n - (int64_t)floor(ratio * (double)n);
    const int64_t words = (n + 31) / 32;
    const int64_t nk_alloc = n_keep > 0 ? n_keep : 1;
    if ((st = ensure(c, c->host,
                     carve_size({12 * (size_t)n, 56 * es * (size_t)n, sizeof(refine_camera) * (size_t)n_views,
                                 4 * (size_t)n, 4 * (size_t)words, 12 * (size_t)nk_alloc,
                                 56 * es * (size_t)nk_alloc, 4 * (size_t)nk_alloc}))))
        return st;
    Carver cv(c->host.p);
    float *d_pos = cv.take<float>(3 * (size_t)n);
    char *d_attr = cv.take<char>(56 * es * (size_t)n);
    refine_camera *d_cams = cv.take<refine_camera>(n_views);
    float *d_scores = cv.take<float>(n);
    uint32_t *d_mask = cv.take<uint32_t>(words);
    float *d_opos = cv.take<float>(3 * (size_t)nk_alloc);
    char *d_oattr = cv.take<char>(56 * es * (size_t)nk_alloc);
    int32_t *d_idx = cv.take<int32_t>(nk_alloc);
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = cudaMemcpyAsync(d_pos, pos_host, 12 * (size_t)n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_attr, attr_host, 56 * es * (size_t)n, cudaMemcpyHostToDevice, s);
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
            e = cudaMemcpyAsync(out_attr_host, d_oattr, 56 * es * (size_t)n_keep, cudaMemcpyDeviceToHost, s);
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
    c->timing = enable != 0;
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

}  // extern "C"

// ==================================================================== batch

struct refine_batch {
    refine_ctx *ctx = nullptr;
    std::vector<refine_job> jobs;
    refine_params params;
    int dtype = REFINE_F32;
    std::vector<ScenePlan> plans;
    std::vector<SceneScratch> sx;
    std::vector<void *> sel_scr, cmp_scr;
    std::vector<int64_t> n_keep;
    std::vector<unsigned int *> kstar;
    std::vector<long long *> total;
    void *scratch = nullptr;
    void *h_res = nullptr;  // pinned read-back area
    ScoreLaunch *d_launch = nullptr;
    long long *d_tile_begin = nullptr;
    unsigned long long *d_counter = nullptr;
    long long total_tiles = 0;
    int max_v = 0;
    int grid = 1;
    cudaStream_t main = nullptr;
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> events;  // fork, join[lanes], fork2, join2[lanes]
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches_per_run = 0;
};

namespace {

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
    e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), m);
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
    if (e == cudaSuccess && !st) {
        BatchLaunch bl;
        bl.scenes = b->d_launch;
        bl.tile_begin = b->d_tile_begin;
        bl.n_scenes = S;
        bl.total_tiles = b->total_tiles;
        bl.counter = b->d_counter;
        bl.status = c->d_status;
        e = launch_score_batch(bl, b->dtype, (b->params.flags & REFINE_FLAG_NO_PROJ) != 0, b->max_v, b->grid, m);
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

}  // namespace

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
    b->dtype = jobs[0].scene.dtype;
    size_t total = carve_size({sizeof(ScoreLaunch) * (size_t)S, sizeof(long long) * (size_t)(S + 1),
                               sizeof(unsigned long long)});
    for (int j = 0; j < S; ++j) {
        const refine_job &jb = jobs[j];
        if ((st = check_score_args(c, &jb.scene, jb.cams_dev, jb.n_views, p, jb.scores_dev))) {
            delete b;
            return fail(c, st, "batch job %d: %s", j, std::string(c->err).c_str());
        }
        if (jb.scene.n < 1 || jb.scene.dtype != b->dtype || jb.n_views > kViewsPerPass || !jb.keep_mask_dev ||
            !(jb.ratio >= 0.0 && jb.ratio < 1.0)) {
            delete b;
            return fail(c, REFINE_EINVAL,
                        "batch job %d: needs n >= 1, one dtype for all jobs, n_views <= %d, a keep mask and a ratio "
                        "in [0, 1)",
                        j, kViewsPerPass);
        }
        const int64_t nk = jb.scene.n - (int64_t)floor(jb.ratio * (double)jb.scene.n);
        if (jb.out_pos_dev && (!jb.out_attr_dev || jb.out_row_stride < nk)) {
            delete b;
            return fail(c, REFINE_EINVAL, "batch job %d: compaction output missing or shorter than n_keep", j);
        }
        b->n_keep.push_back(nk);
        b->plans.push_back(plan_scene(c, &jb.scene, jb.n_views));
        total += scene_bytes(b->plans.back()) + select_bytes(jb.scene.n) + compact_bytes(jb.scene.n) + 768;
        b->max_v = std::max(b->max_v, jb.n_views);
    }
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
    b->d_launch = cv.take<ScoreLaunch>(S);
    b->d_tile_begin = cv.take<long long>(S + 1);
    b->d_counter = cv.take<unsigned long long>(1);
    std::vector<ScoreLaunch> hl(S);
    std::vector<long long> tb(S + 1, 0);
    const long long tile = (long long)kScoreThreads * kScoreGPT;
    for (int j = 0; j < S; ++j) {
        b->sx.push_back(carve_scene(cv, b->plans[j]));
        b->sel_scr.push_back(cv.take<char>(select_bytes(jobs[j].scene.n)));
        b->cmp_scr.push_back(cv.take<char>(compact_bytes(jobs[j].scene.n)));
        hl[j] = make_score_launch(&jobs[j].scene, b->plans[j], b->sx[j], p, 0, jobs[j].scores_dev, nullptr, false,
                                  c->d_status);
        tb[j + 1] = tb[j] + (jobs[j].scene.n + tile - 1) / tile;
    }
    b->kstar.assign(S, nullptr);
    b->total.assign(S, nullptr);
    b->total_tiles = tb[S];
    e = cudaMemcpy(b->d_launch, hl.data(), sizeof(ScoreLaunch) * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tile_begin, tb.data(), sizeof(long long) * (S + 1), cudaMemcpyHostToDevice);
    b->grid = score_batch_grid(c->num_sms, b->dtype, (p.flags & REFINE_FLAG_NO_PROJ) != 0, b->max_v);
    if (b->grid > b->total_tiles) b->grid = (int)b->total_tiles;
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
