// Internals shared by the C-ABI translation units (refine_api.cu, queue.cu):
// the context, scratch planning and the enqueue_* sequences of the score,
// select and compaction passes.  Every enqueue_* issues its launches through
// a caller-supplied runner, so the same sequence serves the plain calls, the
// graph-captured batch and the request queue.
#pragma once
#include <float.h>
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

namespace refine_api {

enum KClass {
    K_FEATURES = 0,
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
    K_SELFTEST,
    K_FMA_PROBE,
    K_NCLASS
};
const char *const kClassName[K_NCLASS] = {"features",
                                          "cells",         "cell_scan",    "cell_scatter",
                                          "score",         "select_pass",  "select_ties",
                                          "select_mask",   "mask_fill",    "compact_count",
                                          "compact_scatter", "selftest",   "fma_probe"};

struct Arena {
    void *p = nullptr;
    size_t cap = 0;
};

struct Pending {
    int cls;
    cudaEvent_t a, b;
};

// Bump allocator over an arena.  Every sub-block starts on a 256-byte boundary of the address space (not
// merely of the offset), so a carved region is aligned even when the arena's
// base is not; carve_size() is a multiple of 256 that covers that padding.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *p) : base(static_cast<char *>(p)) {}
    template <typename T>
    T *take(size_t count)
    {
        const uintptr_t at = (reinterpret_cast<uintptr_t>(base) + off + 255) & ~uintptr_t(255);
        off = at - reinterpret_cast<uintptr_t>(base);
        T *r = reinterpret_cast<T *>(at);
        off += count * sizeof(T);
        return r;
    }
};

inline size_t carve_size(std::initializer_list<size_t> parts)
{
    size_t off = 0;
    for (size_t p : parts) off = ((off + 255) & ~size_t(255)) + p;
    return ((off + 255) & ~size_t(255)) + 256;
}

}  // namespace refine_api

struct refine_ctx {
    int device = 0;
    int num_sms = 0;
    char err[512] = {0};
    int *d_status = nullptr;
    void *h_small = nullptr;  // pinned 4 KB for read-backs
    refine_api::Arena score, select, compact, host;
    int timing = 0;  // 0, REFINE_TIMING_ALL or REFINE_TIMING_SCORE
    std::vector<refine_api::Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[refine_api::K_NCLASS] = {0};
    int64_t launches[refine_api::K_NCLASS] = {0};
    int64_t launch_count = 0;
    refine::ScoreShape shape;  // work-item shape of the score kernels (refine_autotune)
};

namespace refine_api {

inline refine_status fail(refine_ctx *c, refine_status st, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

inline refine_status cuda_fail(refine_ctx *c, cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear non-sticky errors
    return fail(c, e == cudaErrorMemoryAllocation ? REFINE_ENOMEM : REFINE_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

inline refine_status use_device(refine_ctx *c)
{
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != c->device) {
        cudaError_t e = cudaSetDevice(c->device);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    }
    return REFINE_OK;
}

inline refine_status ensure(refine_ctx *c, Arena &a, size_t bytes)
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

inline cudaEvent_t take_event(refine_ctx *c)
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
inline refine_status launch(refine_ctx *c, int cls, cudaStream_t s, F &&f)
{
    cudaEvent_t a = nullptr, b = nullptr;
    const bool timed = c->timing == REFINE_TIMING_ALL || (c->timing == REFINE_TIMING_SCORE && cls == K_SCORE);
    if (timed) {
        a = take_event(c);
        cudaEventRecord(a, s);
    }
    cudaError_t e = f();
    if (e != cudaSuccess) return cuda_fail(c, e, kClassName[cls]);
    if (timed) {
        b = take_event(c);
        cudaEventRecord(b, s);
        c->pending.push_back({cls, a, b});
    }
    c->launch_count++;
    c->launches[cls]++;
    return REFINE_OK;
}

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline refine_status check_params(refine_ctx *c, const refine_params *p)
{
    if (!(p->eta >= FLT_MIN) || !isfinite(p->eta))
        return fail(c, REFINE_EINVAL, "params: eta must be finite and at least FLT_MIN (1.18e-38)");
    for (int k = 0; k < 3; ++k)
        if (!isfinite(p->luma[k])) return fail(c, REFINE_EINVAL, "params: luma must be finite");
    if (!(isfinite(p->e_ln_gem) && p->e_ln_gem != 0.0 && isfinite(p->e_col) && p->e_col != 0.0 &&
          isfinite(p->e_opa) && p->e_opa != 0.0))
        return fail(c, REFINE_EINVAL, "params: calibration constants must be finite and nonzero");
    if (p->max_views < 0) return fail(c, REFINE_EINVAL, "params: max_views must be >= 0");
    return REFINE_OK;
}

inline refine_status check_scene(refine_ctx *c, const refine_scene *s)
{
    if (!s) return fail(c, REFINE_EINVAL, "scene is NULL");
    if (s->n < 0 || s->n > INT32_MAX) return fail(c, REFINE_EINVAL, "scene: n=%lld out of [0, 2^31-1]", (long long)s->n);
    if (!valid_dtype(s->dtype)) return fail(c, REFINE_EINVAL, "scene: unknown dtype %d", s->dtype);
    if (s->n == 0) return REFINE_OK;
    if (!s->pos || !s->attr) return fail(c, REFINE_EINVAL, "scene: NULL pos/attr");
    if (s->row_stride < s->n) return fail(c, REFINE_EINVAL, "scene: row_stride < n");
    if (!aligned16(s->pos) || !aligned16(s->attr)) return fail(c, REFINE_EINVAL, "scene: pos/attr must be 16-byte aligned");
    return REFINE_OK;
}

// Reads back and clears the device status word (synchronises `s`).
inline refine_status read_status(refine_ctx *c, cudaStream_t s)
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
    int V = 0;        // views scored
    int vstride = 1;  // input camera stride (view subsampling)
    int vpp = kViewsPerPass;  // views per pass (the camera block)
    int passes = 1;
    bool multipass = false;
    int nb = 1;    // feature-pass blocks
    int bits = 4;  // processing-order grid resolution
};

struct SceneScratch {
    CamRec *cams;
    PrimRec *recs;
    float2 *partials;  // per feature-pass block, float-float sums
    SceneConsts *consts;
    SceneStats *stats;
    uint2 *cell;  // (cell, slot within the cell) of every primitive
    unsigned *counts;  // order_keys(bits) + 64 words; the two after the keys count the finished blocks of
                       // the cell scan and of the feature pass
    unsigned *off_local;
    unsigned *bsum;
    uint32_t *perm;
    unsigned long long *need;
    unsigned long long *tiles;  // k_score's tile counter
    float2 *running;  // (sum, compensation) per primitive between passes
};

// V input cameras; with 0 < max_views < V every s-th view is scored,
// s = ceil(V / max_views) (Table B.1's view subsampling).  The views scored
// are processed in passes of `vpp` (the camera block of the shape).
inline ScenePlan plan_scene(int64_t n, int V, int max_views = 0, int vpp = kViewsPerPass)
{
    ScenePlan pl;
    pl.n = n;
    pl.vstride = (max_views > 0 && V > max_views) ? (V + max_views - 1) / max_views : 1;
    pl.V = (V + pl.vstride - 1) / pl.vstride;
    pl.vpp = vpp;
    pl.passes = (pl.V + vpp - 1) / vpp;
    pl.multipass = pl.passes > 1;
    pl.nb = feature_blocks(pl.n);
    pl.bits = cell_bits_for(pl.n);
    return pl;
}

inline size_t scene_bytes(const ScenePlan &pl)
{
    const size_t n = (size_t)pl.n, cells = (size_t)order_keys(pl.bits);
    return carve_size({sizeof(CamRec) * (size_t)pl.V, sizeof(PrimRec) * n, sizeof(float2) * kFeatSums * 1024,
                       sizeof(SceneConsts), sizeof(SceneStats), sizeof(uint2) * n,
                       sizeof(unsigned) * (cells + 64), sizeof(unsigned) * cells,
                       sizeof(unsigned) * (cells / kScanCells), sizeof(uint32_t) * n,
                       kCountSlots * sizeof(unsigned long long), sizeof(unsigned long long),
                       pl.multipass ? sizeof(float2) * n : 0});
}

inline SceneScratch carve_scene(Carver &cv, const ScenePlan &pl)
{
    const int64_t n = pl.n;
    const int cells = order_keys(pl.bits);
    SceneScratch x;
    x.cams = cv.take<CamRec>(pl.V);
    x.recs = cv.take<PrimRec>(n);
    x.partials = cv.take<float2>(kFeatSums * 1024);
    x.consts = cv.take<SceneConsts>(1);
    x.stats = cv.take<SceneStats>(1);
    x.cell = cv.take<uint2>(n);
    x.counts = cv.take<unsigned>(cells + 64);
    x.off_local = cv.take<unsigned>(cells);
    x.bsum = cv.take<unsigned>(cells / kScanCells);
    x.perm = cv.take<uint32_t>(n);
    x.need = cv.take<unsigned long long>(kCountSlots);
    x.tiles = cv.take<unsigned long long>(1);
    x.running = pl.multipass ? cv.take<float2>(n) : nullptr;
    return x;
}

// Camera records, content features and lambda, processing order.
template <typename L>
inline refine_status enqueue_prep(refine_ctx *c, L &&run, const refine_scene *sc, const refine_camera *cams,
                           const ScenePlan &pl, const SceneScratch &x, const refine_params &p, bool count,
                           int *status, cudaStream_t s)
{
    const int64_t n = pl.n;
    const int cells = order_keys(pl.bits);
    cudaError_t e = cudaMemsetAsync(x.counts, 0, sizeof(unsigned) * (cells + 64), s);
    if (e == cudaSuccess && count) e = cudaMemsetAsync(x.need, 0, kCountSlots * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
    refine_status st;
    FeatureTail tail;
    tail.cams = cams;
    tail.V = pl.V;
    tail.vstride = pl.vstride;
    tail.cam_out = x.cams;
    tail.p = p;
    tail.cell_bits = pl.bits;
    tail.consts = x.consts;
    tail.stats = x.stats;
    tail.done = x.counts + cells + 1;  // zeroed with the counts above
    if ((st = run(K_FEATURES, [&] {
             return launch_features(sc->pos, sc->attr, sc->dtype, sc->row_stride, n, p.eta, p.luma, x.recs,
                                    x.partials, status, tail, s);
         })))
        return st;
    if ((st = run(K_CELLS, [&] {
             return launch_cells(sc->pos, sc->attr, sc->dtype, sc->row_stride, n, pl.bits, x.consts, x.cell,
                                 x.counts, c->num_sms, s);
         })))
        return st;
    if ((st = run(K_CELL_SCAN,
                  [&] { return launch_cell_scan(x.counts, x.off_local, x.bsum, x.counts + cells, pl.bits, s); })))
        return st;
    return run(K_CELL_SCATTER,
               [&] { return launch_cell_scatter(x.cell, n, x.off_local, x.bsum, x.perm, c->num_sms, s); });
}

inline ScoreLaunch make_score_launch(const refine_scene *sc, const ScenePlan &pl, const SceneScratch &x,
                              const refine_params &p, int v0, float *scores, float *view_sum, bool count, int *status)
{
    ScoreLaunch a;
    a.recs = x.recs;
    a.perm = x.perm;
    a.n = pl.n;
    a.cams = x.cams + v0;
    a.vcount = pl.V - v0 < pl.vpp ? pl.V - v0 : pl.vpp;
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
    a.tiles_taken = nullptr;
    a.status = status;
    a.grid = 0;
    return a;
}

inline refine_status check_score_args(refine_ctx *c, const refine_scene *sc, const refine_camera *cams, int V,
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

inline refine_status score_impl(refine_ctx *c, const refine_scene *sc, const refine_camera *cams, int V,
                         const refine_params *pin, float *scores, float *view_sum, SceneStats **stats_dev,
                         unsigned long long **need_dev, cudaStream_t s)
{
    refine_params p;
    if (pin) p = *pin; else refine_params_default(&p);
    refine_status st = check_score_args(c, sc, cams, V, p, scores);
    if (st || sc->n == 0) return st;
    const ScenePlan pl = plan_scene(sc->n, V, p.max_views, c->shape.views_per_pass);
    if ((st = ensure(c, c->score, scene_bytes(pl)))) return st;
    Carver cv(c->score.p);
    const SceneScratch x = carve_scene(cv, pl);
    if (stats_dev) *stats_dev = x.stats;
    if (need_dev) *need_dev = x.need;
    auto run = [&](int cls, auto &&f) { return launch(c, cls, s, f); };
    if ((st = enqueue_prep(c, run, sc, cams, pl, x, p, need_dev != nullptr, c->d_status, s))) return st;
    for (int v0 = 0; v0 < pl.V; v0 += pl.vpp) {
        ScoreLaunch a = make_score_launch(sc, pl, x, p, v0, scores, view_sum, need_dev != nullptr, c->d_status);
        a.grid = score_grid(c->num_sms, pl.n, a.vcount, c->shape);
        a.tiles_taken = x.tiles;
        const cudaError_t e = cudaMemsetAsync(x.tiles, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
        if ((st = launch(c, K_SCORE, s, [&] { return launch_score(a, c->shape, s); }))) return st;
    }
    return REFINE_OK;
}

// ----------------------------------------------------------------- select
inline size_t select_bytes(int64_t n)
{
    return carve_size({sizeof(SelState), sizeof(unsigned) * (size_t)((n + kTieSeg - 1) / kTieSeg)});
}

// Radix select into the given state; *kstar_dev is NULL when nothing is pruned.
template <typename L>
inline refine_status enqueue_select(refine_ctx *c, L &&run, const float *scores, int64_t n, int64_t n_keep,
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

inline refine_status select_impl(refine_ctx *c, const float *scores, int64_t n, double ratio, uint32_t *mask,
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

inline refine_status read_threshold(refine_ctx *c, unsigned int *kstar_dev, float *thr, cudaStream_t s)
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
inline size_t compact_bytes(int64_t n)
{
    const size_t nseg = (size_t)((n + kCmpSeg - 1) / kCmpSeg);
    return carve_size({sizeof(CmpState), sizeof(unsigned) * nseg, sizeof(unsigned long long) * nseg});
}

template <typename L>
inline refine_status enqueue_compact(refine_ctx *c, L &&run, const refine_scene *in, const uint32_t *mask, float *out_pos,
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
    const CmpShape sshape = compact_shape(c->num_sms, n, in->dtype);
    if ((st = run(K_CMP_SCATTER, [&] {
             return launch_compact_scatter(*in, mask, seg_off, cs, out_pos, out_attr, out_stride, idx, sshape, s);
         })))
        return st;
    *total_dev = &cs->total;
    return REFINE_OK;
}

inline refine_status compact_impl(refine_ctx *c, const refine_scene *in, const uint32_t *mask, float *out_pos,
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

}  // namespace refine_api
