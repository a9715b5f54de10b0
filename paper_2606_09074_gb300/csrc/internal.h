// Host-side declarations of the kernel launchers.  Each launch_* enqueues
// exactly one kernel on `stream` and returns the launch error.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "refine.h"
#include "common.cuh"

namespace refine {

// Cameras processed per score launch at most (144 bytes each in shared
// memory).  A larger view set is split into passes (camera blocks) of
// ScoreShape::views_per_pass views, a multiple of 32; a primitive's running
// Kahan pair (sum, compensation) is carried from pass to pass, so its sum
// is the same whatever the block size.
constexpr int kViewsPerPass = 512;
constexpr int kScoreThreads = 256;     // threads per CTA of k_score

// Work-item shape of the score kernels, chosen per device by the autotuner
// (refine_autotune).  Every primitive's score is computed by one thread with
// the views in a fixed order, whatever tile it is in, so the shape changes
// speed only, never a result.
struct ScoreShape {
    int gpt = 2;          // primitives per thread: a warp's tile is 32 * gpt primitives (1 or 2)
    int threads = 256;    // threads per CTA of the batched kernel (128 or 256); k_score uses kScoreThreads
    int ctas_per_sm = 0;  // cap on resident CTAs per SM of the batched kernel (0 = as many as fit)
    int views_per_pass = kViewsPerPass;  // camera block: views per score pass (32..512, a multiple of 32)
};
bool shape_valid(const ScoreShape &sh);
// An item of the batched kernel: `rounds` warp tiles per warp of the CTA
// (1, 2 or 4), of one scene; the CTA's warps share them out dynamically.
// Large items cost fewer CTA barriers and counter atomics; a launch with
// little work takes smaller ones, so that every CTA gets several items and
// the launch does not end on a few long ones (batch_rounds).  Warp tiles
// stay 32 * gpt aligned within a scene either way.
constexpr int kBatchRounds = 4;
inline int64_t batch_tile(const ScoreShape &sh, int rounds = kBatchRounds)
{
    return (int64_t)sh.threads * sh.gpt * rounds;
}
// The largest item (4, 2 or 1 rounds) that leaves at least 4 items per CTA
// of a grid of `grid` CTAs over scenes of n[0..k) primitives.
inline int batch_rounds(const ScoreShape &sh, const int64_t *n, int k, int grid)
{
    for (int r = kBatchRounds; r > 1; r /= 2) {
        const int64_t t = batch_tile(sh, r);
        int64_t items = 0;
        for (int i = 0; i < k; ++i) items += (n[i] + t - 1) / t;
        if (items >= 4 * (int64_t)grid) return r;
    }
    return 1;
}
constexpr int kFeatThreads = 256;

// Spatial cells for the processing order of k_score: a 2^b x 2^b x 2^b grid
// over the scene's mean +- 3 sigma box, numbered in Morton order, with b the
// largest value in [kMinCellBits, kMaxCellBits] that leaves ~0.5 primitives
// per cell or more (cell_bits_for).  Fine cells keep the counting sort's
// atomics spread out: dense scenes put hundreds of centres in one coarse
// cell, and atomics on one address serialise.
constexpr int kMinCellBits = 4;
constexpr int kMaxCellBits = 7;
constexpr int kScanThreads = 1024;
constexpr int kScanCells = 4 * kScanThreads;  // cells per block of the cell scan (4 per thread)
inline int cell_bits_for(int64_t n)
{
    int b = kMinCellBits;
    while (b < kMaxCellBits && (int64_t(1) << (3 * (b + 1))) <= n * 2) ++b;
    return b;
}
inline int cell_count(int bits) { return 1 << (3 * bits); }
// Keys of the processing order: the cell, plus cell_count(bits) for the
// primitives with large scales (ln s_max > SceneConsts::big_ls), which
// thereby follow all the others.
inline int order_keys(int bits) { return 2 * cell_count(bits); }
constexpr double kSizeSplitSd = 1.28;

// Diagnostic counters of k_score (written only when ScoreLaunch::need is set).
enum {
    kCntTiles = 0,     // (warp tile, view) classifications
    kCntInPairs,       // pairs in tiles classified entirely visible
    kCntOutPairs,      // pairs in tiles classified entirely invisible
    kCntMixedPairs,    // pairs evaluated one by one
    kCntBoundPairs,    // of those: centre outside the image, in the depth range
    kCntExactPairs,    // of those: within the conservative footprint radius
    kCntVisMixed,      // pairs evaluated one by one and found visible
    kCntOpenX,         // pairs evaluated one by one with the u axis open (U computed)
    kCntOpenY,         //   ... with the v axis open (V computed)
    kCntOpenZ,         //   ... with the depth range open (compared)
    kCntBoundX,        // bound-stage pairs with the u axis open
    kCntBoundY,        // bound-stage pairs with the v axis open
    kCntExactX,        // exact-stage pairs whose u extent was needed (centre beyond u)
    kCntExactY,        // exact-stage pairs whose v extent was needed
    kCntExactWarpAxes, // warp-level executions of one axis of the exact test
    kCountSlots
};

// Per-primitive record written by the feature pass, in scene order (64 B):
//   a = (mu.x, mu.y, mu.z, b2)   b2 = 9 s_max^2 (1 + 2^-10), the footprint
//                                bound factor; -(1 + b2) when a scale
//                                underflowed to 0
//   b, c, d.x = L, row-major 3x3 with rows 3 s_k r_k (r_k the k-th column of
//                R(q)), so that L^T L = 9 Sigma
//   d.y = alpha, d.z = m_gem, d.w = m_col
struct __align__(16) PrimRec {
    float4 a, b, c, d;
};
static_assert(sizeof(PrimRec) == 64, "primitive record layout");

struct ScoreLaunch {
    const PrimRec *recs;        // records in scene order
    int64_t n;
    const uint32_t *perm;       // processing order (a permutation of 0..n-1)
    const CamRec *cams;         // this pass's cameras (device, 16-byte aligned)
    int vcount;                 // cameras in this pass
    int first, last;            // first / last pass of the view set
    float eta;
    float inv_views;            // 1 / |V|
    int flags;
    const SceneConsts *consts;
    float2 *running;            // per-primitive running (sum, Kahan compensation) between passes
    float *scores;
    float *view_sum;            // optional
    unsigned long long *need;   // optional diagnostic counters (kCountSlots), see k_score
    unsigned long long *tiles_taken;  // k_score: warp-tile counter, zero before the launch (required;
                                      // k_score_batch takes its items from BatchLaunch::counter)
    int *status;
    int grid;                   // CTAs (persistent)
};

// What the feature pass forms besides the primitive records: the camera
// records of views 0, vstride, 2 vstride, ... (V of them, spread over its
// blocks) and, in its last block, the scene constants (Eq. 18-19, the
// processing-order grid and size split).
struct FeatureTail {
    const refine_camera *cams;
    int V, vstride;
    CamRec *cam_out;
    refine_params p;
    int cell_bits;
    SceneConsts *consts;
    SceneStats *stats;
    unsigned *done;  // count of finished blocks, zero before the launch
};
int feature_blocks(int64_t n);
cudaError_t launch_features(const float *pos, const void *attr, int dtype, int64_t stride, int64_t n,
                            float eta, const float luma[3], PrimRec *recs, float2 *partials, int *status,
                            const FeatureTail &tail, cudaStream_t s);
cudaError_t launch_cells(const float *pos, const void *attr, int dtype, int64_t stride, int64_t n, int cell_bits,
                         const SceneConsts *consts, uint2 *cell, unsigned *counts, int num_sms, cudaStream_t s);
cudaError_t launch_cell_scan(unsigned *counts, unsigned *off_local, unsigned *bsum, unsigned *done, int cell_bits,
                             cudaStream_t s);
cudaError_t launch_cell_scatter(const uint2 *cell, int64_t n,
                                const unsigned *off_local, const unsigned *bsum, uint32_t *perm,
                                int num_sms, cudaStream_t s);
cudaError_t launch_score(const ScoreLaunch &a, const ScoreShape &sh, cudaStream_t s);
int score_grid(int num_sms, int64_t n, int vcount, const ScoreShape &sh);

// FP32 FMA throughput probe (refine_fma_rate): FLOPs of one launch of
// `iters` steps on `num_sms` SMs, and the launch itself (sink: one float,
// never written).
constexpr int kFmaProbeMaxIters = 1 << 20;  // about 65 ms at the nominal FP32 peak
double fma_probe_flops(int num_sms, int iters);
cudaError_t launch_fma_probe(int num_sms, int iters, float *sink, cudaStream_t s);

// Self-test of the bounded mbarrier wait (refine_selftest_wait).
constexpr uint32_t kSelftestMaxBytes = 1024;
cudaError_t launch_wait_selftest(const void *src, uint32_t bytes, uint32_t missing, long long limit, int *status,
                                 cudaStream_t s);

// Batched score launch over the tiles of many scenes (each scene a single
// pass of at most kViewsPerPass views).
struct BatchLaunch {
    const ScoreLaunch *scenes;       // device [n_scenes]
    const long long *tile_begin;     // device [n_scenes + 1], first tile of each scene
    int n_scenes;
    long long total_tiles;
    unsigned long long *counter;     // device, zero before the launch
    int *status;
    int rounds;                      // warp tiles per warp in an item (batch_tile)
};
int score_batch_grid(int num_sms, int max_vcount, const ScoreShape &sh);
cudaError_t launch_score_batch(const BatchLaunch &b, int max_vcount, int grid, const ScoreShape &sh, cudaStream_t s);

// ------------------------------------------------------------- select
struct SelState {
    unsigned int hist[2048];
    unsigned int done;
    unsigned int prefix;
    unsigned int remaining;
    unsigned int count_gt;
    unsigned int kstar;
    unsigned int cnt_eq;
    unsigned int need_ties;
    unsigned int pad;
    long long idx_cut;
};
constexpr int kTieSeg = 4096;
int select_grid(int num_sms, int64_t n);
cudaError_t launch_select_pass(int pass, const float *scores, int64_t n, uint32_t n_keep,
                               SelState *st, bool vec, int grid, int *status, cudaStream_t s);
cudaError_t launch_select_ties(const float *scores, int64_t n, SelState *st, unsigned *seg_cnt,
                               int grid, cudaStream_t s);
cudaError_t launch_select_mask(const float *scores, int64_t n, const SelState *st, uint32_t *mask,
                               int grid, cudaStream_t s);
cudaError_t launch_mask_fill(uint32_t *mask, int64_t n, cudaStream_t s);

// ------------------------------------------------------------- compact
struct CmpState {
    unsigned int done;
    unsigned int ok;
    long long total;
};
constexpr int kCmpSeg = 256;  // elements per compaction segment (8 mask words)
cudaError_t launch_compact_count(const uint32_t *mask, int64_t n, unsigned *seg_cnt,
                                 unsigned long long *seg_off, CmpState *cs, int64_t out_stride,
                                 int grid, int *status, cudaStream_t s);
struct CmpShape {
    int grid;  // CTAs of the scatter
    bool seg;  // k_compact_seg (a warp per segment) rather than k_compact_warp (a warp per mask word)
};
CmpShape compact_shape(int num_sms, int64_t n, int dtype);
cudaError_t launch_compact_scatter(const refine_scene &in, const uint32_t *mask, const unsigned long long *seg_off,
                                   const CmpState *cs, float *out_pos, void *out_attr, int64_t out_stride,
                                   int32_t *out_idx, CmpShape shape, cudaStream_t s);

}  // namespace refine
