// Scoring kernels: camera preparation, the content-feature pass (Eq.
// (features), Eq. 18-19), the spatial processing order, and the N x V
// importance kernel (Eq. 7, Eq. 20).
#include <math.h>

#include "internal.h"

namespace refine {

// ---------------------------------------------------------------------
// Camera preparation: refine_camera -> CamRec (P = K W and p = K t formed
// in double and rounded once), with validation.
// ---------------------------------------------------------------------
__device__ void prep_camera(const refine_camera *__restrict__ cams, int v, int vstride, CamRec *__restrict__ out,
                            int *status)
{
    refine_camera c = cams[(int64_t)v * vstride];
    bool ok = isfinite(c.fx) && isfinite(c.fy) && isfinite(c.cx) && isfinite(c.cy) &&
              isfinite(c.znear) && isfinite(c.zfar) && c.fx > 0.f && c.fy > 0.f &&
              c.width >= 1 && c.height >= 1 && c.znear > 0.f && c.zfar > c.znear;
    for (int k = 0; k < 9; ++k) ok = ok && isfinite(c.R[k]);
    for (int k = 0; k < 3; ++k) ok = ok && isfinite(c.t[k]);
    CamRec r;
    if (!ok) {
        set_status(status, kEinval);
        r.r0 = make_float4(0.f, 0.f, 0.f, 0.f);
        r.r1 = r.r0;
        r.r2 = r.r0;
        r.lim = make_float4(0.f, 0.f, 1.f, 0.f);  // znear > zfar: never visible
        r.k = r.r0;
        r.uw = r.vh = r.tx = r.ty = r.r0;
        out[v] = r;
        return;
    }
    double fx = c.fx, fy = c.fy, cx = c.cx, cy = c.cy;
    r.r0 = make_float4((float)(fx * c.R[0] + cx * c.R[6]), (float)(fx * c.R[1] + cx * c.R[7]),
                       (float)(fx * c.R[2] + cx * c.R[8]), (float)(fx * c.t[0] + cx * c.t[2]));
    r.r1 = make_float4((float)(fy * c.R[3] + cy * c.R[6]), (float)(fy * c.R[4] + cy * c.R[7]),
                       (float)(fy * c.R[5] + cy * c.R[8]), (float)(fy * c.t[1] + cy * c.t[2]));
    r.r2 = make_float4(c.R[6], c.R[7], c.R[8], c.t[2]);
    r.lim = make_float4((float)c.width, (float)c.height, c.znear, c.zfar);
    r.k = make_float4((float)(fx * fx), (float)(fy * fy), c.cx, c.cy);
    const double w = c.width, h = c.height;
    r.uw = make_float4((float)(fx * c.R[0] + (cx - w) * c.R[6]), (float)(fx * c.R[1] + (cx - w) * c.R[7]),
                       (float)(fx * c.R[2] + (cx - w) * c.R[8]), (float)(fx * c.t[0] + (cx - w) * c.t[2]));
    r.vh = make_float4((float)(fy * c.R[3] + (cy - h) * c.R[6]), (float)(fy * c.R[4] + (cy - h) * c.R[7]),
                       (float)(fy * c.R[5] + (cy - h) * c.R[8]), (float)(fy * c.t[1] + (cy - h) * c.t[2]));
    r.tx = make_float4((float)(fx * c.R[0]), (float)(fx * c.R[1]), (float)(fx * c.R[2]), (float)(fx * c.t[0]));
    r.ty = make_float4((float)(fy * c.R[3]), (float)(fy * c.R[4]), (float)(fy * c.R[5]), (float)(fy * c.t[1]));
    out[v] = r;
}

// Eq. (features) -> Eq. 18 -> Eq. 19 in double, by one block (every thread
// calls it); also the grid box (mean +- 3 sigma of the means) and the size
// split of the processing order.
__device__ void finalize_features(const float2 *partials, int nblocks, int64_t n, const refine_params &p,
                                  int cell_bits, SceneConsts *consts, SceneStats *stats)
{
    // each sum k is reduced by one warp over the block partials in a fixed
    // order (lane-strided, then a shuffle tree) in float-float, whichever
    // warp it is, and converted to double once
    __shared__ double red[kFeatSums][1];
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int k = threadIdx.x >> 5; k < kFeatSums; k += nwarps) {
        FF v = {0.f, 0.f};
#pragma unroll 4
        for (int b = lane; b < nblocks; b += 32) {
            const float2 q = __ldcg(partials + (int64_t)b * kFeatSums + k);
            v = ff_add(v, FF{q.x, q.y});
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v = ff_add(v, FF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
        if (lane == 0) red[k][0] = ff_to_double(v);
    }
    __syncthreads();
    // The scalar tail in double, spread over three threads: thread t forms
    // lambda~ of attribute t (Eq. 18), then its lambda, kappa (Eq. 19) and
    // the grid box along axis t, each by the same expression as a one-thread
    // evaluation would use.
    __shared__ double lam_t[3];
    const int t = threadIdx.x;
    const double N = (double)n;
    if (t < 3) {
        double lt;
        if (t == 0) {
            lt = log(red[3][0] / N + (double)p.eta) / p.e_ln_gem;
        } else if (t == 1) {
            const double ybar = red[0][0] / N;
            double fc = red[1][0] / N - ybar * ybar;
            if (fc < 0.0) fc = 0.0;
            lt = fc / p.e_col;
            if (stats) stats->F_col = fc;
        } else {
            lt = (red[2][0] / N) / p.e_opa;
        }
        if (!(lt > 0.0)) lt = 0.0;
        lam_t[t] = lt;
    }
    __syncthreads();
    if (t >= 3) return;  // no barrier follows
    const double tot = (lam_t[0] + lam_t[1]) + lam_t[2];
    const double lambda = ((p.flags & REFINE_FLAG_EQUAL_LAMBDA) || tot == 0.0) ? 1.0 / 3.0 : lam_t[t] / tot;
    const double mean_m = red[4 + t][0] / N;
    double kap = lambda;
    if (p.flags & REFINE_FLAG_NORM_ATTR) kap = mean_m > 0.0 ? lambda / mean_m : 0.0;
    consts->kappa[t] = (float)kap;
    const double mean = red[7 + t][0] / N;
    const double var = red[10 + t][0] / N - mean * mean;
    const double sd = var > 0.0 ? sqrt(var) : 0.0;
    consts->lo[t] = (float)(mean - 3.0 * sd);
    consts->qscale[t] = sd > 0.0 && isfinite(sd) ? (float)((1 << cell_bits) / (6.0 * sd)) : 0.f;
    if (t < 2) consts->pad[t] = 0.f;
    if (t == 0) {
        // The primitives whose ln s_max lies above its scene mean + 1.28 sd
        // (the largest ~10 % for a normal spread) are ordered after all the
        // others, so that the tiles of the rest carry small footprint bounds.
        const double ml = red[13][0] / N, vl = red[14][0] / N - ml * ml;
        const double big = ml + kSizeSplitSd * (vl > 0.0 ? sqrt(vl) : 0.0);
        consts->big_ls = isfinite(big) ? (float)big : INFINITY;
    }
    if (stats) {
        stats->lambda_t[t] = lam_t[t];
        stats->lambda[t] = lambda;
        stats->mean_m[t] = mean_m;
        if (t == 0) {
            stats->F_opa = red[2][0] / N;
            stats->F_gem = red[3][0] / N;
        }
    }
}

// ---------------------------------------------------------------------
// Content features.  One primitive per thread: its 59 attribute rows are
// read with coalesced loads (all in flight at once), its record and its
// feature terms formed (primitive_record), fifteen sums per thread kept in
// float and reduced per block in a fixed float-float order.  The camera
// records (prep_camera, in double) are spread over the blocks, one camera
// per thread, blocks first, before the primitives.  The block that
// finishes last (a count of finished blocks, no waiting) then forms the
// scene constants from all blocks' sums (finalize_features), which saves
// two small launches per scene.
// ---------------------------------------------------------------------
constexpr int kFeatRedLanes = 16;                                 // threads per sum in the block reduction
constexpr int kFeatRedRow = kFeatThreads + kFeatRedLanes;         // padded row: two sums of a warp hit
                                                                  // different banks
static_assert(kFeatSums * kFeatRedLanes <= kFeatThreads, "one reduction thread per (sum, lane)");
static_assert(kFeatThreads % kFeatRedLanes == 0, "whole columns per reduction lane");

template <int DT>
__global__ void __launch_bounds__(kFeatThreads, 4) k_features(const float *__restrict__ pos,
                                                           AttrRows<DT> attr, int64_t S, int64_t n,
                                                           float eta, float l0, float l1, float l2,
                                                           PrimRec *__restrict__ recs,
                                                           float2 *__restrict__ partials, int *status,
                                                           FeatureTail tail)
{
    for (int64_t v = blockIdx.x + (int64_t)gridDim.x * threadIdx.x; v < tail.V;
         v += (int64_t)gridDim.x * blockDim.x)
        prep_camera(tail.cams, (int)v, tail.vstride, tail.cam_out, status);

    FeatSums acc;
#pragma unroll
    for (int k = 0; k < kFeatSums; ++k) acc.s[k] = 0.f;
    acc.bad = 0.f;
    bool zero_q = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float sq = 0.f;
#pragma unroll
        for (int r = 8; r < 56; ++r) {
            const float x = attr.ld(r, i);
            sq = fmaf(x, x, sq);
        }
        float4 ra, rb, rc, rd;
        primitive_record(acc, __ldg(pos + i), __ldg(pos + S + i), __ldg(pos + 2 * S + i), attr.ld(0, i),
                         attr.ld(1, i), attr.ld(2, i), attr.ld(3, i), attr.ld(4, i), attr.ld(5, i), attr.ld(6, i),
                         attr.ld(7, i), attr.ld(8, i), attr.ld(9, i), attr.ld(10, i), sq, eta, l0, l1, l2, ra, rb,
                         rc, rd, zero_q);
        PrimRec *r = recs + i;
        r->a = ra; r->b = rb; r->c = rc; r->d = rd;
    }
    if (!isfinite(acc.bad)) set_status(status, kEnonfinite);
    if (zero_q) set_status(status, kEinval);

    // Block sums in float-float: thread (k, j) adds the values of threads
    // j, j + 16, j + 32, ... of sum k in that order, then the 16 lanes of
    // sum k meet in a shuffle tree (xor 8, 4, 2, 1).
    __shared__ float red[kFeatSums * kFeatRedRow];
#pragma unroll
    for (int k = 0; k < kFeatSums; ++k) red[k * kFeatRedRow + threadIdx.x] = acc.s[k];
    __syncthreads();
    if (threadIdx.x < kFeatSums * kFeatRedLanes) {
        const int k = threadIdx.x / kFeatRedLanes, j = threadIdx.x % kFeatRedLanes;
        const float *col = red + k * kFeatRedRow + j;
        FF v = {col[0], 0.f};
#pragma unroll
        for (int t = kFeatRedLanes; t < kFeatThreads; t += kFeatRedLanes) v = ff_add(v, FF{col[t], 0.f});
        // lanes of other sums in the same warp run the same tree on their own
        // 16-lane groups (xor below 16 stays within a group); the last warp
        // may hold reduction threads in its low lanes only
        constexpr int kRedThreads = kFeatSums * kFeatRedLanes;
        const unsigned grp = (int)(threadIdx.x | 31u) < kRedThreads ? 0xffffffffu : (1u << (kRedThreads & 31)) - 1u;
#pragma unroll
        for (int o = kFeatRedLanes / 2; o > 0; o >>= 1)
            v = ff_add(v, FF{__shfl_xor_sync(grp, v.hi, o), __shfl_xor_sync(grp, v.lo, o)});
        if (j == 0) partials[(int64_t)blockIdx.x * kFeatSums + k] = make_float2(v.hi, v.lo);
    }

    // the last block to finish: scene constants
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(tail.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    finalize_features(partials, gridDim.x, n, tail.p, tail.cell_bits, tail.consts, tail.stats);
}

// A single wave on a 152-SM part (4 CTAs of 256 threads per SM); the grid
// depends only on n, so the per-block sums, and the scene constants, do too.
int feature_blocks(int64_t n)
{
    int64_t b = (n + (int64_t)kFeatThreads * 8 - 1) / ((int64_t)kFeatThreads * 8);
    if (b < 1) b = 1;
    if (b > 608) b = 608;
    return (int)b;
}

cudaError_t launch_features(const float *pos, const void *attr, int dtype, int64_t stride, int64_t n,
                            float eta, const float luma[3], PrimRec *recs, float2 *partials, int *status,
                            const FeatureTail &tail, cudaStream_t s)
{
    const int nb = feature_blocks(n);
    if (dtype == REFINE_BF16)
        k_features<REFINE_BF16><<<nb, kFeatThreads, 0, s>>>(pos, AttrRows<REFINE_BF16>(attr, stride), stride, n, eta,
                                                            luma[0], luma[1], luma[2], recs, partials, status, tail);
    else if (dtype == REFINE_BF16S)
        k_features<REFINE_BF16S><<<nb, kFeatThreads, 0, s>>>(pos, AttrRows<REFINE_BF16S>(attr, stride), stride, n,
                                                             eta, luma[0], luma[1], luma[2], recs, partials, status,
                                                             tail);
    else
        k_features<REFINE_F32><<<nb, kFeatThreads, 0, s>>>(pos, AttrRows<REFINE_F32>(attr, stride), stride, n, eta,
                                                           luma[0], luma[1], luma[2], recs, partials, status, tail);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------
// Processing order.  Primitives are sorted by their cell in a 2^b x 2^b x
// 2^b grid over the mean +- 3 sigma box of the centres, cells numbered in
// Morton order (a counting sort: count, scan, scatter), so that the 32
// lanes of a warp hold nearby primitives and tend to take the same side of
// each view's frustum edges.  The primitives with the largest scales (ln
// s_max above SceneConsts::big_ls) come after all the others, in their own
// cells, so that a tile's footprint bound (set by its largest s_max) is not
// set by a few large primitives among small ones.  The order only affects speed: every
// primitive's score is computed by one thread with the views in a fixed
// order, whatever its position, so the sort need not be stable (the
// count atomics order the primitives of a cell arbitrarily).  Each
// thread keeps kSortU primitives in flight.
// ---------------------------------------------------------------------
constexpr int kSortU = 4;

__device__ __forceinline__ uint32_t spread3(uint32_t x)
{
    uint32_t r = 0;
#pragma unroll
    for (int b = 0; b < kMaxCellBits; ++b) r |= ((x >> b) & 1u) << (3 * b);
    return r;
}

__device__ __forceinline__ uint32_t quantise(float x, float lo, float qs, float top)
{
    return (uint32_t)fminf(fmaxf((x - lo) * qs, 0.f), top);
}

template <int DT>
__global__ void k_cells(const float *__restrict__ pos, AttrRows<DT> attr, int64_t stride, int64_t n,
                        int cell_bits, const SceneConsts *__restrict__ consts, uint2 *__restrict__ cell,
                        unsigned *__restrict__ counts)
{
    const SceneConsts c = *consts;
    const float top = (float)((1 << cell_bits) - 1);
    const uint32_t big_key = 1u << (3 * cell_bits);
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += kSortU * step) {
        float x[kSortU], y[kSortU], z[kSortU], ls[kSortU];
#pragma unroll
        for (int u = 0; u < kSortU; ++u) {
            const int64_t j = i + u * step;
            const bool ok = j < n;
            x[u] = ok ? __ldg(pos + j) : 0.f;
            y[u] = ok ? __ldg(pos + stride + j) : 0.f;
            z[u] = ok ? __ldg(pos + 2 * stride + j) : 0.f;
            ls[u] = ok ? fmaxf(attr.ld(0, j), fmaxf(attr.ld(1, j), attr.ld(2, j))) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kSortU; ++u) {
            const int64_t j = i + u * step;
            if (j >= n) break;
            const uint32_t id = (spread3(quantise(x[u], c.lo[0], c.qscale[0], top)) |
                                 (spread3(quantise(y[u], c.lo[1], c.qscale[1], top)) << 1) |
                                 (spread3(quantise(z[u], c.lo[2], c.qscale[2], top)) << 2)) +
                                (ls[u] > c.big_ls ? big_key : 0u);
            cell[j] = make_uint2(id, atomicAdd(&counts[id], 1u));  // the key and the slot in it
        }
    }
}

static int sort_grid(int num_sms, int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > (int64_t)num_sms * 8) g = (int64_t)num_sms * 8;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_cells(const float *pos, const void *attr, int dtype, int64_t stride, int64_t n, int cell_bits,
                         const SceneConsts *consts, uint2 *cell, unsigned *counts, int num_sms, cudaStream_t s)
{
    const int g = sort_grid(num_sms, n);
    if (dtype == REFINE_BF16)
        k_cells<REFINE_BF16><<<g, 256, 0, s>>>(pos, AttrRows<REFINE_BF16>(attr, stride), stride, n, cell_bits, consts,
                                               cell, counts);
    else if (dtype == REFINE_BF16S)
        k_cells<REFINE_BF16S><<<g, 256, 0, s>>>(pos, AttrRows<REFINE_BF16S>(attr, stride), stride, n, cell_bits,
                                                consts, cell, counts);
    else
        k_cells<REFINE_F32><<<g, 256, 0, s>>>(pos, AttrRows<REFINE_F32>(attr, stride), stride, n, cell_bits, consts,
                                              cell, counts);
    return cudaGetLastError();
}

// Exclusive scan of the cell counts: local offsets within blocks of
// kScanCells cells (4 consecutive cells per thread, one 16-byte load), then
// the last block turns the block totals into block offsets, so cell c
// starts at bsum[c / kScanCells] + off_local[c].
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned x = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += x;
    }
    if (lane == 31) wsum[warp] = s;
    __syncthreads();
    if (warp == 0) {
        unsigned w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned x = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += x;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    const unsigned r = s - v + (warp > 0 ? wsum[warp - 1] : 0u);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_cell_scan(const unsigned *__restrict__ counts,
                                                            unsigned *__restrict__ off_local,
                                                            unsigned *bsum, unsigned *done)
{
    __shared__ unsigned wsum[32];
    __shared__ unsigned is_last, carry;
    const int nblocks = gridDim.x;
    const int64_t c4 = (int64_t)blockIdx.x * kScanThreads + threadIdx.x;  // 4 cells from 4 * c4
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(counts) + c4);
    const unsigned tot = v.x + v.y + v.z + v.w;
    const unsigned ex = block_excl_scan(tot, wsum);
    reinterpret_cast<uint4 *>(off_local)[c4] = make_uint4(ex, ex + v.x, ex + v.x + v.y, ex + v.x + v.y + v.z);
    if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = ex + tot;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(done, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) carry = 0u;
    __syncthreads();
    for (int b0 = 0; b0 < nblocks; b0 += kScanThreads) {
        const int bi = b0 + threadIdx.x;
        const unsigned b = bi < nblocks ? __ldcg(bsum + bi) : 0u;
        const unsigned bex = block_excl_scan(b, wsum) + carry;
        __syncthreads();
        if (bi < nblocks) bsum[bi] = bex;
        if (threadIdx.x == kScanThreads - 1) carry = bex + b;
        __syncthreads();
    }
}

cudaError_t launch_cell_scan(unsigned *counts, unsigned *off_local, unsigned *bsum, unsigned *done, int cell_bits,
                             cudaStream_t s)
{
    k_cell_scan<<<order_keys(cell_bits) / kScanCells, kScanThreads, 0, s>>>(counts, off_local, bsum, done);
    return cudaGetLastError();
}

// Primitive j goes to the start of its cell (block offset + offset within
// the block) plus the slot that its count atomic returned in k_cells.
__global__ void k_cell_scatter(const uint2 *__restrict__ cell, int64_t n, const unsigned *__restrict__ off_local,
                               const unsigned *__restrict__ boff, uint32_t *__restrict__ perm)
{
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += kSortU * step) {
        uint2 c[kSortU];
#pragma unroll
        for (int u = 0; u < kSortU; ++u) {
            const int64_t j = i + u * step;
            c[u] = j < n ? __ldg(cell + j) : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kSortU; ++u) {
            const int64_t j = i + u * step;
            if (j < n) perm[__ldg(boff + c[u].x / kScanCells) + __ldg(off_local + c[u].x) + c[u].y] = (uint32_t)j;
        }
    }
}

cudaError_t launch_cell_scatter(const uint2 *cell, int64_t n, const unsigned *off_local, const unsigned *bsum,
                                uint32_t *perm, int num_sms, cudaStream_t s)
{
    k_cell_scatter<<<sort_grid(num_sms, n), 256, 0, s>>>(cell, n, off_local, bsum, perm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------
// The N x V importance kernel.
//
// One thread owns two primitives (the lanes of a warp hold 64 consecutive
// primitives of the processing order, a "tile") and walks every camera of
// the pass; the camera records are staged once per CTA into shared memory by
// a TMA bulk copy.  For primitive i and view v (Eq. 13-14, Eq. 17, Eq. 20):
//   (U, V, z) = P mu + p                  homogeneous pixel, u = U / z
//   d_u z = max(-U, U - w z)              distance of the centre outside
//   d_v z = max(-V, V - h z)              [0,w] x [0,h], times z
//   in range: znear < z < zfar
//   3-sigma box meets the image  <=>  (max(d_u z, 0) z)^2 <= Qx  and
//                                     (max(d_v z, 0) z)^2 <= Qy
//     with g0 = z P0 - U P2, g1 = z P1 - V P2 (the rows of z^2 J W) and
//     Qx = |L g0|^2 = 9 z^4 S_xx, Qy = |L g1|^2 = 9 z^4 S_yy, L = 3 diag(s)
//     R(q)^T, i.e. Sigma2D = J W Sigma W^T J^T formed through the square
//     root of Sigma (well conditioned in float).
//   det Sigma2D = |L g0 x L g1|^2 / (81 z^8) > 0 whenever all three scales
//     are nonzero (L invertible, g0 and g1 independent); a warp holding a
//     primitive with an underflowed scale evaluates it on every pair.
//   term = vis / (z^2 + eta)              (Eq. 17, one MUFU reciprocal)
//
// Work is skipped only where the outcome is already implied, so every
// decision equals the full test's, bit for bit:
//  * per tile (the bounding box of its 64 centres) and view, a lane classifies
//    one view (32 views at a time) with interval bounds of the linear forms
//    U, V, z, U - w z, V - h z, fx x, fy y over the box, plus a 2^-14
//    relative slack that covers float32 rounding:
//      IN   every centre is in range and inside the image: vis = 1 for all
//      OUT  every centre is out of range, or outside an image edge by more
//           than the footprint bound below: vis = 0, the view is skipped
//      MIXED otherwise: decided pair by pair;
//  * pair by pair, in two warp-uniform stages entered only when some lane
//    needs them: a centre inside the image is visible whatever Sigma2D; a
//    centre outside is first tested against Qx <= 9 s_max^2 ((U - cx z)^2 +
//    fx^2 z^2) (as |g0|^2 = fx^2 (x^2 + z^2); inflated by 2^-10), and only
//    lanes passing that bound need Qx and Qy.
// Views are summed in blocks of 32, in view order (an invisible or skipped
// view adds +0, which changes nothing), and the block sums are added to the
// primitive's total with Kahan compensation, so a primitive's sum does not
// depend on the tile it is in and its rounding error does not grow with V.
// The epilogue forms D_i = alpha_i S_i / |V| * sum_k lambda^k G~_i^k (Eq. 7).
// ---------------------------------------------------------------------
struct PairIn {
    float mx, my, mz;
    float L[9];
    float b2;  // 9 s_max^2 (1 + 2^-10)
};

struct __align__(16) TileBox {
    float cx, cy, cz;  // centre of the box of the tile's centres
    float hx, hy, hz;  // half extents
    float mx, my, mz;  // |centre| + half extent (magnitude bound)
    float b2;          // max over the tile of 9 s_max^2 (1 + 2^-10)
    float pad[2];
};

// The tile box lives in the warp's shared-memory slot while its views are
// scored and is read back for each classification, so that it holds no
// registers across the view loop (the loads are volatile: never hoisted).
__device__ __forceinline__ TileBox load_box(const TileBox *s)
{
    TileBox t;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(s);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(t.cx), "=f"(t.cy), "=f"(t.cz), "=f"(t.hx) : "r"(a));
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(t.hy), "=f"(t.hz), "=f"(t.mx), "=f"(t.my) : "r"(a + 16));
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(t.mz), "=f"(t.b2) : "r"(a + 32));
    return t;
}

constexpr float kTileSlack = 6.103515625e-05f;  // 2^-14

struct Range {
    float lo, hi;
};

// [lo, hi] of a . mu + a0 over the tile box, widened by the slack.
__device__ __forceinline__ Range form_range(const float4 &a, const TileBox &t)
{
    const float mid = fmaf(a.x, t.cx, fmaf(a.y, t.cy, fmaf(a.z, t.cz, a.w)));
    const float rad = fmaf(fabsf(a.x), t.hx, fmaf(fabsf(a.y), t.hy, fabsf(a.z) * t.hz));
    const float mag = fmaf(fabsf(a.x), t.mx, fmaf(fabsf(a.y), t.my, fmaf(fabsf(a.z), t.mz, fabsf(a.w))));
    const float sl = kTileSlack * mag;
    return {mid - rad - sl, mid + rad + sl};
}

// Class of one view for one tile: kClsMixed, kClsIn or kClsOut in the low two
// bits; for MIXED also the axes whose test some centre of the tile may fail
// (kAxX: 0 < u < w, kAxY: 0 < v < h, kAxZ: znear < z < zfar) above them.  An
// axis that is not flagged holds for every centre of the tile, with the same
// float32 slack as the IN class, so a pair's test on it needs no evaluation.
enum { kClsMixed = 0, kClsIn = 1, kClsOut = 2 };
enum { kAxX = 4, kAxY = 8, kAxZ = 16 };

__device__ __forceinline__ int classify(const CamRec &c, const TileBox &t)
{
    const Range z = form_range(c.r2, t);
    if (z.hi < c.lim.z || z.lo > c.lim.w) return kClsOut;
    const Range U = form_range(c.r0, t), V = form_range(c.r1, t);
    const Range UW = form_range(c.uw, t), VH = form_range(c.vh, t);
    const bool zin = z.lo > c.lim.z && z.hi < c.lim.w;
    const bool xin = U.lo > 0.f && UW.hi < 0.f, yin = V.lo > 0.f && VH.hi < 0.f;
    if (zin && xin && yin) return kClsIn;
    const int mixed = kClsMixed | (xin ? 0 : kAxX) | (yin ? 0 : kAxY) | (zin ? 0 : kAxZ);
    if (!(z.lo > 0.f)) return mixed;
    // outside an edge by more than the footprint bound (times z^2)
    const Range TX = form_range(c.tx, t), TY = form_range(c.ty, t);
    const float tx2 = fmaxf(TX.lo * TX.lo, TX.hi * TX.hi), ty2 = fmaxf(TY.lo * TY.lo, TY.hi * TY.hi);
    // per pair the bound reads (d z)^2 > b2 (fx^2 z^2 + tx^2), i.e. d^2 > b2 (fx^2 + (tx / z)^2): over
    // the box d >= d_lo and z >= z_lo > 0, so (d_lo z_lo)^2 > b2 (fx^2 z_lo^2 + max tx^2) suffices
    const float zz = z.lo * z.lo;
    const float bx = t.b2 * fmaf(c.k.x, zz, tx2) * 1.00390625f;  // (1 + 2^-8)
    const float by = t.b2 * fmaf(c.k.y, zz, ty2) * 1.00390625f;
    const float dl = fmaxf(-U.hi, UW.lo) * z.lo;  // > 0 when the box is left or right of the image
    const float dt = fmaxf(-V.hi, VH.lo) * z.lo;
    if ((dl > 0.f && dl * dl > bx) || (dt > 0.f && dt * dt > by)) return kClsOut;
    return mixed;
}

template <bool DET>
__device__ __forceinline__ bool exact_box(const float4 &c0, const float4 &c1, const float4 &c2, float U, float V,
                                          float z, float ex2, float ey2, const PairIn &p)
{
    const float g0x = fmaf(-U, c2.x, z * c0.x), g0y = fmaf(-U, c2.y, z * c0.y), g0z = fmaf(-U, c2.z, z * c0.z);
    const float g1x = fmaf(-V, c2.x, z * c1.x), g1y = fmaf(-V, c2.y, z * c1.y), g1z = fmaf(-V, c2.z, z * c1.z);
    const float a0 = fmaf(p.L[0], g0x, fmaf(p.L[1], g0y, p.L[2] * g0z));
    const float a1 = fmaf(p.L[3], g0x, fmaf(p.L[4], g0y, p.L[5] * g0z));
    const float a2 = fmaf(p.L[6], g0x, fmaf(p.L[7], g0y, p.L[8] * g0z));
    const float b0 = fmaf(p.L[0], g1x, fmaf(p.L[1], g1y, p.L[2] * g1z));
    const float b1 = fmaf(p.L[3], g1x, fmaf(p.L[4], g1y, p.L[5] * g1z));
    const float b2 = fmaf(p.L[6], g1x, fmaf(p.L[7], g1y, p.L[8] * g1z));
    const float Qx = fmaf(a0, a0, fmaf(a1, a1, a2 * a2));
    const float Qy = fmaf(b0, b0, fmaf(b1, b1, b2 * b2));
    bool ok = (ex2 <= Qx) & (ey2 <= Qy);
    if (DET) {
        const float x0 = a1 * b2 - a2 * b1, x1 = a2 * b0 - a0 * b2, x2 = a0 * b1 - a1 * b0;
        ok = ok & ((x0 != 0.f) | (x1 != 0.f) | (x2 != 0.f));
    }
    return ok;
}

struct PairGeom {
    float U, V, z, ex2, ey2;
    bool inz, inside;
};

__device__ __forceinline__ PairGeom pair_geom(const float4 &c0, const float4 &c1, const float4 &c2, const float4 &lim,
                                              const PairIn &p)
{
    PairGeom r;
    r.U = fmaf(c0.x, p.mx, fmaf(c0.y, p.my, fmaf(c0.z, p.mz, c0.w)));
    r.V = fmaf(c1.x, p.mx, fmaf(c1.y, p.my, fmaf(c1.z, p.mz, c1.w)));
    r.z = fmaf(c2.x, p.mx, fmaf(c2.y, p.my, fmaf(c2.z, p.mz, c2.w)));
    const float du = fmaxf(-r.U, fmaf(-lim.x, r.z, r.U));
    const float dv = fmaxf(-r.V, fmaf(-lim.y, r.z, r.V));
    r.inz = (r.z > lim.z) & (r.z < lim.w);
    r.inside = r.inz & (du <= 0.f) & (dv <= 0.f);
    const float ex = fmaxf(du, 0.f) * r.z, ey = fmaxf(dv, 0.f) * r.z;
    r.ex2 = ex * ex;
    r.ey2 = ey * ey;
    return r;
}

// Projection term of a visible (primitive, view) pair.  PM (projection
// mode): 0 = Eq. 17, 1/(z^2 + eta); 1 = Table 3 "w/o P", 1; 2 = Eq. 14 before
// the simplification of Eq. 16, the Jacobian energy Tr(J^T J) = (fx^2 +
// fy^2)/z^2 + ((fx x)^2 + (fy y)^2)/z^4, with fx x and fy y from the camera's
// fx R0 and fy R1 rows (the same arithmetic on every path, so the weight does
// not depend on the tile's classification).
enum { kProjEq17 = 0, kProjNone = 1, kProjFullJ = 2 };

template <int PM>
__device__ __forceinline__ float weight(const CamRec &c, float z, float eta, float mx, float my, float mz)
{
    if (PM == kProjNone) return 1.f;
    // z^2 + eta >= eta >= 2^-126 (checked on the host), so the operand is
    // never subnormal; weights below 2^-126 (z beyond 9.2e18) flush to zero
    if (PM == kProjEq17) return rcp_approx_ftz(fmaf(z, z, eta));
    const float4 tx = c.tx, ty = c.ty, k = c.k;
    const float fxx = fmaf(tx.x, mx, fmaf(tx.y, my, fmaf(tx.z, mz, tx.w)));
    const float fyy = fmaf(ty.x, mx, fmaf(ty.y, my, fmaf(ty.z, mz, ty.w)));
    // explicit rounding intrinsics: never contracted into a neighbouring
    // add, so every path (IN, MIXED, plain, batched) rounds identically
    const float iz2 = rcp_approx(__fmul_rn(z, z));
    return __fmul_rn(fmaf(fmaf(fxx, fxx, __fmul_rn(fyy, fyy)), iz2, __fadd_rn(k.x, k.y)), iz2);
}

__host__ __device__ inline int proj_mode(int flags)
{
    return (flags & REFINE_FLAG_NO_PROJ) ? kProjNone : (flags & REFINE_FLAG_FULL_JACOBIAN) ? kProjFullJ : kProjEq17;
}

template <int PM, bool DET, bool COUNT, int GPT>
__device__ __forceinline__ void mixed_view(const CamRec &c, float eta, const PairIn (&p)[GPT],
                                           const bool (&valid)[GPT], float (&part)[GPT],
                                           unsigned long long (&cnt)[kCountSlots])
{
    const float4 c0 = c.r0, c1 = c.r1, c2 = c.r2, lim = c.lim;
    PairGeom q[GPT];
    bool vis[GPT], out = false;
#pragma unroll
    for (int g = 0; g < GPT; ++g) {
        q[g] = pair_geom(c0, c1, c2, lim, p[g]);
        vis[g] = q[g].inside;
        out |= q[g].inz & !q[g].inside;
        if (COUNT && valid[g]) {
            cnt[kCntMixedPairs] += 1;
            cnt[kCntOpenX] += 1;
            cnt[kCntOpenY] += 1;
            cnt[kCntOpenZ] += 1;
        }
    }
    if (DET || __any_sync(0xffffffffu, out)) {
        const float4 k = c.k;
        bool nearq = false, nq[GPT];
#pragma unroll
        for (int g = 0; g < GPT; ++g) {
            const float tx = fmaf(-k.z, q[g].z, q[g].U), ty = fmaf(-k.w, q[g].z, q[g].V);
            const float zz = q[g].z * q[g].z;
            const bool o = q[g].inz & !q[g].inside;
            nq[g] = o & (q[g].ex2 <= p[g].b2 * fmaf(k.x, zz, tx * tx)) & (q[g].ey2 <= p[g].b2 * fmaf(k.y, zz, ty * ty));
            nearq |= nq[g];
            if (COUNT && valid[g]) {
                cnt[kCntBoundPairs] += o ? 1 : 0;
                cnt[kCntBoundX] += o ? 1 : 0;
                cnt[kCntBoundY] += o ? 1 : 0;
                cnt[kCntExactPairs] += nq[g] ? 1 : 0;
                // the determinant path evaluates both extents of every pair
                cnt[kCntExactX] += q[g].inz ? 1 : 0;
                cnt[kCntExactY] += q[g].inz ? 1 : 0;
            }
        }
        if (DET || __any_sync(0xffffffffu, nearq)) {
#pragma unroll
            for (int g = 0; g < GPT; ++g)
                vis[g] = q[g].inz & exact_box<DET>(c0, c1, c2, q[g].U, q[g].V, q[g].z, q[g].ex2, q[g].ey2, p[g]);
            if (COUNT && (threadIdx.x & 31) == 0) cnt[kCntExactWarpAxes] += 2 * GPT;
        }
    }
#pragma unroll
    for (int g = 0; g < GPT; ++g) {
        part[g] += vis[g] ? weight<PM>(c, q[g].z, eta, p[g].mx, p[g].my, p[g].mz) : 0.f;
        if (COUNT) cnt[kCntVisMixed] += (valid[g] && vis[g]) ? 1 : 0;
    }
}

// A MIXED view of a tile without underflowed scales, evaluated only on the
// axes its classification left open (NX: 0 < u < w, NY: 0 < v < h, NZ: the
// depth range); an axis that holds for every centre of the tile contributes
// d = 0 to the box test, which it then passes for every Sigma2D, so leaving
// it out changes no decision.  The stages are those of the full test, with
// the same expressions (so the same float32 roundings): the centre test; for
// centres outside, the footprint bound; and the exact footprint test, entered
// per primitive slot g and per axis only when some lane of the warp needs it
// (a lane whose bound test failed, or whose centre lies within that axis's
// interval, passes or fails it without evaluation).
template <int PM, bool COUNT, int GPT, bool NX, bool NY, bool NZ>
__device__ __forceinline__ void mixed_view_ax(const CamRec &c, float eta, const PairIn (&p)[GPT],
                                              const bool (&valid)[GPT], float (&part)[GPT],
                                              unsigned long long (&cnt)[kCountSlots])
{
    const float4 c2 = c.r2, lim = c.lim;
    float z[GPT], U[GPT], V[GPT], du[GPT], dv[GPT];
    bool vis[GPT], o[GPT], anyo = false;
#pragma unroll
    for (int g = 0; g < GPT; ++g) {
        z[g] = fmaf(c2.x, p[g].mx, fmaf(c2.y, p[g].my, fmaf(c2.z, p[g].mz, c2.w)));
        bool inside = NZ ? (z[g] > lim.z) & (z[g] < lim.w) : true;
        const bool inz = inside;
        if (NX) {
            const float4 c0 = c.r0;
            U[g] = fmaf(c0.x, p[g].mx, fmaf(c0.y, p[g].my, fmaf(c0.z, p[g].mz, c0.w)));
            du[g] = fmaxf(-U[g], fmaf(-lim.x, z[g], U[g]));
            inside &= du[g] <= 0.f;
        }
        if (NY) {
            const float4 c1 = c.r1;
            V[g] = fmaf(c1.x, p[g].mx, fmaf(c1.y, p[g].my, fmaf(c1.z, p[g].mz, c1.w)));
            dv[g] = fmaxf(-V[g], fmaf(-lim.y, z[g], V[g]));
            inside &= dv[g] <= 0.f;
        }
        vis[g] = inside;
        o[g] = inz & !inside;
        anyo |= o[g];
        if (COUNT && valid[g]) {
            cnt[kCntMixedPairs] += 1;
            cnt[kCntOpenX] += NX ? 1 : 0;
            cnt[kCntOpenY] += NY ? 1 : 0;
            cnt[kCntOpenZ] += NZ ? 1 : 0;
        }
    }
    if (__any_sync(0xffffffffu, anyo)) {
        const float4 k = c.k;
        float ex2[GPT], ey2[GPT];
        bool nq[GPT];
#pragma unroll
        for (int g = 0; g < GPT; ++g) {
            const float zz = z[g] * z[g];
            bool ok = o[g];
            if (NX) {
                const float ex = fmaxf(du[g], 0.f) * z[g];
                ex2[g] = ex * ex;
                const float tx = fmaf(-k.z, z[g], U[g]);
                ok &= ex2[g] <= p[g].b2 * fmaf(k.x, zz, tx * tx);
            }
            if (NY) {
                const float ey = fmaxf(dv[g], 0.f) * z[g];
                ey2[g] = ey * ey;
                const float ty = fmaf(-k.w, z[g], V[g]);
                ok &= ey2[g] <= p[g].b2 * fmaf(k.y, zz, ty * ty);
            }
            nq[g] = ok;
            if (COUNT && valid[g]) {
                cnt[kCntBoundPairs] += o[g] ? 1 : 0;
                cnt[kCntBoundX] += (NX && o[g]) ? 1 : 0;
                cnt[kCntBoundY] += (NY && o[g]) ? 1 : 0;
                cnt[kCntExactPairs] += nq[g] ? 1 : 0;
                cnt[kCntExactX] += (NX && nq[g] && ex2[g] > 0.f) ? 1 : 0;
                cnt[kCntExactY] += (NY && nq[g] && ey2[g] > 0.f) ? 1 : 0;
            }
        }
#pragma unroll
        for (int g = 0; g < GPT; ++g) {
            bool xt = true, yt = true;
            if (NX && __any_sync(0xffffffffu, nq[g] & (ex2[g] > 0.f))) {
                const float4 c0 = c.r0;
                const float gx = fmaf(-U[g], c2.x, z[g] * c0.x), gy = fmaf(-U[g], c2.y, z[g] * c0.y),
                            gz = fmaf(-U[g], c2.z, z[g] * c0.z);
                const float a0 = fmaf(p[g].L[0], gx, fmaf(p[g].L[1], gy, p[g].L[2] * gz));
                const float a1 = fmaf(p[g].L[3], gx, fmaf(p[g].L[4], gy, p[g].L[5] * gz));
                const float a2 = fmaf(p[g].L[6], gx, fmaf(p[g].L[7], gy, p[g].L[8] * gz));
                xt = ex2[g] <= fmaf(a0, a0, fmaf(a1, a1, a2 * a2));
                if (COUNT && (threadIdx.x & 31) == 0) cnt[kCntExactWarpAxes] += 1;
            }
            if (NY && __any_sync(0xffffffffu, nq[g] & (ey2[g] > 0.f))) {
                const float4 c1 = c.r1;
                const float gx = fmaf(-V[g], c2.x, z[g] * c1.x), gy = fmaf(-V[g], c2.y, z[g] * c1.y),
                            gz = fmaf(-V[g], c2.z, z[g] * c1.z);
                const float b0 = fmaf(p[g].L[0], gx, fmaf(p[g].L[1], gy, p[g].L[2] * gz));
                const float b1 = fmaf(p[g].L[3], gx, fmaf(p[g].L[4], gy, p[g].L[5] * gz));
                const float b2 = fmaf(p[g].L[6], gx, fmaf(p[g].L[7], gy, p[g].L[8] * gz));
                yt = ey2[g] <= fmaf(b0, b0, fmaf(b1, b1, b2 * b2));
                if (COUNT && (threadIdx.x & 31) == 0) cnt[kCntExactWarpAxes] += 1;
            }
            vis[g] |= nq[g] & xt & yt;
        }
    }
#pragma unroll
    for (int g = 0; g < GPT; ++g) {
        part[g] += vis[g] ? weight<PM>(c, z[g], eta, p[g].mx, p[g].my, p[g].mz) : 0.f;
        if (COUNT) cnt[kCntVisMixed] += (valid[g] && vis[g]) ? 1 : 0;
    }
}

template <int PM, bool DET, bool COUNT, int GPT>
__device__ __forceinline__ void view_loop(const CamRec *cs, int vcount, float eta, const PairIn (&p)[GPT],
                                          const bool (&valid)[GPT], const TileBox *tbs,
                                          float (&acc)[GPT], float (&comp)[GPT],
                                          unsigned long long (&cnt)[kCountSlots])
{
    const int lane = threadIdx.x & 31;
    int nvalid = 0;
#pragma unroll
    for (int g = 0; g < GPT; ++g) nvalid += __popc(__ballot_sync(0xffffffffu, valid[g]));
    for (int vb = 0; vb < vcount; vb += 32) {
        const int nv = min(32, vcount - vb);
        const unsigned vmask = nv == 32 ? 0xffffffffu : ((1u << nv) - 1u);
        unsigned in_m = 0u, out_m = 0u, ux_m = 0u, uy_m = 0u, uz_m = 0u;
        if (!DET) {
            const TileBox tb = load_box(tbs);
            const int cls = lane < nv ? classify(cs[vb + lane], tb) : (kAxX | kAxY | kAxZ);
            in_m = __ballot_sync(0xffffffffu, (cls & 3) == kClsIn);
            out_m = __ballot_sync(0xffffffffu, (cls & 3) == kClsOut);
            ux_m = __ballot_sync(0xffffffffu, (cls & kAxX) != 0);
            uy_m = __ballot_sync(0xffffffffu, (cls & kAxY) != 0);
            uz_m = __ballot_sync(0xffffffffu, (cls & kAxZ) != 0);
            if (COUNT && lane == 0) {
                cnt[kCntTiles] += nv;
                cnt[kCntInPairs] += (unsigned long long)__popc(in_m & vmask) * nvalid;
                cnt[kCntOutPairs] += (unsigned long long)__popc(out_m & vmask) * nvalid;
            }
        }
        {
            float part[GPT];
#pragma unroll
            for (int g = 0; g < GPT; ++g) part[g] = 0.f;
            unsigned todo = vmask & ~out_m;
            while (todo) {
                const int b = __ffs(todo) - 1;
                todo &= todo - 1u;
                const CamRec &c = cs[vb + b];
                if ((in_m >> b) & 1u) {
                    const float4 c2 = c.r2;
#pragma unroll
                    for (int g = 0; g < GPT; ++g) {
                        const float z = fmaf(c2.x, p[g].mx, fmaf(c2.y, p[g].my, fmaf(c2.z, p[g].mz, c2.w)));
                        part[g] += weight<PM>(c, z, eta, p[g].mx, p[g].my, p[g].mz);
                    }
                } else if (DET) {
                    mixed_view<PM, true, COUNT, GPT>(c, eta, p, valid, part, cnt);
                } else {
                    const unsigned bit = 1u << b;
                    if (uz_m & bit)
                        mixed_view_ax<PM, COUNT, GPT, true, true, true>(c, eta, p, valid, part, cnt);
                    else if (ux_m & uy_m & bit)
                        mixed_view_ax<PM, COUNT, GPT, true, true, false>(c, eta, p, valid, part, cnt);
                    else if (ux_m & bit)
                        mixed_view_ax<PM, COUNT, GPT, true, false, false>(c, eta, p, valid, part, cnt);
                    else
                        mixed_view_ax<PM, COUNT, GPT, false, true, false>(c, eta, p, valid, part, cnt);
                }
            }
            // Kahan-compensated sum of the 32-view partial sums
#pragma unroll
            for (int g = 0; g < GPT; ++g) {
                const float y = part[g] - comp[g];
                const float t = acc[g] + y;
                comp[g] = (t - acc[g]) - y;
                acc[g] = t;
            }
        }
    }
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void fence_proxy_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Scores one warp tile: the 32 * GPT primitives of the processing order
// starting at `base`; `next_base` (or -1) is the tile this warp takes next,
// whose primitives are pulled towards L2 meanwhile.  `tbs` is the warp's
// shared-memory slot for the tile box.
template <int PM, bool COUNT, int GPT>
__device__ __forceinline__ void score_tile(const ScoreLaunch &a, const CamRec *cs, const SceneConsts &sc,
                                           int64_t base, int64_t next_base, TileBox *tbs,
                                           unsigned long long (&cnt)[kCountSlots])
{
    const int lane = threadIdx.x & 31;
    if (next_base >= 0) {
#pragma unroll
        for (int g = 0; g < GPT; ++g) {
            const int64_t j = next_base + g * 32 + lane;
            if (j < a.n) prefetch_l2(a.recs + __ldg(a.perm + j));
        }
    }
    PairIn p[GPT];
    float acc[GPT], comp[GPT];
    bool valid[GPT];
    bool degen = false;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, b2 = 0.f;
#pragma unroll
    for (int g = 0; g < GPT; ++g) {
        const int64_t j = base + g * 32 + lane;
        float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra, rc = ra, rd = ra;
        acc[g] = 0.f;
        comp[g] = 0.f;
        valid[g] = j < a.n;
        if (valid[g]) {
            const int64_t i = __ldg(a.perm + j);
            const PrimRec *r = a.recs + i;
            ra = __ldg(&r->a); rb = __ldg(&r->b); rc = __ldg(&r->c); rd = __ldg(&r->d);
            if (!a.first) {
                const float2 run = a.running[i];
                acc[g] = run.x;
                comp[g] = run.y;
            }
        }
        p[g].mx = ra.x; p[g].my = ra.y; p[g].mz = ra.z; p[g].b2 = ra.w;
        p[g].L[0] = rb.x; p[g].L[1] = rb.y; p[g].L[2] = rb.z; p[g].L[3] = rb.w;
        p[g].L[4] = rc.x; p[g].L[5] = rc.y; p[g].L[6] = rc.z; p[g].L[7] = rc.w;
        p[g].L[8] = rd.x;
        degen |= ra.w < 0.f;
        if (valid[g]) {
            lo[0] = fminf(lo[0], p[g].mx); hi[0] = fmaxf(hi[0], p[g].mx);
            lo[1] = fminf(lo[1], p[g].my); hi[1] = fmaxf(hi[1], p[g].my);
            lo[2] = fminf(lo[2], p[g].mz); hi[2] = fmaxf(hi[2], p[g].mz);
            b2 = fmaxf(b2, p[g].b2);
        }
    }
    if (!__any_sync(0xffffffffu, valid[0])) return;  // warp past the end

    {
        const float l0 = warp_min(lo[0]), l1 = warp_min(lo[1]), l2 = warp_min(lo[2]);
        const float h0 = warp_max(hi[0]), h1 = warp_max(hi[1]), h2 = warp_max(hi[2]);
        const float tb2 = warp_max(b2);
        __syncwarp();  // every lane is done with the previous tile's box
        if (lane == 0) {
            TileBox tb;
            tb.b2 = tb2;
            tb.cx = 0.5f * (l0 + h0); tb.hx = 0.5f * (h0 - l0);
            tb.cy = 0.5f * (l1 + h1); tb.hy = 0.5f * (h1 - l1);
            tb.cz = 0.5f * (l2 + h2); tb.hz = 0.5f * (h2 - l2);
            tb.mx = fabsf(tb.cx) + tb.hx;
            tb.my = fabsf(tb.cy) + tb.hy;
            tb.mz = fabsf(tb.cz) + tb.hz;
            tb.pad[0] = tb.pad[1] = 0.f;
            *tbs = tb;
        }
        __syncwarp();
    }

    if (__any_sync(0xffffffffu, degen))
        view_loop<PM, true, COUNT, GPT>(cs, a.vcount, a.eta, p, valid, tbs, acc, comp, cnt);
    else
        view_loop<PM, false, COUNT, GPT>(cs, a.vcount, a.eta, p, valid, tbs, acc, comp, cnt);

#pragma unroll
    for (int g = 0; g < GPT; ++g) {
        if (!valid[g]) continue;
        const int64_t i = __ldg(a.perm + base + g * 32 + lane);
        if (!a.last) {
            a.running[i] = make_float2(acc[g], comp[g]);
            continue;
        }
        const float Ssum = acc[g] - comp[g];
        if (a.view_sum) a.view_sum[i] = Ssum;
        const float4 rd = __ldg(&a.recs[i].d);  // (L8, alpha, m_gem, m_col)
        const float coupled = fmaf(sc.kappa[0], rd.z, fmaf(sc.kappa[1], rd.w, sc.kappa[2] * rd.y));
        const float A = ((a.flags & REFINE_FLAG_NO_VIS) ? 1.f : rd.y) * (Ssum * a.inv_views);
        a.scores[i] = A * coupled;
    }
}

// A camera block may be staged by one bulk copy chain only if its source is
// 16-byte aligned and it fits the launch's dynamic shared memory.
__device__ __forceinline__ int cams_stageable(const CamRec *cams, int vcount)
{
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    return vcount >= 1 && (reinterpret_cast<uintptr_t>(cams) & 15u) == 0 &&
           (uint64_t)vcount * sizeof(CamRec) <= (uint64_t)dyn;
}

template <int PM, bool COUNT, int GPT>
__global__ void __launch_bounds__(kScoreThreads, COUNT ? 1 : 4) k_score(ScoreLaunch a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ TileBox s_box[kScoreThreads / 32];
    CamRec *cs = reinterpret_cast<CamRec *>(smem_raw);

    // Stage this pass's cameras once per CTA (TMA bulk copy, mbarrier).
    __shared__ int s_ok;
    const uint32_t bytes = (uint32_t)a.vcount * (uint32_t)sizeof(CamRec);
    if (threadIdx.x == 0) {
        s_ok = cams_stageable(a.cams, a.vcount) && a.tiles_taken != nullptr;
        if (s_ok) {
            mbar_init(&bar, 1);
            mbar_expect_tx(&bar, bytes);
            for (uint32_t off = 0; off < bytes; off += 16384u) {
                const uint32_t len = bytes - off < 16384u ? bytes - off : 16384u;
                bulk_g2s(smem_raw + off, reinterpret_cast<const unsigned char *>(a.cams) + off, len, &bar);
            }
        } else {
            set_status(a.status, kEinval);
        }
    }
    __syncthreads();
    if (!s_ok) return;
    if (!mbar_wait_bounded(&bar, 0)) {
        set_status(a.status, kEtimeout);
        mbar_wait_bounded(&bar, 0);  // give the copy a second bound before leaving
        return;
    }

    unsigned long long cnt[kCountSlots];
#pragma unroll
    for (int k = 0; k < kCountSlots; ++k) cnt[k] = 0;
    const SceneConsts sc = *a.consts;
    // Every warp takes its own tiles of 32 * GPT primitives from a counter,
    // one ahead (the records of the next are pulled towards L2 while the
    // current one is scored): warps that draw cheap tiles take more of them,
    // and no warp waits for the others of its CTA.  Tile indices stay below
    // 2^31 (n <= INT32_MAX).
    const int lane = threadIdx.x & 31;
    const int ntiles = (int)((a.n + 32 * GPT - 1) / (32 * GPT));
    int cur = 0;
    if (lane == 0) cur = (int)min((unsigned long long)ntiles, atomicAdd(a.tiles_taken, 1ull));
    cur = __shfl_sync(0xffffffffu, cur, 0);
    while (cur < ntiles) {
        int nxt = 0;
        if (lane == 0) nxt = (int)min((unsigned long long)ntiles, atomicAdd(a.tiles_taken, 1ull));
        nxt = __shfl_sync(0xffffffffu, nxt, 0);
        score_tile<PM, COUNT, GPT>(a, cs, sc, (int64_t)cur * (32 * GPT),
                                   nxt < ntiles ? (int64_t)nxt * (32 * GPT) : -1, &s_box[threadIdx.x >> 5], cnt);
        cur = nxt;
    }
    if (COUNT) {
#pragma unroll
        for (int k = 0; k < kCountSlots; ++k) {
            unsigned long long v = cnt[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && v) atomicAdd(&a.need[k], v);
        }
    }
}

// The batched form: one persistent launch over the tiles of many scenes.
// CTAs take (scene, tile) items from an atomic counter (items are ordered
// by scene); when a CTA moves to another scene it restages that scene's
// cameras by TMA.  Every tile is scored by score_tile exactly as in
// k_score, so a scene's scores are the same alone and in a batch; scenes
// may differ in storage type (the records are float32) and in flags.
template <int GPT, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_score_batch(BatchLaunch b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_scene, s_ok, s_wt;
    __shared__ long long s_base;
    __shared__ TileBox s_box[THREADS / 32];
    CamRec *cs = reinterpret_cast<CamRec *>(smem_raw);
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    unsigned long long cnt[kCountSlots];
    int cur = -1;
    uint32_t phase = 0;
    const int lane = threadIdx.x & 31;
    const int64_t tile = (int64_t)THREADS * GPT * b.rounds;  // primitives per item
    for (;;) {
        if (threadIdx.x == 0) {
            s_wt = 0;
            const unsigned long long item = atomicAdd(b.counter, 1ull);
            int sidx = -1;
            long long base = 0;
            if ((long long)item < b.total_tiles) {
                int lo = 0, hi = b.n_scenes - 1;  // last scene whose first tile <= item
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (b.tile_begin[mid] <= (long long)item) lo = mid; else hi = mid - 1;
                }
                sidx = lo;
                base = ((long long)item - b.tile_begin[lo]) * tile;
            }
            s_scene = sidx;
            s_base = base;
        }
        __syncthreads();
        const int sidx = s_scene;
        const int64_t base = s_base;
        if (sidx < 0) break;
        const ScoreLaunch &a = b.scenes[sidx];
        if (sidx != cur) {
            if (threadIdx.x == 0) {
                s_ok = cams_stageable(a.cams, a.vcount);
                if (s_ok) {
                    fence_proxy_async_shared();
                    const uint32_t bytes = (uint32_t)a.vcount * (uint32_t)sizeof(CamRec);
                    mbar_expect_tx(&bar, bytes);
                    for (uint32_t off = 0; off < bytes; off += 16384u) {
                        const uint32_t len = bytes - off < 16384u ? bytes - off : 16384u;
                        bulk_g2s(smem_raw + off, reinterpret_cast<const unsigned char *>(a.cams) + off, len, &bar);
                    }
                } else {
                    set_status(a.status, kEinval);
                }
            }
            __syncthreads();
            if (!s_ok) {
                cur = -1;
                continue;  // the tile is left unscored; the loop's first barrier orders s_scene
            }
            if (!mbar_wait_bounded(&bar, phase)) {
                // the item left unscored belongs to this scene: its own
                // status word carries the error, and so does the launch's
                set_status(a.status, kEtimeout);
                set_status(b.status, kEtimeout);
                mbar_wait_bounded(&bar, phase);
                return;
            }
            phase ^= 1u;
            cur = sidx;
        }
        const SceneConsts sc = *a.consts;
        const int pm = proj_mode(a.flags);
        // the item's warp tiles go to whichever warp of the CTA is free
        const int wtiles = (int)((min(tile, a.n - base) + 32 * GPT - 1) / (32 * GPT));
        for (;;) {
            int t = 0;
            if (lane == 0) t = atomicAdd(&s_wt, 1);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= wtiles) break;
            const int64_t wbase = base + (int64_t)t * (32 * GPT);
            if (pm == kProjEq17)
                score_tile<kProjEq17, false, GPT>(a, cs, sc, wbase, -1, &s_box[threadIdx.x >> 5], cnt);
            else if (pm == kProjNone)
                score_tile<kProjNone, false, GPT>(a, cs, sc, wbase, -1, &s_box[threadIdx.x >> 5], cnt);
            else
                score_tile<kProjFullJ, false, GPT>(a, cs, sc, wbase, -1, &s_box[threadIdx.x >> 5], cnt);
        }
        __syncthreads();  // the cameras, s_scene and s_wt are free again
    }
}

// Self-test of the bounded wait that guards the camera staging above: one
// thread stages `bytes` by a bulk copy while the barrier expects `bytes +
// missing` bytes.  With missing > 0 the phase cannot complete; the wait gives
// up after `limit` cycles (long after the copy itself has landed) and the
// kernel reports kEtimeout through the status word and returns.
__global__ void k_wait_selftest(const unsigned char *src, uint32_t bytes, uint32_t missing, long long limit,
                                int *status)
{
    __shared__ __align__(16) unsigned char buf[kSelftestMaxBytes];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, bytes + missing);
    bulk_g2s(buf, src, bytes, &bar);
    if (!mbar_wait_bounded(&bar, 0, limit)) {
        set_status(status, kEtimeout);
        mbar_wait_bounded(&bar, 0, limit);
    }
}

cudaError_t launch_wait_selftest(const void *src, uint32_t bytes, uint32_t missing, long long limit, int *status,
                                 cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(static_cast<const unsigned char *>(src), bytes, missing, limit, status);
    return cudaGetLastError();
}

template <int PM, bool COUNT, int GPT>
static const void *score_fn()
{
    return reinterpret_cast<const void *>(&k_score<PM, COUNT, GPT>);
}

template <int PM, int GPT>
static const void *pick_score_pg(bool count)
{
    return count ? score_fn<PM, true, GPT>() : score_fn<PM, false, GPT>();
}

template <int GPT>
static const void *pick_score_g(int pm, bool count)
{
    if (pm == kProjNone) return pick_score_pg<kProjNone, GPT>(count);
    if (pm == kProjFullJ) return pick_score_pg<kProjFullJ, GPT>(count);
    return pick_score_pg<kProjEq17, GPT>(count);
}

static const void *pick_score(int pm, bool count, int gpt)
{
    return gpt == 1 ? pick_score_g<1>(pm, count) : pick_score_g<2>(pm, count);
}

bool shape_valid(const ScoreShape &sh)
{
    return (sh.gpt == 1 || sh.gpt == 2) && (sh.threads == 128 || sh.threads == 256) && sh.ctas_per_sm >= 0 &&
           sh.views_per_pass >= 32 && sh.views_per_pass <= kViewsPerPass && sh.views_per_pass % 32 == 0;
}

int score_grid(int num_sms, int64_t n, int vcount, const ScoreShape &sh)
{
    // Persistent grid: as many CTAs as fit per SM, capped by the tile count.
    int per_sm = 0;
    const size_t smem = (size_t)vcount * sizeof(CamRec);
    const void *fn = pick_score(kProjEq17, false, sh.gpt);
    if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kScoreThreads, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int64_t tile = (int64_t)kScoreThreads * sh.gpt;
    const int64_t tiles = (n + tile - 1) / tile;
    int64_t g = (int64_t)num_sms * per_sm;
    if (g > tiles) g = tiles;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_score(const ScoreLaunch &a, const ScoreShape &sh, cudaStream_t s)
{
    const void *fn = pick_score(proj_mode(a.flags), a.need != nullptr, sh.gpt);
    const size_t smem = (size_t)a.vcount * sizeof(CamRec);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    ScoreLaunch arg = a;
    void *args[] = {&arg};
    return cudaLaunchKernel(fn, dim3(a.grid), dim3(kScoreThreads), args, smem, s);
}

static const void *batch_fn(const ScoreShape &sh)
{
    if (sh.threads == 128)
        return sh.gpt == 1 ? reinterpret_cast<const void *>(&k_score_batch<1, 128>)
                           : reinterpret_cast<const void *>(&k_score_batch<2, 128>);
    return sh.gpt == 1 ? reinterpret_cast<const void *>(&k_score_batch<1, 256>)
                       : reinterpret_cast<const void *>(&k_score_batch<2, 256>);
}

int score_batch_grid(int num_sms, int max_vcount, const ScoreShape &sh)
{
    const void *fn = batch_fn(sh);
    const size_t smem = (size_t)max_vcount * sizeof(CamRec);
    if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, sh.threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    if (sh.ctas_per_sm > 0 && sh.ctas_per_sm < per_sm) per_sm = sh.ctas_per_sm;
    return num_sms * per_sm;
}

cudaError_t launch_score_batch(const BatchLaunch &b, int max_vcount, int grid, const ScoreShape &sh, cudaStream_t s)
{
    const void *fn = batch_fn(sh);
    const size_t smem = (size_t)max_vcount * sizeof(CamRec);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    BatchLaunch arg = b;
    void *args[] = {&arg};
    return cudaLaunchKernel(fn, dim3(grid), dim3(sh.threads), args, smem, s);
}

}  // namespace refine
