// HBM-streaming kernels: the content-feature pass and the compaction, fed by
// TMA bulk copies of 256-primitive row chunks into shared memory (double
// buffered, one mbarrier per stage).  One CTA works through chunks
// b, b + grid, b + 2 grid, ...; the partial chunk at the end of the scene is
// read with plain loads.
#include <math.h>

#include "internal.h"

namespace refine {

constexpr int kChunk = 256;    // primitives per chunk = threads per CTA
constexpr int kStages = 2;     // feature pass: two CTAs per SM, two stages each
constexpr int kCmpStages = 3;  // compaction: one (float32) or two (bfloat16) CTAs per SM

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }

// Waits for every stage that still has copies in flight (bounded), so that a
// CTA never leaves while the copy engine writes its shared memory.
template <int NS>
__device__ __forceinline__ void drain_stages(uint64_t *bars, const int *issued, const int *waited)
{
    for (int s = 0; s < NS; ++s)
        if (issued[s] > waited[s]) mbar_wait_bounded(&bars[s], (uint32_t)(waited[s] & 1));
}

// ------------------------------------------------------------ features
// Rows staged per chunk: mean x, y, z (float32) and attribute rows 0-2
// (log-scale), 7 (opacity logit), 8-55 (SH) in the storage type.
constexpr int kFeatAttrRows = 52;

__device__ __forceinline__ int feat_attr_row(int s) { return s < 3 ? s : s + 4; }

template <typename AT>
struct FeatStage {
    float pos[3][kChunk];
    AT attr[kFeatAttrRows][kChunk];
};

template <typename AT>
__device__ __forceinline__ void issue_feat(FeatStage<AT> *st, uint64_t *bar, const float *pos, const AT *attr,
                                           int64_t S, int64_t base, int lane)
{
    constexpr uint32_t bytes = 3 * kChunk * 4 + kFeatAttrRows * kChunk * sizeof(AT);
    if (lane == 0) mbar_expect_tx(bar, bytes);
    __syncwarp();
    for (int r = lane; r < 3 + kFeatAttrRows; r += 32) {
        if (r < 3)
            bulk_g2s(st->pos[r], pos + r * S + base, kChunk * 4, bar);
        else
            bulk_g2s(st->attr[r - 3], attr + feat_attr_row(r - 3) * S + base, kChunk * sizeof(AT), bar);
    }
}

// Per-primitive feature terms; identical arithmetic to the vector path of
// k_features (same sums, same m_col).
struct FeatSums {
    float s[kFeatSums];
    float bad;
};

__device__ __forceinline__ float feat_terms(FeatSums &acc, float mx, float my, float mz, float ls0, float ls1,
                                            float ls2, float logit, float dc0, float dc1, float dc2, float sumsq,
                                            float eta, float l0, float l1, float l2)
{
    constexpr float kC0 = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
    const float e0 = expf(ls0), e1 = expf(ls1), e2 = expf(ls2);
    const float alpha = 1.f / (1.f + expf(-logit));
    const float y = kC0 * fmaf(l0, dc0, fmaf(l1, dc1, l2 * dc2));
    const float smax = fmaxf(e0, fmaxf(e1, e2)), smin = fminf(e0, fminf(e1, e2));
    const float mg = fmaxf(fmaxf(e0 * e1, e0 * e2), e1 * e2);
    const float mc = sqrtf(sumsq);
    acc.s[0] += y;
    acc.s[1] = fmaf(y, y, acc.s[1]);
    acc.s[2] = fmaf(alpha, 1.f - alpha, acc.s[2]);
    acc.s[3] += smax / (smin + eta);
    acc.s[4] += mg;
    acc.s[5] += mc;
    acc.s[6] += alpha;
    acc.s[7] += mx;
    acc.s[8] += my;
    acc.s[9] += mz;
    acc.s[10] = fmaf(mx, mx, acc.s[10]);
    acc.s[11] = fmaf(my, my, acc.s[11]);
    acc.s[12] = fmaf(mz, mz, acc.s[12]);
    acc.bad = fmaf(mx + my + mz + ls0 + ls1 + ls2 + logit + sumsq, 0.f, acc.bad);
    return mc;
}

template <typename AT>
__global__ void __launch_bounds__(kChunk) k_features_tma(const float *__restrict__ pos, const AT *__restrict__ attr,
                                                         int64_t S, int64_t n, float eta, float l0, float l1,
                                                         float l2, float *__restrict__ m_col,
                                                         double *__restrict__ partials, int *status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FeatStage<AT> *stages = reinterpret_cast<FeatStage<AT> *>(smem_raw);
    __shared__ __align__(8) uint64_t bars[kStages];
    const int t = threadIdx.x, lane = t & 31;
    const int64_t full = n / kChunk;
    const int64_t mine = full > blockIdx.x ? (full - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    int issued[kStages] = {0, 0}, waited[kStages] = {0, 0};
    if (t == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    }
    __syncthreads();
    if (t < 32) {
        for (int s = 0; s < kStages && s < mine; ++s)
            issue_feat(&stages[s], &bars[s], pos, attr, S, (blockIdx.x + (int64_t)s * gridDim.x) * kChunk, lane);
    }
    for (int s = 0; s < kStages && s < mine; ++s) issued[s] = 1;

    FeatSums acc;
#pragma unroll
    for (int k = 0; k < kFeatSums; ++k) acc.s[k] = 0.f;
    acc.bad = 0.f;
    for (int64_t k = 0; k < mine; ++k) {
        const int s = (int)(k % kStages);
        if (!mbar_wait_bounded(&bars[s], (uint32_t)(waited[s] & 1))) {
            set_status(status, kEtimeout);
            drain_stages<kStages>(bars, issued, waited);
            return;
        }
        ++waited[s];
        const FeatStage<AT> &st = stages[s];
        const int64_t i = (blockIdx.x + k * gridDim.x) * kChunk + t;
        float sq = 0.f;
#pragma unroll
        for (int r = 4; r < 7; ++r) {
            const float x = to_f32(st.attr[r][t]);
            sq = fmaf(x, x, sq);
        }
#pragma unroll 15
        for (int r = 7; r < kFeatAttrRows; ++r) {
            const float x = to_f32(st.attr[r][t]);
            sq = fmaf(x, x, sq);
        }
        m_col[i] = feat_terms(acc, st.pos[0][t], st.pos[1][t], st.pos[2][t], to_f32(st.attr[0][t]),
                              to_f32(st.attr[1][t]), to_f32(st.attr[2][t]), to_f32(st.attr[3][t]),
                              to_f32(st.attr[4][t]), to_f32(st.attr[5][t]), to_f32(st.attr[6][t]), sq, eta, l0, l1,
                              l2);
        __syncthreads();  // every thread is done with this stage
        if (k + kStages < mine) {
            if (t < 32) {
                fence_proxy_async_smem();
                issue_feat(&stages[s], &bars[s], pos, attr, S, (blockIdx.x + (k + kStages) * gridDim.x) * kChunk,
                           lane);
            }
            ++issued[s];
        }
    }
    // the partial chunk at the end: the block that would own it, plain loads
    const int64_t tail0 = full * kChunk;
    if (tail0 < n && (full % gridDim.x) == blockIdx.x) {
        const int64_t i = tail0 + t;
        if (i < n) {
            float sq = 0.f;
            for (int r = 8; r < 56; ++r) {
                const float x = ld_attr(attr + r * S + i);
                sq = fmaf(x, x, sq);
            }
            m_col[i] = feat_terms(acc, __ldg(pos + i), __ldg(pos + S + i), __ldg(pos + 2 * S + i), ld_attr(attr + i),
                                  ld_attr(attr + S + i), ld_attr(attr + 2 * S + i), ld_attr(attr + 7 * S + i),
                                  ld_attr(attr + 8 * S + i), ld_attr(attr + 9 * S + i), ld_attr(attr + 10 * S + i),
                                  sq, eta, l0, l1, l2);
        }
    }
    if (!isfinite(acc.bad)) set_status(status, kEnonfinite);

    // fixed-order block reduction in double (shared memory reused)
    __syncthreads();
    double *red = reinterpret_cast<double *>(smem_raw);  // [kFeatSums][kChunk]
#pragma unroll
    for (int k = 0; k < kFeatSums; ++k) red[k * kChunk + t] = (double)acc.s[k];
    __syncthreads();
    for (int h = kChunk / 2; h > 0; h >>= 1) {
        if (t < h) {
#pragma unroll
            for (int k = 0; k < kFeatSums; ++k) red[k * kChunk + t] += red[k * kChunk + t + h];
        }
        __syncthreads();
    }
    if (t < kFeatSums) partials[(int64_t)blockIdx.x * kFeatSums + t] = red[t * kChunk];
}

template <typename AT>
static size_t feat_smem() { return sizeof(FeatStage<AT>) * kStages; }

int feature_tma_blocks(int num_sms, int dtype)
{
    const size_t smem = dtype == REFINE_BF16 ? feat_smem<__nv_bfloat16>() : feat_smem<float>();
    const int per_sm = (int)((227u * 1024u) / (smem + 1024));
    return num_sms * (per_sm < 1 ? 1 : per_sm);
}

cudaError_t launch_features_tma(const float *pos, const void *attr, int dtype, int64_t stride, int64_t n,
                                float eta, const float luma[3], float *m_col, double *partials, int nblocks,
                                int *status, cudaStream_t s)
{
    if (dtype == REFINE_BF16) {
        const size_t smem = feat_smem<__nv_bfloat16>();
        cudaError_t e = cudaFuncSetAttribute(k_features_tma<__nv_bfloat16>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_features_tma<__nv_bfloat16><<<nblocks, kChunk, smem, s>>>(
            pos, static_cast<const __nv_bfloat16 *>(attr), stride, n, eta, luma[0], luma[1], luma[2], m_col,
            partials, status);
    } else {
        const size_t smem = feat_smem<float>();
        cudaError_t e =
            cudaFuncSetAttribute(k_features_tma<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_features_tma<float><<<nblocks, kChunk, smem, s>>>(pos, static_cast<const float *>(attr), stride, n, eta,
                                                            luma[0], luma[1], luma[2], m_col, partials, status);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------- compaction
// Chunk = one compaction segment of 256 elements (8 mask words).
template <typename AT>
struct CmpStage {
    float pos[3][kChunk];
    AT attr[56][kChunk];
};

template <typename AT>
__device__ __forceinline__ void issue_cmp(CmpStage<AT> *st, uint64_t *bar, const float *pos, const AT *attr,
                                          int64_t S, int64_t base, int lane)
{
    constexpr uint32_t bytes = 3 * kChunk * 4 + 56 * kChunk * sizeof(AT);
    if (lane == 0) mbar_expect_tx(bar, bytes);
    __syncwarp();
    for (int r = lane; r < 59; r += 32) {
        if (r < 3)
            bulk_g2s(st->pos[r], pos + r * S + base, kChunk * 4, bar);
        else
            bulk_g2s(st->attr[r - 3], attr + (r - 3) * S + base, kChunk * sizeof(AT), bar);
    }
}

// Builds the kept list of a chunk: list[k] = position within the chunk of
// the k-th kept element; returns the kept count.
__device__ __forceinline__ int kept_list(const uint32_t *mask, int64_t word0, int64_t words, int64_t limit,
                                        int *list, int *wcnt)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t w = word0 + warp;
    uint32_t word = w < words ? __ldg(mask + w) : 0u;
    const int64_t valid = limit - (int64_t)warp * 32;  // elements of this word inside the scene
    if (valid < 32) word &= valid <= 0 ? 0u : ((1u << valid) - 1u);
    const bool keep = (word >> lane) & 1u;
    if (lane == 0) wcnt[warp] = __popc(word);
    __syncthreads();
    int off = 0, total = 0;
#pragma unroll
    for (int k = 0; k < kChunk / 32; ++k) {
        off += k < warp ? wcnt[k] : 0;
        total += wcnt[k];
    }
    if (keep) list[off + __popc(word & ((1u << lane) - 1u))] = t;
    __syncthreads();
    return total;
}

template <typename AT, bool TMA>
__global__ void __launch_bounds__(kChunk) k_compact_stream(const float *__restrict__ pos, const AT *__restrict__ attr,
                                                           int64_t S, int64_t n, const uint32_t *__restrict__ mask,
                                                           const unsigned long long *__restrict__ seg_off,
                                                           const CmpState *cs, float *__restrict__ out_pos,
                                                           AT *__restrict__ out_attr, int64_t OS,
                                                           int32_t *__restrict__ out_idx, int *status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    CmpStage<AT> *stages = reinterpret_cast<CmpStage<AT> *>(smem_raw);
    __shared__ __align__(8) uint64_t bars[kCmpStages];
    __shared__ int list[kChunk];
    __shared__ int wcnt[kChunk / 32];
    if (!cs->ok) return;
    const int t = threadIdx.x, lane = t & 31;
    const int64_t nseg = (n + kChunk - 1) / kChunk;
    const int64_t words = (n + 31) / 32;
    const int64_t full = TMA ? n / kChunk : 0;  // chunks fed by the copy engine
    const int64_t mine = full > blockIdx.x ? (full - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    int issued[kCmpStages] = {}, waited[kCmpStages] = {};
    if (TMA) {
        if (t == 0)
            for (int s = 0; s < kCmpStages; ++s) mbar_init(&bars[s], 1);
        __syncthreads();
        if (t < 32)
            for (int s = 0; s < kCmpStages && s < mine; ++s)
                issue_cmp(&stages[s], &bars[s], pos, attr, S, (blockIdx.x + (int64_t)s * gridDim.x) * kChunk, lane);
        for (int s = 0; s < kCmpStages && s < mine; ++s) issued[s] = 1;
    }
    for (int64_t k = 0; k < mine; ++k) {
        const int s = (int)(k % kCmpStages);
        const int64_t sg = blockIdx.x + k * gridDim.x;
        const int cnt = kept_list(mask, sg * (kChunk / 32), words, n - sg * kChunk, list, wcnt);
        if (!mbar_wait_bounded(&bars[s], (uint32_t)(waited[s] & 1))) {
            set_status(status, kEtimeout);
            drain_stages<kCmpStages>(bars, issued, waited);
            return;
        }
        ++waited[s];
        const CmpStage<AT> &st = stages[s];
        const int64_t o = (int64_t)seg_off[sg];
        if (t < cnt) {
            const int e = list[t];
            if (out_idx) out_idx[o + t] = (int32_t)(sg * kChunk + e);
#pragma unroll
            for (int r = 0; r < 3; ++r) out_pos[r * OS + o + t] = st.pos[r][e];
#pragma unroll 8
            for (int r = 0; r < 56; ++r) out_attr[r * OS + o + t] = st.attr[r][e];
        }
        __syncthreads();  // stage and list free again
        if (k + kCmpStages < mine) {
            if (t < 32) {
                fence_proxy_async_smem();
                issue_cmp(&stages[s], &bars[s], pos, attr, S, (blockIdx.x + (k + kCmpStages) * gridDim.x) * kChunk,
                          lane);
            }
            ++issued[s];
        }
    }
    // segments not fed by the copy engine (the partial last one, or all of
    // them without TMA): plain loads
    for (int64_t sg = full + ((blockIdx.x + gridDim.x - full % gridDim.x) % gridDim.x); sg < nseg; sg += gridDim.x) {
        const int cnt = kept_list(mask, sg * (kChunk / 32), words, n - sg * kChunk, list, wcnt);
        const int64_t o = (int64_t)seg_off[sg];
        if (t < cnt) {
            const int64_t i = sg * kChunk + list[t];
            if (out_idx) out_idx[o + t] = (int32_t)i;
#pragma unroll
            for (int r = 0; r < 3; ++r) out_pos[r * OS + o + t] = __ldg(pos + r * S + i);
            for (int r = 0; r < 56; ++r) out_attr[r * OS + o + t] = attr[r * S + i];
        }
        __syncthreads();
    }
}

template <typename AT>
static size_t cmp_smem() { return sizeof(CmpStage<AT>) * kCmpStages; }

int compact_stream_blocks(int num_sms, int dtype)
{
    const size_t smem = dtype == REFINE_BF16 ? cmp_smem<__nv_bfloat16>() : cmp_smem<float>();
    const int per_sm = (int)((227u * 1024u) / (smem + 2048));
    return num_sms * (per_sm < 1 ? 1 : per_sm);
}

template <typename AT>
static cudaError_t launch_cmp_t(const refine_scene &in, const uint32_t *mask, const unsigned long long *seg_off,
                                const CmpState *cs, float *out_pos, void *out_attr, int64_t out_stride,
                                int32_t *out_idx, bool tma, int grid, int *status, cudaStream_t s)
{
    const AT *attr = static_cast<const AT *>(in.attr);
    AT *oattr = static_cast<AT *>(out_attr);
    if (tma) {
        const size_t smem = cmp_smem<AT>();
        cudaError_t e =
            cudaFuncSetAttribute(k_compact_stream<AT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_compact_stream<AT, true><<<grid, kChunk, smem, s>>>(in.pos, attr, in.row_stride, in.n, mask, seg_off, cs,
                                                              out_pos, oattr, out_stride, out_idx, status);
    } else {
        k_compact_stream<AT, false><<<grid, kChunk, 0, s>>>(in.pos, attr, in.row_stride, in.n, mask, seg_off, cs,
                                                            out_pos, oattr, out_stride, out_idx, status);
    }
    return cudaGetLastError();
}

cudaError_t launch_compact_stream(const refine_scene &in, const uint32_t *mask, const unsigned long long *seg_off,
                                  const CmpState *cs, float *out_pos, void *out_attr, int64_t out_stride,
                                  int32_t *out_idx, bool tma, int grid, int *status, cudaStream_t s)
{
    if (in.dtype == REFINE_BF16)
        return launch_cmp_t<__nv_bfloat16>(in, mask, seg_off, cs, out_pos, out_attr, out_stride, out_idx, tma, grid,
                                           status, s);
    return launch_cmp_t<float>(in, mask, seg_off, cs, out_pos, out_attr, out_stride, out_idx, tma, grid, status, s);
}

}  // namespace refine
