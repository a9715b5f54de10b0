// Compaction, pass 2: the scatter of every row of the kept primitives, in
// one of two forms chosen by compact_shape from the scene's size and type.
//
// Word form (k_compact_warp).  One warp handles one mask word (32
// primitives) at a time; its output offset is the offset of its segment of
// kCmpSeg = 256 primitives (from pass 1, k_compact_count) plus the kept bits
// of the segment's earlier words.  The warp inverts the ranks of the kept
// bits once (lane d of the output reads from the lane holding the d-th kept
// primitive), then moves each of the 59 rows with one coalesced load, one
// shuffle and one contiguous store.  The loads of sixteen float rows, or of
// 28 bfloat16 rows (64-byte warp loads, so more of them must be in flight),
// are issued together.  The CTA is 8 warps with a few hundred bytes of
// shared memory; at 40 registers per thread (FP32 rows) an SM keeps 48 warps
// and their 768 row loads resident, at 64 (bfloat16 rows) 32 warps and 896.
//
// Segment form (k_compact_seg, FP32 attributes only).  One warp owns a
// whole segment (8 mask words); the offsets of its words come from a shuffle
// scan of their kept counts.  Each row moves with 8 coalesced loads (one
// contiguous 1 KB span of the row), 8 shuffles and 8 stores that together
// write one contiguous run of the output row.  Two rows (16 loads) are in
// flight per warp; 80 registers hold the per-word ranks and offsets, so 3
// CTAs of 8 warps fit per SM.  It keeps a quarter of the word form's warps in
// flight, which pays only when each warp has several segments to stream.
//
// No shared-memory staging of the rows in either form.
#include "internal.h"

namespace refine {

constexpr int kCmpWarps = 8;
constexpr int kCmpBatch = 16;      // float rows in flight per warp
constexpr int kCmpBatchB16 = 28;   // bfloat16 rows in flight per warp (56 rows in two steps)

__device__ __forceinline__ float shfl_row(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ __nv_bfloat16 shfl_row(__nv_bfloat16 v, int src)
{
    const unsigned short b = __shfl_sync(0xffffffffu, __bfloat16_as_ushort(v), src);
    return __ushort_as_bfloat16(b);
}

template <typename T, int NR, int B = (sizeof(T) == 2 ? kCmpBatchB16 : kCmpBatch)>
__device__ __forceinline__ void move_rows(const T *__restrict__ in, int64_t S, bool ld, int src, T *__restrict__ out,
                                          int64_t OS, bool st)
{
#pragma unroll 1
    for (int r0 = 0; r0 < NR; r0 += B) {
        T v[B];
#pragma unroll
        for (int k = 0; k < B; ++k) v[k] = (ld && r0 + k < NR) ? in[k * S] : T(0.f);
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const T x = shfl_row(v[k], src);
            if (st && r0 + k < NR) out[k * OS] = x;
        }
        in += B * S;
        out += B * OS;
    }
}

// DT is the storage type of the attribute rows: its float32 rows are moved
// as float, the rest as bfloat16, each block of rows from and to its own
// place in the layout (attr_f32_rows).
template <int DT>
__global__ void __launch_bounds__(32 * kCmpWarps) k_compact_warp(const float *__restrict__ pos,
                                                                 const void *__restrict__ attr, int64_t S, int64_t n,
                                                                 const uint32_t *__restrict__ mask,
                                                                 const unsigned long long *__restrict__ seg_off,
                                                                 const CmpState *cs, float *__restrict__ out_pos,
                                                                 void *__restrict__ out_attr, int64_t OS,
                                                                 int32_t *__restrict__ out_idx)
{
    constexpr int NF = attr_f32_rows(DT), NB = 56 - NF;
    const float *in_f = static_cast<const float *>(attr);
    const __nv_bfloat16 *in_b =
        reinterpret_cast<const __nv_bfloat16 *>(static_cast<const char *>(attr) + (size_t)NF * 4 * (size_t)S);
    float *out_f = static_cast<float *>(out_attr);
    __nv_bfloat16 *out_b = reinterpret_cast<__nv_bfloat16 *>(static_cast<char *>(out_attr) + (size_t)NF * 4 * (size_t)OS);
    __shared__ unsigned char src_of[kCmpWarps][32];
    if (!cs->ok) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    constexpr int kWords = kCmpSeg / 32;
    const int64_t words = (n + 31) / 32;
    for (int64_t w = (int64_t)blockIdx.x * kCmpWarps + wib; w < words; w += (int64_t)gridDim.x * kCmpWarps) {
        // lane k < (w mod 8) holds the k-th earlier word of the segment, lane
        // 31 this word; bits past n cleared
        const int64_t w0 = w & ~(int64_t)(kWords - 1);
        const int64_t wl = lane == 31 ? w : w0 + lane;
        uint32_t word = 0u;
        if (lane == 31 || wl < w) {
            word = __ldg(mask + wl);
            const int64_t valid = n - wl * 32;
            if (valid < 32) word &= (1u << valid) - 1u;
        }
        const uint32_t wk = __shfl_sync(0xffffffffu, word, 31);
        const int kept = __popc(wk);
        if (kept == 0) continue;  // uniform
        const int before = __reduce_add_sync(0xffffffffu, lane == 31 ? 0u : (unsigned)__popc(word));
        const int64_t base = w * 32;
        const int64_t dst = (int64_t)__ldg(seg_off + w / kWords) + before + lane;
        if ((wk >> lane) & 1u) src_of[wib][__popc(wk & ((1u << lane) - 1u))] = (unsigned char)lane;
        __syncwarp();
        const int src = lane < kept ? src_of[wib][lane] : lane;
        __syncwarp();
        const bool ld = base + lane < n;
        const bool st = lane < kept;
        if (out_idx && st) out_idx[dst] = (int32_t)(base + src);
        move_rows<float, 3>(pos + base + lane, S, ld, src, out_pos + dst, OS, st);
        if constexpr (NF > 0) move_rows<float, NF>(in_f + base + lane, S, ld, src, out_f + dst, OS, st);
        if constexpr (NB > 0) move_rows<__nv_bfloat16, NB>(in_b + base + lane, S, ld, src, out_b + dst, OS, st);
    }
}

constexpr int kSegRows = 2;  // rows in flight per warp (8 loads each)

// The 59 rows of one primitive are pos rows 0..2 then attr rows 0..55; for
// FP32 attributes both are float, so one loop walks all 59.
__device__ __forceinline__ const float *seg_row(const float *pos, const float *attr, int64_t S, int r)
{
    return r < 3 ? pos + (int64_t)r * S : attr + (int64_t)(r - 3) * S;
}
__device__ __forceinline__ float *seg_row(float *pos, float *attr, int64_t S, int r)
{
    return r < 3 ? pos + (int64_t)r * S : attr + (int64_t)(r - 3) * S;
}

__global__ void __launch_bounds__(32 * kCmpWarps, 3) k_compact_seg(const float *__restrict__ pos,
                                                                   const float *__restrict__ attr, int64_t S,
                                                                   int64_t n, const uint32_t *__restrict__ mask,
                                                                   const unsigned long long *__restrict__ seg_off,
                                                                   const CmpState *cs, float *__restrict__ out_pos,
                                                                   float *__restrict__ out_attr, int64_t OS,
                                                                   int32_t *__restrict__ out_idx)
{
    constexpr int kWords = kCmpSeg / 32;
    constexpr int kRows = 3 + 56;
    static_assert(kWords == 8, "a segment is 8 mask words");
    __shared__ unsigned char src_of[kCmpWarps][kWords][32];
    if (!cs->ok) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nseg = (n + kCmpSeg - 1) / kCmpSeg;
    const int64_t words = (n + 31) / 32;
    for (int64_t sg = (int64_t)blockIdx.x * kCmpWarps + wib; sg < nseg; sg += (int64_t)gridDim.x * kCmpWarps) {
        // lane w < 8 holds word w of the segment, bits past n cleared
        uint32_t word = 0u;
        {
            const int64_t w = sg * kWords + lane;
            if (lane < kWords && w < words) {
                word = __ldg(mask + w);
                const int64_t valid = n - w * 32;
                if (valid < 32) word &= (1u << valid) - 1u;
            }
        }
        int incl = __popc(word);  // inclusive scan of the kept counts over the 8 words
#pragma unroll
        for (int o = 1; o < kWords; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        const int64_t base = sg * kCmpSeg;
        const int64_t o0 = (int64_t)__ldg(seg_off + sg);
        int kept[kWords], off[kWords], src[kWords];
        bool ld[kWords];
#pragma unroll
        for (int w = 0; w < kWords; ++w) {
            const uint32_t wk = __shfl_sync(0xffffffffu, word, w);
            kept[w] = __popc(wk);
            off[w] = __shfl_sync(0xffffffffu, incl, w) - kept[w];
            if ((wk >> lane) & 1u) src_of[wib][w][__popc(wk & ((1u << lane) - 1u))] = (unsigned char)lane;
            ld[w] = base + 32 * w + lane < n;
        }
        __syncwarp();
#pragma unroll
        for (int w = 0; w < kWords; ++w) src[w] = lane < kept[w] ? src_of[wib][w][lane] : lane;
        __syncwarp();
        if (out_idx)
#pragma unroll
            for (int w = 0; w < kWords; ++w)
                if (lane < kept[w]) out_idx[o0 + off[w] + lane] = (int32_t)(base + 32 * w + src[w]);
        const float *in_p = pos + base + lane, *in_a = attr + base + lane;
        float *out_p = out_pos + o0, *out_a = out_attr + o0;
#pragma unroll 1
        for (int r0 = 0; r0 < kRows; r0 += kSegRows) {
            float v[kSegRows][kWords];
#pragma unroll
            for (int k = 0; k < kSegRows; ++k) {
                const float *in = seg_row(in_p, in_a, S, r0 + k);
#pragma unroll
                for (int w = 0; w < kWords; ++w) v[k][w] = (ld[w] && r0 + k < kRows) ? in[32 * w] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < kSegRows; ++k) {
                if (r0 + k >= kRows) break;  // uniform
                float *out = seg_row(out_p, out_a, OS, r0 + k);
#pragma unroll
                for (int w = 0; w < kWords; ++w) {
                    const float x = shfl_row(v[k][w], src[w]);
                    if (lane < kept[w]) out[off[w] + lane] = x;
                }
            }
        }
    }
}

// The segment form for FP32 rows once every resident warp of it gets two
// segments or more (n of 1.87M or more on 152 SMs); the word form otherwise.
// Measured on 3.5M primitives, FP32 rows: 0.199 ms against 0.249 ms; BF16
// rows: 0.164 ms both; 1M primitives: 0.084 ms against 0.067 ms.  Work is
// dealt round-robin over at most 6 CTAs per SM: for the segment form that is
// two waves of 3, the second filling SMs whose first CTAs finish early.
CmpShape compact_shape(int num_sms, int64_t n, int dtype)
{
    const int64_t nseg = (n + kCmpSeg - 1) / kCmpSeg;
    const bool seg = dtype == REFINE_F32 && nseg >= 2 * (int64_t)num_sms * 3 * kCmpWarps;
    const int64_t units = seg ? nseg : (n + 31) / 32;
    int64_t g = (units + kCmpWarps - 1) / kCmpWarps;
    const int64_t cap = (int64_t)num_sms * 6;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return {(int)g, seg};
}

cudaError_t launch_compact_scatter(const refine_scene &in, const uint32_t *mask, const unsigned long long *seg_off,
                                   const CmpState *cs, float *out_pos, void *out_attr, int64_t out_stride,
                                   int32_t *out_idx, CmpShape shape, cudaStream_t s)
{
    if (in.dtype == REFINE_BF16) {
        k_compact_warp<REFINE_BF16><<<shape.grid, 32 * kCmpWarps, 0, s>>>(
            in.pos, in.attr, in.row_stride, in.n, mask, seg_off, cs, out_pos, out_attr, out_stride, out_idx);
    } else if (in.dtype == REFINE_BF16S) {
        k_compact_warp<REFINE_BF16S><<<shape.grid, 32 * kCmpWarps, 0, s>>>(
            in.pos, in.attr, in.row_stride, in.n, mask, seg_off, cs, out_pos, out_attr, out_stride, out_idx);
    } else {
        const float *a = static_cast<const float *>(in.attr);
        float *oa = static_cast<float *>(out_attr);
        if (shape.seg)
            k_compact_seg<<<shape.grid, 32 * kCmpWarps, 0, s>>>(in.pos, a, in.row_stride, in.n, mask, seg_off, cs,
                                                                out_pos, oa, out_stride, out_idx);
        else
            k_compact_warp<REFINE_F32><<<shape.grid, 32 * kCmpWarps, 0, s>>>(in.pos, a, in.row_stride, in.n, mask,
                                                                             seg_off, cs, out_pos, oa, out_stride,
                                                                             out_idx);
    }
    return cudaGetLastError();
}

}  // namespace refine
