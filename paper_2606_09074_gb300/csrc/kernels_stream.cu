// Compaction, pass 2: the scatter of every row of the kept primitives.
//
// One warp owns one segment of kCmpSeg = 256 primitives (8 mask words) at a
// time; its output offset is the segment's offset from pass 1
// (k_compact_count) plus the kept bits of the segment's earlier words, taken
// with a shuffle scan over the 8 words.  For each word the warp inverts the
// ranks of the kept bits once (lane d of the output reads from the lane
// holding the d-th kept primitive).  Each of the 59 rows then moves with 8
// coalesced loads (one contiguous 1 KB span of the row), 8 shuffles and 8
// stores that together write one contiguous run of the output row, so only
// the two ends of a run are partial sectors.  Two rows (16 loads) are in
// flight per warp; the CTA is 8 warps with 2 KB of shared memory, held to
// 3 CTAs per SM by its launch bounds.  No shared-memory staging of the rows.
#include "internal.h"

namespace refine {

constexpr int kCmpWarps = 8;
__device__ __forceinline__ float shfl_row(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ __nv_bfloat16 shfl_row(__nv_bfloat16 v, int src)
{
    const unsigned short b = __shfl_sync(0xffffffffu, __bfloat16_as_ushort(v), src);
    return __ushort_as_bfloat16(b);
}

constexpr int kSegRows = 2;  // rows in flight per warp (8 loads each)

template <typename T, int NR>
__device__ __forceinline__ void move_rows_seg(const T *__restrict__ in, int64_t S, const bool (&ld)[8],
                                              const int (&src)[8], const int (&kept)[8], T *__restrict__ out,
                                              const int (&off)[8], int64_t OS)
{
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int r0 = 0; r0 < NR; r0 += kSegRows) {
        T v[kSegRows][8];
#pragma unroll
        for (int k = 0; k < kSegRows; ++k)
#pragma unroll
            for (int w = 0; w < 8; ++w)
                v[k][w] = (ld[w] && r0 + k < NR) ? in[(int64_t)k * S + 32 * w] : T(0.f);
#pragma unroll
        for (int k = 0; k < kSegRows; ++k) {
            if (r0 + k >= NR) break;  // uniform
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const T x = shfl_row(v[k][w], src[w]);
                if (lane < kept[w]) out[(int64_t)k * OS + off[w] + lane] = x;
            }
        }
        in += kSegRows * S;
        out += kSegRows * OS;
    }
}

template <typename AT>
__global__ void __launch_bounds__(32 * kCmpWarps, 3) k_compact_seg(const float *__restrict__ pos,
                                                                   const AT *__restrict__ attr, int64_t S, int64_t n,
                                                                   const uint32_t *__restrict__ mask,
                                                                   const unsigned long long *__restrict__ seg_off,
                                                                   const CmpState *cs, float *__restrict__ out_pos,
                                                                   AT *__restrict__ out_attr, int64_t OS,
                                                                   int32_t *__restrict__ out_idx)
{
    constexpr int kWords = kCmpSeg / 32;
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
        move_rows_seg<float, 3>(pos + base + lane, S, ld, src, kept, out_pos + o0, off, OS);
        move_rows_seg<AT, 56>(attr + base + lane, S, ld, src, kept, out_attr + o0, off, OS);
    }
}

// Segments are dealt round-robin over a grid of at most 6 CTAs per SM, twice
// the 3 that the launch bounds keep resident: the second wave fills SMs whose
// first CTAs finish early (3.5M primitives, FP32 rows: 0.214 ms against
// 0.220 ms with one resident wave).
int compact_grid(int num_sms, int64_t n)
{
    const int64_t nseg = (n + kCmpSeg - 1) / kCmpSeg;
    int64_t g = (nseg + kCmpWarps - 1) / kCmpWarps;
    const int64_t cap = (int64_t)num_sms * 6;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_compact_scatter(const refine_scene &in, const uint32_t *mask, const unsigned long long *seg_off,
                                   const CmpState *cs, float *out_pos, void *out_attr, int64_t out_stride,
                                   int32_t *out_idx, int grid, cudaStream_t s)
{
    if (in.dtype == REFINE_BF16)
        k_compact_seg<__nv_bfloat16><<<grid, 32 * kCmpWarps, 0, s>>>(
            in.pos, static_cast<const __nv_bfloat16 *>(in.attr), in.row_stride, in.n, mask, seg_off, cs, out_pos,
            static_cast<__nv_bfloat16 *>(out_attr), out_stride, out_idx);
    else
        k_compact_seg<float><<<grid, 32 * kCmpWarps, 0, s>>>(in.pos, static_cast<const float *>(in.attr),
                                                              in.row_stride, in.n, mask, seg_off, cs, out_pos,
                                                              static_cast<float *>(out_attr), out_stride, out_idx);
    return cudaGetLastError();
}

}  // namespace refine
