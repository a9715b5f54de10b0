// Compaction, pass 2: the scatter of every row of the kept primitives.
//
// One warp handles one mask word (32 primitives) at a time; its output
// offset is the offset of its segment of kCmpSeg = 256 primitives (from pass
// 1, k_compact_count) plus the kept bits of the segment's earlier words.  The
// warp inverts the ranks of the kept bits once (lane d of the output reads
// from the lane holding the d-th kept primitive), then moves each of the 59
// rows with one coalesced load, one shuffle and one contiguous store; the
// loads of sixteen rows are in flight at a time.  No shared-memory staging:
// the CTA is 8 warps with a few hundred bytes of shared memory and 40
// registers per thread, so an SM keeps 48 warps, and their 768 row loads,
// resident.
#include "internal.h"

namespace refine {

constexpr int kCmpWarps = 8;
constexpr int kCmpBatch = 16;  // rows in flight per warp

__device__ __forceinline__ float shfl_row(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ __nv_bfloat16 shfl_row(__nv_bfloat16 v, int src)
{
    const unsigned short b = __shfl_sync(0xffffffffu, __bfloat16_as_ushort(v), src);
    return __ushort_as_bfloat16(b);
}

template <typename T, int NR>
__device__ __forceinline__ void move_rows(const T *__restrict__ in, int64_t S, bool ld, int src, T *__restrict__ out,
                                          int64_t OS, bool st)
{
#pragma unroll 1
    for (int r0 = 0; r0 < NR; r0 += kCmpBatch) {
        T v[kCmpBatch];
#pragma unroll
        for (int k = 0; k < kCmpBatch; ++k) v[k] = (ld && r0 + k < NR) ? in[k * S] : T(0.f);
#pragma unroll
        for (int k = 0; k < kCmpBatch; ++k) {
            const T x = shfl_row(v[k], src);
            if (st && r0 + k < NR) out[k * OS] = x;
        }
        in += kCmpBatch * S;
        out += kCmpBatch * OS;
    }
}

template <typename AT>
__global__ void __launch_bounds__(32 * kCmpWarps) k_compact_warp(const float *__restrict__ pos,
                                                                 const AT *__restrict__ attr, int64_t S, int64_t n,
                                                                 const uint32_t *__restrict__ mask,
                                                                 const unsigned long long *__restrict__ seg_off,
                                                                 const CmpState *cs, float *__restrict__ out_pos,
                                                                 AT *__restrict__ out_attr, int64_t OS,
                                                                 int32_t *__restrict__ out_idx)
{
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
        move_rows<AT, 56>(attr + base + lane, S, ld, src, out_attr + dst, OS, st);
    }
}

// Every warp of the resident grid stays busy to the end: words are dealt
// round-robin (a warp's rows are latency-bound chains, so the load is
// spread over as many warps as fit).
int compact_grid(int num_sms, int64_t n)
{
    const int64_t words = (n + 31) / 32;
    int64_t g = (words + kCmpWarps - 1) / kCmpWarps;
    const int64_t cap = (int64_t)num_sms * 6;  // 6 CTAs of 8 warps fit per SM (40 registers per thread)
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_compact_scatter(const refine_scene &in, const uint32_t *mask, const unsigned long long *seg_off,
                                   const CmpState *cs, float *out_pos, void *out_attr, int64_t out_stride,
                                   int32_t *out_idx, int grid, cudaStream_t s)
{
    if (in.dtype == REFINE_BF16)
        k_compact_warp<__nv_bfloat16><<<grid, 32 * kCmpWarps, 0, s>>>(
            in.pos, static_cast<const __nv_bfloat16 *>(in.attr), in.row_stride, in.n, mask, seg_off, cs, out_pos,
            static_cast<__nv_bfloat16 *>(out_attr), out_stride, out_idx);
    else
        k_compact_warp<float><<<grid, 32 * kCmpWarps, 0, s>>>(in.pos, static_cast<const float *>(in.attr),
                                                              in.row_stride, in.n, mask, seg_off, cs, out_pos,
                                                              static_cast<float *>(out_attr), out_stride, out_idx);
    return cudaGetLastError();
}

}  // namespace refine
