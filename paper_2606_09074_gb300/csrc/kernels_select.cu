// Ratio pruning (Sec. 3.3): radix select of the n_keep-th largest score with
// an index tie-break, keep-mask construction, and stable compaction.
#include "internal.h"

namespace refine {

// Radix digits from the most significant end: 11, 11 and 10 bits.
__host__ __device__ constexpr int pass_shift(int p) { return p == 0 ? 21 : (p == 1 ? 10 : 0); }
__host__ __device__ constexpr int pass_width(int p) { return p == 2 ? 10 : 11; }

constexpr int kSelThreads = 512;

// Inclusive suffix sum over the block (thread t receives the sum of the
// values of threads t..blockDim-1), blockDim == kSelThreads.
__device__ unsigned int block_suffix_sum(unsigned int v, unsigned int *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int x = __shfl_down_sync(0xffffffffu, s, o);
        if (lane + o < 32) s += x;
    }
    if (lane == 0) wsum[warp] = s;
    __syncthreads();
    if (warp == 0) {
        unsigned int w = lane < kSelThreads / 32 ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned int x = __shfl_down_sync(0xffffffffu, w, o);
            if (lane + o < 32) w += x;
        }
        if (lane < kSelThreads / 32) wsum[lane] = w;  // inclusive suffix over warps
    }
    __syncthreads();
    unsigned int after = (warp + 1 < kSelThreads / 32) ? wsum[warp + 1] : 0u;
    unsigned int r = s + after;
    __syncthreads();
    return r;
}

// Inclusive prefix sum over the block.
__device__ unsigned long long block_prefix_sum(unsigned long long v, unsigned long long *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long x = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += x;
    }
    if (lane == 31) wsum[warp] = s;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nw ? wsum[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long x = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += x;
        }
        if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    unsigned long long r = s + (warp > 0 ? wsum[warp - 1] : 0ull);
    __syncthreads();
    return r;
}

// One histogram pass over the keys that match the digits decided so far.
// The last CTA to finish chooses the digit of the n_keep-th largest key.
template <int PASS, bool VEC>
__global__ void __launch_bounds__(kSelThreads) k_select_pass(const float *__restrict__ scores, int64_t n,
                                                             uint32_t n_keep, SelState *st, int *status)
{
    constexpr int SHIFT = pass_shift(PASS), WIDTH = pass_width(PASS), NB = 1 << WIDTH;
    __shared__ unsigned int h[2048];
    __shared__ unsigned int wsum[32];
    __shared__ unsigned int is_last;
    for (int b = threadIdx.x; b < NB; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const unsigned int prefix = PASS == 0 ? 0u : st->prefix;
    bool bad = false;
    // Every lane of a warp runs the same iterations (warp-uniform bounds), so
    // the full-mask match below sees a converged warp; `valid` masks lanes.
    auto add = [&](float f, bool valid) {
        bad |= valid && isnan(f);
        const uint32_t k = score_key(f);
        const bool match = valid && (PASS == 0 ? true : ((k >> (SHIFT + WIDTH)) == prefix));
        // after the first pass few keys still match the digits decided so
        // far: a warp with none skips the grouping
        if (PASS > 0 && !__any_sync(0xffffffffu, match)) return;
        const unsigned int d = (k >> SHIFT) & (NB - 1);
        const unsigned int grp = __match_any_sync(0xffffffffu, match ? d : 0xffffffffu);
        if (match && (__ffs(grp) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&h[d], __popc(grp));
    };
    const int lane = threadIdx.x & 31;
    const int64_t wbase = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    int64_t done_to = 0;
    if (VEC) {
        const int64_t n4 = n / 4;
        const float4 *s4 = reinterpret_cast<const float4 *>(scores);
        for (int64_t i0 = wbase; i0 < n4; i0 += nthr) {
            const int64_t i = i0 + lane;
            const bool valid = i < n4;
            const float4 q = valid ? __ldg(s4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            add(q.x, valid); add(q.y, valid); add(q.z, valid); add(q.w, valid);
        }
        done_to = n4 * 4;
    }
    for (int64_t i0 = done_to + wbase; i0 < n; i0 += nthr) {
        const int64_t i = i0 + lane;
        const bool valid = i < n;
        add(valid ? __ldg(scores + i) : 0.f, valid);
    }
    if (PASS == 0 && bad) set_status(status, kEnonfinite);
    __syncthreads();
    for (int b = threadIdx.x; b < NB; b += blockDim.x)
        if (h[b]) atomicAdd(&st->hist[b], h[b]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(&st->done, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();

    // Choose the bucket: thread t owns bins [t*PER, t*PER + PER).
    constexpr int PER = NB / kSelThreads;
    unsigned int cnt[PER], loc = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        cnt[k] = atomicAdd(&st->hist[threadIdx.x * PER + k], 0u);  // coherent read
        loc += cnt[k];
    }
    const unsigned int remaining = PASS == 0 ? n_keep : st->remaining;
    const unsigned int incl = block_suffix_sum(loc, wsum);  // bins >= my first bin
    const unsigned int excl = incl - loc;                   // bins above my range
    if (excl < remaining && remaining <= incl) {
        unsigned int above = excl;
        for (int k = PER - 1; k >= 0; --k) {
            if (above + cnt[k] >= remaining) {
                const unsigned int digit = threadIdx.x * PER + k;
                const unsigned int rem = remaining - above;
                st->count_gt = (PASS == 0 ? 0u : st->count_gt) + above;
                st->remaining = rem;
                st->prefix = (prefix << WIDTH) | digit;
                if (PASS == 2) {
                    st->kstar = (prefix << WIDTH) | digit;
                    st->cnt_eq = cnt[k];
                    st->need_ties = cnt[k] > rem ? 1u : 0u;
                    st->idx_cut = n;  // refined by k_select_ties when needed
                }
                break;
            }
            above += cnt[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) st->hist[threadIdx.x * PER + k] = 0u;
    if (threadIdx.x == 0) st->done = 0u;
}

int select_grid(int num_sms, int64_t n)
{
    int64_t g = (n + (int64_t)kSelThreads * 8 - 1) / ((int64_t)kSelThreads * 8);
    if (g > 2 * num_sms) g = 2 * num_sms;
    if (g < 1) g = 1;
    return (int)g;
}

template <int PASS>
static cudaError_t launch_pass_t(const float *scores, int64_t n, uint32_t n_keep, SelState *st,
                                 bool vec, int grid, int *status, cudaStream_t s)
{
    if (vec)
        k_select_pass<PASS, true><<<grid, kSelThreads, 0, s>>>(scores, n, n_keep, st, status);
    else
        k_select_pass<PASS, false><<<grid, kSelThreads, 0, s>>>(scores, n, n_keep, st, status);
    return cudaGetLastError();
}

cudaError_t launch_select_pass(int pass, const float *scores, int64_t n, uint32_t n_keep,
                               SelState *st, bool vec, int grid, int *status, cudaStream_t s)
{
    if (pass == 0) return launch_pass_t<0>(scores, n, n_keep, st, vec, grid, status, s);
    if (pass == 1) return launch_pass_t<1>(scores, n, n_keep, st, vec, grid, status, s);
    return launch_pass_t<2>(scores, n, n_keep, st, vec, grid, status, s);
}

// Index tie-break: when more keys equal k* than remain to be kept, find the
// index of the `remaining`-th such key in index order.  Segments of kTieSeg
// elements are counted; the last CTA locates the segment and the element.
__global__ void __launch_bounds__(kSelThreads) k_select_ties(const float *__restrict__ scores, int64_t n,
                                                             SelState *st, unsigned *seg_cnt)
{
    if (!st->need_ties) return;
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned int is_last;
    __shared__ long long found_seg;
    __shared__ unsigned long long seg_base;
    const uint32_t kstar = st->kstar;
    const int64_t nseg = (n + kTieSeg - 1) / kTieSeg;
    for (int64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        unsigned int c = 0;
        const int64_t e1 = min(n, (sg + 1) * (int64_t)kTieSeg);
        for (int64_t i = sg * (int64_t)kTieSeg + threadIdx.x; i < e1; i += blockDim.x)
            c += score_key(__ldg(scores + i)) == kstar;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        __shared__ unsigned int red[kSelThreads / 32];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int t = 0;
            for (int w = 0; w < kSelThreads / 32; ++w) t += red[w];
            seg_cnt[sg] = t;
        }
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(&st->done, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const unsigned long long target = st->remaining;  // 1-based rank among equal keys
    if (threadIdx.x == 0) found_seg = -1;
    __syncthreads();
    unsigned long long run = 0;
    for (int64_t c0 = 0; c0 < nseg; c0 += blockDim.x) {
        const int64_t sg = c0 + threadIdx.x;
        const unsigned long long v = sg < nseg ? atomicAdd(&seg_cnt[sg], 0u) : 0ull;
        const unsigned long long incl = block_prefix_sum(v, wsum) + run;
        if (sg < nseg && incl - v < target && target <= incl) {
            found_seg = sg;
            seg_base = incl - v;
        }
        __syncthreads();
        if (found_seg >= 0) break;
        // the running total is the inclusive sum of the chunk's last thread
        __shared__ unsigned long long chunk_end;
        if (threadIdx.x == blockDim.x - 1) chunk_end = incl;
        __syncthreads();
        run = chunk_end;
        __syncthreads();
    }
    const int64_t sg = found_seg;
    if (sg >= 0) {
        unsigned long long base = seg_base;
        const int64_t e1 = min(n, (sg + 1) * (int64_t)kTieSeg);
        for (int64_t i0 = sg * (int64_t)kTieSeg; i0 < e1; i0 += blockDim.x) {
            const int64_t i = i0 + threadIdx.x;
            const unsigned long long eq = (i < e1 && score_key(__ldg(scores + i)) == kstar) ? 1ull : 0ull;
            const unsigned long long incl = block_prefix_sum(eq, wsum) + base;
            if (eq && incl == target) st->idx_cut = i;
            __shared__ unsigned long long cend;
            if (threadIdx.x == blockDim.x - 1) cend = incl;
            __syncthreads();
            base = cend;
            __syncthreads();
            if (base >= target) break;
        }
    }
    if (threadIdx.x == 0) st->done = 0u;
}

cudaError_t launch_select_ties(const float *scores, int64_t n, SelState *st, unsigned *seg_cnt,
                               int grid, cudaStream_t s)
{
    k_select_ties<<<grid, kSelThreads, 0, s>>>(scores, n, st, seg_cnt);
    return cudaGetLastError();
}

// Keep mask: a warp builds kMaskWords consecutive 32-element words per
// step, their loads issued together.
constexpr int kMaskWords = 4;

__global__ void k_select_mask(const float *__restrict__ scores, int64_t n, const SelState *st,
                              uint32_t *__restrict__ mask)
{
    const uint32_t kstar = st->kstar;
    const long long cut = st->idx_cut;
    const int64_t words = (n + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w0 = warp0 * kMaskWords; w0 < words; w0 += nwarps * kMaskWords) {
        float v[kMaskWords];
#pragma unroll
        for (int u = 0; u < kMaskWords; ++u) {
            const int64_t i = (w0 + u) * 32 + lane;
            v[u] = i < n ? __ldg(scores + i) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kMaskWords; ++u) {
            const int64_t i = (w0 + u) * 32 + lane;
            const uint32_t k = score_key(v[u]);
            const bool keep = i < n && (k > kstar || (k == kstar && i <= cut));
            const uint32_t word = __ballot_sync(0xffffffffu, keep);
            if (lane == 0 && w0 + u < words) mask[w0 + u] = word;
        }
    }
}

cudaError_t launch_select_mask(const float *scores, int64_t n, const SelState *st, uint32_t *mask,
                               int grid, cudaStream_t s)
{
    k_select_mask<<<grid, 256, 0, s>>>(scores, n, st, mask);
    return cudaGetLastError();
}

__global__ void k_mask_fill(uint32_t *mask, int64_t n)
{
    const int64_t words = (n + 31) / 32;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rem = n - w * 32;
        mask[w] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
}

cudaError_t launch_mask_fill(uint32_t *mask, int64_t n, cudaStream_t s)
{
    int64_t words = (n + 31) / 32;
    int grid = (int)((words + 255) / 256);
    if (grid > 1024) grid = 1024;
    if (grid < 1) grid = 1;
    k_mask_fill<<<grid, 256, 0, s>>>(mask, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------
// Compaction, pass 1.  Segment s covers elements [s*kCmpSeg, (s+1)*kCmpSeg)
// (8 mask words).  Kept elements are counted per segment and the last CTA
// turns the counts into exclusive offsets; the scatter of every row is
// k_compact_warp or k_compact_seg.
// ---------------------------------------------------------------------
constexpr int kCmpThreads = 1024;

__global__ void __launch_bounds__(kCmpThreads) k_compact_count(const uint32_t *__restrict__ mask, int64_t n,
                                                               unsigned *seg_cnt, unsigned long long *seg_off,
                                                               CmpState *cs, int64_t out_stride, int *status)
{
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned int is_last;
    const int64_t words = (n + 31) / 32;
    const int64_t nseg = (n + kCmpSeg - 1) / kCmpSeg;
    constexpr int kWords = kCmpSeg / 32;
    for (int64_t sg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sg < nseg;
         sg += (int64_t)gridDim.x * blockDim.x) {
        unsigned c = 0;
#pragma unroll
        for (int k = 0; k < kWords; ++k) {
            const int64_t w = sg * kWords + k;
            if (w < words) {
                uint32_t word = __ldg(mask + w);
                const int64_t valid = n - w * 32;  // bits past n do not count
                if (valid < 32) word &= (1u << valid) - 1u;
                c += __popc(word);
            }
        }
        seg_cnt[sg] = c;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(&cs->done, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // thread t takes kCmpScanU consecutive segment counts per chunk (read
    // from L2, where the other blocks' counts are)
    constexpr int kCmpScanU = 4;
    unsigned long long run = 0;
    __shared__ unsigned long long chunk_end;
    for (int64_t c0 = 0; c0 < nseg; c0 += (int64_t)blockDim.x * kCmpScanU) {
        const int64_t sg0 = c0 + (int64_t)threadIdx.x * kCmpScanU;
        unsigned v[kCmpScanU];
        unsigned long long local = 0;
#pragma unroll
        for (int u = 0; u < kCmpScanU; ++u) {
            v[u] = sg0 + u < nseg ? __ldcg(seg_cnt + sg0 + u) : 0u;
            local += v[u];
        }
        const unsigned long long incl = block_prefix_sum(local, wsum) + run;
        unsigned long long o = incl - local;
#pragma unroll
        for (int u = 0; u < kCmpScanU; ++u) {
            if (sg0 + u < nseg) seg_off[sg0 + u] = o;
            o += v[u];
        }
        if (threadIdx.x == blockDim.x - 1) chunk_end = incl;
        __syncthreads();
        run = chunk_end;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        cs->total = (long long)run;
        cs->ok = run <= (unsigned long long)out_stride ? 1u : 0u;
        if (!cs->ok) set_status(status, kEinval);
        cs->done = 0u;
    }
}

cudaError_t launch_compact_count(const uint32_t *mask, int64_t n, unsigned *seg_cnt,
                                 unsigned long long *seg_off, CmpState *cs, int64_t out_stride,
                                 int grid, int *status, cudaStream_t s)
{
    k_compact_count<<<grid, kCmpThreads, 0, s>>>(mask, n, seg_cnt, seg_off, cs, out_stride, status);
    return cudaGetLastError();
}

}  // namespace refine
