// refine_select_noalloc: ratio pruning for callers that must not allocate.
//
// Some callers cannot call cudaMalloc at all: plug-ins hosted by an engine
// that owns every device allocation, and real-time loops whose memory is
// fixed at start-up.  They cannot create a refine_ctx either (creating one
// allocates).  This entry point runs the same radix-select
// kernels as refine_select, but its scratch -- the histogram/selection state
// and the per-segment tie counts -- lives in the fixed device array below,
// which every GPU that loads the library holds until the process exits.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "internal.h"

using namespace refine;

namespace {

// Largest scene this entry point accepts.
constexpr int64_t kNoallocMaxN = int64_t(1) << 26;  // 67,108,864 primitives
constexpr int64_t kNoallocMaxSeg = (kNoallocMaxN + kTieSeg - 1) / kTieSeg;

struct NoallocScratch {
    SelState state;
    int status;
    int pad[63];
    unsigned seg[kNoallocMaxSeg];
};

// The scratch (about 74 KB).  Shared by every call on a device.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

void put_err(char *buf, size_t len, const char *msg)
{
    if (buf && len) snprintf(buf, len, "%s", msg);
}

}  // namespace

extern "C" refine_status refine_select_noalloc(const float *scores_dev, int64_t n, double ratio,
                                               uint32_t *keep_mask_dev, float *threshold_out,
                                               int64_t *n_keep_out, char *errbuf, size_t errlen,
                                               refine_stream_t stream)
{
    put_err(errbuf, errlen, "");
    if (n < 0 || n > kNoallocMaxN) {
        char m[160];
        snprintf(m, sizeof m, "refine_select_noalloc: n=%lld exceeds the fixed scratch limit of %lld primitives",
                 (long long)n, (long long)kNoallocMaxN);
        put_err(errbuf, errlen, m);
        return REFINE_EINVAL;
    }
    if (!(ratio >= 0.0 && ratio < 1.0)) {
        put_err(errbuf, errlen, "refine_select_noalloc: ratio must lie in [0, 1)");
        return REFINE_EINVAL;
    }
    const int64_t n_keep = n - (int64_t)floor(ratio * (double)n);
    if (n_keep_out) *n_keep_out = n_keep;
    if (n == 0) {
        if (threshold_out) *threshold_out = -INFINITY;
        return REFINE_OK;
    }
    if (!scores_dev || !keep_mask_dev) {
        put_err(errbuf, errlen, "refine_select_noalloc: NULL scores or mask");
        return REFINE_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        put_err(errbuf, errlen, "refine_select_noalloc: no current CUDA device");
        return REFINE_ECUDA;
    }
    // The array's device address on the current device, looked up on every
    // call (after the first call on a device, which loads the library's
    // device code there, a host-side lookup), so that it always belongs to
    // the device's current context.  In host code g_noalloc_scratch names a
    // host-side stand-in, never the device memory.
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char m[200];
        snprintf(m, sizeof m, "refine_select_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        put_err(errbuf, errlen, m);
        return REFINE_ECUDA;
    }
    NoallocScratch *scr = static_cast<NoallocScratch *>(p);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) num_sms = 1;
    const int64_t n_prune = n - n_keep;
    if (n_prune == 0) {
        e = launch_mask_fill(keep_mask_dev, n, s);
        if (e != cudaSuccess) {
            put_err(errbuf, errlen, cudaGetErrorString(e));
            return REFINE_ECUDA;
        }
        if (threshold_out) *threshold_out = -INFINITY;
        return REFINE_OK;
    }
    // The previous call's state is still in the array: clear what the
    // kernels expect to start at zero (selection state and status word).
    e = cudaMemsetAsync(scr, 0, offsetof(NoallocScratch, seg), s);
    const bool vec = (reinterpret_cast<uintptr_t>(scores_dev) & 15u) == 0;
    const int grid = select_grid(num_sms, n);
    for (int pass = 0; pass < 3 && e == cudaSuccess; ++pass)
        e = launch_select_pass(pass, scores_dev, n, (uint32_t)n_keep, &scr->state, vec, grid, &scr->status, s);
    if (e == cudaSuccess) e = launch_select_ties(scores_dev, n, &scr->state, scr->seg, grid, s);
    if (e == cudaSuccess) e = launch_select_mask(scores_dev, n, &scr->state, keep_mask_dev, grid, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        put_err(errbuf, errlen, cudaGetErrorString(e));
        return REFINE_ECUDA;
    }
    if (threshold_out) {
        unsigned int kstar = 0;
        int status = 0;
        e = cudaMemcpyAsync(&kstar, &scr->state.kstar, sizeof kstar, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &scr->status, sizeof status, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            put_err(errbuf, errlen, cudaGetErrorString(e));
            return REFINE_ECUDA;
        }
        if (status == kEnonfinite) {
            put_err(errbuf, errlen, "refine_select_noalloc: NaN score");
            return REFINE_ENONFINITE;
        }
        *threshold_out = key_to_score(kstar);
    }
    return REFINE_OK;
}
