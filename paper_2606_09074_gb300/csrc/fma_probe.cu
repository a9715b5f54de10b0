// FP32 FMA throughput probe.
//
// The score kernel is bound by FP32 instruction issue, and its roofline is
// stated against the nominal FP32 peak that the unit counts and the clock
// give (SMs x 128 lanes x 2 FLOPs x clock).  This kernel measures the rate
// the device sustains on independent FMA chains at the clock it runs, as a
// measured denominator beside the nominal one.  It reads no memory and
// writes none (its one store is never taken).
#include "internal.h"

namespace refine {

namespace {

constexpr int kProbeChains = 8;     // independent FMA chains per thread
constexpr int kProbeThreads = 256;  // threads per CTA
constexpr int kProbeCtasPerSm = 8;  // 64 resident warps per SM

// Each thread advances kProbeChains independent chains x <- x a + b.  With
// 0 < a < 1 and b >= 0 every chain stays positive and bounded, so the sum is
// never -1 and the store never happens, but the compiler cannot know that
// and keeps every FMA.
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(float *sink, int iters, float a, float b)
{
    float x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += x[k];
    if (s == -1.f) *sink = s;
}

}  // namespace

double fma_probe_flops(int num_sms, int iters)
{
    return 2.0 * kProbeChains * (double)iters * (double)num_sms * kProbeCtasPerSm * kProbeThreads;
}

cudaError_t launch_fma_probe(int num_sms, int iters, float *sink, cudaStream_t s)
{
    k_fma_probe<<<num_sms * kProbeCtasPerSm, kProbeThreads, 0, s>>>(sink, iters, 0.999f, 1e-3f);
    return cudaGetLastError();
}

}  // namespace refine
