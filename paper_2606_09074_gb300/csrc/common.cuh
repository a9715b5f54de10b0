// Internal device/host definitions shared by the librefine translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace refine {

// Device status codes; the values match refine_status in include/refine.h.
enum : int { kOk = 0, kEinval = 1, kEnonfinite = 4, kEtimeout = 5 };

// Bound on every device-side wait: ~1 s at the maximum SM clock.
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ void set_status(int *status, int code)
{
    atomicCAS(status, 0, code);  // the first error wins
}

// Derived camera record (144 bytes).  With the intrinsic matrix K and the
// world-to-camera rotation rows R0, R1, R2 (Eq. 13), each row a linear form
// (a, a0) evaluated as a . mu + a0:
//   U = P0 mu + p0, V = P1 mu + p1, z = R2 mu + t2   (P = K W, p = K t),
//   pixel (u, v) = (U / z, V / z).
struct __align__(16) CamRec {
    float4 r0;   // U:        (fx R0 + cx R2, fx t0 + cx t2)
    float4 r1;   // V:        (fy R1 + cy R2, fy t1 + cy t2)
    float4 r2;   // z:        (R2, t2)
    float4 lim;  // (width, height, znear, zfar)
    float4 k;    // (fx^2, fy^2, cx, cy)
    float4 uw;   // U - w z:  (P0 - w R2, p0 - w t2)
    float4 vh;   // V - h z:  (P1 - h R2, p1 - h t2)
    float4 tx;   // fx x:     (fx R0, fx t0)
    float4 ty;   // fy y:     (fy R1, fy t1)
};
static_assert(sizeof(CamRec) == 144, "camera record layout");

// Per-scene constants produced by the content-feature pass (Eq. 18-19) and
// the quantisation of the processing-order grid.
struct SceneConsts {
    float kappa[3];   // lambda^k / mean(m^k)  (or lambda^k without NORM_ATTR)
    float lo[3];      // grid origin (mean - 3 sigma per axis)
    float qscale[3];  // cells per unit length per axis
    float pad[3];
};

// Scene statistics (host-visible copy of refine_scene_stats).
struct SceneStats {
    double F_col, F_opa, F_gem;
    double lambda_t[3];
    double lambda[3];
    double mean_m[3];
};

// Number of float sums the content-feature pass reduces per block:
// y, y^2, a(1-a), gem ratio, m_gem, m_col, m_opa, mu (3), mu^2 (3).
constexpr int kFeatSums = 13;

// ---------------------------------------------------------------- loads
__device__ __forceinline__ float ld_attr(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_attr(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}

// --------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared through the TMA engine, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    uint64_t gsrc;
    asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(gsrc) : "l"(src));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of `bar` for at most kWaitCycles; returns false
// on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

// Fast reciprocal on the MUFU pipe (max error 1 ulp).
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Order-preserving map of a float score to an unsigned key (-0 maps as +0).
__device__ __forceinline__ uint32_t score_key(float f)
{
    uint32_t b = __float_as_uint(f);
    if (b == 0x80000000u) b = 0u;
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__host__ __device__ inline float key_to_score(uint32_t k)
{
    uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    float f;
#ifdef __CUDA_ARCH__
    f = __uint_as_float(b);
#else
    __builtin_memcpy(&f, &b, 4);
#endif
    return f;
}

}  // namespace refine
