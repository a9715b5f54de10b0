// Internal device/host definitions shared by the librefine translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "refine.h"

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
    float big_ls;     // ln s_max above which a primitive is ordered with the large ones
    float pad[2];
};

// Scene statistics (host-visible copy of refine_scene_stats).
struct SceneStats {
    double F_col, F_opa, F_gem;
    double lambda_t[3];
    double lambda[3];
    double mean_m[3];
};

// Number of float sums the content-feature pass reduces per block:
// y, y^2, a(1-a), gem ratio, m_gem, m_col, m_opa, mu (3), mu^2 (3), and
// ln s_max with its square (for the size split of the processing order).
constexpr int kFeatSums = 15;

// Float-float numbers: an unevaluated sum hi + lo of two floats, added on
// the FP32 pipes (the FP64 rate of this part is 1/64 of the FP32 rate).
// Each addition keeps the rounding error of its leading sum exactly
// (Knuth's TwoSum) and renormalises with Dekker's FastTwoSum, so a sum of
// many terms carries about 44 significant bits.  Every step is an explicit
// round-to-nearest add, never contracted, and the addition is commutative
// bit for bit, so a fixed reduction order gives fixed bits.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, t);
    return {hi, __fsub_rn(t, __fsub_rn(hi, s))};
}

// The value as a double (exact: hi and lo do not overlap).
__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

// Per-thread content-feature sums (kFeatSums of them) and a non-finite trap.
struct FeatSums {
    float s[kFeatSums];
    float bad;  // accumulates x * 0, which is NaN iff some x was not finite
};

// Activation of one primitive (Eq. 1) and its feature terms (the readings R1,
// R3: y = C0 (l . dc) is the luma minus its constant offset 0.5 sum(l);
// gem = max(s) / (min(s) + eta); m_gem = product of the two largest scales;
// m_col = |SH|_2; m_opa = alpha).  Adds to the thirteen sums and returns the
// primitive's record (layout: PrimRec in internal.h).  *zero_q is set for a
// zero quaternion (then R = I).
__device__ __forceinline__ void primitive_record(FeatSums &acc, float mx, float my, float mz, float ls0, float ls1,
                                                 float ls2, float qw, float qx, float qy, float qz, float logit,
                                                 float dc0, float dc1, float dc2, float sumsq, float eta, float l0,
                                                 float l1, float l2, float4 &ra, float4 &rb, float4 &rc, float4 &rd,
                                                 bool &zero_q)
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
    const float lsmax = fmaxf(ls0, fmaxf(ls1, ls2));
    acc.s[13] += lsmax;
    acc.s[14] = fmaf(lsmax, lsmax, acc.s[14]);
    acc.bad = fmaf(mx + my + mz + ls0 + ls1 + ls2 + qw + qx + qy + qz + logit + sumsq, 0.f, acc.bad);

    const float qn2 = fmaf(qw, qw, fmaf(qx, qx, fmaf(qy, qy, qz * qz)));
    if (!(qn2 > 0.f)) {
        zero_q = true;
        qw = 1.f; qx = qy = qz = 0.f;
    } else {
        const float r = rsqrtf(qn2);
        qw *= r; qx *= r; qy *= r; qz *= r;
    }
    const float s0 = 3.f * e0, s1 = 3.f * e1, s2 = 3.f * e2;
    const float sm = fmaxf(s0, fmaxf(s1, s2));
    float b2 = sm * sm * 1.0009765625f;
    if ((s0 == 0.f) | (s1 == 0.f) | (s2 == 0.f)) b2 = -(1.f + b2);
    // the rows of L are the columns of R(q) scaled by 3 s_k
    ra = make_float4(mx, my, mz, b2);
    rb = make_float4(s0 * (1.f - 2.f * (qy * qy + qz * qz)), s0 * (2.f * (qx * qy + qw * qz)),
                     s0 * (2.f * (qx * qz - qw * qy)), s1 * (2.f * (qx * qy - qw * qz)));
    rc = make_float4(s1 * (1.f - 2.f * (qx * qx + qz * qz)), s1 * (2.f * (qy * qz + qw * qx)),
                     s2 * (2.f * (qx * qz + qw * qy)), s2 * (2.f * (qy * qz - qw * qx)));
    rd = make_float4(s2 * (1.f - 2.f * (qx * qx + qy * qy)), alpha, mg, mc);
}

// ------------------------------------------------------ row layouts
// The 56 attribute rows of a storage type: rows [0, attr_f32_rows) are
// float32, the rest bfloat16, one block of rows after the other, each row
// `stride` elements of its own type (REFINE_F32: all 56 rows float32;
// REFINE_BF16: all bfloat16; REFINE_BF16S: the 3 log-scale rows float32).
__host__ __device__ constexpr int attr_f32_rows(int dtype)
{
    return dtype == REFINE_F32 ? 56 : (dtype == REFINE_BF16S ? 3 : 0);
}
__host__ __device__ constexpr bool valid_dtype(int dtype)
{
    return dtype == REFINE_F32 || dtype == REFINE_BF16 || dtype == REFINE_BF16S;
}
// Bytes of one element column of the 56 rows (236 - 12 = 224, 112 or 118).
__host__ __device__ constexpr size_t attr_col_bytes(int dtype)
{
    return (size_t)attr_f32_rows(dtype) * 4 + (size_t)(56 - attr_f32_rows(dtype)) * 2;
}

// ---------------------------------------------------------------- loads
__device__ __forceinline__ float ld_attr(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_attr(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}

// Read access to the 56 attribute rows of storage type DT (REFINE_F32,
// REFINE_BF16 or REFINE_BF16S), each row widened to float on load.  The row
// index is a compile-time constant wherever the kernels unroll over rows,
// so the choice of block (float32 or bfloat16) costs nothing.
template <int DT>
struct AttrRows {
    const float *f;          // the float32 rows [0, attr_f32_rows(DT))
    const __nv_bfloat16 *b;  // the bfloat16 rows after them
    int64_t S;               // row stride in elements

    __host__ __device__ AttrRows(const void *attr, int64_t stride)
        : f(static_cast<const float *>(attr)),
          b(reinterpret_cast<const __nv_bfloat16 *>(static_cast<const char *>(attr) +
                                                    (size_t)attr_f32_rows(DT) * 4 * (size_t)stride)),
          S(stride)
    {
    }
    __device__ __forceinline__ float ld(int r, int64_t i) const
    {
        return r < attr_f32_rows(DT) ? ld_attr(f + (int64_t)r * S + i)
                                     : ld_attr(b + (int64_t)(r - attr_f32_rows(DT)) * S + i);
    }
};

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

// Waits for phase `parity` of `bar` for at most `limit` SM clock cycles;
// returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit = kWaitCycles)
{
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
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

// The same reciprocal without the handling of subnormal operands and
// results: a single MUFU operation, against several instructions for the
// form above.  Equal to rcp_approx for x in [2^-126, 2^126]; above that the
// result (below 2^-126) flushes to zero.
__device__ __forceinline__ float rcp_approx_ftz(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
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
