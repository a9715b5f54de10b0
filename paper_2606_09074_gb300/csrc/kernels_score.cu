// Scoring kernels: camera preparation, the content-feature pass (Eq.
// (features), Eq. 18-19) and the N x V importance kernel (Eq. 7, Eq. 20).
#include <math.h>

#include "internal.h"

namespace refine {

// Degree-0 real spherical-harmonic basis constant 1 / (2 sqrt(pi)).
constexpr float kSH_C0 = 0.28209479177387814f;

// ---------------------------------------------------------------------
// Camera preparation: refine_camera -> CamRec (P = K W and p = K t formed
// in double and rounded once), with validation.
// ---------------------------------------------------------------------
__global__ void k_cam_prep(const refine_camera *__restrict__ cams, int V, CamRec *__restrict__ out,
                           int *status)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    refine_camera c = cams[v];
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
    out[v] = r;
}

cudaError_t launch_cam_prep(const refine_camera *cams, int V, CamRec *out, int *status,
                            cudaStream_t s)
{
    k_cam_prep<<<(V + 127) / 128, 128, 0, s>>>(cams, V, out, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------
// Content features.  Per primitive (R1, R3 of the oracle's readings):
//   y     = C0 (l . dc)           luma minus its constant offset 0.5 sum(l)
//   a     = sigmoid(logit)
//   s     = exp(log-scale)
//   gem   = max(s) / (min(s) + eta)
//   m_gem = product of the two largest scales, m_col = |SH|_2, m_opa = a
// Sums per thread in float, per block in a fixed double tree; the block
// partials are reduced by k_features_finalize in a fixed order, so the
// result depends only on n and the storage type.
// ---------------------------------------------------------------------
template <typename AT, int K>
struct RowLoad;

template <>
struct RowLoad<float, 4> {
    __device__ static void load(const float *row, int64_t i, float (&v)[4])
    {
        float4 q = __ldg(reinterpret_cast<const float4 *>(row + i));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};

template <>
struct RowLoad<__nv_bfloat16, 8> {
    __device__ static void load(const __nv_bfloat16 *row, int64_t i, float (&v)[8])
    {
        uint4 q = __ldg(reinterpret_cast<const uint4 *>(row + i));
        uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = __uint_as_float(w[k] << 16);
            v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
};

struct FeatAcc {
    float s[kFeatSums];
    float bad;  // accumulates x * 0, which is NaN iff some x was not finite
};

__device__ __forceinline__ void feat_accumulate(FeatAcc &acc, float ls0, float ls1, float ls2,
                                                float logit, float dc0, float dc1, float dc2,
                                                float sumsq, float eta, float l0, float l1,
                                                float l2, float &m_col)
{
    float s0 = expf(ls0), s1 = expf(ls1), s2 = expf(ls2);
    float a = 1.f / (1.f + expf(-logit));
    float y = kSH_C0 * fmaf(l0, dc0, fmaf(l1, dc1, l2 * dc2));
    float smax = fmaxf(s0, fmaxf(s1, s2)), smin = fminf(s0, fminf(s1, s2));
    float mg = fmaxf(fmaxf(s0 * s1, s0 * s2), s1 * s2);
    m_col = sqrtf(sumsq);
    acc.s[0] += y;
    acc.s[1] = fmaf(y, y, acc.s[1]);
    acc.s[2] = fmaf(a, 1.f - a, acc.s[2]);
    acc.s[3] += smax / (smin + eta);
    acc.s[4] += mg;
    acc.s[5] += m_col;
    acc.s[6] += a;
    acc.bad = fmaf(ls0 + ls1 + ls2 + logit, 0.f, acc.bad);
}

template <typename AT, int K>
__global__ void __launch_bounds__(kFeatThreads) k_features(const AT *__restrict__ attr, int64_t stride,
                                                           int64_t n, float eta, float l0, float l1,
                                                           float l2, float *__restrict__ m_col,
                                                           double *__restrict__ partials,
                                                           int *status)
{
    FeatAcc acc;
#pragma unroll
    for (int k = 0; k < kFeatSums; ++k) acc.s[k] = 0.f;
    acc.bad = 0.f;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * K;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * K; base < n; base += step) {
        if constexpr (K > 1) {
          if (base + K <= n) {
            float ls[3][K], lg[K], dc[3][K], sq[K], v[K];
#pragma unroll
            for (int r = 0; r < 3; ++r) RowLoad<AT, K>::load(attr + r * stride, base, ls[r]);
            RowLoad<AT, K>::load(attr + 7 * stride, base, lg);
#pragma unroll
            for (int r = 0; r < 3; ++r) RowLoad<AT, K>::load(attr + (8 + r) * stride, base, dc[r]);
#pragma unroll
            for (int k = 0; k < K; ++k)
                sq[k] = fmaf(dc[0][k], dc[0][k], fmaf(dc[1][k], dc[1][k], dc[2][k] * dc[2][k]));
#pragma unroll 5
            for (int r = 11; r < 56; ++r) {
                RowLoad<AT, K>::load(attr + r * stride, base, v);
#pragma unroll
                for (int k = 0; k < K; ++k) sq[k] = fmaf(v[k], v[k], sq[k]);
            }
            float mc[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                feat_accumulate(acc, ls[0][k], ls[1][k], ls[2][k], lg[k], dc[0][k], dc[1][k],
                                dc[2][k], sq[k], eta, l0, l1, l2, mc[k]);
                acc.bad = fmaf(sq[k], 0.f, acc.bad);
            }
#pragma unroll
            for (int k = 0; k < K; ++k) m_col[base + k] = mc[k];
            continue;
          }
        }
        {
            for (int64_t i = base; i < n && i < base + K; ++i) {
                float sq = 0.f;
                for (int r = 8; r < 56; ++r) {
                    float x = ld_attr(attr + r * stride + i);
                    sq = fmaf(x, x, sq);
                }
                float mc;
                feat_accumulate(acc, ld_attr(attr + i), ld_attr(attr + stride + i),
                                ld_attr(attr + 2 * stride + i), ld_attr(attr + 7 * stride + i),
                                ld_attr(attr + 8 * stride + i), ld_attr(attr + 9 * stride + i),
                                ld_attr(attr + 10 * stride + i), sq, eta, l0, l1, l2, mc);
                acc.bad = fmaf(sq, 0.f, acc.bad);
                m_col[i] = mc;
            }
        }
    }
    if (!isfinite(acc.bad)) set_status(status, kEnonfinite);

    __shared__ double red[kFeatSums][kFeatThreads];
#pragma unroll
    for (int k = 0; k < kFeatSums; ++k) red[k][threadIdx.x] = (double)acc.s[k];
    __syncthreads();
    for (int s = kFeatThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int k = 0; k < kFeatSums; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x < kFeatSums) partials[(int64_t)blockIdx.x * kFeatSums + threadIdx.x] = red[threadIdx.x][0];
}

int feature_blocks(int64_t n, int dtype)
{
    const int64_t per_block = (int64_t)kFeatThreads * (dtype == REFINE_BF16 ? 8 : 4) * 4;
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

cudaError_t launch_features(const void *attr, int dtype, int64_t stride, int64_t n, float eta,
                            const float luma[3], float *m_col, double *partials, bool vec,
                            int *status, cudaStream_t s)
{
    int nb = feature_blocks(n, dtype);
    if (dtype == REFINE_BF16) {
        const __nv_bfloat16 *a = static_cast<const __nv_bfloat16 *>(attr);
        if (vec)
            k_features<__nv_bfloat16, 8><<<nb, kFeatThreads, 0, s>>>(a, stride, n, eta, luma[0], luma[1],
                                                                      luma[2], m_col, partials, status);
        else
            k_features<__nv_bfloat16, 1><<<nb, kFeatThreads, 0, s>>>(a, stride, n, eta, luma[0], luma[1],
                                                                      luma[2], m_col, partials, status);
    } else {
        const float *a = static_cast<const float *>(attr);
        if (vec)
            k_features<float, 4><<<nb, kFeatThreads, 0, s>>>(a, stride, n, eta, luma[0], luma[1], luma[2],
                                                             m_col, partials, status);
        else
            k_features<float, 1><<<nb, kFeatThreads, 0, s>>>(a, stride, n, eta, luma[0], luma[1], luma[2],
                                                             m_col, partials, status);
    }
    return cudaGetLastError();
}

// Eq. (features) -> Eq. 18 -> Eq. 19, in double, one block.
__global__ void k_features_finalize(const double *__restrict__ partials, int nblocks, int64_t n,
                                    refine_params p, SceneConsts *consts, SceneStats *stats)
{
    __shared__ double red[kFeatSums][256];
    double loc[kFeatSums];
#pragma unroll
    for (int k = 0; k < kFeatSums; ++k) loc[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < kFeatSums; ++k) loc[k] += partials[(int64_t)b * kFeatSums + k];
#pragma unroll
    for (int k = 0; k < kFeatSums; ++k) red[k][threadIdx.x] = loc[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < kFeatSums; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double N = (double)n;
    SceneStats st;
    double ybar = red[0][0] / N;
    st.F_col = red[1][0] / N - ybar * ybar;
    if (st.F_col < 0.0) st.F_col = 0.0;
    st.F_opa = red[2][0] / N;
    st.F_gem = red[3][0] / N;
    for (int k = 0; k < 3; ++k) st.mean_m[k] = red[4 + k][0] / N;
    st.lambda_t[0] = log(st.F_gem + (double)p.eta) / p.e_ln_gem;
    st.lambda_t[1] = st.F_col / p.e_col;
    st.lambda_t[2] = st.F_opa / p.e_opa;
    double tot = 0.0;
    for (int k = 0; k < 3; ++k) {
        if (!(st.lambda_t[k] > 0.0)) st.lambda_t[k] = 0.0;
        tot += st.lambda_t[k];
    }
    SceneConsts c;
    for (int k = 0; k < 3; ++k) {
        st.lambda[k] = ((p.flags & REFINE_FLAG_EQUAL_LAMBDA) || tot == 0.0) ? 1.0 / 3.0
                                                                             : st.lambda_t[k] / tot;
        double kap = st.lambda[k];
        if (p.flags & REFINE_FLAG_NORM_ATTR) kap = st.mean_m[k] > 0.0 ? st.lambda[k] / st.mean_m[k] : 0.0;
        c.kappa[k] = (float)kap;
    }
    c.pad = 0.f;
    *consts = c;
    if (stats) *stats = st;
}

cudaError_t launch_features_finalize(const double *partials, int nblocks, int64_t n,
                                     const refine_params *p, SceneConsts *consts,
                                     SceneStats *stats, cudaStream_t s)
{
    k_features_finalize<<<1, 256, 0, s>>>(partials, nblocks, n, *p, consts, stats);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------
// The N x V importance kernel.
//
// One thread owns GPT primitives and walks every camera of the pass, the
// camera records staged once per CTA into shared memory by a TMA bulk copy.
// For primitive i and view v (Eq. 13-14, Eq. 17, Eq. 20):
//   (U, V, z) = P mu + p                                (homogeneous pixel)
//   g0 = z P0 - U P2,  g1 = z P1 - V P2                 (z^2 J W rows)
//   Qx = |L g0|^2 = 9 z^4 S_xx,  Qy = |L g1|^2 = 9 z^4 S_yy
//        with L = 3 diag(s) R^T, i.e. Sigma2D = J W Sigma W^T J^T formed
//        through the square root of Sigma (well conditioned in float)
//   the 3-sigma box meets [0,w] x [0,h]  <=>  (d_u z^2)^2 <= Qx and
//        (d_v z^2)^2 <= Qy, d_u = max(0, -u, u - w) written as
//        max(0, -U, U - w z) / z, so no division is needed
//   det Sigma2D = |L g0 x L g1|^2 / (81 z^8) > 0 holds whenever all three
//        scales are nonzero (L invertible, g0 and g1 independent); only a
//        warp holding a primitive with an underflowed scale evaluates it
//   term = vis / (z^2 + eta)                            (Eq. 17, one MUFU)
// Views are summed in blocks of 16 into a running total (fixed order).
// The epilogue forms D_i = alpha_i S_i / |V| * sum_k lambda^k G~_i^k.
// ---------------------------------------------------------------------
template <bool NOPROJ, bool DET>
__device__ __forceinline__ float pair_term(const float4 &c0, const float4 &c1, const float4 &c2,
                                           const float4 &lim, float mx, float my, float mz,
                                           const float (&L)[9], float eta)
{
    const float U = fmaf(c0.x, mx, fmaf(c0.y, my, fmaf(c0.z, mz, c0.w)));
    const float V = fmaf(c1.x, mx, fmaf(c1.y, my, fmaf(c1.z, mz, c1.w)));
    const float z = fmaf(c2.x, mx, fmaf(c2.y, my, fmaf(c2.z, mz, c2.w)));
    const float g0x = fmaf(-U, c2.x, z * c0.x), g0y = fmaf(-U, c2.y, z * c0.y),
                g0z = fmaf(-U, c2.z, z * c0.z);
    const float g1x = fmaf(-V, c2.x, z * c1.x), g1y = fmaf(-V, c2.y, z * c1.y),
                g1z = fmaf(-V, c2.z, z * c1.z);
    const float a0 = fmaf(L[0], g0x, fmaf(L[1], g0y, L[2] * g0z));
    const float a1 = fmaf(L[3], g0x, fmaf(L[4], g0y, L[5] * g0z));
    const float a2 = fmaf(L[6], g0x, fmaf(L[7], g0y, L[8] * g0z));
    const float b0 = fmaf(L[0], g1x, fmaf(L[1], g1y, L[2] * g1z));
    const float b1 = fmaf(L[3], g1x, fmaf(L[4], g1y, L[5] * g1z));
    const float b2 = fmaf(L[6], g1x, fmaf(L[7], g1y, L[8] * g1z));
    const float Qx = fmaf(a0, a0, fmaf(a1, a1, a2 * a2));
    const float Qy = fmaf(b0, b0, fmaf(b1, b1, b2 * b2));
    const float du = fmaxf(fmaxf(-U, fmaf(-lim.x, z, U)), 0.f) * z;
    const float dv = fmaxf(fmaxf(-V, fmaf(-lim.y, z, V)), 0.f) * z;
    bool vis = (z > lim.z) & (z < lim.w) & (du * du <= Qx) & (dv * dv <= Qy);
    if (DET) {
        const float x0 = a1 * b2 - a2 * b1, x1 = a2 * b0 - a0 * b2, x2 = a0 * b1 - a1 * b0;
        vis = vis & ((x0 != 0.f) | (x1 != 0.f) | (x2 != 0.f));
    }
    const float w = NOPROJ ? 1.f : rcp_approx(fmaf(z, z, eta));
    return vis ? w : 0.f;
}

template <int GPT, bool NOPROJ, bool DET>
__device__ __forceinline__ void view_loop(const CamRec *cs, int vcount, float eta,
                                          const float (&mx)[GPT], const float (&my)[GPT],
                                          const float (&mz)[GPT], const float (&L)[GPT][9],
                                          float (&acc)[GPT])
{
    for (int v0 = 0; v0 < vcount; v0 += 16) {
        const int vend = min(v0 + 16, vcount);
        float part[GPT];
#pragma unroll
        for (int g = 0; g < GPT; ++g) part[g] = 0.f;
#pragma unroll 2
        for (int v = v0; v < vend; ++v) {
            const float4 c0 = cs[v].r0, c1 = cs[v].r1, c2 = cs[v].r2, lim = cs[v].lim;
#pragma unroll
            for (int g = 0; g < GPT; ++g)
                part[g] += pair_term<NOPROJ, DET>(c0, c1, c2, lim, mx[g], my[g], mz[g], L[g], eta);
        }
#pragma unroll
        for (int g = 0; g < GPT; ++g) acc[g] += part[g];
    }
}

template <typename AT, int GPT, bool NOPROJ>
__global__ void __launch_bounds__(kScoreThreads) k_score(ScoreLaunch a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    CamRec *cs = reinterpret_cast<CamRec *>(smem_raw);
    const AT *attr = static_cast<const AT *>(a.attr);
    const int64_t S = a.stride;

    // Stage this pass's cameras once per CTA (TMA bulk copy, mbarrier).
    const uint32_t bytes = (uint32_t)a.vcount * (uint32_t)sizeof(CamRec);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, bytes);
        for (uint32_t off = 0; off < bytes; off += 16384u) {
            uint32_t len = bytes - off < 16384u ? bytes - off : 16384u;
            bulk_g2s(smem_raw + off, reinterpret_cast<const unsigned char *>(a.cams) + off, len, &bar);
        }
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0)) {
        set_status(a.status, kEtimeout);
        mbar_wait_bounded(&bar, 0);  // give the copy a second bound before leaving
        return;
    }

    const int64_t tile = (int64_t)blockDim.x * GPT;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < a.n; base += (int64_t)gridDim.x * tile) {
        float mx[GPT], my[GPT], mz[GPT], L[GPT][9], acc[GPT];
        bool degen = false;
#pragma unroll
        for (int g = 0; g < GPT; ++g) {
            const int64_t i = base + threadIdx.x + (int64_t)g * blockDim.x;
            float ls0 = 0.f, ls1 = 0.f, ls2 = 0.f, qw = 1.f, qx = 0.f, qy = 0.f, qz = 0.f;
            mx[g] = my[g] = mz[g] = 0.f;
            acc[g] = 0.f;
            if (i < a.n) {
                mx[g] = __ldg(a.pos + i);
                my[g] = __ldg(a.pos + S + i);
                mz[g] = __ldg(a.pos + 2 * S + i);
                ls0 = ld_attr(attr + i);
                ls1 = ld_attr(attr + S + i);
                ls2 = ld_attr(attr + 2 * S + i);
                qw = ld_attr(attr + 3 * S + i);
                qx = ld_attr(attr + 4 * S + i);
                qy = ld_attr(attr + 5 * S + i);
                qz = ld_attr(attr + 6 * S + i);
                if (!a.first) acc[g] = a.running[i];
                float chk = fmaf(mx[g] + my[g] + mz[g] + ls0 + ls1 + ls2 + qw + qx + qy + qz, 0.f, 0.f);
                if (!isfinite(chk)) set_status(a.status, kEnonfinite);
            }
            const float qn2 = fmaf(qw, qw, fmaf(qx, qx, fmaf(qy, qy, qz * qz)));
            if (!(qn2 > 0.f)) {
                if (i < a.n) set_status(a.status, kEinval);
                qw = 1.f; qx = qy = qz = 0.f;
            } else {
                const float r = rsqrtf(qn2);
                qw *= r; qx *= r; qy *= r; qz *= r;
            }
            const float s0 = 3.f * expf(ls0), s1 = 3.f * expf(ls1), s2 = 3.f * expf(ls2);
            degen |= (s0 == 0.f) | (s1 == 0.f) | (s2 == 0.f);
            // columns of R(q) scaled by 3 s_k form the rows of L
            L[g][0] = s0 * (1.f - 2.f * (qy * qy + qz * qz));
            L[g][1] = s0 * (2.f * (qx * qy + qw * qz));
            L[g][2] = s0 * (2.f * (qx * qz - qw * qy));
            L[g][3] = s1 * (2.f * (qx * qy - qw * qz));
            L[g][4] = s1 * (1.f - 2.f * (qx * qx + qz * qz));
            L[g][5] = s1 * (2.f * (qy * qz + qw * qx));
            L[g][6] = s2 * (2.f * (qx * qz + qw * qy));
            L[g][7] = s2 * (2.f * (qy * qz - qw * qx));
            L[g][8] = s2 * (1.f - 2.f * (qx * qx + qy * qy));
        }

        if (__any_sync(0xffffffffu, degen))
            view_loop<GPT, NOPROJ, true>(cs, a.vcount, a.eta, mx, my, mz, L, acc);
        else
            view_loop<GPT, NOPROJ, false>(cs, a.vcount, a.eta, mx, my, mz, L, acc);

#pragma unroll
        for (int g = 0; g < GPT; ++g) {
            const int64_t i = base + threadIdx.x + (int64_t)g * blockDim.x;
            if (i >= a.n) continue;
            if (!a.last) {
                a.running[i] = acc[g];
                continue;
            }
            const float Ssum = acc[g];
            if (a.view_sum) a.view_sum[i] = Ssum;
            const float e0 = expf(ld_attr(attr + i)), e1 = expf(ld_attr(attr + S + i)),
                        e2 = expf(ld_attr(attr + 2 * S + i));
            const float alpha = 1.f / (1.f + expf(-ld_attr(attr + 7 * S + i)));
            const float mg = fmaxf(fmaxf(e0 * e1, e0 * e2), e1 * e2);
            const SceneConsts c = *a.consts;
            const float coupled = fmaf(c.kappa[0], mg, fmaf(c.kappa[1], a.m_col[i], c.kappa[2] * alpha));
            const float A = ((a.flags & REFINE_FLAG_NO_VIS) ? 1.f : alpha) * (Ssum * a.inv_views);
            a.scores[i] = A * coupled;
        }
    }
}

template <typename AT, int GPT, bool NOPROJ>
static const void *score_fn()
{
    return reinterpret_cast<const void *>(&k_score<AT, GPT, NOPROJ>);
}

static const void *pick_score(int dtype, int gpt, bool noproj)
{
    if (dtype == REFINE_BF16) {
        if (gpt == 2) return noproj ? score_fn<__nv_bfloat16, 2, true>() : score_fn<__nv_bfloat16, 2, false>();
        return noproj ? score_fn<__nv_bfloat16, 1, true>() : score_fn<__nv_bfloat16, 1, false>();
    }
    if (gpt == 2) return noproj ? score_fn<float, 2, true>() : score_fn<float, 2, false>();
    return noproj ? score_fn<float, 1, true>() : score_fn<float, 1, false>();
}

int score_grid(int num_sms, int64_t n, int vcount, int gpt)
{
    // Persistent grid: as many CTAs as fit per SM (occupancy query), capped
    // by the number of tiles.
    int per_sm = 0;
    const void *fn = pick_score(REFINE_F32, gpt, false);
    size_t smem = (size_t)vcount * sizeof(CamRec);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kScoreThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t tiles = (n + (int64_t)kScoreThreads * gpt - 1) / ((int64_t)kScoreThreads * gpt);
    int64_t g = (int64_t)num_sms * per_sm;
    if (g > tiles) g = tiles;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_score(const ScoreLaunch &a, cudaStream_t s)
{
    const void *fn = pick_score(a.dtype, a.gpt, (a.flags & REFINE_FLAG_NO_PROJ) != 0);
    size_t smem = (size_t)a.vcount * sizeof(CamRec);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    ScoreLaunch arg = a;
    void *args[] = {&arg};
    return cudaLaunchKernel(fn, dim3(a.grid), dim3(kScoreThreads), args, smem, s);
}

}  // namespace refine
