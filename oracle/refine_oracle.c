/*
 * FP64 CPU oracle for REFINE's rendering-free primitive importance, ratio
 * pruning and compaction (arXiv 2606.09074, Sec. 3.2-3.3).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares no source,
 * header, table or helper with the CUDA library and is deliberately slow and
 * literal: every quantity is formed the way the paper writes it (explicit
 * matrices, explicit square roots, a comparison sort), in double precision.
 *
 * Readings of the paper used here (the paper is silent or ambiguous on each):
 *   R1  The attribute subsets G~^k of Eq. 7 are scalar magnitudes:
 *       gem = product of the two largest activated scales (the "area"),
 *       col = L2 norm of all 48 SH coefficients, opa = alpha.  With the
 *       NORM_ATTR flag each is divided by its scene mean (a zero mean gives 0).
 *   R2  The expectations E[.] of Eq. 18 are caller-supplied constants.
 *       A negative lambda~ is clamped to 0; if all three are 0, lambda = 1/3.
 *   R3  The luma Y_i of Eq. (features) is BT.601 luma of the SH DC colour
 *       0.5 + C0*dc, C0 = 1/(2 sqrt(pi)); F_col is the population variance.
 *   R4  One eta (0.05) serves Eq. 17 and Eq. 18 / (features).
 *   R5  A view contributes to Eq. 20 only when the primitive reaches its
 *       image: znear < z < zfar, det Sigma2D > 0 and the 3-sigma axis-aligned
 *       box [u +- 3 sqrt(S_xx)] x [v +- 3 sqrt(S_yy)] meets the closed
 *       rectangle [0,w] x [0,h], with Sigma2D = J W Sigma W^T J^T (EWA,
 *       Eq. 13-14).  No low-pass dilation.
 *   R6  |V| in Eq. 20 counts every view, visible or not.
 *   R8  Ratio pruning (Sec. 3.3): n_prune = floor(beta * N) in double;
 *       primitives are kept in order (score desc, index asc); the threshold
 *       is the smallest kept score, or -inf when nothing is pruned.
 *
 * Parity band: besides each score, the oracle reports which (primitive, view)
 * visibility decisions lie so close to a boundary that a float32 evaluation
 * may legitimately take the other side (see orc_visible).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NO_VIS        (1 << 0)  /* Table 3 "w/o V": alpha -> 1 in Eq. 20 */
#define ORC_NO_PROJ       (1 << 1)  /* Table 3 "w/o P": P -> 1 in Eq. 20     */
#define ORC_EQUAL_LAMBDA  (1 << 2)  /* Table 3 "Equal lambda^k"             */
#define ORC_NORM_ATTR     (1 << 3)  /* R1: G~^k = m^k / mean(m^k)           */
#define ORC_FULL_JAC      (1 << 4)  /* Eq. 14 before Eq. 16: P = Tr(J^T J)  */

/* Relative width of the band inside which a float32 evaluation of a
 * visibility decision may differ from this FP64 one (64 float32 ulps). */
#define ORC_BAND 3.814697265625e-06 /* 2^-18 */
/* The determinant test is flagged only where double rounding itself is in
 * doubt (det / (S_xx S_yy) below 1e-12). */
#define ORC_DET_BAND 1e-12

typedef struct {
    double R[9];              /* world-to-camera rotation W, row-major    */
    double t[3];              /* world-to-camera translation              */
    double fx, fy, cx, cy;    /* Eq. 13: f_x, f_y, principal point u_x,u_y */
    double width, height;     /* image size in pixels                     */
    double znear, zfar;       /* depth range                              */
} orc_camera;

typedef struct {
    double eta;               /* Eq. 17 stability constant                */
    double e_ln_gem;          /* Eq. 18: E[ln F_gem]                      */
    double e_col;             /* Eq. 18: E[F_col]                         */
    double e_opa;             /* Eq. 18: E[F_opa]                         */
    double luma[3];           /* R3 luma weights                          */
    int flags;
} orc_params;

typedef struct {
    double F_col, F_opa, F_gem;       /* Eq. (features)             */
    double lambda_t[3];               /* Eq. 18 (gem, col, opa)     */
    double lambda[3];                 /* Eq. 19 (gem, col, opa)     */
    double mean_m[3];                 /* R1 scene means of m^k      */
} orc_stats;

/* ---------------------------------------------------------------- Eq. 1 */

/* Activation of one primitive read from the SoA parameter block g[59][stride]:
 * alpha = sigmoid(logit), s = exp(log-scale), q normalised, R(q) and
 * Sigma = R diag(s^2) R^T. */
void orc_activate(const double *g, int64_t stride, int64_t i,
                  double *alpha, double s[3], double Rq[9], double Sigma[9])
{
    double w = g[6 * stride + i], x = g[7 * stride + i];
    double y = g[8 * stride + i], z = g[9 * stride + i];
    double qn = sqrt(w * w + x * x + y * y + z * z);
    w /= qn; x /= qn; y /= qn; z /= qn;
    Rq[0] = 1.0 - 2.0 * (y * y + z * z); Rq[1] = 2.0 * (x * y - w * z);       Rq[2] = 2.0 * (x * z + w * y);
    Rq[3] = 2.0 * (x * y + w * z);       Rq[4] = 1.0 - 2.0 * (x * x + z * z); Rq[5] = 2.0 * (y * z - w * x);
    Rq[6] = 2.0 * (x * z - w * y);       Rq[7] = 2.0 * (y * z + w * x);       Rq[8] = 1.0 - 2.0 * (x * x + y * y);
    for (int k = 0; k < 3; ++k) s[k] = exp(g[(3 + k) * stride + i]);
    *alpha = 1.0 / (1.0 + exp(-g[10 * stride + i]));
    double M[9]; /* M = R diag(s^2) */
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * s[c] * s[c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += M[3 * r + k] * Rq[3 * c + k];
            Sigma[3 * r + c] = acc;
        }
}

/* ------------------------------------------------------- Eq. 13 and 14 */

/* Camera-space centre (x, y, z) = W mu + t. */
void orc_to_camera(const orc_camera *c, const double mu[3], double tc[3])
{
    for (int r = 0; r < 3; ++r)
        tc[r] = c->R[3 * r] * mu[0] + c->R[3 * r + 1] * mu[1] + c->R[3 * r + 2] * mu[2] + c->t[r];
}

/* Eq. 13: Pi(x, y, z) = (f_x x / z + u_x, f_y y / z + u_y). */
void orc_project(const orc_camera *c, const double tc[3], double uv[2])
{
    uv[0] = c->fx * tc[0] / tc[2] + c->cx;
    uv[1] = c->fy * tc[1] / tc[2] + c->cy;
}

/* Eq. 14: the 2x3 Jacobian J_Pi of Eq. 13 at (x, y, z), row-major. */
void orc_projection_jacobian(const orc_camera *c, const double tc[3], double J[6])
{
    double x = tc[0], y = tc[1], z = tc[2];
    J[0] = c->fx / z; J[1] = 0.0;       J[2] = -c->fx * x / (z * z);
    J[3] = 0.0;       J[4] = c->fy / z; J[5] = -c->fy * y / (z * z);
}

/* EWA projected covariance Sigma2D = J W Sigma W^T J^T (2x2, row-major). */
void orc_cov2d(const orc_camera *c, const double tc[3], const double Sigma[9], double S2[4])
{
    double J[6], T[6], TS[6];
    orc_projection_jacobian(c, tc, J);
    for (int r = 0; r < 2; ++r)        /* T = J W */
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m) acc += J[3 * r + m] * c->R[3 * m + k];
            T[3 * r + k] = acc;
        }
    for (int r = 0; r < 2; ++r)        /* T Sigma */
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m) acc += T[3 * r + m] * Sigma[3 * m + k];
            TS[3 * r + k] = acc;
        }
    for (int r = 0; r < 2; ++r)        /* (T Sigma) T^T */
        for (int k = 0; k < 2; ++k) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m) acc += TS[3 * r + m] * T[3 * k + m];
            S2[2 * r + k] = acc;
        }
}

/* R5: does the primitive (camera-space centre tc, covariance Sigma) reach
 * the image of camera c?  *border is set when any of the three decisions is
 * within the float32 parity band. */
int orc_visible(const orc_camera *c, const double mu[3], const double Sigma[9], int *border)
{
    double tc[3], uv[2], S2[4];
    double Mx = fabs(c->t[0]), My = fabs(c->t[1]), Mz = fabs(c->t[2]);
    for (int k = 0; k < 3; ++k) {
        Mx += fabs(c->R[k] * mu[k]);
        My += fabs(c->R[3 + k] * mu[k]);
        Mz += fabs(c->R[6 + k] * mu[k]);
    }
    orc_to_camera(c, mu, tc);
    double z = tc[2];
    *border = 0;
    if (fabs(z - c->znear) <= ORC_BAND * Mz || fabs(z - c->zfar) <= ORC_BAND * Mz) *border = 1;
    if (!(z > c->znear && z < c->zfar)) return 0;

    orc_project(c, tc, uv);
    orc_cov2d(c, tc, Sigma, S2);
    double det = S2[0] * S2[3] - S2[1] * S2[2];
    if (det <= ORC_DET_BAND * S2[0] * S2[3]) *border = 1;
    if (!(det > 0.0)) return 0;

    double rx = 3.0 * sqrt(S2[0]), ry = 3.0 * sqrt(S2[3]);
    /* rounding scale of a float32 evaluation of u and v, in pixels */
    double su = (c->fx * Mx + (fabs(c->cx) + fabs(uv[0])) * Mz) / z + c->width + rx;
    double sv = (c->fy * My + (fabs(c->cy) + fabs(uv[1])) * Mz) / z + c->height + ry;
    double m0 = uv[0] + rx, m1 = c->width - (uv[0] - rx);
    double m2 = uv[1] + ry, m3 = c->height - (uv[1] - ry);
    if (fabs(m0) <= ORC_BAND * su || fabs(m1) <= ORC_BAND * su ||
        fabs(m2) <= ORC_BAND * sv || fabs(m3) <= ORC_BAND * sv)
        *border = 1;
    return m0 >= 0.0 && m1 >= 0.0 && m2 >= 0.0 && m3 >= 0.0;
}

/* ------------------------------------------------------ Eq. (features) */

static double max3(const double s[3]) { double m = s[0]; if (s[1] > m) m = s[1]; if (s[2] > m) m = s[2]; return m; }
static double min3(const double s[3]) { double m = s[0]; if (s[1] < m) m = s[1]; if (s[2] < m) m = s[2]; return m; }

/* R1 magnitudes of one primitive: m[0] = gem (two largest scales' product),
 * m[1] = col (|c|_2 over 48 SH coefficients), m[2] = opa (alpha). */
void orc_magnitudes(const double *g, int64_t stride, int64_t i, double m[3])
{
    double alpha, s[3], Rq[9], Sigma[9];
    orc_activate(g, stride, i, &alpha, s, Rq, Sigma);
    double d[3] = {s[0], s[1], s[2]};   /* sort descending */
    for (int a = 0; a < 2; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (d[b] > d[a]) { double tmp = d[a]; d[a] = d[b]; d[b] = tmp; }
    m[0] = d[0] * d[1];
    double acc = 0.0;
    for (int r = 11; r < 59; ++r) acc += g[r * stride + i] * g[r * stride + i];
    m[1] = sqrt(acc);
    m[2] = alpha;
}

/* Eq. (features), Eq. 18 and Eq. 19 over the whole scene. */
void orc_scene_stats(const double *g, int64_t stride, int64_t n, const orc_params *p, orc_stats *st)
{
    const double C0 = 0.28209479177387814; /* degree-0 real SH basis constant 1/(2 sqrt(pi)) */
    double sumY = 0.0, sumOpa = 0.0, sumGem = 0.0, sumM[3] = {0.0, 0.0, 0.0};
    memset(st, 0, sizeof *st);
    for (int64_t i = 0; i < n; ++i) {
        double alpha, s[3], Rq[9], Sigma[9], m[3];
        orc_activate(g, stride, i, &alpha, s, Rq, Sigma);
        double Y = 0.0;
        for (int ch = 0; ch < 3; ++ch) Y += p->luma[ch] * (0.5 + C0 * g[(11 + ch) * stride + i]);
        sumY += Y;
        sumOpa += alpha * (1.0 - alpha);
        sumGem += max3(s) / (min3(s) + p->eta);
        orc_magnitudes(g, stride, i, m);
        for (int k = 0; k < 3; ++k) sumM[k] += m[k];
    }
    if (n == 0) {
        for (int k = 0; k < 3; ++k) st->lambda[k] = 1.0 / 3.0;
        return;
    }
    double Ybar = sumY / (double)n, var = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double Y = 0.0;
        for (int ch = 0; ch < 3; ++ch) Y += p->luma[ch] * (0.5 + C0 * g[(11 + ch) * stride + i]);
        var += (Y - Ybar) * (Y - Ybar);
    }
    st->F_col = var / (double)n;
    st->F_opa = sumOpa / (double)n;
    st->F_gem = sumGem / (double)n;
    for (int k = 0; k < 3; ++k) st->mean_m[k] = sumM[k] / (double)n;

    /* Eq. 18 (gem, col, opa) with R2's clamp */
    st->lambda_t[0] = log(st->F_gem + p->eta) / p->e_ln_gem;
    st->lambda_t[1] = st->F_col / p->e_col;
    st->lambda_t[2] = st->F_opa / p->e_opa;
    double tot = 0.0;
    for (int k = 0; k < 3; ++k) {
        if (!(st->lambda_t[k] > 0.0)) st->lambda_t[k] = 0.0;
        tot += st->lambda_t[k];
    }
    /* Eq. 19 */
    for (int k = 0; k < 3; ++k)
        st->lambda[k] = (p->flags & ORC_EQUAL_LAMBDA) || tot == 0.0 ? 1.0 / 3.0 : st->lambda_t[k] / tot;
}

/* ----------------------------------------------------- Eq. 7 and Eq. 20 */

/* Importance D(G_i) of every primitive.
 *   g       [59][stride] FP64 parameters, n primitives
 *   cams    V cameras
 *   scores  out [n]    D_i (Eq. 7 with Eq. 20's weights)
 *   S       out [n]    sum over views of vis * P (Eq. 17), i.e. Eq. 20's
 *                      bracket without alpha and 1/|V| (may be NULL)
 *   S_sure  out [n]    the same sum over non-borderline pairs only (may be NULL)
 *   nborder out [n]    number of borderline pairs (may be NULL)
 *   bterms  out [n][4] the first four borderline pairs' terms (may be NULL)
 *   st      out        scene statistics (may be NULL) */
void orc_score_subset(const double *g, int64_t stride, int64_t n, const int64_t *idx, int64_t m_out,
                      const orc_camera *cams, int V, const orc_params *p, double *scores, double *S,
                      double *S_sure, int32_t *nborder, double *bterms, orc_stats *st_out);

void orc_score(const double *g, int64_t stride, int64_t n, const orc_camera *cams, int V,
               const orc_params *p, double *scores, double *S, double *S_sure,
               int32_t *nborder, double *bterms, orc_stats *st_out)
{
    orc_score_subset(g, stride, n, NULL, n, cams, V, p, scores, S, S_sure, nborder, bterms, st_out);
}

/* As orc_score, but the outputs cover only the m_out primitives listed in
 * idx (all n when idx is NULL); the scene statistics still come from all n
 * primitives.  Output arrays are indexed 0 .. m_out-1. */
void orc_score_subset(const double *g, int64_t stride, int64_t n, const int64_t *idx, int64_t m_out,
                      const orc_camera *cams, int V, const orc_params *p, double *scores, double *S,
                      double *S_sure, int32_t *nborder, double *bterms, orc_stats *st_out)
{
    orc_stats st;
    orc_scene_stats(g, stride, n, p, &st);
    if (st_out) *st_out = st;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t o = 0; o < m_out; ++o) {
        int64_t i = idx ? idx[o] : o;
        double alpha, s[3], Rq[9], Sigma[9], m[3];
        double mu[3] = {g[i], g[stride + i], g[2 * stride + i]};
        orc_activate(g, stride, i, &alpha, s, Rq, Sigma);
        double sum = 0.0, sure = 0.0;
        int nb = 0;
        for (int v = 0; v < V; ++v) {
            int border = 0;
            int vis = orc_visible(&cams[v], mu, Sigma, &border);
            double tc[3];
            orc_to_camera(&cams[v], mu, tc);
            double P;
            if (p->flags & ORC_NO_PROJ) {
                P = 1.0;
            } else if (p->flags & ORC_FULL_JAC) {                       /* Eq. 14: ||J_Pi||_F^2 */
                double J[6];
                orc_projection_jacobian(&cams[v], tc, J);
                P = 0.0;
                for (int k = 0; k < 6; ++k) P += J[k] * J[k];
            } else {
                P = 1.0 / (tc[2] * tc[2] + p->eta);                        /* Eq. 17 */
            }
            if (vis) sum += P;
            if (border) {
                if (bterms && nb < 4) bterms[4 * o + nb] = P;
                ++nb;
            } else if (vis) {
                sure += P;
            }
        }
        if (S) S[o] = sum;
        if (S_sure) S_sure[o] = sure;
        if (nborder) nborder[o] = nb;
        double vis_alpha = (p->flags & ORC_NO_VIS) ? 1.0 : alpha;          /* Eq. 12, T = 1 */
        double A = vis_alpha * sum / (double)V;                            /* Eq. 20 / lambda */
        orc_magnitudes(g, stride, i, m);
        double coupled = 0.0;                                              /* Eq. 7 */
        for (int k = 0; k < 3; ++k) {
            double Gt = m[k];
            if (p->flags & ORC_NORM_ATTR) Gt = st.mean_m[k] > 0.0 ? m[k] / st.mean_m[k] : 0.0;
            coupled += st.lambda[k] * Gt;
        }
        scores[o] = A * coupled;
    }
}

/* ------------------------------------------------------------- Sec. 3.3 */

static const double *g_sort_scores;

/* keep order: score descending, then index ascending */
static int orc_keep_order(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    double si = g_sort_scores[i], sj = g_sort_scores[j];
    if (si > sj) return -1;
    if (si < sj) return 1;
    return (i > j) - (i < j);
}

/* Global ranking and removal of the bottom floor(beta N) primitives.
 * mask: out, ceil(n/32) words, bit (i % 32) of word i / 32 set when kept.
 * Returns n_keep; *threshold is the smallest kept score (-inf if none pruned). */
int64_t orc_select(const double *scores, int64_t n, double beta, uint32_t *mask, double *threshold)
{
    int64_t n_prune = (int64_t)floor(beta * (double)n);
    int64_t n_keep = n - n_prune;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    g_sort_scores = scores;
    qsort(order, (size_t)n, sizeof(int64_t), orc_keep_order);
    memset(mask, 0, sizeof(uint32_t) * (size_t)((n + 31) / 32));
    for (int64_t r = 0; r < n_keep; ++r) mask[order[r] / 32] |= 1u << (order[r] % 32);
    *threshold = (n_prune > 0 && n_keep > 0) ? scores[order[n_keep - 1]] : -INFINITY;
    free(order);
    return n_keep;
}

/* Stable gather of the kept primitives: every one of the `rows` rows of
 * `in` (element size `esize` bytes, row stride `stride` elements) is copied
 * in index order into `out` (row stride `out_stride`); idx receives the
 * original indices.  Returns the number kept. */
int64_t orc_compact(const void *in, int64_t stride, int64_t n, int rows, int esize,
                    const uint32_t *mask, void *out, int64_t out_stride, int32_t *idx)
{
    int64_t j = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!((mask[i / 32] >> (i % 32)) & 1u)) continue;
        for (int r = 0; r < rows; ++r)
            memcpy((char *)out + ((size_t)r * (size_t)out_stride + (size_t)j) * (size_t)esize,
                   (const char *)in + ((size_t)r * (size_t)stride + (size_t)i) * (size_t)esize,
                   (size_t)esize);
        if (idx) idx[j] = (int32_t)i;
        ++j;
    }
    return j;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}
