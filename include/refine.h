/*
 * refine.h -- C ABI of librefine, a GB300 (sm_103a) implementation of the
 * rendering-free primitive importance pass of REFINE (arXiv 2606.09074):
 * per-primitive Hessian-weight scoring (Sec. 3.2, Eq. 7 and Eq. 20), ratio
 * pruning by global rank (Sec. 3.3) and compaction of the kept primitives.
 *
 * Conventions shared by every entry point
 *  - Every function returns a refine_status; REFINE_OK is 0.  On failure a
 *    human-readable message is available from refine_last_error(ctx).
 *    Nothing aborts the process.
 *  - "_dev" pointers are CUDA device pointers on the context's device;
 *    "_host" pointers are host memory (pinned host memory makes the copies
 *    asynchronous and fast; pageable memory works but is slower).
 *  - The caller owns every buffer it passes.  The library never frees or
 *    retains caller buffers after a call returns.  Scratch memory is owned
 *    by the context, grows on demand and is released by refine_ctx_destroy.
 *  - Work is enqueued on the caller's stream and is asynchronous unless a
 *    function says it synchronises.  A context is not thread-safe: calls on
 *    one context must be issued from one thread and ordered on one stream,
 *    because they share the context's scratch memory.
 *  - Errors found by device code (NaN / Inf inputs, invalid cameras, a
 *    bounded wait that ran out) are recorded in a device status word and
 *    reported by the next synchronising call (refine_select with a
 *    threshold_out, refine_compact with an n_keep_out, refine_ctx_check).
 *  - Sizes: 0 <= n <= 2^31 - 1 primitives; 1 <= n_views <= 65535.
 */
#ifndef REFINE_H
#define REFINE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *refine_stream_t;

typedef enum refine_status {
    REFINE_OK = 0,
    REFINE_EINVAL = 1,      /* bad argument (NULL, size or ratio out of range, misaligned) */
    REFINE_ENOMEM = 2,      /* device or pinned allocation failed                          */
    REFINE_ECUDA = 3,       /* CUDA runtime error; details in refine_last_error            */
    REFINE_ENONFINITE = 4,  /* NaN or Inf in an input that the device read                 */
    REFINE_ETIMEOUT = 5,    /* a bounded device wait ran out                               */
    REFINE_EBUSY = 6,
    REFINE_ECANCELLED = 7,
    REFINE_ENOTFOUND = 8
} refine_status;

/* Storage type of primitive rows 3..58 (positions are always float32).
 *   REFINE_F32    all 56 attribute rows float32 (224 B per primitive)
 *   REFINE_BF16   all 56 attribute rows bfloat16 (112 B)
 *   REFINE_BF16S  the 3 log-scale rows float32, the other 53 rows bfloat16
 *                 (12 + 106 = 118 B): the rows are laid out as 3 float32
 *                 rows of row_stride elements followed, at byte offset
 *                 12 * row_stride, by 53 bfloat16 rows of row_stride
 *                 elements.  The bfloat16 rounding of the log-scales is what
 *                 moves the keep mask of the BF16 form most (its error grows
 *                 with |ln s| and m_gem carries two scales); this form keeps
 *                 them exact for 6 more bytes per primitive. */
enum { REFINE_F32 = 0, REFINE_BF16 = 1, REFINE_BF16S = 2 };

/* refine_params.flags */
#define REFINE_FLAG_NO_VIS       (1 << 0) /* Table 3 "w/o V": alpha -> 1 in Eq. 20          */
#define REFINE_FLAG_NO_PROJ      (1 << 1) /* Table 3 "w/o P": 1/(z^2+eta) -> 1 in Eq. 20    */
#define REFINE_FLAG_EQUAL_LAMBDA (1 << 2) /* Table 3 "Equal lambda^k": lambda^k = 1/3       */
#define REFINE_FLAG_NORM_ATTR    (1 << 3) /* G~^k = m^k / mean_j(m^k_j) (default on)        */
#define REFINE_FLAG_FULL_JACOBIAN (1 << 4) /* projection term of Eq. 14 before the Eq. 16 *
                                            * simplification: Tr(J^T J) = (fx^2+fy^2)/z^2 *
                                            * + ((fx x)^2+(fy y)^2)/z^4 instead of        *
                                            * 1/(z^2+eta); NO_PROJ takes precedence       */

/* Defaults.  eta is the paper's stability constant (Eq. 17, Sec. 3.2).  The
 * paper calibrates lambda~ by expectations E[.] (Eq. 18) without printing
 * them; these are ln F_gem, F_col and F_opa of 1,000,000 synthetic
 * core-shell primitives (seed 12345) computed in FP64. */
#define REFINE_DEFAULT_ETA      0.05
#define REFINE_DEFAULT_E_LN_GEM (-0.4889612576346142)
#define REFINE_DEFAULT_E_COL    0.008896804239666543
#define REFINE_DEFAULT_E_OPA    0.1515067583205341

/* A pinhole camera (Eq. 13).  80 bytes.  R (row-major) and t map world
 * points to camera space with OpenCV axes (x right, y down, z forward):
 * x_cam = R x_world + t.  Pixel (u, v) = (fx x/z + cx, fy y/z + cy); the
 * image is the closed rectangle [0, width] x [0, height].  Requirements:
 * all fields finite, fx, fy > 0, width, height >= 1, 0 < znear < zfar. */
typedef struct refine_camera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear, zfar;
} refine_camera;

/* A scene of n primitives in structure-of-arrays form (Eq. 1: mean, scale,
 * rotation, SH colour, opacity -- 59 parameters per primitive).
 *   pos   device, float32 [3][row_stride]: rows 0-2, mean x, y, z
 *   attr  device, [56][row_stride] in `dtype` (float32, bfloat16, or the
 *           mixed layout of REFINE_BF16S):
 *           row 0-2   log-scale
 *           row 3-6   rotation quaternion (w, x, y, z), need not be unit
 *           row 7     opacity logit
 *           row 8-10  SH DC (r, g, b)
 *           row 11-55 SH degree 1-3, 15 coefficients x 3 channels
 *   row_stride  elements between consecutive rows, >= n (the stride counts
 *           elements of each row's own type).
 * pos and attr must be 16-byte aligned. */
typedef struct refine_scene {
    int64_t n;
    int32_t dtype;
    int32_t reserved;
    const float *pos;
    const void *attr;
    int64_t row_stride;
} refine_scene;

/* Method parameters.  Fill with refine_params_default() and override. */
typedef struct refine_params {
    float eta;        /* Eq. 17 and Eq. 18 stability constant (>= FLT_MIN, finite)  */
    float luma[3];    /* weights of the perceptual luma Y of the SH DC colour          */
    double e_ln_gem;  /* Eq. 18 calibration E[ln F_gem] (nonzero)                      */
    double e_col;     /* Eq. 18 calibration E[F_col]    (nonzero)                      */
    double e_opa;     /* Eq. 18 calibration E[F_opa]    (nonzero)                      */
    int32_t flags;    /* REFINE_FLAG_*                                                 */
    int32_t max_views; /* view subsampling (Table B.1 scores 64 views): with          *
                        * 0 < max_views < n_views, views 0, s, 2s, ... are scored,    *
                        * s = ceil(n_views / max_views), and |V| in Eq. 20 is their   *
                        * count; 0 = every view (default)                             */
} refine_params;

/* Scene statistics computed on the device (Eq. (features), Eq. 18-19). */
typedef struct refine_scene_stats {
    double F_col, F_opa, F_gem;
    double lambda_t[3];  /* unnormalised lambda~ (gem, col, opa), negatives clamped to 0 */
    double lambda[3];    /* Eq. 19 (gem, col, opa)                                        */
    double mean_m[3];    /* scene means of the magnitudes m^gem, m^col, m^opa             */
    /* How the (primitive, view) pairs were decided (work accounting):        */
    int64_t pairs;           /* n * n_views                                                */
    int64_t tile_views;      /* (tile of 64 primitives, view) classifications              */
    int64_t in_pairs;        /* pairs in tiles found entirely in range and in the image    */
    int64_t out_pairs;       /* pairs in tiles found entirely invisible                    */
    int64_t mixed_pairs;     /* pairs decided one by one                                   */
    int64_t bound_pairs;     /* of those: centre in the depth range but outside the image  */
    int64_t footprint_pairs; /* of those: within the conservative footprint radius, so the
                                exact J W Sigma W^T J^T test decided them                  */
    int64_t visible_mixed_pairs; /* pairs decided one by one and found visible             */
    int64_t open_u_pairs;    /* pairs decided one by one whose tile left 0 < u < w open    */
    int64_t open_v_pairs;    /* ... 0 < v < h open                                        */
    int64_t open_z_pairs;    /* ... znear < z < zfar open                                 */
    int64_t bound_u_pairs;   /* bound-stage pairs with 0 < u < w open                     */
    int64_t bound_v_pairs;   /* bound-stage pairs with 0 < v < h open                     */
    int64_t exact_u_pairs;   /* exact-test pairs whose centre lies beyond 0 < u < w, so
                                the u extent of the footprint was formed                  */
    int64_t exact_v_pairs;   /* ... beyond 0 < v < h, the v extent formed                 */
    int64_t exact_warp_axes; /* warp-level evaluations of one extent of the exact test
                                (32 lanes each): how densely the exact test ran           */
} refine_scene_stats;

typedef struct refine_ctx refine_ctx;

/* Library version string. */
const char *refine_version(void);

/* Fills *out with eta = 0.05, BT.601 luma (0.299, 0.587, 0.114), the
 * default E[.] constants and flags = REFINE_FLAG_NORM_ATTR.  EINVAL if out
 * is NULL. */
refine_status refine_params_default(refine_params *out);

/* Creates a context bound to CUDA device `device` (it becomes current on
 * the calling thread).  *out receives the handle.  EINVAL for a bad device
 * or NULL out; ECUDA if the device cannot be initialised. */
refine_status refine_ctx_create(refine_ctx **out, int device);

/* Frees the context's scratch memory and the context.  NULL is a no-op.
 * Synchronises the context's device first. */
void refine_ctx_destroy(refine_ctx *ctx);

/* Message of the last failure on this context ("" if none).  The string is
 * owned by the context and valid until its next call. */
const char *refine_last_error(const refine_ctx *ctx);

/* Importance score D(G_i) of every primitive (Sec. 3.2: Eq. 7 with the
 * Hessian weights of Eq. 20, lambda^k from Eq. 18-19, the projection term
 * of Eq. 17 and, for each view, the visibility of the primitive's 3-sigma
 * footprint under the EWA projected covariance J W Sigma W^T J^T, Eq. 13-14).
 *   scene       primitives (see refine_scene), device memory
 *   cams_dev    device array of n_views refine_camera records
 *   params      host pointer; NULL means refine_params_default()
 *   scores_dev  device float32 [scene->n], written
 * Asynchronous on `stream`.  Input NaN/Inf and invalid cameras are
 * reported through the device status word (ENONFINITE / EINVAL). */
refine_status refine_score(refine_ctx *ctx, const refine_scene *scene,
                           const refine_camera *cams_dev, int32_t n_views,
                           const refine_params *params, float *scores_dev,
                           refine_stream_t stream);

/* refine_score plus diagnostics.
 *   view_sum_dev  device float32 [n] or NULL: sum over views of
 *                 vis * 1/(z^2+eta) (Eq. 20's bracket without alpha, 1/|V|)
 *   stats_out     host pointer or NULL: scene statistics; when non-NULL the
 *                 call synchronises `stream` to return them. */
refine_status refine_score_ex(refine_ctx *ctx, const refine_scene *scene,
                              const refine_camera *cams_dev, int32_t n_views,
                              const refine_params *params, float *scores_dev,
                              float *view_sum_dev, refine_scene_stats *stats_out,
                              refine_stream_t stream);

/* Ratio pruning by global rank (Sec. 3.3): the bottom floor(ratio * n)
 * primitives are pruned, ranking by score and breaking ties by index
 * (among equal scores the higher index is pruned first; -0 equals +0).
 *   scores_dev     device float32 [n] (NaN rejected with ENONFINITE)
 *   ratio          pruning ratio beta in [0, 1)
 *   keep_mask_dev  device uint32 [ceil(n/32)], written: bit (i % 32) of word
 *                  i / 32 is set when primitive i is kept; bits >= n are 0
 *   threshold_out  host, or NULL: the smallest kept score (-inf when nothing
 *                  is pruned).  Non-NULL makes the call synchronise.
 *   n_keep_out     host, or NULL: n - floor(ratio * n) (known on the host,
 *                  no synchronisation)
 * Uses context scratch memory (radix-select histograms and state). */
refine_status refine_select(refine_ctx *ctx, const float *scores_dev, int64_t n, double ratio,
                            uint32_t *keep_mask_dev, float *threshold_out, int64_t *n_keep_out,
                            refine_stream_t stream);

/* Stable compaction of the kept primitives (Sec. 3.3, "saving primitives"):
 * every one of the 59 rows of the kept primitives, in index order.
 *   in             the scene (device)
 *   keep_mask_dev  device uint32 [ceil(n/32)] as written by refine_select
 *   out_pos_dev    device float32 [3][out_row_stride]
 *   out_attr_dev   device [56][out_row_stride] in in->dtype (the same row
 *                  layout as the input, with out_row_stride)
 *   out_row_stride >= number of kept primitives
 *   kept_idx_dev   device int32 [n_keep] original indices, or NULL
 *   n_keep_out     host or NULL; non-NULL synchronises and returns the count
 * The kept count must not exceed out_row_stride; the kernel writes nothing
 * beyond it and reports EINVAL through the status word if it would. */
refine_status refine_compact(refine_ctx *ctx, const refine_scene *in,
                             const uint32_t *keep_mask_dev, float *out_pos_dev,
                             void *out_attr_dev, int64_t out_row_stride,
                             int32_t *kept_idx_dev, int64_t *n_keep_out,
                             refine_stream_t stream);

/* The whole pass from host memory: copies the scene (pos_host float32
 * [3][n], attr_host [56][n] in `dtype`, both row-contiguous) and cameras to
 * the device, scores, selects and compacts, and copies back the kept
 * primitives (out_pos_host [3][n_keep], out_attr_host [56][n_keep]), their
 * indices (out_idx_host int32 [n_keep], or NULL) and the scores
 * (scores_host float32 [n], or NULL).  Device buffers are context scratch.
 * Synchronises `stream` before returning; *n_keep_out and *threshold_out
 * (either may be NULL) receive the kept count and threshold. */
refine_status refine_prune_host(refine_ctx *ctx, int64_t n, int32_t dtype,
                                const float *pos_host, const void *attr_host,
                                const refine_camera *cams_host, int32_t n_views,
                                const refine_params *params, double ratio,
                                float *out_pos_host, void *out_attr_host,
                                int32_t *out_idx_host, float *scores_host,
                                int64_t *n_keep_out, float *threshold_out,
                                refine_stream_t stream);

/* ------------------------------------------------------------ batches
 * Many scenes in one go: per-scene preparation (content features, lambda,
 * processing order) and per-scene selection and compaction run on parallel
 * streams, and all scenes are scored by persistent kernel launches over a
 * (scene, tile, camera block) work list: one launch per camera block level,
 * launch p scoring the p-th block of views of every scene that has one
 * (a single launch when every scene has at most camera_block views).  The
 * whole batch is captured into a CUDA graph on its first run and replayed
 * afterwards, so a run costs one graph launch.  Scores, masks and compacted
 * outputs are bit-identical to the per-scene entry points. */

/* One scene of a batch; every pointer is device memory owned by the caller
 * and must stay valid (and unchanged in address) for the batch's life. */
typedef struct refine_job {
    refine_scene scene;            /* primitives (see refine_scene)                      */
    const refine_camera *cams_dev; /* n_views camera records                             */
    int32_t n_views;               /* 1 .. 65535                                          */
    int32_t reserved;
    double ratio;                  /* pruning ratio in [0, 1)                             */
    float *scores_dev;             /* [n] written                                         */
    uint32_t *keep_mask_dev;       /* [ceil(n/32)] written                                */
    float *out_pos_dev;            /* [3][out_row_stride] or NULL to skip compaction      */
    void *out_attr_dev;            /* [56][out_row_stride] in scene.dtype                 */
    int64_t out_row_stride;        /* >= n - floor(ratio n)                               */
    int32_t *kept_idx_dev;         /* [n_keep] or NULL                                    */
} refine_job;

typedef struct refine_batch refine_batch;

/* Builds a batch of n_jobs scenes (1 <= n_jobs <= 4096, n >= 1 and
 * n_views <= 65535 each, storage types may differ; the jobs array is copied),
 * with the context's shape at this call (camera block included).  Allocates
 * all scratch up front (released by refine_batch_destroy).  EINVAL on a bad
 * job (refine_last_error(ctx) names it), ENOMEM if the scratch does not fit. */
refine_status refine_batch_create(refine_ctx *ctx, const refine_job *jobs, int32_t n_jobs,
                                  const refine_params *params, refine_batch **out);

/* Enqueues a run of the whole batch on `stream` (asynchronous).  The first
 * run records the CUDA graph (it must not be called while `stream` is being
 * captured); later runs launch it. */
refine_status refine_batch_run(refine_batch *batch, refine_stream_t stream);

/* Synchronises `stream` and returns, per job, the kept count and the
 * threshold of the last run (either pointer may be NULL), plus any device
 * error recorded since the last check. */
refine_status refine_batch_results(refine_batch *batch, int64_t *n_keep_out, float *threshold_out,
                                   refine_stream_t stream);

/* Number of kernels one run launches. */
int64_t refine_batch_launches(const refine_batch *batch);

/* Releases the batch (synchronising its device first).  NULL is a no-op. */
void refine_batch_destroy(refine_batch *batch);

/* ------------------------------------------------------------ autotuner
 * Work-item shape of the score kernels.  A warp scores a tile of 32 or 64
 * consecutive primitives of the processing order against every view; the
 * batched kernel hands out CTA-sized items of such tiles, and the views are
 * taken in camera blocks (passes) of `camera_block` views.  Every
 * primitive's score is computed by one thread with the views in a fixed
 * order, whatever tile it is in, and its running Kahan pair is carried
 * from one camera block to the next, so the shape changes speed only:
 * results are bit-identical for every shape. */
typedef struct refine_shape {
    int32_t tile;         /* primitives per warp tile: 32 or 64 (default 64)            */
    int32_t cta_threads;  /* threads per CTA of the batched kernel: 128 or 256          */
    int32_t ctas_per_sm;  /* cap on resident CTAs per SM (batched kernel), 0 = all fit */
    int32_t camera_block; /* views per score pass: 32..512, a multiple of 32 (default
                             512); a scene with more views is scored in passes, and a
                             batch scores pass p of all its scenes in one launch       */
    double ms;            /* refine_autotune: measured time of the batched score launches */
} refine_shape;

/* Times the batched score launches of `jobs` (as refine_batch_create takes
 * them; their scores are written) under every candidate shape -- tile 64 or
 * 32, CTAs of 256 or 128 threads, all CTAs that fit per SM or a cap, and
 * camera blocks of 512, 256 and 128 views (a block that would split no scene
 * differently from a larger one is not tried again) -- `reps` runs each
 * after one warm-up, and makes the fastest the context's shape
 * (used by refine_score and by batches and queues created afterwards).
 * *best_out (may be NULL) receives it; table_out (may be NULL) receives up to
 * table_cap candidates in the order tried, *table_count their number.
 * EINVAL for bad jobs or reps < 1. */
refine_status refine_autotune(refine_ctx *ctx, const refine_job *jobs, int32_t n_jobs,
                              const refine_params *params, int32_t reps, refine_shape *best_out,
                              refine_shape *table_out, int32_t table_cap, int32_t *table_count);

/* Reads or sets the context's shape (EINVAL for a shape outside the
 * candidates: tile 32 or 64, cta_threads 128 or 256, ctas_per_sm >= 0,
 * camera_block 32..512 in steps of 32). */
refine_status refine_ctx_get_shape(const refine_ctx *ctx, refine_shape *out);
refine_status refine_ctx_set_shape(refine_ctx *ctx, const refine_shape *shape);

/* ------------------------------------------------------ request queue
 * A serving loop for pruning requests (Sec. 3.3 applied to a stream of
 * scenes).  Three native threads own the GPU work:
 *   - the dispatcher admits pending requests in arrival order while the
 *     device bytes of the admitted ones fit the queue's HBM budget and a
 *     slot is free; each admitted request gets a slot (its own CUDA stream)
 *     and one device block from the queue's memory pool, into which its
 *     scene and cameras are copied at once (the copies of all requests go
 *     through one input-copy stream, in admission order, so that each ends
 *     as early as the link allows), and its preparation follows on its
 *     slot stream;
 *   - the scorer batches continuously: as soon as the previous batched
 *     launch has ended, ONE persistent launch scores every request whose
 *     preparation has ended (those requests form a round; a request with
 *     more views than the camera block has its further blocks scored right
 *     after it, in order, on the same stream); selection and compaction
 *     then run on the requests' slot streams and the copies back on one
 *     output-copy stream.  Requests that arrive while others are on the GPU
 *     thus join the next launch, and their copies overlap the others'
 *     kernels;
 *   - the completion thread retires requests whose GPU work has finished:
 *     it finishes copies into pageable host buffers, records the result,
 *     frees the device block and returns its bytes to the budget.
 * A request's results are bit-identical to refine_score + refine_select +
 * refine_compact on the same scene, whatever else is in flight. */
typedef struct refine_queue refine_queue;

/* One pruning request.  Every pointer is host memory owned by the caller;
 * inputs are read, and outputs written, between submission and the moment
 * the request's result is reported by refine_queue_poll, so all of them
 * must stay valid until then.  Page-locked buffers (cudaHostAlloc or
 * cudaHostRegister) are copied asynchronously; pageable ones are copied by
 * the queue's threads synchronously, which is slower. */
typedef struct refine_request {
    int64_t n;                       /* primitives, 1 .. 2^31 - 1                           */
    int32_t dtype;                   /* REFINE_F32, REFINE_BF16 or REFINE_BF16S (attr rows) */
    int32_t n_views;                 /* 1 .. 65535                                          */
    const float *pos_host;           /* [3][n] float32 means                               */
    const void *attr_host;           /* [56][n] in dtype, rows as in refine_scene          */
    const refine_camera *cams_host;  /* [n_views]                                          */
    double ratio;                    /* pruning ratio in [0, 1)                            */
    const refine_params *params;     /* NULL = the queue's parameters; copied at submit    */
    uint32_t *keep_mask_host;        /* [ceil(n/32)] or NULL                               */
    float *scores_host;              /* [n] or NULL                                        */
    float *out_pos_host;             /* [3][n_keep] compacted means, or NULL (no compaction) */
    void *out_attr_host;             /* [56][n_keep] in dtype; needed with out_pos_host    */
    int32_t *kept_idx_host;          /* [n_keep] original indices, or NULL                 */
} refine_request;

/* Result of one request.  Times are host steady-clock instants in ms since
 * the queue was created: submission, admission (device block granted) and
 * completion (every output in host memory). */
typedef struct refine_result {
    refine_status status;  /* of this request: OK, ENONFINITE, EINVAL (bad camera), ECUDA, ECANCELLED */
    int32_t round_size;    /* requests scored by the same launch                                   */
    int64_t n_keep;        /* n - floor(ratio n)                                                    */
    float threshold;       /* as refine_select                                                      */
    float reserved;
    double submit_ms, admit_ms, done_ms;
    /* The request's device timeline, in ms of device time since the queue
     * was created (a different clock from the three above; -1 where the
     * request did not get that far): its copy in ended, its preparation
     * ended, the batched score launch that scored it ended, its selection
     * and compaction ended, its copy out ended. */
    double copied_ms, prepped_ms, scored_ms, computed_ms, read_ms;
} refine_result;

typedef struct refine_queue_stats {
    int64_t submitted, admitted, completed, rounds;
    int64_t pending, in_flight;
    uint64_t bytes_in_use, peak_bytes, budget_bytes;
    int32_t max_round, slots;
    int64_t kernel_launches;
    double dispatch_ms;  /* host time the dispatcher spent issuing rounds (API calls)  */
    double retire_ms;    /* host time the completion thread spent retiring requests   */
} refine_queue_stats;

/* Device bytes one request holds while admitted (scene, cameras, scratch,
 * scores, mask and, with compact != 0, the compacted rows), for the
 * smallest camera block (so an upper bound for any queue's shape); 0 for
 * arguments out of range. */
uint64_t refine_queue_footprint(int64_t n, int32_t dtype, int32_t n_views, double ratio, int32_t compact);

/* Creates a queue on ctx's device (ctx itself is not used by the queue's
 * threads and may keep serving other calls).  hbm_budget_bytes bounds the
 * sum of the footprints of admitted requests; max_slots (1 .. 64) bounds
 * their number.  params NULL = refine_params_default().  EINVAL on bad
 * arguments, ENOMEM/ECUDA if streams, pools or threads cannot be made. */
refine_status refine_queue_create(refine_ctx *ctx, uint64_t hbm_budget_bytes, int32_t max_slots,
                                  const refine_params *params, refine_queue **out);

/* Enqueues a request (the struct and *params are copied) and returns its
 * ticket.  EINVAL for a malformed request, ENOMEM if its footprint alone
 * exceeds the budget, ECANCELLED after refine_queue_destroy began.  Never
 * blocks on the GPU. */
refine_status refine_queue_submit(refine_queue *q, const refine_request *req, uint64_t *ticket);

/* Waits up to timeout_ms (0 = do not wait, < 0 = no limit) for the request
 * with this ticket and, when it is done, fills *out and retires the ticket.
 * Returns OK (see out->status for the request's own outcome), ETIMEOUT if it
 * is not done yet, ENOTFOUND for an unknown or already retired ticket. */
refine_status refine_queue_poll(refine_queue *q, uint64_t ticket, refine_result *out, int32_t timeout_ms);

/* Like refine_queue_poll for whichever request finishes first: waits up to
 * timeout_ms for any submitted request to be done, then fills *ticket_out
 * and *out and retires that ticket (among several done, the lowest ticket).
 * Lets a server take results in completion order, so that a long request
 * does not hold up the output buffers of the short ones that finish after
 * it.  ETIMEOUT if none is done in time, ENOTFOUND if no request is
 * outstanding. */
refine_status refine_queue_poll_any(refine_queue *q, uint64_t *ticket_out, refine_result *out, int32_t timeout_ms);

refine_status refine_queue_stats_get(refine_queue *q, refine_queue_stats *out);

/* Text of the last failure the queue's threads met while issuing GPU work
 * ("" if none).  The string is owned by the queue and valid until the next
 * call on it. */
const char *refine_queue_last_error(refine_queue *q);

/* Stops admitting, cancels pending requests, waits for the admitted ones,
 * joins the threads and frees everything.  NULL is a no-op. */
void refine_queue_destroy(refine_queue *q);

/* Ratio pruning without any allocation.  The paper has no counterpart; this
 * entry point exists for callers that cannot allocate device memory --
 * plug-ins whose host engine owns every device allocation, real-time loops
 * whose memory is fixed at start-up -- and so cannot create a refine_ctx.
 *
 * Same inputs, outputs and result as refine_select (same kernels), but no
 * context: it runs on the calling thread's current device and keeps its
 * scratch (selection state and tie counts) in a fixed device array of about
 * 74 KB inside the library, which every GPU that loads the library holds
 * until the process exits.  It calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *   n        0 <= n <= 67,108,864 (2^26); larger n returns REFINE_EINVAL
 *   errbuf   host buffer of errlen bytes for a message, or NULL
 * Every call looks up the array's device address (cudaGetSymbolAddress) on
 * the calling thread's current device; the first call on a device also
 * loads the library's device code there.  Every call on a device shares the
 * one array and each call resets it: calls whose work overlaps on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 * NaN scores are
 * reported (REFINE_ENONFINITE) only when threshold_out is non-NULL, which
 * makes the call synchronise `stream`. */
refine_status refine_select_noalloc(const float *scores_dev, int64_t n, double ratio,
                                    uint32_t *keep_mask_dev, float *threshold_out,
                                    int64_t *n_keep_out, char *errbuf, size_t errlen,
                                    refine_stream_t stream);

/* ------------------------------------------------------------ scene files
 * Host-side I/O of scenes in the PLY layout of 3D Gaussian Splatting
 * checkpoints, the format in which a pruned scene is saved ("saving
 * primitives", Sec. 4.2): binary little-endian, one float32 vertex per
 * primitive with properties x y z nx ny nz f_dc_0-2 f_rest_0-44 opacity
 * scale_0-2 rot_0-3 (log-scales, quaternion w x y z, opacity logit, f_rest
 * channel-major).  Rows map to refine_scene rows one to one (normals are
 * written as 0 and ignored on reading). */

/* Writes n primitives from host rows pos_host [3][row_stride] (float32) and
 * attr_host [56][row_stride] (dtype, any storage type; bfloat16 is widened
 * exactly).  EINVAL
 * for bad arguments or a file that cannot be written. */
refine_status refine_write_ply(const char *path, int64_t n, int32_t dtype, const float *pos_host,
                               const void *attr_host, int64_t row_stride);

/* Reads a scene PLY.  With pos_host and attr_host NULL only *n_out is set;
 * otherwise the rows are written to pos_host [3][row_stride] and attr_host
 * [56][row_stride], both float32, row_stride >= n.  Properties are matched by
 * name, in any order, extra ones ignored.  EINVAL for a file that is not
 * binary little-endian with one float32 vertex element holding them all. */
refine_status refine_read_ply(const char *path, int64_t *n_out, float *pos_host, float *attr_host,
                              int64_t row_stride);

/* Synchronises `stream` and returns (then clears) the device status word:
 * REFINE_OK, or the first error a kernel recorded since the last check. */
refine_status refine_ctx_check(refine_ctx *ctx, refine_stream_t stream);

/* Instrumentation.  With timing enabled kernel launches are bracketed by
 * CUDA events on their stream: enable = REFINE_TIMING_ALL brackets every
 * launch, REFINE_TIMING_SCORE only the score kernel's (two events per score
 * pass, so that a timed loop is barely perturbed; each event pair costs
 * about 2 us of stream time), 0 none.  refine_ctx_kernel_times
 * synchronises, then reports the accumulated device milliseconds and launch
 * counts per kernel class (names[i], ms[i], launches[i] for i < *count,
 * at most `cap` entries) and resets them.  refine_ctx_launch_count returns
 * the number of kernels the context has launched since creation. */
#define REFINE_TIMING_ALL   1
#define REFINE_TIMING_SCORE 2
refine_status refine_ctx_set_timing(refine_ctx *ctx, int enable);
refine_status refine_ctx_kernel_times(refine_ctx *ctx, const char **names, double *ms,
                                      int64_t *launches, int32_t cap, int32_t *count);
int64_t refine_ctx_launch_count(const refine_ctx *ctx);

/* Self-test of failure detection on the device (no counterpart in the
 * paper: it tests the bounded wait that guards the score kernels' TMA
 * camera staging, without faulting or hanging the GPU).  A one-thread kernel
 * stages `bytes` bytes of context scratch into shared memory by a bulk copy
 * whose mbarrier expects bytes + missing_bytes.
 *   bytes          16..1024, a multiple of 16
 *   missing_bytes  0..65536: with 0 the wait completes and the call returns
 *                  REFINE_OK; otherwise the barrier phase can never complete,
 *                  the wait gives up after wait_cycles SM clock cycles and
 *                  the call returns REFINE_ETIMEOUT, read from the device
 *                  status word like any device error (which it then clears)
 *   wait_cycles    1..2e9 (about a second at the maximum SM clock)
 * Synchronises `stream`.  The context stays usable afterwards. */
refine_status refine_selftest_wait(refine_ctx *ctx, uint32_t bytes, uint32_t missing_bytes,
                                   int64_t wait_cycles, refine_stream_t stream);

/* Measured FP32 FMA throughput of the context's device: the denominator
 * that the score kernel's roofline (an FP32-issue-bound kernel, no dense
 * contraction) is compared with, beside the nominal SMs x 128 lanes x 2 x
 * clock.  The paper has no counterpart.  A grid of 8 CTAs of 256 threads per
 * SM runs `iters` steps of 8 independent FMA chains per thread with no
 * memory traffic; one launch runs untimed, the next is timed with CUDA
 * events on `stream`.
 *   iters        1 .. 2^20 (2^17 takes about 8 ms on a 152-SM part)
 *   flops_per_s  2 FLOPs per FMA / elapsed seconds, at whatever SM clock the
 *                device ran (required)
 *   ms_out       the timed launch's duration, or NULL
 * Synchronises `stream`.  EINVAL for iters out of range. */
refine_status refine_fma_rate(refine_ctx *ctx, int32_t iters, double *flops_per_s, double *ms_out,
                              refine_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* REFINE_H */
