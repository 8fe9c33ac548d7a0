/* gsblitz.h -- C ABI of the GB300 (sm_103a) 3D Gaussian Splatting hot path.
 *
 * Implements the per-iteration render of BlitzGS (arXiv 2605.13794) on one GPU:
 *   gs_preprocess  view gate (Sec. 3.3, Eq. 1-3) + EWA projection and SH colour
 *                  (App. A: "projected to screen-space ellipses", c_i(d) by SH)
 *   gs_bin_sort    tile/depth keys and a device radix sort (App. A: tile-based,
 *                  depth-ordered projected Gaussians)
 *   gs_render_fwd  front-to-back alpha compositing (App. A, Eq. for C(p), T_i)
 *   gs_render_bwd  its adjoint and the adjoint of the projection, plus the
 *                  scale regulariser of Eq. 5
 *   gs_importance  the instrumented colourless sweep of Sec. 3.2 / Fig. 2:
 *                  w = sum_p alpha T, a = qualifying pixels, s, c^rad, c^vis, Cull
 *   gs_photometric_loss  L1 + lambda (1 - SSIM) of Eq. 4
 *   gs_adam_step   the optimizer step of "standard 3DGS" training (also fused
 *                  with compact gradient rows, and with deferred zero-gradient
 *                  steps: gs_adam_lazy_enable / gs_adam_flush)
 *   gs_render_fwd_importance  the forward and the importance raster in one pass
 *   gs_prune_sample, gs_prune_mass, gs_compact, gs_densify, gs_count_views
 *                  the model-level passes of Sec. 3.2-3.3 (pruning Pass 1 and 2,
 *                  density control with the phi reweighting, LOD inheritance)
 *   gs_visible_set_static  a view's Cull column without any allocation
 *   gs_kernel_timing, gs_kernel_time  event timing of the rasterisers
 *   gs_graph_*     capture and replay of a sequence of calls as a CUDA graph
 *
 * Conventions for every call:
 *   - Every pointer argument that names an array is a DEVICE pointer unless the
 *     comment says "host".  Arrays are owned by the caller; the library never
 *     frees or retains them beyond the call.
 *   - Calls are asynchronous on the given stream and allocate nothing: all
 *     scratch lives in a gs_workspace created once by gs_workspace_create.
 *     The one exception is gs_visible_set_static, which takes no workspace:
 *     its scratch is a fixed device array of the library, and its kernel
 *     errors come back through its own error_out word, not gs_sync_status.
 *     A NULL stream means the legacy default stream.
 *   - A workspace is not thread-safe on the host: the calls on one workspace
 *     are issued from one thread at a time (their GPU work may still overlap
 *     where a call says so, as gs_importance on a second stream).
 *   - Every call returns a gs_status.  Argument errors are reported at once.
 *     Errors found by kernels (capacity overflow, a bounded wait that gave up)
 *     are recorded in the workspace's device error word, returned by the next
 *     gs_sync_status call and reported in gs_counts.error by
 *     gs_workspace_counts; the outputs of the failing step are then
 *     undefined.  The library never aborts, exits or traps.  gs_last_error()
 *     describes the last error of the calling thread.
 *   - Floating point is FP32: the projected mean is carried as a pair of
 *     floats (double-float), and the few scalar reductions (loss, importance
 *     masses) are exact fixed-point or FP64 sums.
 */
#ifndef GSBLITZ_H
#define GSBLITZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gs_stream; /* same handle as cudaStream_t */
typedef struct gs_workspace gs_workspace;

#define GS_MAX_CAMERAS 64
#define GS_TILE 16
#define GS_MAX_ADAM_GROUPS 16

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = -1, /* bad argument (NULL, size, alignment) */
    GS_ERR_OOM = -2,         /* workspace allocation failed */
    GS_ERR_CAPACITY = -3,    /* a workspace capacity was exceeded; see gs_counts */
    GS_ERR_CUDA = -4,        /* a CUDA runtime call failed */
    GS_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    GS_ERR_DEVICE = -6       /* other device-side error */
} gs_status;

/* Workspace capacities.  Records are active (Gaussian, camera) pairs after
 * the view gate and culling; instances are (record, tile) pairs. */
typedef struct {
    int64_t max_gaussians;
    int64_t max_records;
    int64_t max_instances;
    int64_t max_tiles;    /* sum over the cameras of one call of tiles_x * tiles_y */
    int64_t max_pixels;   /* sum over the cameras of one call of width * height */
    int32_t max_cameras;  /* <= GS_MAX_CAMERAS */
    int32_t flags;        /* GS_CAP_* bits */
} gs_capacity;

/* gs_capacity.flags: a workspace for rendering and importance only.  It holds
 * no gradient storage (36 -> 8 bytes per instance, no per-record gradient
 * rows, no loss maps); the backward, the loss and the compact Adam step
 * return GS_ERR_INVALID_ARG on it. */
#define GS_CAP_FORWARD_ONLY 1
/* gs_capacity.flags: also hold scratch for the model-level calls (pruning,
 * compaction, densification; about 28 bytes per Gaussian of max_gaussians). */
#define GS_CAP_MODEL_OPS 2

/* Gaussian parameters, one row per Gaussian for each attribute (the layout of
 * PyTorch 3DGS code), FP32:
 *   mean          [n][3]     world-space centre mu
 *   log_scale     [n][3]     log of the per-axis standard deviations
 *   quat          [n][4]     rotation (w, x, y, z); normalised before use
 *   opacity_logit [n]        opacity = sigmoid(opacity_logit)
 *   sh            [n][16][3] degree-3 SH: coefficient, then channel
 *   lod           [n]        uint8 LOD level (Sec. 3.3); NULL = all level 0
 * Rows keep a Gaussian's attribute contiguous, so the sparse passes (only
 * active Gaussians) read few cache sectors while the dense passes stay
 * coalesced.  Base pointers must be 16-byte aligned. */
typedef struct {
    int64_t n;
    const float *mean;
    const float *log_scale;
    const float *quat;
    const float *opacity_logit;
    const float *sh;
    const uint8_t *lod;
} gs_gaussians;

/* Gradients with the layout of gs_gaussians (no lod). */
typedef struct {
    float *mean;
    float *log_scale;
    float *quat;
    float *opacity_logit;
    float *sh;
} gs_gaussian_grads;

/* Pinhole camera: x_cam = R x_world + t (R row-major), looking along +z,
 * image x right and y down.  Pixel (px, py) is centred at (px + 0.5, py + 0.5);
 * (cx, cy) is the principal point.  campos is the camera centre in world
 * coordinates (-R^T t), used by the LOD gate (Eq. 1) and the SH direction. */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float campos[3];
    int32_t width, height;
} gs_camera;

/* Cull modes (gs_render_params.cull_enable).  GS_CULL_DROP removes a culled
 * Gaussian from the view at the gate.  GS_CULL_MARK keeps it and marks its
 * record: gs_render_fwd and the backward treat a marked record as absent (the
 * same images and gradients as GS_CULL_DROP; its gradient is zero and it is
 * not in the visible set of Eq. 5), while gs_importance scores every record
 * as with GS_CULL_OFF -- so one preprocess and one gs_bin_sort serve both the
 * masked training render and the unmasked importance sweep of a view. */
enum { GS_CULL_OFF = 0, GS_CULL_DROP = 1, GS_CULL_MARK = 2 };

/* Render parameters; gs_default_params fills the standard values. */
typedef struct {
    int32_t tile_w;      /* tile width in pixels; tile_w x tile_h is one of 16x16 (GS_TILE, the */
    int32_t tile_h;      /* 3DGS tiling), 32x8, 8x32, 32x16, 16x8, 8x16 */
    int32_t lod_enable;  /* distance LOD gate of Eq. 1-2 */
    int32_t lod_Lmax;    /* L_max(t) of Eq. 1 */
    int32_t cull_enable; /* per-view Cull column of Eq. 3: GS_CULL_OFF, GS_CULL_DROP or GS_CULL_MARK */
    float bg[3];         /* background colour, added as T_final * bg */
    float alpha_min;     /* 1/255: fragments with alpha below are skipped */
    float alpha_max;     /* 0.99: alpha = min(alpha_max, o G') */
    float T_min;         /* 1e-4: a pixel stops before T would drop below */
    float dilation;      /* 0.3 added to the diagonal of the 2D covariance */
    float znear;         /* 0.2: Gaussians with camera z <= znear are culled */
    float fov_clamp;     /* 1.3: Jacobian evaluated at x/z clamped to fov_clamp * tan(fov/2) */
    float lod_d0;        /* d0 of Eq. 1 */
    float lod_f;         /* f of Eq. 1 (2) */
    float eps_score;     /* epsilon of the importance score s_i (Sec. 3.2) */
    float vis_mass;      /* 0.99: c^vis keeps the top vis_mass of each view's w mass */
} gs_render_params;

/* Device-side counters of the last preprocess / bin_sort, read by
 * gs_workspace_counts (which synchronises the stream). */
typedef struct {
    int64_t n_records;        /* active (Gaussian, camera) pairs */
    int64_t n_instances;      /* (record, tile) pairs */
    int64_t n_visible;        /* Gaussians with at least one record (not marked culled) */
    int64_t records_needed;   /* equals n_records unless capacity was exceeded */
    int64_t instances_needed; /* equals n_instances unless capacity was exceeded */
    int32_t error;            /* device error word: 0 or a gs_status */
    int32_t error_site;       /* kernel that set it (implementation detail) */
    int64_t fragments;        /* sum over pixels of the list entries up to and including the pixel's
                                 last composited one: the (pixel, entry) pairs the backward walks.
                                 Counted by gs_render_bwd, reset by gs_preprocess */
    int64_t composited;       /* those of the pairs above that composite (alpha >= alpha_min) */
    int64_t n_candidates;     /* Gaussians the view gate passed on to the projection */
} gs_counts;

typedef struct {
    float *param;
    const float *grad;
    float *m;
    float *v;
    int64_t n;
    float lr, beta1, beta2, eps;
} gs_adam_group;

/* Internal buffers exposed for inspection (debugging, tests).  Pointers are
 * device pointers owned by the workspace; counts are capacities.  Records are
 * stored in (Gaussian, camera) order, so a Gaussian's records are contiguous. */
typedef enum {
    GS_BUF_REC_GAUSSIAN = 0, /* uint32 [max_records]: Gaussian of each record */
    GS_BUF_REC_CAMERA = 1,   /* uint16 [max_records]: camera of each record */
    GS_BUF_REC_RECT = 2,     /* uint32 [max_records][2]: x0|y0<<16, x1|y1<<16 (tiles) */
    GS_BUF_REC_TILES = 3,    /* uint32 [max_records]: tiles touched */
    GS_BUF_REC_DEPTH = 4,    /* uint32 [max_records]: FP32 bits of camera z */
    GS_BUF_REC_XY_CONIC = 5, /* float4 [max_records]: u, v (the floats nearest the projected mean), A, k */
    GS_BUF_REC_C_OPAC_RG = 6,/* float4 [max_records]: D, opacity, r, g */
    GS_BUF_REC_B_LO = 7,     /* float4 [max_records]: b, u_lo, v_lo, 0; the mean is u + u_lo, v + v_lo.
                              * The conic is held as A (x + k y)^2 + D y^2, i.e. k = B / A and
                              * D = C - B^2 / A of the conic (A, B; B, C). */
    GS_BUF_SORTED_VALUES = 8,/* uint32 [max_instances]: record of each sorted instance */
    GS_BUF_TILE_RANGES = 9,  /* uint32 [max_tiles][2]: [start, end) of each tile */
    GS_BUF_N_CONTRIB = 10    /* uint32 [max_pixels]: last composited entry + 1 */
} gs_buffer_id;

void gs_default_params(gs_render_params *p);
const char *gs_last_error(void);
/* Number of CUDA kernels this library has launched in this process (all
 * workspaces, all threads); for launch accounting in benchmarks. */
int64_t gs_kernel_launches(void);

/* Creates a workspace on the current CUDA device.  cap: host pointer. */
int gs_workspace_create(const gs_capacity *cap, gs_workspace **out);
int gs_workspace_destroy(gs_workspace *ws);
/* Bytes of device memory a workspace with these capacities holds. */
int64_t gs_workspace_bytes(const gs_capacity *cap);
/* Execution tuning that leaves every result unchanged: keys ranked per block
 * by the radix passes of gs_bin_sort and gs_importance, 1024, 2048 or 4096;
 * 0 (the default) picks by the size of each sort (1024 up to 2^18 keys of
 * capacity, 2048 up to 2^20, 4096 above).  Applies to the calls made after it. */
int gs_workspace_set_sort_chunk(gs_workspace *ws, int32_t keys_per_block);

/* View gate, projection and colour of every Gaussian for each of n_cams
 * cameras (host array, <= GS_MAX_CAMERAS).  cull: device bit array
 * [n_cams][ceil(n/32)], bit i%32 of word i/32 set = Gaussian i culled in that
 * view (Eq. 3); may be NULL when params->cull_enable == 0.  The Gaussian
 * arrays must stay unchanged until gs_render_bwd of the same step.
 * Equivalent to gs_upload_cameras followed by gs_preprocess_uploaded. */
int gs_preprocess(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams, int32_t n_cams,
                  const uint32_t *cull, const gs_render_params *params, gs_stream stream);

/* The two halves of gs_preprocess, for CUDA graphs.  gs_upload_cameras
 * validates the cameras (host array), lays out their tiles (params->tile_w,
 * tile_h) and pixels, and copies the table to the workspace's device copy on
 * the stream; it must not be called while the stream is being captured
 * (GS_ERR_INVALID_ARG).  Every later kernel reads the cameras from that device
 * copy, so a graph that captured gs_preprocess_uploaded and the calls after
 * it renders whatever cameras were uploaded before its launch, provided they
 * have the widths and heights (hence the tiles and pixels) of the cameras
 * uploaded when it was captured.  gs_preprocess_uploaded takes the render
 * parameters of this pass; their tile shape and fov_clamp must be those of
 * the upload. */
int gs_upload_cameras(gs_workspace *ws, const gs_camera *cams, int32_t n_cams, const gs_render_params *params,
                      gs_stream stream);
int gs_preprocess_uploaded(gs_workspace *ws, const gs_gaussians *g, const uint32_t *cull,
                           const gs_render_params *params, gs_stream stream);

/* Tile keys, device radix sort by (camera, tile, depth, record), tile ranges. */
int gs_bin_sort(gs_workspace *ws, gs_stream stream);

/* Front-to-back compositing.  rgb_out: [sum over cameras of 3*H*W], camera c's
 * planar [3][H][W] image at offset 3 * (pixels of cameras < c).  T_out: final
 * transmittance [sum of H*W], same camera order; may be NULL. */
int gs_render_fwd(gs_workspace *ws, float *rgb_out, float *T_out, gs_stream stream);

/* gs_render_fwd and the importance sweep's raster in one walk of the lists:
 * the image, T_final and n_contrib of gs_render_fwd, and each record's w and a
 * (the raster and per-record sums of gs_importance, Sec. 3.2), bit for bit
 * both.  With GS_CULL_MARK the image skips the marked records while the
 * scores take every record.  The next gs_importance on the same binning then
 * only selects (it skips its raster); a gs_preprocess or gs_bin_sort clears
 * this.  The scores survive gs_render_bwd of the same binning. */
int gs_render_fwd_importance(gs_workspace *ws, float *rgb_out, float *T_out, gs_stream stream);

/* Adjoint of preprocess + compositing for dL_drgb (layout of rgb_out).
 * g must be the arrays given to gs_preprocess.  grads: written (accumulate=0,
 * every Gaussian, zeros where no record) or added to (accumulate=1).
 * absgrad: [n], += |dL/d(u,v)| per record (densification statistic); may be
 * NULL.  scale_reg_beta > 0 adds beta * mean over visible Gaussians of the
 * smallest scale (Eq. 5) to the loss; its value goes to *scale_reg_value
 * (device float, may be NULL). */
int gs_render_bwd(gs_workspace *ws, const gs_gaussians *g, const float *dL_drgb, const gs_gaussian_grads *grads,
                  int32_t accumulate, float *absgrad, float scale_reg_beta, float *scale_reg_value,
                  gs_stream stream);

/* Backward into the workspace: as gs_render_bwd, but each Gaussian's 59
 * parameter gradients (mean, log-scale, quat, opacity, SH, in that order) are
 * kept as one compact row in the workspace, only for Gaussians with a record;
 * nothing is written for the others.  Consumed by gs_adam_step_compact. */
int gs_render_bwd_compact(gs_workspace *ws, const gs_gaussians *g, const float *dL_drgb, float *absgrad,
                          float scale_reg_beta, float *scale_reg_value, gs_stream stream);

/* One Adam step (Kingma and Ba, bias-corrected; step counts from 1) of every
 * Gaussian with the gradients of the last gs_render_bwd_compact: Gaussians
 * without a record take a zero-gradient step.  The arrays of g are UPDATED in
 * place (the const of gs_gaussians does not apply here); m and v are the first
 * and second moments in the layout of g; lr: learning rates of mean,
 * log-scale, quat, opacity and SH.  One streaming pass reads and writes the
 * parameters and both moments (24 bytes per parameter) and never a dense
 * gradient array.  step >= 1 is the step number (and sets the workspace's
 * device step counter); step == 0 takes one past the device counter and
 * advances it, so a captured optimizer step counts on every graph replay. */
int gs_adam_step_compact(gs_workspace *ws, const gs_gaussians *g, const gs_gaussian_grads *m,
                         const gs_gaussian_grads *v, const float lr[5], float beta1, float beta2, float eps,
                         int32_t step, gs_stream stream);

/* Deferred zero-gradient Adam steps.  Dense Adam moves every parameter every
 * step, also those of Gaussians without a gradient.  Once enabled, a
 * Gaussian's parameters and moments are kept as of the step in last_step[i]
 * and brought up to date only when it is next used -- by gs_preprocess (its
 * candidates), by gs_adam_step_compact (before its next gradient step) or by
 * gs_adam_flush -- by replaying exactly the zero-gradient steps it missed, so
 * every value equals dense Adam's bit for bit.  Parameters read by anything
 * else (the caller, the model-level calls, a checkpoint) must be flushed
 * first.  gs_preprocess then UPDATES the Gaussian arrays it is given.
 *   m, v: the moments gs_adam_step_compact will be given (same arrays);
 *   last_step: [n] int32, set by the caller to the current step (0 before the
 *     first step) when enabling; drift: [2][n] float, zeroed by the caller (per
 *     Gaussian, bounds on how far its mean and its largest log-scale can still
 *     move, which widen the view gate);
 *   max_steps: steps the workspace keeps coefficients for (40 bytes each);
 *   every moment array 16-byte aligned (as the parameter arrays);
 *   needs beta1 < sqrt(beta2).  Allocates the step history (once, here). */
int gs_adam_lazy_enable(gs_workspace *ws, const gs_gaussian_grads *m, const gs_gaussian_grads *v, int32_t *last_step,
                        float *drift, float beta1, float beta2, float eps, int32_t max_steps);
int gs_adam_lazy_disable(gs_workspace *ws);
/* Brings every Gaussian up to the current step (no-op when not enabled). */
int gs_adam_flush(gs_workspace *ws, const gs_gaussians *g, gs_stream stream);

/* gs_render_bwd_compact followed by gs_adam_step_compact: the backward fused
 * with the optimizer step, no gradient array materialised. */
int gs_render_bwd_adam(gs_workspace *ws, const gs_gaussians *g, const float *dL_drgb, const gs_gaussian_grads *m,
                       const gs_gaussian_grads *v, const float lr[5], float beta1, float beta2, float eps,
                       int32_t step, float *absgrad, float scale_reg_beta, float *scale_reg_value, gs_stream stream);

/* Instrumented colourless sweep over the binned cameras (Sec. 3.2, Fig. 2).
 * Per camera v and Gaussian i: w[v][i] = sum over composited pixels of alpha T,
 * a[v][i] = number of those pixels (w, a: [n_cams][n], written, may be NULL).
 * Accumulated over views (+=): s_accum[i] += w/(a + eps) when a > 0,
 * crad_accum[i] += 1 when the Gaussian has a record (in frustum, radius > 0),
 * cvis_accum[i] += 1 when w lies in the view's top vis_mass of w mass.
 * cull_out: [n_cams][ceil(n/32)] written, bit = 1 - c^vis.  Any of the
 * accumulators may be NULL.
 * Concurrency: gs_importance reads only the binning and the records, and its
 * scratch (importance slots, selection sort and scans) is its own, so it may
 * run on a second stream, ordered after gs_bin_sort by an event, while
 * gs_render_fwd, gs_photometric_loss, gs_render_bwd(_compact),
 * gs_adam_step(_compact) and gs_render_bwd_adam run on the first.  The next
 * gs_preprocess, gs_bin_sort or gs_render_fwd_importance on the workspace
 * must be ordered after it, and cull_out must not be read meanwhile. */
int gs_importance(gs_workspace *ws, float *w, uint32_t *a, float *s_accum, uint32_t *crad_accum,
                  uint32_t *cvis_accum, uint32_t *cull_out, gs_stream stream);

/* Eq. 4 over a batch of planar images [batch][3][H][W]:
 * loss = mean_b (1 - lambda) mean|I - I*| + lambda (1 - SSIM(I, I*)), SSIM with
 * an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2, zero padding.
 * Writes *loss_out (device float) and dL_dimage (same layout).  Uses the
 * workspace's scratch (max_pixels must cover batch * H * W). */
int gs_photometric_loss(gs_workspace *ws, const float *image, const float *target, int32_t batch, int32_t height,
                        int32_t width, float lambda, float *loss_out, float *dL_dimage, gs_stream stream);

/* One Adam step (Kingma and Ba, bias-corrected) over n_groups (host array,
 * <= GS_MAX_ADAM_GROUPS) parameter groups; step counts from 1. */
int gs_adam_step(const gs_adam_group *groups, int32_t n_groups, int32_t step, gs_stream stream);

/* ---- model level (Sec. 3.2 simplification passes, density control with the
 * Sec. 3.3 LOD inheritance).  These calls need a workspace created with
 * GS_CAP_MODEL_OPS and n <= max_gaussians. */

/* A whole model: parameters in the rows of gs_gaussians plus the Adam moments
 * (rows of the same shapes; members of m and v may be NULL, then they are not
 * carried, or read as zero) and the LOD labels (NULL: all level 0). */
typedef struct {
    int64_t n;
    float *mean;
    float *log_scale;
    float *quat;
    float *opacity_logit;
    float *sh;
    uint8_t *lod;
    gs_gaussian_grads m;
    gs_gaussian_grads v;
} gs_model;

/* Pass 1 of Sec. 3.2: keeps k of n Gaussians by importance-weighted sampling
 * without replacement (probability proportional to s at every draw), drawn as
 * exponential clocks: Gaussian i fires at expo[i] / s[i], expo[i] ~ Exp(1)
 * supplied by the caller, and the k earliest are kept (equal times by lower
 * index; s = 0 fires after every s > 0).  keep_bits: [ceil(n/32)] written. */
int gs_prune_sample(gs_workspace *ws, const float *s, const float *expo, int64_t n, int64_t k, uint32_t *keep_bits,
                    gs_stream stream);

/* Pass 2 of Sec. 3.2: keeps the smallest prefix of Gaussians by descending s
 * (equal s by lower index) whose summed s reaches mass (0.99) of the total;
 * s = 0 is never kept.  The prefix sums are FP64 in a fixed association. */
int gs_prune_mass(gs_workspace *ws, const float *s, int64_t n, float mass, uint32_t *keep_bits, gs_stream stream);

/* Order-preserving compaction: the rows of src whose keep bit is set, written
 * to dst (capacity dst_capacity rows; its n is ignored); *n_out (device
 * int64) receives the count.  src and dst must not overlap. */
int gs_compact(gs_workspace *ws, const gs_model *src, const uint32_t *keep_bits, gs_model *dst, int64_t dst_capacity,
               int64_t *n_out, gs_stream stream);

/* Density control (standard 3DGS clone / split) with the phi reweighting of
 * Sec. 3.2: a Gaussian is selected when (absgrad / denom) * cvis / (crad + eps)
 * >= grad_threshold (absgrad: summed |dL/d(u,v)| of its records, as
 * gs_render_bwd accumulates it; denom: views with a record, see
 * gs_count_views; cvis, crad: gs_importance's accumulators).  Output, in
 * parent order: a Gaussian with opacity < min_opacity is removed; an
 * unselected one is kept; a selected one whose largest scale is <= dense_scale
 * is kept and followed by a copy; a larger one is replaced by two children
 * mu + R(q) (s * z_c), log-scale - log(split_shrink), the other parameters
 * copied, LOD level + 1 (capped at n_levels - 1) -- the inheritance rule of
 * Sec. 3.3 (a clone keeps its parent's level).  noise: [n][2][3] N(0,1)
 * samples z_c, supplied by the caller.  Kept and cloned parents keep their
 * Adam moments, new Gaussians start from zero.  dst needs up to 2n rows. */
typedef struct {
    float grad_threshold;
    float dense_scale;
    float min_opacity;
    float split_shrink; /* 1.6 */
    float eps;          /* 1e-6 */
    int32_t n_levels;   /* LOD labels 0..n_levels-1 */
} gs_densify_params;
int gs_densify(gs_workspace *ws, const gs_model *src, const float *absgrad, const uint32_t *denom,
               const uint32_t *cvis, const uint32_t *crad, const float *noise, const gs_densify_params *params,
               gs_model *dst, int64_t dst_capacity, int64_t *n_out, gs_stream stream);

/* counts[i] += number of cameras of the last gs_preprocess in which Gaussian i
 * has a record not marked culled (the densification denominator of a training
 * step). */
int gs_count_views(gs_workspace *ws, uint32_t *counts, gs_stream stream);

/* The Cull column of one view (the selection step of gs_importance) without
 * any allocation and without a workspace.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory -- code
 * where a cudaMalloc is forbidden or would stall other work (it can
 * synchronise the device), such as a latency-critical serving thread, a host
 * callback or a plugin whose memory belongs to another allocator.
 *   w        [n] device: the view's per-Gaussian alpha-weights (gs_importance's w)
 *   cull_out [ceil(n/32)] device, written: bit = 1 - c^vis (top vis_mass of the w mass)
 *   cvis_accum [n] device, += 1 where visible; may be NULL
 *   error_out [1] device, may be NULL: written with the call's device error,
 *            a gs_status cast to uint32_t (0 = GS_OK; GS_ERR_TIMEOUT if a
 *            bounded wait of the sort gave up, and then every Gaussian is
 *            left culled)
 * The selection is gs_importance's own (the same stable sort and exact
 * fixed-point prefix sums), so the column equals gs_importance's bit for bit.
 * n <= 2^20: the scratch (about 24.6 MB) is one fixed device array of the
 * library, which every GPU that loads its module keeps until the process
 * exits; larger n is rejected with GS_ERR_CAPACITY.  The first call on a
 * device looks the array's device address up (cudaGetSymbolAddress, with that
 * device current), so make that first call before any stream capture.  All
 * calls share the array: calls whose work overlaps on the GPU race and must be
 * serialised by the caller.  Asynchronous on stream. */
int gs_visible_set_static(const float *w, int64_t n, float vis_mass, uint32_t *cull_out, uint32_t *cvis_accum,
                          uint32_t *error_out, gs_stream stream);

/* Measured throughput of the arithmetic pipes the compositing kernels are
 * bound by, for roofline fractions.  The paper has no counterpart: this is a
 * measurement utility.  Runs three short kernels (FP32 FMA chains, the same
 * as packed FP32x2 FMA, and ex2.approx) on every SM of the current device,
 * times each with CUDA events on `stream` and synchronises with it.
 *   fp32_fma_flops    FLOP/s of scalar FFMA (2 per FMA)
 *   fp32x2_fma_flops  FLOP/s of packed FP32x2 FMA (4 per instruction)
 *   ex2_per_s         ex2.approx results per second (special-function unit)
 *   sms               the device's multiprocessor count */
typedef struct {
    double fp32_fma_flops;
    double fp32x2_fma_flops;
    double ex2_per_s;
    int32_t sms;
} gs_alu_peak;
int gs_alu_peaks(gs_alu_peak *out, gs_stream stream);

/* Bound on the waits of gs_importance's selection sorts: each wait of a
 * block on its predecessors in a sort pass gives up after `spins` polls
 * (0 restores the default, 2^22) and sets GS_ERR_TIMEOUT (reported by
 * gs_sync_status).  The sort's output order is then wrong but every write
 * stays inside its buffers, and the selection's later kernels skip their
 * work, so the Cull column comes out with every Gaussian culled.  The next
 * call after gs_clear_error runs normally.  Host-side setting, read when a
 * call is issued (a captured graph keeps the value it was captured with).
 * The paper has no counterpart: it exists so that the bounded waits can be
 * exercised. */
int gs_workspace_set_spin_limit(gs_workspace *ws, uint64_t spins);

/* Kernel timing, for measurement.  While on, each launch of the timed kernels
 * below is bracketed by a CUDA event pair recorded on the stream it is launched
 * on; a launch issued under stream capture gets a pair of event nodes in the
 * graph, which each replay records again (so they hold the last replay's
 * time).  Turning timing on discards earlier records; the first 64 launches of
 * each kernel are recorded.  gs_kernel_time synchronises those events and
 * returns the summed device time (ms) and the number of timed launches of one
 * kernel (of a captured launch: after at least one replay).  Off by default.
 * gs_kernel_timing's `kernels` selects what is timed: 0 turns timing off,
 * otherwise a mask of (1 << GS_KT_*) bits (GS_KT_ALL: every kernel); each
 * event pair between kernels of a captured graph costs the launch overlap of
 * programmatic dependent launch there, so time only what is read.
 * The events belong to the workspace (created on first use, destroyed with
 * it), so a captured graph stays valid while timing is turned off and on; the
 * pairs are numbered again from the first each time timing is turned on. */
enum {
    GS_KT_RENDER_FWD = 0,      /* gs_render_fwd's compositing kernel */
    GS_KT_RENDER_BWD = 1,      /* the compositing adjoint (per (record, tile) slots) */
    GS_KT_IMPORTANCE = 2,      /* the importance sweep's rasteriser */
    GS_KT_GATE = 3,            /* the view gate's pass over every Gaussian (gs_preprocess) */
    GS_KT_PROJECT = 4,         /* the projection of the gate's candidates (gs_preprocess) */
    GS_KT_BIN_COUNT = 5,       /* gs_bin_sort: each record's first instance and the tile counts */
    GS_KT_BIN_SORT = 6,        /* gs_bin_sort: tile ranges, scatter by tile and the per-tile depth sort */
    GS_KT_REDUCE_SLOTS = 7,    /* the per-record sum of the adjoint's gradient slots */
    GS_KT_PREPROCESS_BWD = 8,  /* the projection adjoint (per Gaussian) */
    GS_KT_SSIM_FWD = 9,        /* gs_photometric_loss: the SSIM statistics and coefficient maps */
    GS_KT_SSIM_BWD = 10,       /* gs_photometric_loss: the gradient from the coefficient maps */
    GS_KT_ADAM_GRAD = 11,      /* the deferred Adam's step of the Gaussians with records */
    GS_KT_COUNT = 12,
    GS_KT_ALL = (1 << 12) - 1 /* mask of every timed kernel */
};
int gs_kernel_timing(gs_workspace *ws, int32_t kernels);
int gs_kernel_time(gs_workspace *ws, int32_t kernel, double *total_ms, int64_t *launches);

/* CUDA graph of a sequence of calls, with per-kernel priorities.
 * gs_graph_capture_begin starts a thread-local capture on stream (not the
 * legacy NULL stream); the calls that follow on it, and on streams that join it
 * through events, are recorded, not run.  gs_graph_capture_end ends the capture
 * (every joined stream must have been joined back), instantiates the graph and
 * returns it in *out (host handle owned by the caller; NULL on error).  Every
 * kernel of this library carries the priority of the stream it was launched
 * on, and the graph runs each kernel at that priority whatever stream it is
 * launched into: a step captured on a high-priority stream, with a side sweep
 * on a low-priority stream, keeps the side sweep out of the critical path's
 * way.  gs_graph_launch enqueues one run on stream; gs_graph_destroy frees the
 * graph (NULL is ignored) once its runs have completed. */
typedef struct gs_graph gs_graph;
int gs_graph_capture_begin(gs_stream stream);
int gs_graph_capture_end(gs_stream stream, gs_graph **out);
int gs_graph_launch(gs_graph *graph, gs_stream stream);
int gs_graph_destroy(gs_graph *graph);

/* Synchronises the stream and returns the device error word as a status. */
int gs_sync_status(gs_workspace *ws, gs_stream stream);
/* Synchronises the stream and reads the counters (host pointer out). */
int gs_workspace_counts(gs_workspace *ws, gs_counts *out, gs_stream stream);
/* Clears the device error word. */
int gs_clear_error(gs_workspace *ws, gs_stream stream);
/* Device pointer and element capacity of an internal buffer. */
int gs_workspace_buffer(gs_workspace *ws, int32_t which, void **ptr, int64_t *count);

#ifdef __cplusplus
}
#endif
#endif /* GSBLITZ_H */
