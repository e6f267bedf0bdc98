/*
 * gsr.h -- C ABI of libgsr, a differentiable tile-based Gaussian-splatting
 * rasterizer for sm_103a (GB300).
 *
 * What it computes: the renderer that the per-keyframe optimisation of
 * "On-the-fly Large-scale 3D Reconstruction from Multi-Camera Rigs" runs every
 * iteration (Sec. 3.3, "Optimization": Gaussian parameters and camera
 * parameters are updated jointly; SH gradients are detached for the camera
 * update; Table 3 attributes 113.3 of 185 ms per keyframe to it).  The paper
 * uses the 3D Gaussian Splatting renderer it cites without restating it; the
 * operations below are that renderer:
 *
 *   preprocess   EWA projection of each (view, Gaussian) to a 2D conic,
 *                SH -> RGB, opacity, screen radius and tile rectangle;
 *   sort         (view, tile, depth) 64-bit keys, ties by Gaussian index;
 *   ranges       [start, end) of each tile's list;
 *   blend        per pixel, front to back: alpha = min(0.99, sigma exp(P)),
 *                entries with alpha < 1/255 skipped, stop before the entry
 *                that would take the transmittance below 1e-4;
 *   backward     exact adjoint (decisions frozen) to the Gaussian parameters
 *                and the per-view se(3) pose (left perturbation
 *                V <- exp(delta^) V, delta = (rho, omega)), with the SH
 *                viewing direction held constant for the pose.
 *
 * Every discrete decision is taken in binary32 with a documented operation
 * order (explicitly rounded multiply/add/divide/sqrt and fused multiply-add);
 * the exponentials are the library's own binary32 routines.
 *
 * Conventions.  All pointers to per-Gaussian and per-pixel arrays are DEVICE
 * pointers owned by the caller; the structs themselves and the view matrices
 * live in HOST memory.  Views follow OpenCV axes (x right, y down, z forward);
 * viewmat is the row-major 4x4 world-to-camera matrix [R | t].  Output images
 * of all views are concatenated: view v starts at pixel offset
 * P_v = sum_{w<v} W_w H_w; rgb is planar per view ([3][H][W] at 3 P_v),
 * depth/alpha are [H][W] at P_v.  Depth is not normalised (divide by alpha
 * for the expected depth).  Background bg is added to rgb only.
 *
 * Errors.  Every function returns a gsr_status; nothing aborts or throws
 * across the ABI.  On error, gsr_last_error() describes it.  Device-side
 * failures (a bounded wait that ran out, an internal capacity overflow) are
 * reported through a status word the library reads back after the work.
 *
 * Threading.  A gsr_ctx is not thread-safe; use one per host thread.  All
 * device work is enqueued on the caller's stream.
 */
#ifndef GSR_H
#define GSR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GSR_API __attribute__((visibility("default")))
#else
#define GSR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int gsr_status;
#define GSR_OK                 0
#define GSR_ERR_INVALID_ARG    1   /* bad pointer, size, view or config       */
#define GSR_ERR_CAPACITY       2   /* internal buffers were too small and the
                                      call ran with GSR_FLAG_NO_SYNC: grow with
                                      gsr_reserve() and call again            */
#define GSR_ERR_CUDA           3   /* a CUDA runtime call failed              */
#define GSR_ERR_TIMEOUT        4   /* a bounded device wait ran out           */
#define GSR_ERR_NOT_SUPPORTED  5   /* e.g. more than GSR_MAX_VIEWS views      */
#define GSR_ERR_OUT_OF_MEMORY  6

#define GSR_MAX_VIEWS 64

/* config.flags */
#define GSR_FLAG_NO_SYNC 1u  /* never synchronise the stream inside a call:
                                capacity overflows are then reported by
                                gsr_check() instead of being retried (needed
                                for CUDA-graph capture)                       */
#define GSR_FLAG_PROFILE 2u  /* record CUDA events between the phases of
                                every call; read with gsr_get_stats()         */
#define GSR_FLAG_NO_PAIR_COUNTS 4u  /* the forward blend skips its per-pixel
                                pair counters: fwd_pairs and blended_pairs of
                                gsr_saved_info read 0 after such a forward
                                (images, lists and gradients are unchanged)  */

/* phases timed under GSR_FLAG_PROFILE */
#define GSR_PHASE_PREPROCESS     0
#define GSR_PHASE_DEPTH_SORT     1
#define GSR_PHASE_DUPLICATE      2
#define GSR_PHASE_TILE_SORT      3
#define GSR_PHASE_RANGES         4
#define GSR_PHASE_BLEND_FWD      5
#define GSR_PHASE_BWD_CLEAR      6
#define GSR_PHASE_BLEND_BWD      7
#define GSR_PHASE_PREPROCESS_BWD 8
#define GSR_NUM_PHASES           9

typedef struct gsr_ctx gsr_ctx;
typedef struct gsr_saved gsr_saved;

typedef struct {
    int tile_w, tile_h;   /* screen tile: 16x16, 32x8 or 8x32                 */
    int blend_batch;      /* Gaussians staged in shared memory per batch:
                             128, 256 or 512                                  */
    int sh_degree;        /* 0 .. 3                                           */
    float near_plane;     /* records with camera z <= near are culled (0.2)   */
    float bg[3];          /* background colour                                */
    uint32_t flags;       /* GSR_FLAG_*                                       */
    int blend_batch_bwd;  /* Gaussians staged per batch by the backward blend:
                             0 (the forward's blend_batch), 128 (default),
                             256 or 512                                       */
    float list_prefix;    /* how the forward builds the tile lists:
                             >= 1 (default): one round, every tile's full
                             list;
                             f in (0, 1): two rounds.  The first lists only
                             the first ceil(f V) of the V visible records in
                             depth order -- a prefix of every tile's list --
                             and renders with them; a tile all of whose
                             pixels stop within its prefix is final (the
                             rest of its list is never read), the others are
                             listed in full and rendered again by the second
                             round.  Images, contributor counts and gradients
                             are those of one round; only the lists of the
                             tiles finished in the first round end early;
                             0: two rounds with f chosen from the saturation
                             statistics of the last forward that synchronised
                             (one round until there is one).  Two rounds need
                             twice the list memory.                          */
} gsr_config;

typedef struct {
    int64_t n;                    /* number of Gaussians                     */
    const float* means;           /* [n][3] world position                    */
    const float* log_scales;      /* [n][3] log of the axis scales            */
    const float* quats;           /* [n][4] (w, x, y, z), need not be unit    */
    const float* opacity_logits;  /* [n]    opacity = sigmoid(logit)          */
    const float* sh;              /* [n][(D+1)^2][3] SH coefficients          */
} gsr_gaussians;

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;         /* pinhole intrinsics in pixels             */
    float viewmat[16];            /* row-major world-to-camera, host memory   */
    const uint32_t* subset;       /* device: strictly ascending Gaussian
                                     indices rendered by this view, or NULL
                                     for all n                                */
    int64_t subset_count;         /* entries in subset (ignored if NULL)     */
} gsr_view;

typedef struct {
    float* rgb;     /* device [sum 3 W H]  */
    float* depth;   /* device [sum W H]    */
    float* alpha;   /* device [sum W H]    */
} gsr_outputs;

typedef struct {
    /* device, same shapes as gsr_gaussians; overwritten (not accumulated)   */
    float* means;
    float* log_scales;
    float* quats;
    float* opacity_logits;
    float* sh;
    float* pose;    /* device [n_views][6] = (d rho, d omega), or NULL        */
    float* focal;   /* device [n_views][2] = (dL/dfx, dL/dfy), or NULL        */
} gsr_grads;

/* Counters and sizes of the last forward that filled a gsr_saved. */
typedef struct {
    int64_t n_records;      /* sum over views of the Gaussians considered     */
    int64_t n_visible;      /* records that survived culling                  */
    int64_t n_instances;    /* M = (record, tile) instances in the sorted
                               lists: the tiles of each record's 3-sigma
                               rectangle that some pixel centre of can reach
                               alpha >= 1/255 (tile culling)                 */
    int64_t n_tiles;        /* sum over views of the tile-grid sizes          */
    int64_t n_pixels;       /* sum over views of W H                          */
    int64_t fwd_pairs;      /* (pixel, entry) pairs examined by the forward   */
    int64_t bwd_pairs;      /* sum of per-pixel contributor counts            */
    int tile_w, tile_h, blend_batch;
    int64_t blended_pairs;  /* (pixel, entry) pairs actually composited       */
    int64_t warp_entries_fwd; /* (32-pixel warp, entry) iterations left after
                                 culling, forward / last backward           */
    int64_t warp_entries_bwd;
    int64_t n_instances_full; /* tiles of the 3-sigma rectangles before culling */
    int64_t grad_rows;      /* (Gaussian, view group) gradient rows the last
                               backward wrote: the Gaussians with a visible
                               record, once per group of views sharing a subset */
    float list_prefix;      /* the first round's record fraction of the
                               forward (1: one round)                         */
    int64_t n_instances_second; /* of n_instances, those of the second round  */
    int64_t open_tiles;     /* tiles the first round left to the second        */
    int64_t list_span;      /* list positions used: n_instances for one round;
                               for two, the second region's start plus its
                               instances (the ranges index this space)        */
} gsr_saved_info;

/* Library statistics.  launches counts the kernels libgsr has launched in
 * this process.  phase_ms[p] is the total device time of phase p over the
 * profiled calls since the previous gsr_get_stats, calls[p] their number. */
typedef struct {
    int64_t launches;
    double phase_ms[GSR_NUM_PHASES];
    int64_t calls[GSR_NUM_PHASES];
} gsr_stats;

/* Fill *cfg with the defaults: 16x16 tiles, batch 256, SH degree 3,
 * near 0.2, black background, no flags. */
GSR_API void gsr_config_default(gsr_config* cfg);

/* Create a context (workspace owner) for the current CUDA device.  *out is
 * NULL on failure.  The context allocates device memory lazily, on the
 * first call that needs it, and grows it when a call needs more. */
GSR_API gsr_status gsr_create(gsr_ctx** out, const gsr_config* cfg);
GSR_API void gsr_destroy(gsr_ctx* ctx);
GSR_API const char* gsr_last_error(const gsr_ctx* ctx);

/* Replace the configuration (tile shape, batch, SH degree, ...).  Saved
 * states filled under the old configuration stay valid for their backward. */
GSR_API gsr_status gsr_set_config(gsr_ctx* ctx, const gsr_config* cfg);
GSR_API gsr_status gsr_get_config(const gsr_ctx* ctx, gsr_config* cfg);

/* A saved state holds what one forward leaves for its backward: projected
 * records, the sorted tile lists and ranges, per-pixel final transmittance
 * and contributor counts.  Owned by the caller, tied to its context. */
GSR_API gsr_status gsr_saved_create(gsr_ctx* ctx, gsr_saved** out);
GSR_API void gsr_saved_destroy(gsr_saved* saved);
GSR_API gsr_status gsr_saved_get_info(const gsr_saved* saved, gsr_saved_info* info);

/* Pre-size the internal buffers for a batch: visible records and tile
 * instances (after tile culling; the rectangle instances before culling are
 * sized at four times that).  Optional; calls grow buffers by themselves
 * unless GSR_FLAG_NO_SYNC is set, and gsr_check grows them after a
 * GSR_ERR_CAPACITY. */
GSR_API gsr_status gsr_reserve(gsr_ctx* ctx, gsr_saved* saved, int64_t visible, int64_t instances);

/* Forward: render n_views views (1 .. GSR_MAX_VIEWS) of the Gaussians.
 * All views go through one preprocess launch (Gaussian-major within runs of
 * consecutive views sharing a subset), one sort and one persistent blend
 * launch over every (view, tile).  stream is a cudaStream_t (NULL = legacy
 * default stream).  Unless GSR_FLAG_NO_SYNC is set, the call waits for the
 * stream once at the end to read the status word, and if an internal buffer
 * was too small it grows it and runs again. */
GSR_API gsr_status gsr_forward(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_view* views, int n_views,
                       const gsr_outputs* out, gsr_saved* saved, void* stream);

/* Backward of the forward that filled `saved` (same g and views).
 * dl_drgb is required; dl_ddepth and dl_dalpha may be NULL (zero).  All
 * gradients in *grads are overwritten.  Parameter gradients sum over views;
 * pose gradients are per view.  The clearing of *grads runs on a stream of
 * the context, forked from `stream` after its queued work and joined back
 * before the gradients are written (events recorded in stream order, so the
 * call can be captured into a CUDA graph); to the caller, all work is
 * ordered on `stream`. */
GSR_API gsr_status gsr_backward(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_view* views, int n_views,
                        gsr_saved* saved, const float* dl_drgb, const float* dl_ddepth,
                        const float* dl_dalpha, const gsr_grads* grads, void* stream);

/* Wait for the stream and report the status word of the calls enqueued on
 * `saved` since the last check (GSR_ERR_CAPACITY, GSR_ERR_TIMEOUT or OK). */
GSR_API gsr_status gsr_check(gsr_ctx* ctx, gsr_saved* saved, void* stream);

/* Insertion probability and scale initialisation of new Gaussians
 * (Sec. 3.2, Eq. 4-6), for a batch of views:
 *   P(I) = min(|| LoG_sigma * I ||, 1) per pixel (Euclidean norm of the three
 *   colour channels' responses), P_a = max(P(I) - P(I~), 0) for the ground
 *   truth I and the rendering I~; a Gaussian is inserted where P_a > tau_a,
 *   with scale S = d / (2 sqrt(P(I)) f), d the caller's distance map and f the
 *   view's fx.
 * The LoG is sampled at integer offsets within ceil(3 sigma), shifted to zero
 * mean; image edges are clamped.  The decision P_a > tau_a is taken in
 * binary32 with a fixed order (see gsr_insert.cu).
 * Layout (device arrays, views concatenated in order, as gsr_outputs):
 *   gt, rendered  [sum_v 3 W_v H_v] float, planar RGB per view
 *   depth, p_a, scale  [sum_v W_v H_v] float (scale 0 where nothing is inserted)
 *   index  [index_cap] uint32: the concatenated pixel indices of the inserted
 *          pixels, ascending (the first index_cap of them); may be NULL if
 *          count is NULL
 *   count  one uint64 (device): the number of inserted pixels; NULL skips the
 *          index list
 * Only views[v].width, height and fx are read.  Asynchronous on stream;
 * GSR_ERR_NOT_SUPPORTED if sigma is outside (0, 7/3]. */
typedef struct {
    float sigma;   /* LoG standard deviation in pixels (default 1)              */
    float tau_a;   /* insertion threshold (default 0.2, the paper's tau_a)      */
} gsr_insert_params;

GSR_API void gsr_insert_params_default(gsr_insert_params* params);
GSR_API gsr_status gsr_insertion(gsr_ctx* ctx, const gsr_insert_params* params, const gsr_view* views, int n_views,
                                 const float* gt, const float* rendered, const float* depth, float* p_a,
                                 float* scale, uint32_t* index, int64_t index_cap, unsigned long long* count,
                                 void* stream);

/* Rig chain (Sec. 3.1): gradients of a multi-camera rig's parameters from
 * the per-view ones gsr_backward wrote.  View i's world-to-camera pose is
 * V_i = A_i V_m(k): A_i = [R_i | t_i] the fixed transform from the central
 * camera of keyframe k = keyframe_of_view[i] to camera i, V_m(k) that central
 * camera's pose (for camera-to-world poses this is T_i = T_m T_(i->m)).  With
 * the left-perturbation convention of gsr_grads.pose,
 *   central[k]      = sum over views i of keyframe k of
 *                     (R_i^T g_rho_i, R_i^T (g_omega_i - t_i x g_rho_i))
 *   camera_rel[c]   = sum over views i of rig camera c = camera_of_view[i]
 *                     of g_i: the gradient of A_c under the left
 *                     perturbation A_c <- exp(delta^) A_c (Sec. 3.3 optimises
 *                     the relative transforms of the non-central cameras)
 *   camera_focal[c] = sum over views i of rig camera c of (dL/dfx_i, dL/dfy_i)
 * Sums are taken in binary64 in ascending view order and rounded once.
 *   pose_grads      device [n_views][6] float (gsr_grads.pose)
 *   focal_grads     device [n_views][2] float (gsr_grads.focal); may be NULL
 *                   with camera_focal
 *   keyframe_of_view, camera_of_view  host [n_views] int32 in [0, n_keyframes)
 *                   and [0, n_cameras); camera_of_view may be NULL when
 *                   camera_rel and camera_focal are
 *   rel             host [n_views][12] float, row-major [R_i | t_i] (3 x 4)
 *   central         device [n_keyframes][6] float, overwritten; may be NULL
 *   camera_rel      device [n_cameras][6] float, overwritten; may be NULL
 *   camera_focal    device [n_cameras][2] float, overwritten; may be NULL
 * The host tables are copied into the launch before the call returns.
 * n_views, n_keyframes, n_cameras <= GSR_MAX_VIEWS (GSR_ERR_NOT_SUPPORTED
 * beyond), an index out of range is GSR_ERR_INVALID_ARG.  Asynchronous on
 * stream. */
GSR_API gsr_status gsr_rig_chain(gsr_ctx* ctx, int n_views, const float* pose_grads, const float* focal_grads,
                                 const int32_t* keyframe_of_view, const int32_t* camera_of_view, const float* rel,
                                 int n_keyframes, int n_cameras, float* central, float* camera_rel,
                                 float* camera_focal, void* stream);

/* Inter-camera Gaussian merging (Sec. 3.2, Eq. 7-8) for camera i of a rig.
 * The Gaussians built from cameras 0 .. i-1 ("existing") are reprojected into
 * camera i and each is paired with the sampled pixel (from gsr_insertion)
 * that contains its projected mean, when |z' - d_i| <= tau_d (z' its camera
 * depth, d_i the depth map there).  Each sampled pixel whose group is not
 * empty keeps one primitive, the one of smallest image-space scale
 * S f / depth (S: an existing Gaussian's largest scale, or the sample's
 * Eq. 6 scale; f = fx), ties to the existing Gaussian of lowest index; the
 * kept primitive takes the mean SH DC colour of the group (a sample's own
 * colour is its ground-truth pixel), and a kept sample moves to the group's
 * mean depth with its scale following the depth.  Pairing, the depth gate and
 * the choice are taken in binary32 with a fixed order (see gsr_merge.cu).
 * Inputs (device): means, log_scales [n_existing][3]; sh: the DC of Gaussian g
 * at sh + g * sh_stride (sh_stride = 3 (D+1)^2 for gsr_gaussians.sh);
 * sample_pixels [n_samples] pixel indices (y W + x) of camera i, distinct
 * (an index >= W H gets sample_action -1 and no other output);
 * scale_map, depth_map [H][W]; gt [3][H][W].  Only the view's width, height,
 * intrinsics and viewmat are read.  Outputs in gsr_merge_outputs (device;
 * sample_action required, the others may be NULL).  n_existing < 2^31.
 * Asynchronous on stream; the workspace belongs to the context. */
typedef struct {
    float tau_d;        /* depth gate in metres (default 0.5; the paper gives no value) */
    float near_plane;   /* existing Gaussians at camera depth <= near_plane are not
                           reprojected (default 0.2)                                   */
} gsr_merge_params;

#define GSR_MERGE_INSERT    0   /* sample: no group; insert it as it is              */
#define GSR_MERGE_MERGED    1   /* sample: dropped, an existing Gaussian is kept     */
#define GSR_MERGE_REPLACES  2   /* sample: kept, its group's Gaussians are removed   */
#define GSR_MERGE_UNTOUCHED 0   /* existing: not paired                              */
#define GSR_MERGE_REMOVED   1   /* existing: dropped from its group                  */
#define GSR_MERGE_KEPT      2   /* existing: kept, with the group's mean colour      */
typedef struct {
    int32_t* sample_action;    /* [n_samples] GSR_MERGE_INSERT / MERGED / REPLACES        */
    float* sample_means;       /* [n_samples][3] world position at sample_depth           */
    float* sample_scale;       /* [n_samples] Eq. 6 scale at sample_depth                  */
    float* sample_depth;       /* [n_samples] camera depth (group mean for REPLACES)       */
    float* sample_dc;          /* [n_samples][3] SH DC (group mean for REPLACES)           */
    int32_t* existing_action;  /* [n_existing] GSR_MERGE_UNTOUCHED / REMOVED / KEPT        */
    float* existing_dc;        /* [n_existing][3] the group's mean SH DC, written for the
                                  KEPT rows only (the others are left as they are)        */
} gsr_merge_outputs;

GSR_API void gsr_merge_params_default(gsr_merge_params* params);
GSR_API gsr_status gsr_merge(gsr_ctx* ctx, const gsr_merge_params* params, const gsr_view* view,
                             int64_t n_existing, const float* means, const float* log_scales, const float* sh,
                             int64_t sh_stride, int64_t n_samples, const uint32_t* sample_pixels,
                             const float* scale_map, const float* depth_map, const float* gt,
                             const gsr_merge_outputs* out, void* stream);

/* Frequency-based scheduling (Sec. 3.3, Eq. 9-12).
 *
 * gsr_dft_energy: for each image, X(I) = sum over all frequencies (i, j) of
 * the Euclidean norm over the three colour channels of the unnormalised 2-D
 * DFT of each channel (Eq. 10, 11).  An image with factor n > 1 is first
 * box-downsampled: the transformed image is floor(height/n) x floor(width/n),
 * each pixel the mean of an n x n block (the level-n ground truth I^n of
 * Eq. 12).  FP32 transform, FP64 sums, one float per image into x (device
 * [n_images]).  Sizes after downsampling up to GSR_DFT_MAX_DIM in each
 * direction (GSR_ERR_NOT_SUPPORTED beyond); an empty image gives 0.  The
 * first use of a transform length builds its twiddle table (a synchronous
 * upload: make that first call outside stream capture).  Asynchronous on
 * stream otherwise; the workspace (half spectra, at most 512 MB or one
 * image's) belongs to the context, so calls on one context must not overlap.
 *
 * gsr_frequency_schedule: per frame f (device arrays of n_frames floats)
 *   r_f       = x_gt_f / x_rendered_f        (Eq. 9, binary32)
 *   r_level_f = x_gt_level_f / x_rendered_f  (Eq. 12, binary32)
 *   level_up_f = r_level_f < tau_f (1 or 0; 0 for NaN): raise the
 *               ground-truth resolution by one level
 * and n_samples frames drawn with probability proportional to r: weights
 * r_f (NaN -> 0, capped at 1e30; all 1 if none is positive), cumulative sums
 * c_f in frame order in binary32, sample s = the first f with
 * c_f > uniforms[s] * c_last (binary32), else the last frame of positive
 * weight; uniforms are the caller's draws in [0, 1).  x_gt_level, r_level
 * and level_up may be NULL together; r and samples may be NULL (samples
 * with uniforms).  n_frames in [1, GSR_SCHED_MAX_FRAMES].  Asynchronous. */
#define GSR_DFT_MAX_DIM      4096
#define GSR_SCHED_MAX_FRAMES 4096
typedef struct {
    const float* data;   /* device, planar RGB [3][height][width]              */
    int width, height;   /* of data                                            */
    int factor;          /* box-downsampling factor n >= 1 before the DFT      */
} gsr_image;

GSR_API gsr_status gsr_dft_energy(gsr_ctx* ctx, const gsr_image* images, int n_images, float* x, void* stream);
GSR_API gsr_status gsr_frequency_schedule(gsr_ctx* ctx, int n_frames, const float* x_gt, const float* x_gt_level,
                                          const float* x_rendered, float tau_f, const float* uniforms,
                                          int n_samples, float* r, float* r_level, int32_t* level_up,
                                          int32_t* samples, void* stream);

/* L1 photometric loss helper: loss = mean |rgb - target| over all n values,
 * dl_drgb = sign(rgb - target) / n.  loss_out (device, one float) may be
 * NULL.  rgb, target, dl_drgb are device arrays of n floats. */
GSR_API gsr_status gsr_l1_loss_grad(const float* rgb, const float* target, int64_t n, float* dl_drgb,
                            float* loss_out, void* stream);

/* Autotuner: time forward+backward for every tile shape in
 * {16x16, 32x8, 8x32} x blend batch in {128, 256, 512} on this batch (with
 * the given upstream gradient), then the backward's own batch
 * (blend_batch_bwd) for the fastest, keep the fastest in the context's
 * configuration and return it in *best (may be NULL).  Results are cached
 * per batch signature (view sizes, subset sizes, SH degree). */
GSR_API gsr_status gsr_tune(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_view* views, int n_views,
                    const gsr_outputs* out, gsr_saved* saved, const float* dl_drgb,
                    const gsr_grads* grads, gsr_config* best, void* stream);

/* Parity exports (copies into caller device buffers, enqueued on stream).
 *  keys     [S] uint64 (global tile << 32 | float bits of camera z),
 *  vals     [S] uint32 record index in view-major numbering
 *           (sum_{w<v} count_w + position in view v's subset),
 *  ranges   [n_tiles][2] uint32 [start, end), (0, 0) for an empty tile,
 * with S = gsr_saved_info.list_span list positions (M = n_instances after a
 * one-round forward).  After a two-round forward the positions between the
 * first region's instances and the second region's start hold keys 0 and
 * vals 0xffffffff; each tile's range lies in one region.
 * Any pointer may be NULL. */
GSR_API gsr_status gsr_debug_lists(gsr_saved* saved, uint64_t* keys, uint32_t* vals, uint32_t* ranges,
                           void* stream);

/* Positions [first, first + count) of the sorted list (same encoding as
 * gsr_debug_lists), e.g. one tile's range; count is clipped to the list. */
GSR_API gsr_status gsr_debug_list_slice(gsr_saved* saved, int64_t first, int64_t count, uint64_t* keys,
                                        uint32_t* vals, void* stream);

/* Per-record export in view-major numbering, for the n_records records:
 *  rec    [n_records][16] float: u, v, qa, qb, qc, sigma, z, (pad), r, g, b,
 *         (pad x 5) where (qa, qb, qc) = -log2(e) (c0/2, c1, c2/2) for the
 *         conic (c0, c1, c2); zero for culled records;
 *  rect   [n_records][4] int32 tile rectangle x0, y0, x1, y1 (0 if culled);
 *  flags  [n_records] uint32: bit0 culled.  Any pointer may be NULL. */
GSR_API gsr_status gsr_debug_records(gsr_saved* saved, float* rec, int32_t* rect, uint32_t* flags, void* stream);

/* Per-pixel saved state: T_final [n_pixels] float, n_contrib [n_pixels]
 * uint32 (list position of the last blended entry + 1). */
GSR_API gsr_status gsr_debug_pixels(gsr_saved* saved, float* t_final, uint32_t* n_contrib, void* stream);

/* Per-record 2D gradients of the last backward on `saved`, view-major:
 * [n_records][12] = du, dv, dqa, dqb, dqc, dsigma, dz, (pad), dr, dg, db, (pad). */
GSR_API gsr_status gsr_debug_record_grads(gsr_saved* saved, float* grec, void* stream);

/* Device-wait limit and a test-only fault of the look-back (failure
 * detection, tested without a GPU fault).  Every device-side wait of the
 * context's later calls (mbarrier waits on bulk copies, decoupled look-back
 * spins) gives up after wait_ns nanoseconds (0 = the default, 2 s), sets the
 * timeout bit of the call's status word and lets its kernel finish; every
 * kernel after it in the call then skips its work, and the call (or
 * gsr_check) returns GSR_ERR_TIMEOUT.  flags: 0, or GSR_DEBUG_WITHHOLD_PREFIX:
 * in the forward's preprocess, the first block of the single-pass scan over
 * the visible records never publishes its prefix, so every later block's wait
 * runs out (for tests of the timeout path; the forward then returns
 * GSR_ERR_TIMEOUT).  Unknown flags: GSR_ERR_INVALID_ARG.  Takes effect from
 * the next call; not for concurrent use with calls on the same context. */
#define GSR_DEBUG_WITHHOLD_PREFIX 1u
GSR_API gsr_status gsr_debug_set_wait(gsr_ctx* ctx, uint64_t wait_ns, uint32_t flags);

/* The automatic list mode's rule (list_prefix 0), a host computation exposed
 * so that it can be checked without a GPU.  A forward that synchronises
 * records two histograms over the share x of its V visible records taken in
 * depth order, in GSR_LIST_BUCKETS buckets with edges gsr_list_bucket_edge(b)
 * (geometric, 2^-12 for b = 0 up to 1 for b = GSR_LIST_BUCKETS):
 *   sat_hist[GSR_LIST_BUCKETS + 1]: list lengths of the tiles by the share
 *     of the records they needed before every pixel stopped, the last entry
 *     for tiles that never saturated;
 *   inst_hist[GSR_LIST_BUCKETS]: kept instances by their record's share.
 * Returns the first-round fraction the next forwards use: an edge in (0, 1),
 * 1 for one round, or -1 when inst_hist is empty (no measurement: the mode
 * keeps its previous choice).  The cost model is stated in gsr_api.cu. */
#define GSR_LIST_BUCKETS 64
GSR_API float gsr_list_prefix_choice(const uint64_t* sat_hist, const uint64_t* inst_hist, uint64_t visible);
GSR_API double gsr_list_bucket_edge(int b);

/* Allocation-free forward render.  The paper has no counterpart to this; it
 * is for callers that cannot allocate device memory while they render: a
 * process that reserves its whole device budget up front, or code running
 * where cudaMalloc is not permitted.  It computes the same rgb, depth and
 * alpha images as gsr_forward for the same configuration, but keeps no saved
 * state (there is no backward for it) and needs no context: its workspace is
 * a fixed array of GSR_NOALLOC_SCRATCH_BYTES compiled into libgsr, which every
 * GPU that loads the library holds until the process exits.
 *   - The first call on each device looks up that array's device address (with
 *     the device current); make that first call before any stream capture.
 *   - Batches beyond the limits below are rejected with GSR_ERR_NOT_SUPPORTED
 *     before any device work.  The instance count is only known on the
 *     device: if it exceeds GSR_NOALLOC_MAX_INSTANCES the call returns
 *     GSR_ERR_CAPACITY and the images are incomplete.
 *   - The call waits for `stream` at its end to read the status word.
 *   - All calls share the array and it keeps the last call's contents; the
 *     call clears what must start at zero.  Calls whose work overlaps on the
 *     GPU (other streams, other host threads) race on it: serialise them.
 * Of cfg.flags only GSR_FLAG_NO_PAIR_COUNTS applies; cfg.list_prefix is
 * ignored (the lists are built in one round).  Nothing is allocated, on the
 * device or through any allocating library routine. */
#define GSR_NOALLOC_MAX_RECORDS   65536     /* sum over views of the Gaussians considered */
#define GSR_NOALLOC_MAX_INSTANCES 524288    /* (Gaussian, tile) instances after tile
                                               culling; the 3-sigma rectangles
                                               before it may hold 8x as many   */
#define GSR_NOALLOC_MAX_PIXELS    524288    /* sum over views of width x height      */
#define GSR_NOALLOC_MAX_TILES     8192      /* sum over views of the tile-grid sizes */
#define GSR_NOALLOC_SCRATCH_BYTES (20u << 20)
GSR_API gsr_status gsr_forward_noalloc(const gsr_config* cfg, const gsr_gaussians* g, const gsr_view* views,
                                       int n_views, const gsr_outputs* out, void* stream);

/* Read (and reset) the statistics; waits for the profiled calls' events. */
GSR_API gsr_status gsr_get_stats(gsr_ctx* ctx, gsr_stats* stats);

/* Library version string. */
GSR_API const char* gsr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GSR_H */
