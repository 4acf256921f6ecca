/*
 * gs.h -- C ABI of the GB300 (sm_103a) hot path of On-the-Fly GS (arxiv 2503.13086).
 *
 * On every Local & Semi-Global iteration (Sec. IV-C) the paper optimises a 3D Gaussian
 * Splatting field (Sec. III, Eq. 1-2) with the original 3DGS rasterizer (Sec. V-A), an
 * L1 + D-SSIM loss (Eq. 10), a splatting-parallel backward (Sec. IV-D) and Adam whose position
 * learning rate is the per-image rate of Eq. 6-8.  Each arriving image first extends the field
 * (Sec. IV-B) and is scheduled by hierarchical image weighting (Eq. 3-4) and the iteration
 * allocation of Eq. 5.
 *
 * Two layers:
 *   gs_raster_*  stateless rasterizer calls on caller-owned device buffers (forward, loss,
 *                backward, Adam) for parity checks and autograd wrappers;
 *   gs_field_* / gs_add_image / gs_select_neighbors / gs_optimize_step / gs_integrate /
 *                gs_render  a session that keeps the field, its Adam state and the registered
 *                images resident on the device.
 *
 * Conventions
 *   - Every call returns gs_status; on failure gs_last_error() gives a thread-local message.
 *     No call aborts the process.  GS_ERR_TIMEOUT means a bounded device-side wait gave up; the
 *     context stays usable and the affected outputs are unspecified.
 *   - "device" pointers are CUDA device addresses on the current device, "host" pointers are
 *     ordinary (preferably pinned) host memory.  The caller owns every pointer it passes; the
 *     library copies what it keeps before the call returns (host data) or before work queued on
 *     the stream after the call runs (device data).
 *   - Stream arguments are cudaStream_t passed as void* (NULL = legacy default stream).  Device
 *     work is asynchronous on that stream unless a call returns a host value, in which case the
 *     call synchronises the stream.
 *   - Gaussian parameters are fp32, component-major with a row stride (a multiple of 32):
 *       params[c * stride + i], i < n <= stride,
 *       c = 0..2 mean (x, y, z), 3..5 log-scale, 6..9 quaternion (w, x, y, z, any norm > 0),
 *       10 opacity logit, 11 + 3 k + ch SH coefficient k = 0..15 of colour channel ch = 0..2.
 *   - Images are fp32 planar 3 x H x W (CHW), values nominally in [0, 1].  Several views are
 *     packed back to back in view order.  Per-pixel buffers are H x W per view, packed likewise.
 *   - Pixel (px, py) is sampled at the continuous image point (px, py); u = fx x/z + cx.
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

#define GS_NUM_PARAMS 59
#define GS_TILE 16

typedef enum gs_status {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1, /* a pointer, size or id is out of range */
  GS_ERR_OOM = 2,         /* a device or pinned allocation failed */
  GS_ERR_BUDGET = 3,      /* the call would exceed the field's hbm_budget_bytes */
  GS_ERR_CAPACITY = 4,    /* a fixed capacity (views per step, image count) is exceeded */
  GS_ERR_CUDA = 5,        /* a CUDA runtime call or kernel launch failed */
  GS_ERR_TIMEOUT = 6,     /* a bounded device-side wait expired */
  GS_ERR_STATE = 7,       /* call out of order (e.g. backward without a forward) */
  GS_ERR_IO = 8,          /* a file could not be written or read, or is not a saved field */
  GS_ERR_INTERNAL = 9     /* a consistency check failed: a device buffer was written past its end */
} gs_status;

/* Pinhole camera.  R is the row-major world->camera rotation and t the translation
 * (x_cam = R x_world + t, OpenCV axes: +z forward, +y down).  fx, fy, cx, cy in pixels. */
typedef struct gs_camera {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
} gs_camera;

/* Thread-local description of the last failure of this thread (never NULL). */
GS_API const char* gs_last_error(void);

/* Library version string. */
GS_API const char* gs_version(void);

/* ----------------------------------------------------------------------------------------
 * Stateless rasterizer (Sec. III Eq. 1-2; Sec. IV-D; Eq. 10).
 * A gs_raster owns only workspaces (projection records, sorted lists, backward checkpoints);
 * gs_raster_backward differentiates the most recent gs_raster_forward of the same object.
 * One gs_raster must not be used from two streams at once.
 * ---------------------------------------------------------------------------------------- */
typedef struct gs_raster gs_raster;

GS_API gs_status gs_raster_create(gs_raster** out);
GS_API gs_status gs_raster_destroy(gs_raster* r);

/* K1-K6 for n_views cameras (host array, n_views <= 32).  Writes, per view packed back to back:
 *   out_image (device, 3 H W floats per view): sum_i c_i alpha_i T_i + T_final bg,
 *   out_T     (device, H W floats, nullable): final transmittance,
 *   out_last  (device, H W uint32): 1 + index in the tile list of the last Gaussian blended,
 *   out_gp    (device, H W uint32, nullable): number of Gaussians blended into the pixel (G_p of
 *             Eq. 9).
 * out_pairs (host, nullable) receives the Gaussian-pixel pairs evaluated: per pixel, the list
 * entries visited up to and including the one that stopped it.  Synchronises the stream once
 * to size the instance buffers. */
GS_API gs_status gs_raster_forward(gs_raster* r, void* stream, const float* params, int64_t n, int64_t stride,
                            const gs_camera* cams, int n_views, const float bg[3], float* out_image,
                            float* out_T, uint32_t* out_last, uint32_t* out_gp, uint64_t* out_pairs);

/* Weights of the loss terms of Eq. 10: lambda_l1 L1 + lambda_ssim D-SSIM + lambda_load L_load. */
typedef struct gs_loss_weights {
  float lambda_l1, lambda_ssim, lambda_load;
} gs_loss_weights;

/* K7 on the views of the last forward (Eq. 10): L = mean over views of
 * lambda_l1 mean|X - Y| + lambda_ssim (1 - mean SSIM(X, Y)) (11x11 Gaussian window, sigma 1.5,
 * zero padding, C1 = 0.01^2, C2 = 0.03^2, means over 3 H W), plus lambda_load L_load when that weight
 * is > 0.  w (host, nullable; NULL = 3DGS's 0.8 / 0.2 / 0) must hold weights >= 0
 * (GS_ERR_INVALID_ARG otherwise).  image/target (device) are packed like out_image.  out_dimage
 * (device, nullable) receives dL/dimage.  out_loss (host, nullable) receives L and synchronises.
 * May be called again on the same forward (e.g. with other weights). */
GS_API gs_status gs_raster_loss(gs_raster* r, void* stream, const float* image, const float* target,
                                const gs_loss_weights* w, float* out_dimage, double* out_loss);

/* K8 + K9: gradients of a scalar loss with respect to the parameters of the last forward,
 * given dL/dimage (device, packed like out_image).  image and last are the forward's outputs.
 * With a load weight > 0 in the last gs_raster_loss, the gradient of lambda_load L_load (Eq. 9,
 * through the soft count, see gs_field_config) is added; that needs the forward's out_gp
 * (GS_ERR_STATE without it).
 * out_grads (device, 59 x stride, row stride = stride) is overwritten for i < n.  out_grad2d
 * (device, nullable, 9 floats per record, record = view * stride + i) receives per view the 2D
 * gradient (d mean2d x, y; d conic a, b, c; d opacity; d rgb).  May be called again on the same
 * forward (another dL/dimage). */
GS_API gs_status gs_raster_backward(gs_raster* r, void* stream, const float* params, const float* image,
                             const uint32_t* last, const float* dimage, float* out_grads, float* out_grad2d);

/* K10: Adam (torch.optim.Adam's bias-corrected update) over 59 x stride device arrays.
 * lr[6] per parameter group: 0 mean, 1 log-scale, 2 quaternion, 3 opacity, 4 SH DC, 5 SH rest.
 * step >= 1 is the step count used for bias correction. */
GS_API gs_status gs_adam_step(void* stream, float* params, const float* grads, float* m, float* v, int64_t n,
                       int64_t stride, const float lr[6], float beta1, float beta2, float eps, int64_t step);

/* Copy a workspace buffer of the last forward to host memory (parity checks).  which:
 *   0 mean  (float4 per record: u, v, ex, ey: the 1/255 cutoff box half extents)
 *   1 conic (float4: -a/2, -b, -c/2, -ln(255 opacity))
 *   2 rgb   (float4: r, g, b, opacity)              3 depth (float)
 *   4 radius (int32)                                5 rect (uint32 x2: x0|x1<<16, y0|y1<<16)
 *   6 count (uint32 tiles touched)                  7 offsets (uint32)
 *   8 keys  (uint64, sorted, m_total of them)       9 values (uint32 record index, sorted)
 *  10 ranges (uint32 x2 per global tile)           11 clamp bits (uint8)
 *  12 instance gradients of the last backward (float x12 per instance, emission order)
 * Records are view * stride + i for the forward's views.  *out_bytes gets the size; with
 * host_dst == NULL only the size is returned.  Synchronises the raster's stream. */
GS_API gs_status gs_raster_read(gs_raster* r, int which, void* host_dst, size_t capacity_bytes, size_t* out_bytes);

/* Per-kernel device time (ms) of the raster's last forward + loss + backward when timing is on:
 * [0] K1 project, [1] K2 scan, [2] K3 emit, [3] K4 sort, [4] K5 ranges, [5] K6 blend forward,
 * [6] K7 loss, [7] K8 blend backward, [8] K9(+K10) project backward. */
GS_API gs_status gs_raster_set_timing(gs_raster* r, int enable);
GS_API gs_status gs_raster_kernel_times(gs_raster* r, float out_ms[9]);

/* Tile shape and blend batch.  The paper renders with the 3DGS tile binning (Sec. III, Sec. V-A)
 * and states no tile size; 3DGS uses 16 x 16.  tile_w x tile_h is the tile of the rect rule
 * ([floor((u - r)/tile_w), floor((u + r + tile_w - 1)/tile_w)), same for y) and of the blend
 * CTA (one thread per pixel), so it decides which Gaussians enter a pixel's list: a Gaussian whose
 * 1/255 footprint reaches past its 3-sigma square can enter or miss a pixel depending on the grid,
 * so the tile shape is part of the result (the oracle takes the same shape).  batch is the
 * number of sorted Gaussians the forward stages in shared memory per round; it does not change
 * any result.  gs_tiling_candidates lists the compiled combinations (out may be NULL to query
 * the count; the first one, 16 x 16 with batch 256, is the default); any other combination is
 * GS_ERR_INVALID_ARG.  gs_raster_set_tiling applies to the raster's next forward. */
typedef struct gs_tiling {
  int32_t tile_w, tile_h, batch;
} gs_tiling;
GS_API gs_status gs_tiling_candidates(gs_tiling* out, int32_t capacity, int32_t* out_n);
GS_API gs_status gs_raster_set_tiling(gs_raster* r, const gs_tiling* t);

/* ----------------------------------------------------------------------------------------
 * Session: the field, its Adam state and the registered images stay on the device.
 * ---------------------------------------------------------------------------------------- */
typedef struct gs_field gs_field;

typedef struct gs_field_config {
  int32_t T_I;              /* iterations per arriving image (paper: 200) */
  int32_t N_m;              /* key images incl. the new one (paper: 10) */
  int32_t T_a;              /* iterations for an image to be "trained" (Eq. 7; paper: 200) */
  int32_t batch_views;      /* views per optimisation step in gs_integrate (1 = per-view) */
  int32_t use_graph;        /* replay each step from a captured CUDA graph */
  int32_t async_steps;      /* gs_integrate enqueues up to this many steps between host syncs (1 = sync each) */
  float eta0, etaf;         /* Eq. 6 initial / final position rate (1.6e-4, 1.6e-6) */
  float lambda_ssim;        /* D-SSIM weight (0.2) */
  float lr_scale, lr_rot, lr_opacity, lr_sh_dc, lr_sh_rest; /* other Adam groups (3DGS) */
  float beta1, beta2, adam_eps;
  float add_dist_thresh;    /* new-point distance test threshold; <= 0: 0.01 x scene extent */
  float scene_extent;       /* position-rate scale; <= 0: 1.1 x camera spread (at least 1) */
  float bg[3];
  uint64_t seed;            /* semi-global selection and slot order (SplitMix64) */
  uint64_t hbm_budget_bytes;/* 0 = unlimited */
  int64_t initial_capacity; /* Gaussians */
  gs_tiling tiling;         /* all zero: autotuned per class of view set (gs_field_autotune); else fixed */
  int32_t batch_scaling;    /* steps over B > 1 views: 0 = mean of their Eq. 8 rates, Adam as configured;
                               1 = also lr x sqrt(B) and betas ^ B (the large-batch rule of Zhao et al.
                               2024 for 3DGS), which keeps per-view progress with B x fewer steps */
  float lambda_l1;          /* Eq. 10 L1 weight; -1 = 1 - lambda_ssim (3DGS: 0.8) */
  float lambda_load;        /* Eq. 10 weight of L_load (Eq. 9, std of G_p over the N pixels some Gaussian
                               reaches, all views of the step).  The loss takes the count G_p; the
                               gradient takes the count's derivative through the soft count, the sum
                               of the alphas of the pixel's blended Gaussians, times
                               dL_load/dG_p = (G_p - mean) / (N std).  The paper's preset:
                               lambda_l1 0.47, lambda_ssim 0.12, lambda_load 0.41.  Default 0. */
  int32_t densify_stats;    /* 1: every step accumulates the statistics gs_field_densify uses */
  int32_t sparse_adam;      /* 1: a step's Adam updates only the Gaussians with instances in one of
                               its views (later 3DGS releases' sparse Adam; bias correction by the
                               field's step count); 0 (default): all, as the original dense Adam */
  int32_t debug_canaries;   /* 1: after every run of steps, check the guard words behind every device
                               buffer of the field (256 bytes of 0xA5 each, written when the buffer
                               is allocated and never by a kernel) and fail with GS_ERR_INTERNAL,
                               naming the buffer, if one changed.  Synchronises once per run of
                               steps.  0 (default): off */
} gs_field_config;

/* Paper defaults (Sec. V-A, implementation details): T_I 200, N_m 10, T_a 200, eta 1.6e-4 -> 1.6e-6;
 * batch 1; loss weights 0.8 L1 + 0.2 D-SSIM (3DGS; the paper's 0.47 / 0.12 / 0.41 is a preset);
 * group rates 5e-3 / 1e-3 / 0.05 / 2.5e-3 / 1.25e-4 and Adam (0.9, 0.999, 1e-15) of the original
 * 3DGS ("all other settings"); tiling auto. */
GS_API void gs_field_config_default(gs_field_config* cfg);

/* A new session: the 3DGS field the paper trains while images arrive (Sec. III; the field of
 * Phase 2, Sec. IV-A), empty, with its Adam state and image registry, on `stream` (a
 * cudaStream_t; NULL = a non-blocking stream of the field's own, as graph capture needs one).
 * cfg (host) is copied.  GS_ERR_INVALID_ARG for an invalid configuration (T_I, N_m, T_a,
 * batch_views outside 1..32, non-positive rates, weights < 0, a tiling not among
 * gs_tiling_candidates), GS_ERR_OOM / GS_ERR_BUDGET when initial_capacity cannot be reserved.
 * *out (host) receives the field, owned by the caller until gs_field_destroy. */
GS_API gs_status gs_field_init(const gs_field_config* cfg, void* stream, gs_field** out);
/* Release every device and host resource of the field (waits for its stream); NULL is ignored. */
GS_API gs_status gs_field_destroy(gs_field* f);

/* Replace the field's Gaussians (host, component-major, src_stride >= n); Adam state is
 * zeroed and the Adam step count reset. */
GS_API gs_status gs_field_set_gaussians(gs_field* f, const float* host_params, int64_t n, int64_t src_stride);
/* Copy the field's parameters (and optionally Adam m, v; nullable) to host, dst_stride >= n. */
GS_API gs_status gs_field_get_gaussians(gs_field* f, float* host_params, float* host_m, float* host_v,
                                 int64_t dst_stride, int64_t* out_n);

/* Register an arriving image (Sec. IV-B; the inputs per image of Sec. III: its pose from the SfM,
 * the image and its new sparse points with their matches): pose and intrinsics, the target image
 * rgb_hwc (H x W x 3 interleaved fp32 in [0, 1], the layout image decoders produce; host or device
 * per rgb_on_device; transposed on the device into the planar layout the loss reads; a page-locked
 * host image is read by that layout kernel directly over the host link, other host memory is first
 * copied to a device staging buffer), and its
 * sparse points (host: xyz n_pts x 3, rgb n_pts x 3 in [0, 1], track ids n_pts; any may be NULL when
 * n_pts == 0).  Points farther than add_dist_thresh from every existing sparse point become new
 * Gaussians (3DGS initialisation); track ids (the co-visibility of Sec. IV-C: a track is one
 * sparse point seen by several images) shared with earlier images define the overlap matrix M
 * (shared / min count).  Synchronises the field's stream (the number of new Gaussians is read
 * back), so every host input has been read when it returns.  *out_image_id (host, nullable)
 * receives the image's id (0, 1, ... in arrival order).  GS_ERR_BUDGET when growing the field would
 * exceed hbm_budget_bytes; GS_ERR_CAPACITY beyond 4096 images. */
GS_API gs_status gs_add_image(gs_field* f, const gs_camera* cam, const float* rgb_hwc, int rgb_on_device,
                              const float* pts_xyz, const float* pts_rgb, int32_t n_pts, const int32_t* pt_track_ids,
                              int32_t* out_image_id);
/* The same with the target already planar (3 x H x W), e.g. a render of another field. */
GS_API gs_status gs_add_image_chw(gs_field* f, const gs_camera* cam, const float* rgb_chw, int rgb_on_device,
                                  const float* pts_xyz, const float* pts_rgb, int32_t n_pts,
                                  const int32_t* pt_track_ids, int32_t* out_image_id);

/* Replace a registered image's target (rgb_hwc, H x W x 3 interleaved, nullable) and/or its pose
 * (cam, nullable; same size), e.g. a refined pose (Sec. IV-A, Phase 3).  Asynchronous on the
 * field's stream: a host image in pinned memory is read by the kernel the call enqueues, so it must
 * stay unchanged until the field's next synchronising call (the next gs_optimize_step) returns;
 * pageable host memory is read before the call returns. */
GS_API gs_status gs_set_image(gs_field* f, int32_t image_id, const gs_camera* cam, const float* rgb_hwc,
                              int rgb_on_device);
/* The same with a planar (3 x H x W) target. */
GS_API gs_status gs_set_image_chw(gs_field* f, int32_t image_id, const gs_camera* cam, const float* rgb_chw,
                                  int rgb_on_device);

/* Eq. 3-4: hierarchical weights from image_id over M; returns image_id first, then up to k
 * neighbours by decreasing weight (ties: lower id).  out_ids / out_w hold k + 1 entries. */
GS_API gs_status gs_select_neighbors(gs_field* f, int32_t image_id, int32_t k, int32_t* out_ids, float* out_w,
                              int32_t* out_n);

/* One Local & Semi-Global optimisation iteration (Sec. IV-C; the 3DGS iteration of Sec. III, Eq.
 * 1-2 forward, Eq. 10 loss, the splatting-parallel backward of Sec. IV-D) over n_views registered
 * views (host array of ids, 1..32): render, loss (mean over views), backward, Adam with the
 * position rate = mean over the views of Eq. 8's rate x scene extent; then T_j += 1 for every
 * view (Eq. 7).  One view is the paper's iteration; several are the batched step.  out_loss (host,
 * nullable) receives the loss.  Synchronises the field's stream once (it checks that the step
 * completed: instance buffers that overflowed are grown and the step re-run).  Errors:
 * GS_ERR_INVALID_ARG (bad ids), GS_ERR_CAPACITY (views), GS_ERR_STATE (no Gaussians),
 * GS_ERR_TIMEOUT (a bounded device wait gave up), GS_ERR_CUDA. */
GS_API gs_status gs_optimize_step(gs_field* f, const int32_t* view_ids, int32_t n_views, float* out_loss);

typedef struct gs_integrate_stats {
  int32_t iterations;      /* view-iterations run (T_I) */
  int32_t steps;           /* optimisation steps (iterations / batch_views, rounded up) */
  int32_t key_images;      /* N_m actually selected */
  int32_t new_gaussians;   /* not used by gs_integrate; set by the caller's bookkeeping */
  double mean_loss;        /* mean of the step losses */
  uint64_t pairs;          /* Gaussian-pixel pairs of all steps */
} gs_integrate_stats;

/* Local & Semi-Global optimisation for a new image (Sec. IV-C): Eq. 3-4 weights, Eq. 5
 * allocation of T_I / 2 iterations over the N_m key images, T_I / 2 spread evenly over the
 * other registered images (remainder to a seeded random subset), a seeded slot order, and
 * ceil(T_I / batch_views) calls of the optimisation step. */
GS_API gs_status gs_integrate(gs_field* f, int32_t image_id, gs_integrate_stats* out_stats);

/* Phase 1 of the method (Sec. IV-A, the initial training before images stream in; the paper: the
 * first 30 images, 2000 iterations, "all other settings" of 3DGS): `iterations` view-iterations over
 * the registered images, batch_views per step, each view drawn uniformly from them (SplitMix64
 * seeded with seed ^ 0x5048415345310000, a draw in [0, n) is next() mod n).  The position rate is
 * 3DGS's exponential schedule, exp((1 - u) ln eta0 + u ln etaf) with u = min(step / max_steps, 1)
 * over the phase-1 steps (3DGS: max_steps 30000), times the scene extent; the other groups keep
 * their rates.  T_j counts these iterations (Eq. 7).  out_stats as for gs_integrate.
 * Called after the last arrival it is also the "rapid additional optimisation" of Phase 3
 * (Sec. IV-A) over all registered images; refined poses, where a caller has them, are set first
 * with gs_set_image. */
GS_API gs_status gs_initial_training(gs_field* f, int32_t iterations, int32_t max_steps, gs_integrate_stats* out_stats);

/* Render the field from any camera (the forward of Eq. 1-2 without a loss; Sec. III's output,
 * the trained field, viewed): out_rgb_chw (device, 3 x H x W fp32, written), out_T (device,
 * H x W final transmittance, nullable).  Synchronises the field's stream.  GS_ERR_INVALID_ARG for a
 * NULL or invalid camera, GS_ERR_STATE for an empty field. */
GS_API gs_status gs_render(gs_field* f, const gs_camera* cam, float* out_rgb_chw, float* out_T);

/* The size of the field and the device memory it holds (Sec. III's output is the field; the
 * memory is what admission by HBM budget counts): *n_gaussians and *bytes_in_use (host, each
 * nullable).  Host-only. */
GS_API gs_status gs_field_stats(const gs_field* f, size_t* n_gaussians, size_t* bytes_in_use);

typedef struct gs_field_info {
  int64_t n_gaussians;
  int64_t capacity;
  int64_t n_images;
  int64_t adam_step;
  uint64_t bytes_in_use;   /* device bytes owned by the field (parameters, Adam, images, workspaces) */
  uint64_t last_pairs;     /* Gaussian-pixel pairs evaluated in the last step (per pixel, up to its stop) */
  uint64_t last_blended;   /* Gaussian-pixel pairs blended in the last step (sum of G_p) */
  int64_t last_instances;  /* Gaussian-tile instances of the last step */
  int32_t last_kernels;    /* kernel launches of the last step */
  int32_t pad;
  double last_loss;
  double last_load_std;    /* Eq. 9 L_load of the last step: std of G_p over the pixels with G_p > 0 */
  gs_tiling last_tiling;   /* tile shape and blend batch of the last step */
  int32_t pad2;
  double last_run_ms;      /* device time of the last run of steps: CUDA events on the field's stream before
                              its first and after its last step (its own readback not included) */
  int64_t last_run_steps;  /* steps of that run */
  uint64_t last_h2d_bytes; /* host->device bytes the library staged for that run (step parameters, views) */
  uint64_t last_d2h_bytes; /* device->host bytes it read back after that run (ledger, control block) */
} gs_field_info;
/* Everything gs_field_stats gives and the bookkeeping of the last step (host-only). */
GS_API gs_status gs_field_info_get(const gs_field* f, gs_field_info* out);

/* Per-image bookkeeping: T_j (iterations trained, Eq. 7) and the overlap row M[image, :]. */
GS_API gs_status gs_image_info(const gs_field* f, int32_t image_id, int32_t* out_T, float* out_M_row, int32_t row_len);

/* The schedule of one arrival on the host, with no session and no GPU (planning, tests): for the
 * arriving image new_id, given the overlap matrix M (host, n x n, row-major, M[i][j] in [0, 1]) and
 * the images' iteration counts T (host, n, Eq. 7), the Eq. 3-4 weights, the N_m key images (highest
 * weight first, ties to the lower id), the T_I view slots of Eq. 5 plus the semi-global half in
 * their seeded order (cfg supplies T_I, N_m and seed), and Eq. 8's rate of every image (cfg supplies
 * eta0, etaf and T_a) -- the computation gs_integrate runs for a session.
 *   out_slots  (host, cfg->T_I int32)         the image of each iteration slot; *out_n_slots = T_I
 *   out_keys   (host, cfg->N_m int32, nullable) the key images; *out_n_keys of them
 *   out_w      (host, n float, nullable)       Eq. 3-4 weights (0 for images new_id cannot reach)
 *   out_lr     (host, n float, nullable)       Eq. 8 rates
 * GS_ERR_INVALID_ARG for n < 1, new_id outside [0, n), T_I or N_m < 1, or a NULL required pointer. */
GS_API gs_status gs_schedule_plan(const gs_field_config* cfg, const float* M, const int32_t* T, int32_t n,
                                  int32_t new_id, int32_t* out_slots, int32_t* out_n_slots, int32_t* out_keys,
                                  int32_t* out_n_keys, float* out_w, float* out_lr);

/* The learning rate of Eq. 8 for image_id under the current T_j (diagnostics and tests). */
GS_API gs_status gs_image_lr(const gs_field* f, int32_t image_id, float* out_lr);

/* Device-side checkpoint of the trainable state: parameters, Adam moments and step count, and
 * each image's iteration count T_j.  gs_field_restore returns the field to the last snapshot
 * (Gaussians added since are dropped; registered images are kept).  GS_ERR_STATE if no
 * snapshot exists.  The snapshot lives in device memory owned by the field. */
GS_API gs_status gs_field_snapshot(gs_field* f);
GS_API gs_status gs_field_restore(gs_field* f);

/* Adaptive density control of the original 3DGS (kept among "all other settings" of 3DGS, Sec.
 * V-A; 3DGS Sec. 5.2).  With densify_stats set, every step adds, per Gaussian and per view in
 * which it has instances, the norm of its view-space mean gradient (the pixel-space gradient
 * scaled by (W/2, H/2)) and a count.  gs_field_densify then clones every Gaussian whose mean norm
 * is >= grad_thresh and whose largest scale is <= percent_dense x extent, splits the larger ones
 * into 2 children (mean + R(q) (s * z), z standard normal from a counter-based generator, every
 * log-scale lowered by log 1.6), prunes every result with opacity < min_opacity or largest scale
 * > max_scale x extent, orders the field as kept originals, clones, children, gives the new
 * Gaussians zero Adam moments and clears the statistics.  extent = the configured scene extent
 * (1.1 x camera spread by default).  3DGS's values: 2e-4, 0.01, 0.005, 0.1.  Synchronises. */
typedef struct gs_densify_params {
  float grad_thresh, percent_dense, min_opacity, max_scale;
} gs_densify_params;
typedef struct gs_densify_result {
  int64_t n_before, n_after, cloned, split, pruned;
} gs_densify_result;
GS_API gs_status gs_field_densify(gs_field* f, const gs_densify_params* p, gs_densify_result* out);
/* The accumulated statistics (host arrays of n floats each; either may be NULL). */
GS_API gs_status gs_field_densify_stats(gs_field* f, float* host_norm_sum, float* host_count);

/* Host-side fault injection for the guard-word check (debug_canaries): overwrites one guard word
 * behind the index-th allocated device buffer of the session (0 .. buffers - 1, a fixed order over
 * the session's, its images' and its rasterizer's buffers) with 0, as a kernel writing past that
 * buffer's end would.  The write lies inside the allocation.  out_name (host, name_cap bytes,
 * nullable) receives the buffer's name.  The next run of steps with debug_canaries set fails with
 * GS_ERR_INTERNAL naming it; the guard stays changed (the session is for testing only afterwards).
 * Synchronous. */
GS_API gs_status gs_field_corrupt_guard(gs_field* f, int32_t index, char* out_name, int32_t name_cap);

/* Checkpoint / resume of a whole session in a file (the paper keeps the field and optimiser state
 * of a session; Sec. IV).  gs_field_save writes the configuration, the Gaussians with their Adam
 * moments and step count, every registered image (camera, pixels, sparse-point tracks, T_j), the
 * overlap matrix, the sparse points of the field update and the densification statistics and
 * round count; it synchronises the field's stream.
 * gs_field_load creates a new field from such a file on `stream` (NULL: a stream of its own); a
 * session resumed from a file continues exactly as the saved one would (with a fixed tiling: bit
 * for bit).  Not saved: the snapshot of gs_field_snapshot, timing state, autotuned tilings.
 * Errors: GS_ERR_IO (file, format), GS_ERR_OOM / GS_ERR_BUDGET as for the calls that build a
 * field. */
GS_API gs_status gs_field_save(gs_field* f, const char* path);
GS_API gs_status gs_field_load(const char* path, void* stream, gs_field** out);

/* Enable per-kernel timing on the field's steps; gs_field_kernel_times returns the summed
 * device ms per kernel (same order as gs_raster_kernel_times) and the number of steps. */
GS_API gs_status gs_field_set_timing(gs_field* f, int enable);
GS_API gs_status gs_field_kernel_times(gs_field* f, float out_ms[9], int64_t* out_steps);

/* Autotuner of the tile shape and blend batch (the paper gives none; see gs_tiling).  Times every
 * compiled candidate on the field's current state and the given views (host array, 1..32 image
 * ids): one sizing pass, one warm-up, then `reps` (>= 1) back-to-back runs of a whole step --
 * projection, scan, key emission, sort, ranges, blend forward, loss, blend backward and the
 * projection backward -- except that the projection backward writes nothing (no Adam update,
 * which costs the same for every tiling), so the field's parameters, moments and T_j are
 * unchanged.  The
 * fastest candidate (best device time per run) becomes the tiling of every later step whose view
 * set falls in the same class -- same device, same power of two of the total pixels -- in every
 * session of the process whose configured tiling is auto (all zero); a session with a fixed
 * tiling keeps it.  With an auto tiling, gs_optimize_step / gs_integrate run this (reps = 3) on
 * the first step of a class no session has tuned yet, so results then depend on the timings; fix
 * the tiling for runs that must be reproducible bit for bit.  Synchronises the field's stream.
 * gs_autotune_clear forgets every class (thread-safe).  out (host, nullable):
 * the choice, and per candidate its tiling and ms (INFINITY if it could not run, e.g. out of
 * the HBM budget). */
#define GS_MAX_TILINGS 16
typedef struct gs_autotune_result {
  gs_tiling chosen;
  int32_t n_candidates;
  gs_tiling candidates[GS_MAX_TILINGS];
  float ms[GS_MAX_TILINGS];
} gs_autotune_result;
GS_API gs_status gs_field_autotune(gs_field* f, const int32_t* view_ids, int32_t n_views, int32_t reps,
                                   gs_autotune_result* out);
GS_API gs_status gs_autotune_clear(void);

/* ----------------------------------------------------------------------------------------
 * Failure detection of the device-side waits.  The paper has no counterpart.
 * ---------------------------------------------------------------------------------------- */

/* The two inter-CTA waits of a step (the decoupled look-back of the K2 scan and of each K4 sort
 * pass) spin a bounded number of times; a wait that gives up sets an error bit in the step's
 * control block and its CTA finishes its work with the prefix it has, so the kernel returns and the
 * context stays usable, and the step reports GS_ERR_TIMEOUT.  This call runs each wait once on a
 * two-tile problem by a single CTA that holds the second tile: the first tile is never started,
 * so the wait can only end by giving up.
 *   spin_limit  rounds of the look-back before giving up; 0 = the limit the steps use
 *   out_error   (host, 2 uint32) error bits of the scan's and the sort pass's run; bit 0 (value 1)
 *               set = the wait gave up
 *   out_ms      (host, 2 float, nullable) device time of each run
 * Synchronous.  Allocates about 0.3 MB of device memory and frees it before returning.
 * Returns GS_OK when both runs completed (whatever they report), GS_ERR_CUDA otherwise. */
GS_API gs_status gs_wait_probe(uint32_t spin_limit, uint32_t out_error[2], float out_ms[2]);

/* The loss forward that follows the blend forward in a step starts each block once the tiles under
 * its window are flagged complete, and its last CTA once every blend-forward warp has counted its
 * pair and G_p totals; both waits poll a bounded number of times, and one that gives up sets the
 * same error bit (the step reports GS_ERR_TIMEOUT) and lets the kernel finish.  This call runs the
 * loss forward once on a one-block 32 x 48 view whose tiles are never flagged and whose forward
 * warps never count themselves, so both waits can only end by giving up.
 *   spin_limit  polls of each wait before giving up; 0 = the limit the steps use
 *   out_error   (host, 1 uint32) the run's error bits; bit 0 (value 1) set = a wait gave up
 *   out_ms      (host, 1 float, nullable) device time of the run
 * Synchronous.  Allocates about 90 KB of device memory and frees it before returning.  Returns
 * GS_OK when the run completed (whatever it reports), GS_ERR_CUDA otherwise. */
GS_API gs_status gs_loss_wait_probe(uint32_t spin_limit, uint32_t* out_error, float* out_ms);

/* ----------------------------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart: this is a deployment variant.
 * ---------------------------------------------------------------------------------------- */

/* Exclusive prefix sum of n uint32 tile counts (the scan K2 runs inside gs_raster_forward),
 * for callers that cannot allocate device memory: code running while another component owns the
 * device allocator, or on a path where an allocation's implicit synchronisation is not allowed.
 * It calls no cudaMalloc, cudaFree or allocating library routine; its scratch is a 65 KiB array
 * in the library's own device memory, which every GPU that loads the library keeps until exit.
 *   counts      (device, n uint32, 16-byte aligned)          input
 *   out_offsets (device, n uint32, 16-byte aligned)          out_offsets[i] = sum of counts[0..i)
 *   out_total   (device, one uint64, nullable)               sum of all counts (UINT64_MAX: see below)
 * n may be 0 .. 2^24 (GS_ERR_CAPACITY beyond); the sum must fit in 32 bits for the offsets.
 * Asynchronous on stream.  The first call on a device also looks up the scratch array's device
 * address; make that first call before any stream capture.  All calls share the one scratch
 * array: calls that can overlap on the GPU (other streams, other threads) race and give wrong
 * results, so serialise them.  The look-back waits are bounded; if one gives up, the offsets are
 * unspecified and *out_total is set to UINT64_MAX (a sum of 32-bit counts never reaches it), so a
 * caller that passes out_total can tell; nothing is read back to the host. */
GS_API gs_status gs_scan_noalloc(void* stream, const uint32_t* counts, int64_t n, uint32_t* out_offsets,
                                 uint64_t* out_total);

#ifdef __cplusplus
}
#endif

#endif /* GS_H_ */
