/*
 * gs.h -- C ABI of libgs, the GB300 (sm_103a) differentiable Gaussian-splatting
 * mapping step of VIGS-SLAM (arXiv 2512.02293, Sec. 3.3 "Gaussian Splatting
 * Mapping", Eq. 6).
 *
 * One mapping iteration is
 *     gs_project -> gs_bin_sort -> gs_render_fwd -> gs_loss -> gs_render_bwd -> gs_adam_step
 * or, with the loss fused into the rasterisers,
 *     gs_project -> gs_bin_sort -> gs_render_fwd_loss -> gs_render_bwd_raster_loss
 *     -> gs_project_bwd -> gs_adam_step
 * over one or more keyframe views ("views").
 *
 * Conventions that hold for every call
 *  - The caller owns all memory.  libgs never allocates device or host memory;
 *    scratch space is passed in as a workspace of gs_workspace_size() bytes.
 *  - Pointers inside the structs below are DEVICE pointers to contiguous,
 *    row-major arrays unless stated otherwise; `gs_camera` arrays, parameter
 *    structs and the structs themselves live in HOST memory and are read
 *    during the call only.
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = the legacy default stream), performs no host synchronisation and no
 *    allocation, and may be captured into a CUDA graph.  Exceptions:
 *    gs_read_device_status synchronises `stream`; gs_loss_noalloc and the
 *    test hook gs_mlp_set_wait_polls carry their own notes.
 *  - Errors detectable on the host (NULL pointers, negative sizes, unsupported
 *    tile sizes, too many views, a too-small workspace) return a non-zero
 *    gs_status before anything is launched.  Errors found on the device
 *    (key-capacity overflow) are recorded in the caller's device status word
 *    (gs_bins.status) and read back with gs_read_device_status outside any
 *    graph.  A launch failure returns GS_ERR_CUDA.
 *  - Entries: a Gaussian i seen from view v is entry e = v * n + i, where n is
 *    the number of Gaussians.  Per-entry arrays have n_views * n rows.
 *  - Pixels: view v's pixels follow those of views 0..v-1; colour images are
 *    planar per view ([3][H_v][W_v] starting at 3 * pix_base(v)), single-channel
 *    images start at pix_base(v) = sum_{u<v} W_u H_u.  Pixel (u, v) is sampled
 *    at (u + 0.5, v + 0.5).
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_ABI_VERSION 6
#define GS_MAX_VIEWS 32

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,   /* bad pointer, size or parameter (host check) */
    GS_ERR_CAPACITY = 2,      /* more (tile, Gaussian) keys than gs_bins.key_capacity */
    GS_ERR_CUDA = 3,          /* a CUDA launch or runtime call failed */
    GS_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    GS_ERR_NUMERIC = 5,       /* non-finite value where a finite one is required */
    GS_ERR_UNSUPPORTED = 6    /* valid request this build does not implement */
} gs_status;

/* Pinhole keyframe camera.  The pose is camera-to-world: x_world = R_wc x_cam
 * + t_wc, the convention of the keyframe poses (R_k, t_k) in Sec. 3.3 "Loop
 * Closure Gaussian Update".  Camera axes: x right, y down, z forward. */
typedef struct gs_camera {
    float fx, fy, cx, cy;     /* focal lengths and principal point, pixels */
    int32_t width, height;    /* image size, pixels (each >= 1) */
    float R_wc[9];            /* rotation, row-major */
    float t_wc[3];            /* camera centre in world coordinates */
} gs_camera;

/* Rendering parameters.  The paper fixes none of these (Sec. 3.3 defers the
 * renderer to 3D Gaussian splatting); the values noted are the defaults the
 * binding uses. */
typedef struct gs_render_params {
    int32_t tile;             /* tile edge in pixels: 8, 16 or 32 (16) */
    float near_plane;         /* Gaussians with camera z <= near are culled (0.2) */
    float alpha_min;          /* splats with alpha < alpha_min are skipped (1/255) */
    float alpha_max;          /* alpha = min(alpha_max, o exp(power)) (0.99) */
    float T_cut;              /* a pixel stops before blending a splat that would
                                 take its transmittance below T_cut (1e-4) */
    float dilation;           /* added to the diagonal of the 2D covariance, px^2 (0.3) */
    float radius_sigma;       /* splat radius = ceil(radius_sigma sqrt(lambda_max)) (3) */
    float bg[3];              /* background colour (0, 0, 0) */
    int32_t sh_degree;        /* 0: direct RGB colour (Sec. 3.3); 3: degree-3 SH */
    int32_t splat_stages;     /* batches of 32 splats a warp of the forward rasteriser
                                 holds at once: 2 (the next batch in flight in
                                 registers) or 3 (the next two in flight through a
                                 shared-memory ring); 0: the library chooses (3 when a
                                 launch has at most 256 pixel blocks per SM, else 2).
                                 Results do not depend on it (0) */
    int32_t block_masks;      /* 1: gs_bin_sort writes gs_bins.masks and the
                                 rasterisers read them instead of testing every list
                                 entry against their pixel block; 0: no masks, the
                                 rasterisers test.  The render calls must be given
                                 the value the gs_bin_sort call that made `bins` was
                                 given.  Results do not depend on it (1) */
    int32_t cull_tiles;       /* 1: gs_bin_sort keeps only the (entry, tile) pairs
                                 whose splat can reach 0.99 alpha_min somewhere in
                                 the tile's box of pixel centres (the rasterisers'
                                 culling test at tile granularity); 0: every tile of
                                 the entry's rectangle.  Images, depth and T_final
                                 do not depend on it; n_contrib counts list
                                 positions, so it counts those of the shorter list
                                 with 1 (the same last blended splat) */
} gs_render_params;

/* The Gaussian map G (Sec. 3.3 "Preliminary"), structure of arrays, device. */
typedef struct gs_gaussians {
    const float* mean;            /* [n][3] world position mu */
    const float* quat;            /* [n][4] rotation (w, x, y, z), normalised inside */
    const float* log_scale;       /* [n][3] per-axis log standard deviation */
    const float* opacity_logit;   /* [n] opacity o = sigmoid(logit) */
    const float* color;           /* [n][3] RGB (sh_degree 0) or [n][16][3] SH coefficients */
    int64_t n;                    /* number of Gaussians, 0 <= n < 2^31 / n_views */
} gs_gaussians;

/* Per-entry output of gs_project (device, caller-allocated, n_views * n rows). */
typedef struct gs_projected {
    float* xy;                /* [E][2] projected mean, pixels */
    float* conic_o;           /* [E][4] inverse 2D covariance (A, B, C) and opacity */
    float* rgbd;              /* [E][4] colour (r, g, b) and camera z of the mean */
    int32_t* rect;            /* [E][4] covered tiles x0, y0, x1, y1 (x1, y1 exclusive) */
    int32_t* radius;          /* [E] splat radius in pixels, 0 if culled */
    uint32_t* tiles_touched;  /* [E] (x1 - x0) * (y1 - y0), 0 if culled */
} gs_projected;

/* Binned, depth-sorted splat lists (device, caller-allocated). */
typedef struct gs_bins {
    uint64_t* keys;           /* [key_capacity] (global tile << 32) | bits(float z) */
    uint32_t* vals;           /* [key_capacity] entry index e */
    int64_t key_capacity;     /* number of slots in keys / vals */
    uint32_t* ranges;         /* [total_tiles][2] [start, end) of each tile's list */
    uint32_t* num_keys;       /* [1] number of keys M the projection produced */
    int32_t* status;          /* [4] [0] device status word (gs_status), sticky; [1..3]
                                 work counters of the persistent rasterisers: zero
                                 before the first render call, and every render
                                 launch leaves them zero */
    uint32_t* masks;          /* [key_capacity] per key, bit b: the splat can reach
                                 pixel block b of its tile (8 x 4 pixel blocks,
                                 row-major within the tile; tile / 8 x tile / 4
                                 bits): its weight reaches 0.99 alpha_min somewhere
                                 in the block's box of pixel centres (the
                                 rasterisers' own culling test, as a conservative
                                 superset); written by gs_bin_sort and read by the
                                 rasterisers when gs_render_params.block_masks is
                                 set */
} gs_bins;

/* Rendered images and the per-pixel checkpoint the backward pass uses. */
typedef struct gs_image {
    float* color;             /* [3 * P] planar per view (see Pixels above) */
    float* depth;             /* [P] alpha-blended camera z of the means */
    float* T_final;           /* [P] transmittance after the last blended splat */
    uint32_t* n_contrib;      /* [P] splats visited up to the last blended one */
} gs_image;

/* Gradients; same layouts as gs_gaussians.  `pose` is [n_views][6], the
 * gradient w.r.t. xi = (rho, phi) of the left perturbation T_cw <- Exp(xi) T_cw
 * of each view's world-to-camera pose at xi = 0; it may be NULL. */
typedef struct gs_grads {
    float* mean;
    float* quat;
    float* log_scale;
    float* opacity_logit;
    float* color;
    float* pose;
} gs_grads;

/* One Adam parameter group (device arrays of n floats). */
typedef struct gs_adam_group {
    float* param;
    const float* grad;
    float* m;
    float* v;
    int64_t n;
    float lr;
    int32_t reserved;         /* must be 0 */
} gs_adam_group;

/* ABI version of the loaded library (GS_ABI_VERSION). */
int32_t gs_abi_version(void);

/* Human-readable name of a status code (static string). */
const char* gs_status_string(int32_t status);

/* Tiles of all views for the given tile size (host computation). */
int64_t gs_total_tiles(const gs_camera* cams, int32_t n_views, int32_t tile);

/* Pixels of all views (host computation). */
int64_t gs_total_pixels(const gs_camera* cams, int32_t n_views);

/* Bytes of workspace that gs_bin_sort, gs_loss and gs_render_bwd need for
 * n Gaussians, these views and a key capacity; one buffer of this size may be
 * shared by all three calls on the same stream. Returns 0 on invalid input. */
size_t gs_workspace_size(int64_t n, int32_t n_views, const gs_camera* cams,
                         const gs_render_params* params, int64_t key_capacity);

/* EWA projection of every Gaussian into every view (Sec. 3.3 "Preliminary":
 * mean mu, covariance Sigma = R(q) diag(exp(log_scale))^2 R(q)^T, opacity
 * sigmoid(logit), colour).  p_c = R_wc^T (mu - t_wc); entries with
 * z <= near_plane, a non-positive 2D determinant or no covered tile are culled
 * (radius = tiles_touched = 0).  conic = inverse of J W Sigma W^T J^T +
 * dilation I with J the perspective Jacobian at p_c.
 * Errors: GS_ERR_INVALID_ARG on NULL pointers, n < 0, n_views outside
 * [1, GS_MAX_VIEWS], bad params; GS_ERR_CUDA on launch failure. */
int32_t gs_project(const gs_gaussians* g, const gs_camera* cams, int32_t n_views,
                   const gs_render_params* params, gs_projected* out, void* stream);

/* gs_project with each view's pose moved on the device first: xi is a device
 * array [n_views][6] of pose tangents (rho, phi) and view v is rendered from
 * Exp(xi_v) T_cw (rotation by Rodrigues' formula, translation to first order:
 * T_cw <- (Exp(phi) R_cw, Exp(phi) t_cw + rho)), the left perturbation whose
 * gradient gs_project_bwd reports (Sec. 3.3 poses; the pose tangent of the
 * differentiable renderer).  It lets a caller render at a pose held in device
 * memory without reading it back to the host.  xi = NULL is gs_project.
 * Errors: as gs_project. */
int32_t gs_project_perturbed(const gs_gaussians* g, const gs_camera* cams, int32_t n_views,
                             const gs_render_params* params, const float* xi, gs_projected* out, void* stream);

/* Tile binning and depth sort.  The paper does not describe this step: Sec. 3.3
 * renders with the 3D Gaussian splatting rasteriser it builds on, whose
 * compositing visits each tile's splats front to back.  Here: one key
 * (global tile << 32) | bits(float z) with value e per (entry e, covered tile),
 * in the order of a stable ascending sort of the entry-ordered list by key
 * (so within a tile by depth, ties in z by entry index), and [start, end) of
 * each tile in it.  With params->cull_tiles the covered tiles are those of the
 * rectangle that the splat can reach at 0.99 alpha_min (see gs_render_params).
 * Built without a global sort: per-tile counts, a prefix over the tiles, a
 * scatter of (bits(z), e) into each tile's segment, and a sort of every segment
 * (six launches; a seventh writes the block masks).  Global tile of view v = tile_base(v) +
 * ty * tiles_x(v) + tx with tile_base(v) = tiles of views 0..v-1.  Writes M to
 * *bins->num_keys;
 * if M > key_capacity it sets *bins->status = GS_ERR_CAPACITY and the outputs
 * are undefined (grow the capacity to M and call again).
 * `ws` must hold gs_workspace_size(...) bytes.
 * Errors: GS_ERR_INVALID_ARG on NULL pointers or a small workspace. */
int32_t gs_bin_sort(const gs_projected* proj, int64_t n, const gs_camera* cams, int32_t n_views,
                    const gs_render_params* params, gs_bins* bins, void* ws, size_t ws_bytes,
                    void* stream);

/* Front-to-back alpha compositing of colour and depth per pixel (Sec. 3.3:
 * pixel colour by alpha blending the visible Gaussians; colour I_hat and depth
 * D_hat rendered per keyframe): over the pixel's tile list, power =
 * -1/2 (A dx^2 + C dy^2) - B dx dy with (dx, dy) = sample - xy; splats with
 * power > 0 or alpha = min(alpha_max, o exp(power)) < alpha_min are skipped; the
 * pixel stops before a splat with T (1 - alpha) < T_cut; C += c alpha T,
 * D += z alpha T, T *= 1 - alpha.  colour = C + T bg.  Also writes T_final and
 * n_contrib (the checkpoint gs_render_bwd starts from).
 * Errors: GS_ERR_INVALID_ARG on NULL pointers. */
int32_t gs_render_fwd(const gs_projected* proj, const gs_bins* bins, const gs_camera* cams,
                      int32_t n_views, const gs_render_params* params, gs_image* img, void* stream);

/* Colour and depth terms of Eq. 6 per view: L_c = mean over 3 W H of
 * |I_hat - I|, L_d = mean over pixels with D > 0 of |D_hat - D| (sign(0) = 0).
 * Writes dL/dI_hat = lambda_c sign / (3 W H) and dL/dD_hat = lambda_d sign / n_valid
 * (0 where D <= 0) for every view, and loss_terms[2 v] = L_c, [2 v + 1] = L_d
 * (unweighted; device, [n_views][2]).  Target layouts equal gs_image's.
 * Errors: GS_ERR_INVALID_ARG on NULL pointers or a small workspace. */
int32_t gs_loss(const gs_image* img, const float* target_color, const float* target_depth,
                const gs_camera* cams, int32_t n_views, float lambda_c, float lambda_d,
                float* dL_dcolor, float* dL_ddepth, float* loss_terms,
                void* ws, size_t ws_bytes, void* stream);

/* Allocation-free variant of gs_loss, for callers that cannot allocate device
 * memory for a workspace (no counterpart in the paper; it exists for such
 * callers only).  Examples: processes that must keep a fixed, pre-planned
 * device-memory budget (an embedded or real-time tracker that may not grow its
 * footprint after start-up); a plugin inside a host application that owns the
 * device allocator and forbids any other allocation; code running where an
 * allocation call is not allowed at that moment.
 * Same arguments, outputs and errors as gs_loss, without the workspace: the
 * per-view accumulators live in a static device array of
 * GS_NOALLOC_LOSS_MAX_VIEWS x 4 floats that every device loading the library
 * keeps until exit.  n_views > GS_NOALLOC_LOSS_MAX_VIEWS returns
 * GS_ERR_INVALID_ARG.  The call allocates nothing (no cudaMalloc / cudaFree /
 * allocating library routine).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  The address is cached for
 * the life of the process: after cudaDeviceReset (or anything else that
 * destroys the device's primary context and reloads the library's module) the
 * cached address is stale, and calling gs_loss_noalloc again is not supported.
 * Each call zeroes the
 * accumulators before use, but all calls on a device share them: calls whose
 * executions overlap on the GPU (different streams, no ordering) race. */
#define GS_NOALLOC_LOSS_MAX_VIEWS 32
int32_t gs_loss_noalloc(const gs_image* img, const float* target_color, const float* target_depth,
                        const gs_camera* cams, int32_t n_views, float lambda_c, float lambda_d,
                        float* dL_dcolor, float* dL_ddepth, float* loss_terms, void* stream);

/* Backward of gs_render_fwd and gs_project: gradient of the loss whose image
 * gradients are dL_dcolor / dL_ddepth, summed over views, w.r.t. every Gaussian
 * parameter and each view's pose tangent.  The compositing is walked back to
 * front from the per-pixel checkpoint (T_final, n_contrib); no per-splat state
 * is read from the forward pass.  Adds lambda_iso times the gradient of the
 * isotropic regulariser L_iso = (1/n) sum_i sum_j |s_ij - mean_j s_ij|,
 * s = exp(log_scale) (the MonoGS form Sec. 3.3 cites); if iso_loss is not NULL
 * it receives L_iso (device scalar).  All gradient arrays are OVERWRITTEN.
 * Gradient at the non-smooth points: 0 for culled entries, skipped splats and
 * splats whose alpha is clamped at alpha_max; SH colours clamped at 0 pass no
 * gradient.
 * Errors: GS_ERR_INVALID_ARG on NULL pointers or a small workspace. */
int32_t gs_render_bwd(const gs_gaussians* g, const gs_projected* proj, const gs_bins* bins,
                      const gs_image* img, const float* dL_dcolor, const float* dL_ddepth,
                      const gs_camera* cams, int32_t n_views, const gs_render_params* params,
                      float lambda_iso, gs_grads* grads, float* iso_loss,
                      void* ws, size_t ws_bytes, void* stream);

/* The two halves of gs_render_bwd, callable on their own (gs_render_bwd is
 * exactly gs_render_bwd_raster into its workspace followed by gs_project_bwd).
 *
 * gs_render_bwd_raster: zeroes grad2d and accumulates, per entry, the gradient
 * of the loss w.r.t. the projected quantities: grad2d[e] = {d xy (2), d conic
 * (A, B, C), d opacity, d z, 0, d rgb (3), 0} (12 floats, 16-byte aligned).
 * gs_project_bwd: chain rule from grad2d (summed over views) to the Gaussian
 * parameters and each view's pose tangent, plus lambda_iso dL_iso (see
 * gs_render_bwd); OVERWRITES grads.
 * Errors: GS_ERR_INVALID_ARG on NULL or misaligned pointers. */
int32_t gs_render_bwd_raster(const gs_projected* proj, const gs_bins* bins, const gs_image* img,
                             const float* dL_dcolor, const float* dL_ddepth, const gs_camera* cams,
                             int32_t n_views, const gs_render_params* params, int64_t n, float* grad2d,
                             void* stream);
int32_t gs_project_bwd(const gs_gaussians* g, const gs_camera* cams, int32_t n_views,
                       const gs_render_params* params, const float* grad2d, float lambda_iso,
                       gs_grads* grads, float* iso_loss, void* stream);
/* gs_project_bwd at the poses moved by the device tangents xi ([n_views][6], as
 * gs_project_perturbed; the pose gradient is that of a further left
 * perturbation of the moved pose).  xi = NULL is gs_project_bwd. */
int32_t gs_project_bwd_perturbed(const gs_gaussians* g, const gs_camera* cams, int32_t n_views,
                                 const gs_render_params* params, const float* xi, const float* grad2d,
                                 float lambda_iso, gs_grads* grads, float* iso_loss, void* stream);

/* The colour and depth terms of Eq. 6 fused into the rasterisers (the same
 * values as gs_render_fwd + gs_loss + gs_render_bwd_raster, without the two
 * loss passes over the images and without materialised gradient images).
 *
 * gs_render_fwd_loss: gs_render_fwd, and per view sum |I_hat - I|,
 * sum over D > 0 of |D_hat - D| and the count of D > 0 into loss_ws (per-CTA
 * partial sums, added up by the launch's last CTA); writes loss_terms[2 v] = L_c,
 * [2 v + 1] = L_d as gs_loss does.  Uses bins->status[3] as its ticket (zero
 * before the first call, left zero).
 * gs_render_bwd_raster_loss: gs_render_bwd_raster with each pixel's dL/dI_hat =
 * lambda_c sign(I_hat - I) / (3 W H) and dL/dD_hat = lambda_d sign(D_hat - D) /
 * n_valid (0 where D <= 0) formed from img, the targets and the totals that the
 * preceding gs_render_fwd_loss left in loss_ws (bit-identical to gs_loss's).
 * Follow it with gs_project_bwd.
 * loss_ws: device, 256-byte aligned, gs_fused_loss_workspace_size(n_views)
 * bytes, zero-filled before its first use; it carries the totals from the
 * forward to the backward call, so the two calls must use the same workspace,
 * targets and views.  It also carries the order in which the rasterisers take
 * their 8 x 4 pixel blocks when a launch has few of them per SM (at most 65536
 * blocks): the backward pass sorts the blocks by the forward's per-block depth,
 * deepest first, and the next forward pass on the same workspace and block count
 * reuses that order.  The order changes only which warp takes which block.
 * Errors: GS_ERR_INVALID_ARG on NULL or misaligned pointers, non-finite lambdas
 * or a small workspace. */
size_t gs_fused_loss_workspace_size(int32_t n_views);
int32_t gs_render_fwd_loss(const gs_projected* proj, const gs_bins* bins, const gs_camera* cams,
                           int32_t n_views, const gs_render_params* params, gs_image* img,
                           const float* target_color, const float* target_depth, float* loss_terms,
                           void* loss_ws, size_t loss_ws_bytes, void* stream);
int32_t gs_render_bwd_raster_loss(const gs_projected* proj, const gs_bins* bins, const gs_image* img,
                                  const float* target_color, const float* target_depth, float lambda_c,
                                  float lambda_d, const void* loss_ws, size_t loss_ws_bytes,
                                  const gs_camera* cams, int32_t n_views, const gs_render_params* params,
                                  int64_t n, float* grad2d, void* stream);

/* Adam with bias correction over n_groups parameter groups in one launch (the
 * optimiser step of each mapping iteration, Sec. 3.3 "Map Management"; the
 * paper does not name the optimiser).  d_step is a device int32[2]: d_step[0]
 * is the number of steps taken so far (the step applied is d_step[0] + 1 and
 * d_step[0] is incremented by the call), d_step[1] is internal and must be 0
 * before the first call.  m and v are updated in place.
 * Errors: GS_ERR_INVALID_ARG on NULL pointers, n < 0, n_groups outside [1, 8]. */
int32_t gs_adam_step(const gs_adam_group* groups, int32_t n_groups, float beta1, float beta2,
                     float eps, int32_t* d_step, void* stream);

/* One whole mapping iteration of the fused path in one call: gs_project,
 * gs_bin_sort (workspace ws), gs_render_fwd_loss (loss_ws),
 * gs_render_bwd_raster_loss (2D gradients in ws, which the sort no longer
 * needs), gs_project_bwd and gs_adam_step, issued in that order on `stream`
 * with the arguments below (each as documented for its call).  ws must hold
 * gs_workspace_size() bytes for these Gaussians, views and key capacity and be
 * 256-byte aligned, else GS_ERR_INVALID_ARG before anything is issued.  Returns
 * the first non-GS_OK status of the six; the calls after it are not issued. */
typedef struct gs_mapping_step_args {
    const gs_gaussians* gaussians;
    const gs_camera* cams;
    const gs_render_params* params;
    gs_projected* proj;
    gs_bins* bins;
    gs_image* img;
    gs_grads* grads;
    const float* target_color;
    const float* target_depth;
    float* loss_terms;            /* [n_views][2] */
    float* iso_loss;              /* device scalar or NULL */
    void* ws;
    size_t ws_bytes;
    void* loss_ws;
    size_t loss_ws_bytes;
    const gs_adam_group* adam_groups;
    int32_t* d_step;
    int32_t n_views;
    int32_t n_adam_groups;
    float lambda_c, lambda_d, lambda_iso;
    float beta1, beta2, adam_eps;
} gs_mapping_step_args;
int32_t gs_mapping_step(const gs_mapping_step_args* args, void* stream);

/* ------------------------------------------------------------------------
 * Learned initialiser of inserted Gaussians (keyframe insertion, Sec. 3.3
 * "Map Management": the paper initialises a new Gaussian's opacity to 0.5 and
 * leaves its shape to the mapper; this network predicts the shape).
 * A perceptron GS_MLP_IN -> GS_MLP_HIDDEN -> GS_MLP_HIDDEN -> GS_MLP_OUT with
 * GELU (x Phi(x), exact form) after both hidden layers:
 *     Z1 = bf16(W1 x + b1), H1 = bf16(gelu(Z1)), Z2 = bf16(W2 H1 + b2),
 *     H2 = bf16(gelu(Z2)), y = W3 H2 + b3,
 * with BF16 weights and inputs and FP32 accumulation (tensor cores).
 * x is a 7 x 7 RGB-D patch (see gs_extract_patches), y = (3 log-scale offsets,
 * 4 quaternion components in the camera frame, 1 opacity logit).
 *
 * BF16 values are passed as uint16_t bit patterns.  Input rows are
 * GS_MLP_IN_STRIDE values long (16-byte aligned rows); only the first
 * GS_MLP_IN are read. */
#define GS_MLP_IN 196
#define GS_MLP_IN_STRIDE 208
#define GS_MLP_HIDDEN 128
#define GS_MLP_OUT 8

/* FP32 master parameters (device): W1 [128][196], b1 [128], W2 [128][128],
 * b2 [128], W3 [8][128], b3 [8], row-major (row = output unit). */
typedef struct gs_mlp_params {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
} gs_mlp_params;

/* BF16 GEMM operands made by gs_mlp_pack (device, caller-owned, 16-byte
 * aligned): W1a [128][208] (W1 | b1 | 0), W2a [128][144] (W2 | b2 | 0),
 * W3a [16][144] (rows 0..7: W3 | b3 | 0; rows 8..15: 0), W2t [128][128] = W2^T;
 * and, because every pre-activation is a BF16 value, the activation tabulated
 * over all 65536 BF16 inputs z (indexed by the bit pattern): gelu_tab [65536]
 * = bf16(gelu(z)) (BF16) and dgelu_tab [65536] = gelu'(z) (FP32), evaluated in
 * FP32 with the exact erf form. */
typedef struct gs_mlp_packed {
    uint16_t *W1a, *W2a, *W3a, *W2t;
    uint16_t* gelu_tab;
    float* dgelu_tab;
} gs_mlp_packed;

/* FP32 gradients (device), same shapes as gs_mlp_params. */
typedef struct gs_mlp_grads {
    float *W1, *b1, *W2, *b2, *W3, *b3;
} gs_mlp_grads;

/* Round the master parameters to the BF16 operands.
 * Errors: GS_ERR_INVALID_ARG on NULL or misaligned pointers. */
int32_t gs_mlp_pack(const gs_mlp_params* params, const gs_mlp_packed* packed, void* stream);

/* Forward pass over n samples X [n][GS_MLP_IN_STRIDE] (BF16).  Writes Y [n][8]
 * (FP32) if Y is not NULL.  Training: Z1, Z2 [n][128] (BF16 pre-activations,
 * needed by gs_mlp_bwd) if not NULL; with targets T [n][8] (FP32) also
 * dY = 2 loss_scale (Y - T) [n][8] and *loss += loss_scale sum (Y - T)^2 (the
 * caller zeroes *loss; loss_scale = 1 / (8 n) gives the mean squared error).
 * d_status: device int32 status word (GS_ERR_TIMEOUT if a bounded wait gave up).
 * One CTA per SM walks tiles of 128 samples, two in flight: X tiles copied by
 * TMA into a two-stage ring, tcgen05 MMAs with accumulators and the hidden
 * activations in tensor memory, issued by one control warp while 16 warps run
 * the epilogues.  Errors: GS_ERR_INVALID_ARG on NULL / misaligned pointers,
 * n < 0, T without dY and loss; GS_ERR_CUDA if the tensor maps of X cannot be
 * made (the driver entry point is missing, or n > 2^31 - 129). */
int32_t gs_mlp_fwd(const gs_mlp_packed* packed, const uint16_t* X, int64_t n, float* Y, uint16_t* Z1,
                   uint16_t* Z2, const float* T, float* dY, float* loss, float loss_scale, int32_t* d_status,
                   void* stream);

/* Backward pass: gradients of sum(dY * Y) with respect to all parameters, from
 * the inputs X, the forward's Z1, Z2 and dY (all [n][...] as above).
 * OVERWRITES `grads` (zeroed, then accumulated over the batch).  Rounding:
 * dZ2 = bf16((W3^T dY) * gelu'(Z2)), dZ1 = bf16((W2^T dZ2) * gelu'(Z1)).
 * Every contraction runs on the tensor cores (dY enters as three BF16 parts
 * whose sum is dY, so its products stay exact); X arrives by TMA.
 * Errors: as gs_mlp_fwd. */
int32_t gs_mlp_bwd(const gs_mlp_packed* packed, const uint16_t* X, const uint16_t* Z1, const uint16_t* Z2,
                   const float* dY, int64_t n, const gs_mlp_grads* grads, int32_t* d_status, void* stream);

/* Test hook of the bounded device-side waits (no counterpart in the paper).
 * gs_mlp_fwd and gs_mlp_bwd wait on mbarriers for their tensor-core MMAs, each
 * wait at most this many polls; a wait that runs out lets the kernel wait
 * (bounded again) for the MMAs and copies it has in flight, record
 * GS_ERR_TIMEOUT in *d_status, release its tensor memory and return, so the
 * context stays usable.  Sets the limit of the launches issued after the call
 * (process-wide; 0 makes the first wait give up at once; a negative value
 * restores the default GS_MLP_WAIT_POLLS_DEFAULT) and returns the previous
 * limit, or -1 (nothing changed) above 2^32 - 1.  The limit is read when a
 * launch is issued, so a captured graph keeps the value of its capture. */
#define GS_MLP_WAIT_POLLS_DEFAULT 67108864u
int64_t gs_mlp_set_wait_polls(int64_t polls);

/* ------------------------------------------------------------------------
 * Keyframe insertion (Sec. 3.3 "Map Management").  A keyframe is one view:
 * colour [3][H][W] and depth [H][W] (device, FP32, planar), its gs_camera, and
 * n sample pixels uv [n][2] (device int32, (u, v) = (column, row)).  Samples
 * outside the image record GS_ERR_INVALID_ARG in *d_status (if not NULL). */

/* Writable destination rows of a map (device): row offset + k receives the
 * Gaussian of sample k.  Same layouts as gs_gaussians; capacity = rows. */
typedef struct gs_map_slots {
    float* mean;
    float* quat;
    float* log_scale;
    float* opacity_logit;
    float* color;
    int64_t capacity;
} gs_map_slots;

/* Network input of each sample: X [n][GS_MLP_IN_STRIDE] BF16.  Window pixel
 * p = 7 (dy + 3) + (dx + 3), dx, dy in [-3, 3], is pixel (u + dx, v + dy)
 * clamped to the image; X[4p .. 4p+2] = its RGB, X[4p+3] = its relative depth
 * (d_p - d_c) f / (7 d_c) with f = (fx + fy) / 2, d_c the sample's depth, 0 where
 * either depth is <= 0; the centre's depth slot (p = 24) holds log d_c (0 if
 * d_c <= 0).  X[196] = 1, X[197..207] = 0.  Values rounded to nearest BF16.
 * Errors: GS_ERR_INVALID_ARG on NULL / misaligned pointers, n < 0, bad camera. */
int32_t gs_extract_patches(const float* color, const float* depth, const gs_camera* cam, const int32_t* uv,
                           int64_t n, uint16_t* X, int32_t* d_status, void* stream);

/* New Gaussians at the samples, written to rows offset .. offset + n - 1 of dst.
 * Heuristic (Y == NULL): mean = back-projection of the pixel centre at its
 * depth d, isotropic log_scale = log(d stride / f) (f = (fx + fy) / 2),
 * identity rotation, opacity logit 0 (opacity 0.5, Sec. 3.3), colour = pixel
 * RGB (sh_degree 3: the DC coefficient (rgb - 0.5) / Y00, others 0).
 * Learned (Y [n][8] from gs_mlp_fwd): log_scale = heuristic + Y[0..2],
 * rotation = R_wc composed with the normalised camera-frame quaternion Y[3..6],
 * opacity logit = Y[7].  A sample with depth <= 0 becomes an inert Gaussian
 * (logit -30, log_scale -10) at the camera centre.
 * Errors: GS_ERR_INVALID_ARG on NULL pointers, n < 0, stride <= 0,
 * offset + n > capacity, sh_degree not 0 or 3, bad camera. */
int32_t gs_insert_gaussians(const float* color, const float* depth, const gs_camera* cam, const int32_t* uv,
                            int64_t n, float stride, const float* Y, const gs_map_slots* dst, int64_t offset,
                            int32_t sh_degree, int32_t* d_status, void* stream);

/* Loop-closure Gaussian update (Sec. 3.3 "Loop Closure Gaussian Update",
 * Eq. 7 and Eq. 8), in place on map rows 0 .. map->capacity - 1.  Gaussian i is
 * anchored to keyframe anchor[i] (device int32 [n], in [0, n_keyframes));
 * pose_before / pose_after (device float [n_keyframes][12]) hold each
 * keyframe's camera-to-world rotation (row-major, 9) and position (3) before
 * and after the pose-graph optimisation; scale_change (device float
 * [n_keyframes]) its scale factor ds_k > 0.  Then
 *     mean <- R+ (ds (R-)^T (mean - t-)) + t+,
 *     Sigma <- R+ ds^2 (R-)^T Sigma R- (R+)^T, i.e. quat <- q(R+ (R-)^T) * quat
 *     (Hamilton product, norm kept) and log_scale <- log_scale + log ds;
 * opacity and colour are unchanged.  A Gaussian with an out-of-range anchor or a
 * non-positive ds is left unchanged and GS_ERR_INVALID_ARG is recorded in
 * *d_status (if not NULL).  quat rows must be 16-byte aligned.
 * Errors: GS_ERR_INVALID_ARG on NULL / misaligned pointers, capacity < 0,
 * n_keyframes < 1. */
int32_t gs_loop_closure_update(const gs_map_slots* map, const int32_t* anchor, const float* pose_before,
                               const float* pose_after, const float* scale_change, int32_t n_keyframes,
                               int32_t* d_status, void* stream);

/* ------------------------------------------------------------------------
 * Dense visual bundle adjustment of the tracker (Sec. 3.2, "Vision Residual"
 * Eq. 2, "Frontend Tracking: Local Bundle Adjustment" Eq. 4): one
 * Levenberg-Marquardt step over a window of keyframes.
 *   r = u*_ij - Pi(T_j T_i^-1 Pi^-1(u, d_i(u))) for every edge (i, j) and every
 *   pixel u of keyframe i's h x w grid (sampled at pixel centres); cost
 *   sum w r^2.  Variables: the left perturbations xi_k = (rho, phi) of the poses
 *   k >= n_fixed (T_k <- Exp(xi_k) T_k; rotation exact, translation to first
 *   order) and every inverse depth of every keyframe that is an edge source.
 *   (H + lambda diag(H) + eps I) delta = -g with H = J^T W J, g = J^T W r,
 *   solved through the Schur complement of the diagonal inverse-depth block.
 * With gs_ba_problem.imu set, the inertial factor of Eq. 3 between consecutive
 * keyframes joins the same system (each free keyframe then also has a velocity
 * and a bias variable); see the fields below. */
typedef struct gs_ba_problem {
    float* poses;            /* [K][12] world-to-camera R (row-major) and t; updated */
    float* disp;             /* [K][h][w] inverse depths; updated */
    const float* targets;    /* [E][h][w][2] target pixel coordinates u*_ij */
    const float* weights;    /* [E][h][w][2] confidences w_ij (>= 0) */
    const int32_t* ii;       /* [E] edge sources (device) */
    const int32_t* jj;       /* [E] edge targets (device) */
    int32_t n_keyframes, n_edges, height, width;
    int32_t n_fixed;         /* the first n_fixed poses are held (gauge) */
    float fx, fy, cx, cy;    /* intrinsics of the h x w grid */
    int32_t* status;         /* device status word: bad edge indices record
                                GS_ERR_INVALID_ARG, more than 15 edges out of one
                                keyframe GS_ERR_UNSUPPORTED, a reduced system
                                that is not positive definite GS_ERR_NUMERIC */
    /* Inertial factor (Eq. 3) between consecutive keyframes k, k + 1; imu NULL
     * = vision only.  The camera frame is taken as the IMU body frame.  With the
     * factor, every free keyframe also has a velocity and a bias variable.
     * imu: [K - 1][GS_BA_IMU_FLOATS] per pair: dR (9, row-major), dp (3), dv (3),
     *      J_rot (9, w.r.t. the gyro bias), J_pos (18, 3 x 6 w.r.t. the bias
     *      (b_g, b_a)), J_vel (18), dt (1), information (225, 15 x 15 over
     *      (r_rot, r_pos, r_vel, r_bias)); the velocity term's bias correction
     *      takes the full bias, as the position term's does.
     * vel: [K][3] world-frame velocities, updated; bias: [K][6] (b_g, b_a),
     * updated; bias_hat: [K][6] the biases the pre-integration was linearised
     * at; gravity: g in the world frame. */
    const float* imu;
    float* vel;
    float* bias;
    const float* bias_hat;
    float gravity[3];
} gs_ba_problem;

#define GS_BA_IMU_FLOATS 286

/* Workspace bytes of gs_ba_step (inertial != 0: with the inertial factor). */
size_t gs_ba_workspace_size(int32_t n_keyframes, int32_t n_edges, int32_t height, int32_t width, int32_t n_fixed,
                            int32_t inertial);

/* One step; *cost (device float) receives sum w r^2 at the poses and inverse
 * depths (and the inertial terms) before the step.  At most 31 free keyframes
 * (15 with the inertial factor) and at most 15 edges with the same source
 * keyframe.  With the inertial factor the first n_fixed keyframes keep their
 * pose, velocity and bias.
 * Errors: GS_ERR_INVALID_ARG on NULL pointers, bad sizes, a too-small or
 * misaligned workspace, lambda < 0, eps < 0, imu given without vel, bias or
 * bias_hat; GS_ERR_UNSUPPORTED above 31 free keyframes (15 with the inertial
 * factor). */
int32_t gs_ba_step(const gs_ba_problem* problem, float lambda, float eps, float* cost, void* ws, size_t ws_bytes,
                   void* stream);

/* Measurement helper, no part of the method: reads buf[n] (device FP32,
 * 16-byte aligned, n a multiple of 4) `reps` times over in one launch with
 * 16-byte loads cached in L2 only, and adds the sum of everything read to
 * *out (device FP32), so the loads cannot be dropped.  With buf smaller than
 * the L2 cache, n * 4 * reps bytes over the launch's time is the L2 read
 * bandwidth: the denominator of the binning stage's L2 roofline.
 * Errors: GS_ERR_INVALID_ARG on NULL pointers, n <= 0, n % 4 != 0, reps < 1,
 * misalignment. */
int32_t gs_l2_read_probe(const float* buf, int64_t n, int32_t reps, float* out, void* stream);

/* Synchronises `stream`, copies the device status word to *host_status and
 * returns GS_OK (or GS_ERR_CUDA if the copy failed).  Not capturable. */
int32_t gs_read_device_status(const int32_t* d_status, void* stream, int32_t* host_status);

#ifdef __cplusplus
}
#endif

#endif /* GS_H_ */
