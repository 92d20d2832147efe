/*
 * gs2d.h -- C ABI of the GB300 (sm_103a) 2D Gaussian (surfel) splatting
 * rasterizer: the hot path of CityGaussianV2 (arXiv 2411.00771).
 *
 * The library renders a surfel scene from a pinhole camera (per-surfel
 * preprocess, (tile, depth) sort, front-to-back compositing), differentiates
 * the render by a hand-written adjoint, evaluates the L1 + D-SSIM + depth
 * losses, and computes the decomposed-gradient densification statistics
 * (Eq. 2) and the elongation filter.
 *
 * Conventions (all entry points):
 *  - Every call returns gs_status: GS_OK (0) or a negative error code.  No
 *    call aborts the process.  gs_last_error() returns a thread-local text
 *    of the last failure.
 *  - "device" pointers are CUDA global-memory addresses on the current
 *    device; "host" pointers are CPU memory.  Unless stated, buffers are
 *    owned by the caller and must stay valid until the work queued on
 *    `stream` has completed.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is queued asynchronously on it.  gs_render reads one
 *    4-byte count back to the host and therefore synchronises the stream
 *    once per call.
 *  - Arrays are FP32, C order.  Surfel parameters are structure-of-arrays:
 *    mu [N][3], quat [N][4] as (w, x, y, z) (normalised inside), scale [N][2]
 *    (activated, > 0), opacity [N] (activated, in [0, 1]), sh [N][K][3] with
 *    K = (sh_degree + 1)^2 real spherical-harmonic coefficients per channel
 *    (index l*l + l + m, Condon-Shortley phase).
 *  - Images are planar: plane p of an H x W image is at offset p*H*W.
 *  - Errors detected on the device (instance-count capacity) are reported
 *    by the call that launched the work after its one synchronisation.
 */
#ifndef GS2D_H
#define GS2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int gs_status;
enum {
  GS_OK = 0,
  GS_ERR_ARG = -1,      /* invalid argument (null pointer, bad size, ...)   */
  GS_ERR_OOM = -2,      /* an allocation through the allocator failed         */
  GS_ERR_CAPACITY = -3, /* a size limit of the library was exceeded           */
  GS_ERR_CUDA = -4,     /* a CUDA runtime call or kernel launch failed        */
  GS_ERR_TIMEOUT = -5,  /* a bounded wait ran out                             */
  GS_ERR_STATE = -6     /* call made on an object in the wrong state          */
};

/* Planes of a render, [GS_OUT_PLANES][H][W] FP32 (Eq. 1 of Sec. 3.1 for the
 * colour; Sec. 3.1 "2D Gaussian Splatting" for distortion and normal;
 * Sec. 3.2 for inverse depth; Sec. 5.1 for median depth):
 *   R, G, B       sum_i w_i c_i + T_final * bg, w_i = alpha_i prod_{j<i}(1 - alpha_j)
 *   ALPHA         sum_i w_i
 *   DEPTH         sum_i w_i z_i   (expected depth times alpha; divide by ALPHA)
 *   INVDEPTH      sum_i w_i / z_i (inverse depth for the depth loss)
 *   MEDIAN        z of the last blended pair entered with transmittance > 0.5
 *   NX, NY, NZ    sum_i w_i n_i (view-space normals facing the camera)
 *   DISTORTION    sum_i 2 w_i (z_i A_{i-1} - Z_{i-1}) (depth distortion)
 *   T_FINAL       transmittance after the last blended pair
 * The first GS_ADJ_PLANES planes are differentiable; an adjoint set has the
 * same layout without T_FINAL. */
enum {
  GS_PLANE_R = 0, GS_PLANE_G = 1, GS_PLANE_B = 2, GS_PLANE_ALPHA = 3,
  GS_PLANE_DEPTH = 4, GS_PLANE_INVDEPTH = 5, GS_PLANE_MEDIAN = 6,
  GS_PLANE_NX = 7, GS_PLANE_NY = 8, GS_PLANE_NZ = 9, GS_PLANE_DISTORTION = 10,
  GS_PLANE_T_FINAL = 11, GS_OUT_PLANES = 12, GS_ADJ_PLANES = 11
};
/* bit masks of adjoint planes */
#define GS_MASK_RGB 0x7u
#define GS_MASK_ALL 0x7FFu

/* Pinhole camera: world-to-camera rotation R (row-major) and translation t,
 * x_cam = R x_world + t; the camera looks down +z, x right, y down.  Pixel
 * (i, j) samples the point (i + 0.5, j + 0.5).  Host struct, read during the
 * call. */
typedef struct {
  double R[9];
  double t[3];
  double fx, fy, cx, cy;
  int32_t width, height;
} gs_camera;

/* Rasterizer constants.  gs_default_settings() fills the values used
 * throughout: near 0.2, alpha_min 1/255, T_min 1e-4, alpha_max 0.99,
 * rho_max 9 (3-sigma support), screen_inv_sigma2 2 (antialiasing filter of
 * variance 1/2 pixel^2), black background. */
typedef struct {
  float near_plane;
  float alpha_min;
  float T_min;
  float alpha_max;
  float rho_max;
  float screen_inv_sigma2;
  float bg[3];
} gs_settings;

/* Device-memory allocator used for every buffer the library allocates.
 * alloc returns a device pointer (NULL on failure) usable on `stream`;
 * free releases it in stream order.  A zeroed struct selects
 * cudaMallocAsync / cudaFreeAsync. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx, void* stream);
  void (*free)(void* ptr, size_t bytes, void* ctx, void* stream);
  void* ctx;
} gs_allocator;

typedef struct {
  int64_t n;                 /* number of surfels, >= 0, < 2^31             */
  int32_t sh_degree;         /* 0..3                                         */
  const float* mu;           /* device [n][3]                                */
  const float* quat;         /* device [n][4]                                */
  const float* scale;        /* device [n][2]                                */
  const float* opacity;      /* device [n]                                   */
  const float* sh;           /* device [n][(d+1)^2][3]                       */
  gs_settings settings;
  gs_allocator allocator;
} gs_scene_desc;

typedef struct gs_scene gs_scene;
typedef struct gs_frame gs_frame;

/* Sec. 3.1: the surfel scene (mu, rotation, (s_u, s_v), opacity, SH).  The
 * parameter arrays are borrowed, not copied: they must stay valid and hold
 * the current values whenever work of this scene runs.  Returns GS_ERR_ARG
 * for bad sizes or null arrays (arrays may be null when n == 0). */
gs_status gs_default_settings(gs_settings* out);
gs_status gs_create_scene(gs_scene** out, const gs_scene_desc* desc);
/* Re-point the borrowed parameter arrays (after densification changes n). */
gs_status gs_set_params(gs_scene* scene, int64_t n, const float* mu, const float* quat,
                        const float* scale, const float* opacity, const float* sh);
gs_status gs_destroy_scene(gs_scene* scene);

/* Render one view (Eq. 1 with the 2DGS surfel model, Sec. 3.1-3.2).
 *  out:       device [GS_OUT_PLANES][H][W] FP32, written entirely.
 *  n_contrib: device [H][W] int32 number of blended pairs, or NULL.
 *  saved:     if non-NULL, receives a frame holding what gs_backward and
 *             gs_densify_accumulate need; the frame keeps a pointer to `out`
 *             (its ALPHA and DEPTH planes are read by the backward), so `out`
 *             must stay unchanged until the frame is released.
 * Synchronises `stream` once (to size the tile lists). */
gs_status gs_render(gs_scene* scene, const gs_camera* cam, float* out, int32_t* n_contrib,
                    gs_frame** saved, void* stream);
gs_status gs_frame_release(gs_frame* frame, void* stream);

typedef struct {
  int64_t n_instances;      /* (surfel, tile) pairs in the tile lists        */
  int64_t n_visible;        /* surfels with a non-empty tile rectangle       */
  int64_t pairs_evaluated;  /* list entries the forward blend evaluated      */
  int64_t pairs_blended;    /* pairs that entered the composite              */
  int64_t bwd_pairs_evaluated; /* list entries the last backward replayed    */
  int64_t bwd_warp_entries;    /* (warp, entry) steps with a blended pair     */
  int64_t bwd_warp_lanes;      /* blended pairs summed over those steps       */
  int32_t tiles_x, tiles_y;
  int64_t n_candidates;     /* surfels the conservative cull kept (sorted)   */
} gs_frame_info;
/* Counters of a frame (synchronises `stream`). */
gs_status gs_frame_get_info(gs_frame* frame, gs_frame_info* info, void* stream);

/* Debug / parity access to the frame's tile lists: copies (device to
 * device) up to `cap` sorted surfel indices into `values` (device int32)
 * and [tiles_x*tiles_y][2] int32 ranges into `ranges` (device), and the
 * per-surfel tile rectangles [n][4] (tx0, ty0, tx1, ty1) into `rects`
 * (device int32, may be NULL). */
gs_status gs_frame_copy_lists(gs_frame* frame, int32_t* values, int64_t cap, int32_t* ranges,
                              int32_t* rects, void* stream);

/* Debug / parity access to what the tile binning (Eq. 1's front-to-back
 * order needs every surfel listed in each tile its {rho <= rho_max} set
 * reaches) was computed from, per surfel, so that a checker can rebuild the
 * tile lists and ranges independently:
 *  geom:       device [n][14] 32-bit words (may be NULL), the FP32 footprint
 *              shape: words 0-3 the projected centre as two-float sums
 *              (c_x hi, c_x lo, c_y hi, c_y lo); words 4-9 the ellipse
 *              {rho_obj <= rho_max} relative to c, (d - e0)^T G^-1 (d - e0) <= 1
 *              given as (e0_x, e0_y, hy = sqrt(G22), t = G12 / sqrt(G11),
 *              slope = G12 / G22, wsc = sqrt(det G) / G22), hy < 0 when the
 *              disk has no ellipse; words 10-13 (int32) the pixel-centre box
 *              [ilo, ihi] x [jlo, jhi] of the whole footprint, clipped to the
 *              image.  A tile row lists the tile columns whose pixel centres
 *              in that row band meet the ellipse or the screen-filter disk
 *              |d| <= sqrt(rho_max / screen_inv_sigma2), each side widened
 *              by an FP32 rounding margin;
 *  depth:      device float [n] (may be NULL), the FP32 centre depth that
 *              orders each tile's list (ties by surfel index);
 *  tile_count: device int32 [n] (may be NULL), the number of tiles listing
 *              the surfel; geom and depth are defined only where it is > 0.
 * Asynchronous on `stream`; GS_ERR_ARG for a null frame. */
gs_status gs_frame_copy_cover(gs_frame* frame, int32_t* geom, float* depth, int32_t* tile_count,
                              void* stream);

/* Sec. 3.1 and 3.2 losses: L1 = mean |C - C*|, SSIM with an 11x11 Gaussian
 * window (sigma 1.5, zero padded, C1 = 0.01^2, C2 = 0.03^2) averaged over
 * pixels and channels, L_depth = mean |I - I*| on inverse depth;
 * total = w_l1 L1 + w_ssim (1 - SSIM) + w_depth L_depth.
 *  out:            device [GS_OUT_PLANES][H][W] (a render).
 *  target_rgb:     device [3][H][W].  target_invdepth: device [H][W] or NULL.
 *  adj_total:      device [GS_ADJ_PLANES][H][W]; planes R, G, B and (when
 *                  target_invdepth is given) INVDEPTH are written with
 *                  d total / d plane; other planes are not touched.
 *  adj_ssim, adj_l1: device [GS_ADJ_PLANES][H][W] or NULL; planes R, G, B
 *                  receive the adjoint of the weighted SSIM term and of the
 *                  weighted L1 term (their sum is adj_total's colour).
 *  losses:         device float[4] = L1, SSIM, L_depth, total. */
typedef struct {
  float w_l1, w_ssim, w_depth;
} gs_loss_weights;
gs_status gs_loss(int32_t width, int32_t height, const float* out, const float* target_rgb,
                  const float* target_invdepth, const gs_loss_weights* w, float* adj_total,
                  float* adj_ssim, float* adj_l1, float* losses, void* stream);

/* gs_loss without any device allocation.  (The paper has no counterpart:
 * this is a service for callers that cannot allocate device memory when
 * they need the loss, e.g. code running under an external memory manager
 * that owns the whole GPU, or a real-time loop that must not stall on or
 * fail an allocation.)
 * Same arguments, results and kernels as gs_loss, but the scratch lives in
 * one fixed device array inside the library (about 9.5 MB, reserved on
 * every GPU that loads the library until the process exits), so:
 *  - the image may have at most 512 * 512 pixels and sides of at most 4096;
 *    larger images return GS_ERR_CAPACITY with a message (use gs_loss);
 *  - the first call on a device looks up the array's device address on that
 *    device (no allocation); make that first call before any stream
 *    capture on that device;
 *  - every call shares the array: calls whose GPU work can overlap (other
 *    streams, other threads) race and must be serialised by the caller. */
gs_status gs_loss_noalloc(int32_t width, int32_t height, const float* out,
                          const float* target_rgb, const float* target_invdepth,
                          const gs_loss_weights* w, float* adj_total, float* adj_ssim,
                          float* adj_l1, float* losses, void* stream);

/* Parameter gradients, device, same shapes as the parameters.  gs_backward
 * ADDS into them (like accumulating .grad); a null pointer skips that
 * parameter.  The arrays must not overlap one another or the parameters. */
typedef struct {
  float* mu;
  float* quat;
  float* scale;
  float* opacity;
  float* sh;
} gs_param_grads;

/* Hand-written adjoint of gs_render (reverse replay per pixel from the
 * saved final transmittance).
 *  adj_sets:    host array of n_sets (1..3) device pointers, each
 *               [GS_ADJ_PLANES][H][W]; set 0 drives the parameter gradients.
 *  plane_masks: host array of n_sets bit masks of the planes that are
 *               non-zero in each set (bit p = plane p); sets after the first
 *               may use only the colour planes (mask within GS_MASK_RGB).
 *  grads:       parameter gradients to accumulate into (set 0).
 *  screen_grads: device [n_sets][N][2] or NULL: ADDS, per set, the gradient
 *               of that set's loss with respect to a screen-space translation
 *               of each surfel's opacity footprint (pixels), the view-space
 *               position gradient used by densification (Sec. 3.1, Eq. 2). */
gs_status gs_backward(gs_scene* scene, gs_frame* frame, const float* const* adj_sets,
                      const uint32_t* plane_masks, int32_t n_sets, const gs_param_grads* grads,
                      float* screen_grads, void* stream);

/* Decomposed densification statistics (Sec. 3.2, Eq. 2).  For every surfel
 * visible in the frame (non-empty tile rectangle):
 *   stats[n][s] += || screen_grads[s][n] ||_2 for s < min(n_sets, 3),
 *   stats[n][3] += 1.
 * Set order: 0 total loss, 1 SSIM term, 2 L1 term.  stats: device [N][4]. */
gs_status gs_densify_accumulate(gs_scene* scene, gs_frame* frame, const float* screen_grads,
                                int32_t n_sets, float* stats, void* stream);

/* DGD selection (Sec. 3.2, Eq. 2) with the elongation filter (Sec. 3.2):
 *   k   = max(omega * avg_n(S_tot/cnt) / avg_n(S_ssim/cnt), 1) over cnt > 0
 *         (k = 1 if the SSIM average is 0),
 *   g_n = k * S_ssim/cnt (0 when cnt = 0),
 *   eta_n = min(s_u, s_v) / max(s_u, s_v),
 *   mask_n = (cnt > 0) and (g_n >= grad_thr) and (eta_n >= eta_thr).
 *  stats: device [n][4]; scale: device [n][2]; mask: device uint8 [n];
 *  g_out: device float [n] or NULL; k_out: device float[1] or NULL. */
gs_status gs_densify_select(int64_t n, const float* stats, const float* scale, float omega,
                            float grad_thr, float eta_thr, uint8_t* mask, float* g_out,
                            float* k_out, void* stream);

/* Elongation filter alone (Sec. 3.2): keep[n] = eta_n >= eta_thr. */
gs_status gs_elongation_filter(int64_t n, const float* scale, float eta_thr, uint8_t* keep,
                               void* stream);

/* ---- Training-loop terms --------------------------------------------------
 *
 * gs_geometry_loss: the geometric terms that 2DGS adds to the loss and the
 * paper keeps (Sec. 3.1; weights in Sec. 5.1: 0.0125 for the normal term, 0
 * for the distortion).  Depth-normal consistency, per pixel L = A - N~ . N_r:
 * A the alpha plane, N_r the rendered normal planes (weight-summed, view
 * space) and N~ the unit normal of the surface at the pixel, the cross product
 * of the central differences of the points P = median depth * (ray through the
 * pixel centre) of its four neighbours, turned towards the camera; interior
 * pixels whose four neighbours have a depth and a non-degenerate cross product
 * count.  Depth distortion: the distortion plane.  losses (device FP32 [2]) =
 * (w_normal * mean of L, w_dist * mean of the distortion plane) over all W*H
 * pixels; their adjoints (alpha, median, normal, distortion planes) are ADDED
 * to adj (device FP32 [11][H][W]); out is a render ([12][H][W]) of `cam`
 * (W x H).  Asynchronous; allocates 16 B per pixel of scratch.
 *
 * gs_adam_step: one bias-corrected Adam update of n FP32 values in place:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * param -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps);
 * step >= 1 counts updates from 1.  Asynchronous. */
gs_status gs_geometry_loss(int32_t W, int32_t H, const gs_camera* cam, const float* out, float w_normal,
                           float w_dist, float* adj, float* losses, void* stream);

/* Densification: the clone / split / prune step of the training schedule the
 * paper keeps from CityGaussian (Sec. 5.1), driven by the selection of Eq. 2
 * and the elongation filter (Sec. 3.2).
 *
 * gs_densify_plan: per surfel an action (device uint8 [n]): 0 drop, 1 keep,
 * 2 clone, 3 split.  A surfel with select[i] != 0 and (keep NULL or keep[i] !=
 * 0) (select: gs_densify_select's mask; keep: gs_elongation_filter's) is
 * cloned when max(scale) <= dense_thr and split otherwise; any other is
 * dropped when opacity < min_opacity, else kept.  raw != 0: scale holds
 * log-scales and opacity logits (the thresholds are mapped accordingly).  offset (device uint32 [n]) = the first output row of each surfel
 * (rows follow the source order: keep 1 row, clone 2 (itself, then the copy),
 * split 2 children, drop 0); *n_out (host) = the number of output rows.  Reads
 * that count back (synchronises the stream).
 *
 * gs_densify_apply: writes the n_out rows (device arrays of the same layouts as
 * the scene parameters, activated scale and opacity).  A split child j of
 * surfel i sits at mu + t_u s_u xi[i][j][0] + t_v s_v xi[i][j][1] (t_u, t_v the
 * first two columns of the surfel's rotation; xi device FP32 [n][2][2], the
 * caller's standard normal draws) with scales s / 1.6 (log-scales minus ln 1.6
 * when raw != 0); everything else is copied.  src[r] (device int32 [n_out]) = the source surfel of row r;
 * fresh[r] (device uint8 [n_out]) = 1 for rows whose optimizer state starts
 * afresh (clone copies and split children).
 *
 * gs_gather_rows: out[r][k] = fresh[r] ? 0 : in[src[r]][k] for width k
 * (fresh may be NULL: no row is fresh); remaps per-surfel state (optimizer
 * moments, accumulators) after densification.
 *
 * gs_activate / gs_activate_grad: the trained parametrisation scale =
 * exp(log_scale) ([n][2]), opacity = sigmoid(logit) ([n]), and the chain of
 * gradients through it in place (grad_scale *= scale, grad_opacity *=
 * opacity (1 - opacity)).  All asynchronous except gs_densify_plan. */
gs_status gs_densify_plan(int64_t n, const uint8_t* select, const uint8_t* keep, const float* scale,
                          const float* opacity, int32_t raw, float dense_thr, float min_opacity,
                          uint8_t* action, uint32_t* offset, int64_t* n_out, void* stream);
gs_status gs_densify_apply(int64_t n, int32_t sh_degree, int32_t raw, const uint8_t* action,
                           const uint32_t* offset,
                           const float* xi, const float* mu, const float* quat, const float* scale,
                           const float* opacity, const float* sh, float* mu_out, float* quat_out,
                           float* scale_out, float* opacity_out, float* sh_out, int32_t* src,
                           uint8_t* fresh, void* stream);
gs_status gs_gather_rows(int64_t n_out, int32_t width, const int32_t* src, const uint8_t* fresh,
                         const float* in, float* out, void* stream);
gs_status gs_activate(int64_t n, const float* log_scale, const float* logit_opacity, float* scale,
                      float* opacity, void* stream);
gs_status gs_activate_grad(int64_t n, const float* scale, const float* opacity, float* grad_scale,
                           float* grad_opacity, void* stream);
gs_status gs_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr, float beta1,
                       float beta2, float eps, int32_t step, void* stream);

/* ---- Trim contribution and pruning (Sec. 3.3) ------------------------------
 *
 * gs_contribution: the single-view contribution of every surfel, Eq. 3,
 *   C_{n,k} = (1/|P_k|) sum over p in P_k of alpha_n^gamma T_n(p)^(1-gamma),
 * where P_k is the surfel's projected region in view k (the pixels inside its
 * 3-sigma support rho <= rho_max, occluded or not), alpha_n the opacity the
 * compositing applies to the pair (0 below the alpha cutoff and behind the
 * pixel's transmittance stop) and T_n(p) the transmittance in front of it.
 * The view is preprocessed and ordered exactly as gs_render does (the same
 * tile lists and compositing decisions) but no image is written.
 *   gamma:       in [0, 1]; the paper's value is 0.5.
 *   contrib:     device FP32 [N] or NULL; weight * C_{n,k} is ADDED (C = 0
 *                where |P_k| = 0).  With weight = 1/|V_m| over the views of a
 *                block this accumulates Eq. 4's average.
 *   view_sum, view_count: device [N] (FP32, uint32) or NULL; when given they
 *                are overwritten with this view's sum and |P_k| (0 for
 *                surfels outside the view).
 * At least one output must be given.  Reads one 4-byte count back (like
 * gs_render); otherwise asynchronous on `stream`.  Errors: GS_ERR_ARG
 * (null scene/camera/outputs, gamma outside [0, 1], bad camera), GS_ERR_OOM,
 * GS_ERR_CAPACITY, GS_ERR_CUDA.
 *
 * gs_prune_by_contribution: percentile pruning, Sec. 3.3.  With
 * k = ceil(ratio * n) clamped to [0, n], the bound is the k-th smallest value
 * of contrib (device FP32 [n]); keep[i] (device uint8 [n]) = contrib[i] >
 * bound, so every surfel at or below the bound is removed, ties and
 * never-observed (0) surfels included.  k = 0 keeps everything and the bound
 * is -inf.  bound: device FP32 [1] or NULL.  ratio must be in [0, 1] (the
 * paper uses 0.025 and, in its ablation, 0.1).  Asynchronous; allocates a
 * 1 KB scratch through the default allocator. */
gs_status gs_contribution(gs_scene* scene, const gs_camera* camera, float gamma, float weight,
                          float* contrib, float* view_sum, uint32_t* view_count, void* stream);
gs_status gs_prune_by_contribution(int64_t n, const float* contrib, double ratio, uint8_t* keep,
                                   float* bound, void* stream);

/* ---- Visible frequency of points (Sec. 4, crop volume estimation) -------
 *
 * gs_visibility_count: for each of n points (device FP32 [n][3], world
 * coordinates), ADDS to counts[j] (device uint32 [n]) the number of the
 * n_views cameras (host array) in which the point is visible as a Gaussian
 * primitive of a rasterizer: an isotropic 3D Gaussian of standard deviation
 * sigma (world units) that lies in front of near_plane and whose projected
 * footprint's 3-sigma square overlaps the image.  The footprint covariance is
 * sigma^2 J J^T + lowpass I (J the Jacobian of the perspective projection at
 * the point; lowpass the rasterizer's screen-space dilation in px^2, 0.3 in
 * the usual 3DGS rasterizer); the half-width is 3 sqrt(largest eigenvalue).
 * Occlusion plays no part (the rasterizer's per-primitive visible mask).  FP32;
 * a decision within about 1e-6 (relative) of its threshold may go either way.
 * Asynchronous; the cameras are copied to the device before the call returns.
 *
 * gs_visibility_bounds: keep[j] = (counts[j] >= min_count) (device uint8 [n]);
 * zrange (device FP32 [2]) = lowest and highest world z among the kept points,
 * NaN when none is kept.  The paper then fits an alpha shape to the kept
 * points' ground projection (not part of this library). */
gs_status gs_visibility_count(int64_t n, const float* points, float sigma, const gs_camera* cams,
                              int32_t n_views, float near_plane, float lowpass, uint32_t* counts,
                              void* stream);
gs_status gs_visibility_bounds(int64_t n, const float* points, const uint32_t* counts, uint32_t min_count,
                               uint8_t* keep, float* zrange, void* stream);

/* ---- Vector quantisation of SH and compressed scenes (Sec. 3.3) ------------
 *
 * After the blocks are merged, the surfels of least contribution (Eq. 4,
 * gs_contribution over the training views) have their SH vector replaced by
 * the nearest entry of a K-means codebook; every other attribute is stored in
 * IEEE binary16 (Appendix C: codebook size 8192, quantisation ratio 0.4).
 * keep (device uint8 [n]) names the surfels that keep their own SH (non-zero);
 * the others are quantised: gs_prune_by_contribution's keep at the
 * quantisation ratio selects exactly the paper's set.
 * A vector is the surfel's whole SH row, C = 3 (deg+1)^2 values, rounded to
 * binary16; codebook entries are binary16 too.
 *
 * gs_vq_kmeans: Lloyd's K-means over the m surfels with keep[i] == 0
 * (surfel-index order).
 *   sh:        device FP32 [n][(deg+1)^2][3].
 *   K >= 1 entries; iters >= 0 update steps; entry j starts as the vector at
 *              position floor(u_j m) (u_j = init_u[j], device FP32 [K], the
 *              caller's uniform draws in [0, 1); FP64 product; clamped to
 *              [0, m - 1]).
 *   Each step assigns every vector to argmin_j ||x - c_j||^2 (the lowest j
 *   among equal scores; scores are evaluated in FP32 from the binary16 values,
 *   so two entries within about 1e-5 relative of each other may go either
 *   way) and then sets each entry with vectors to
 *   rn16((double(exact sum) * 2^-24) / count) (exact sums: order-independent
 *   and reproducible); an entry without vectors keeps its value.  A final
 *   assignment to the last codebook follows the iters steps.
 *   codebook:  device binary16 [K][C] (output).
 *   assign:    device int32 [n] (output): the entry of each quantised surfel,
 *              -1 for the others.
 *   objective: device FP64 [iters + 1] or NULL: sum over vectors of the
 *              squared distance to their entry, after each assignment.
 *   method:    0 chooses, 1 tensor cores (tcgen05; K a multiple of 256),
 *              2 CUDA cores (FP32).
 *   m_out:     host, optional: m.
 * Synchronises the stream twice (to size the work, and to read the error
 * flag at the end).  Errors: GS_ERR_ARG (bad sizes, method 1 with K not a
 * multiple of 256, SH or centroid values outside binary16), GS_ERR_OOM,
 * GS_ERR_CUDA (includes a kernel pipeline that timed out).
 *
 * gs_vq_assign: one assignment of the quantised vectors to a given codebook
 * (device binary16 [K][C]); assign as above.  Synchronises once.
 *
 * gs_vq_pack: the compressed render layout.  quat16 [n][4], scale16 [n][2],
 * opacity16 [n] = rn16 of quat, scale, opacity (device FP32, activated
 * values); sh_row [n]: assign[i] for quantised surfels, K + (rank of i among
 * the kept surfels) otherwise; sh_table: the K codebook rows, then the kept
 * surfels' rn16 SH rows ([K + n][C] capacity, device).  *rows_out (host) =
 * K + number kept.  Synchronises once.  GS_ERR_ARG if a value leaves the
 * binary16 range or an assign entry is outside [0, K).
 *
 * gs_create_compressed_scene: a render-only scene over a compressed layout
 * (borrowed arrays as in gs_create_scene): mu FP32 [n][3]; quat binary16
 * [n][4] (8-byte aligned); scale binary16 [n][2] (4-byte aligned, activated);
 * opacity binary16 [n]; sh_row uint32 [n]; sh_table binary16 [sh_rows][C].
 * gs_render, gs_contribution and the server accept it and compute exactly as
 * on the FP32 scene whose values are the binary16 ones; gs_backward and
 * gs_densify_accumulate return GS_ERR_ARG.  Checks every sh_row against
 * sh_rows (synchronises `stream` once); GS_ERR_ARG when one is out of range. */
gs_status gs_vq_kmeans(int64_t n, int32_t sh_degree, const float* sh, const uint8_t* keep, int32_t K,
                       int32_t iters, const float* init_u, uint16_t* codebook, int32_t* assign, double* objective,
                       int32_t method, int64_t* m_out, void* stream);
gs_status gs_vq_assign(int64_t n, int32_t sh_degree, const float* sh, const uint8_t* keep, int32_t K,
                       const uint16_t* codebook, int32_t* assign, int32_t method, void* stream);
gs_status gs_vq_pack(int64_t n, int32_t sh_degree, const float* quat, const float* scale, const float* opacity,
                     const float* sh, const uint8_t* keep, const int32_t* assign, int32_t K,
                     const uint16_t* codebook, uint16_t* quat16, uint16_t* scale16, uint16_t* opacity16,
                     uint32_t* sh_row, uint16_t* sh_table, int64_t* rows_out, void* stream);

typedef struct {
  int64_t n;
  int32_t sh_degree;
  const float* mu;
  const uint16_t* quat;
  const uint16_t* scale;
  const uint16_t* opacity;
  const uint32_t* sh_row;
  const uint16_t* sh_table;
  int64_t sh_rows;
  gs_settings settings;
  gs_allocator allocator;
} gs_compressed_scene_desc;
gs_status gs_create_compressed_scene(gs_scene** out, const gs_compressed_scene_desc* desc, void* stream);

/* ---- Serving: continuous batching of forward renders ------------------
 * (the serving loop built on the rasterizer; the paper has no serving
 * component of its own.)
 * A server owns a worker thread, `max_slots` CUDA streams on the device
 * current at creation, and device buffers (per-surfel records, sort buffers,
 * tile lists) that stay resident between requests and grow on demand; their
 * total never exceeds `budget_bytes`.  Requests are queued in submission
 * order and admitted into free slots when their buffers fit the budget;
 * stages of different requests overlap on the device and the views whose
 * tile lists are ready are blended together by one persistent launch.  A
 * request that cannot fit even alone fails with GS_ERR_CAPACITY.  Results
 * equal gs_render's for the same scene and camera.
 *  alloc:  device allocator for the server's buffers (NULL: cudaMallocAsync).
 * Scenes are registered with gs_server_add_scene before requests name them
 * and must outlive the server; their parameters must not change while
 * requests are in flight. */
typedef struct gs_server gs_server;
typedef struct {
  int32_t scene;       /* id from gs_server_add_scene                        */
  gs_camera camera;    /* copied at submission                               */
  float* out;          /* device [GS_OUT_PLANES][H][W], caller-owned; written */
                       /* when gs_server_wait returns GS_OK                    */
  int32_t* n_contrib;  /* device [H][W] or NULL                              */
} gs_request;
typedef struct {
  int64_t completed, failed, queued, in_flight;
  int64_t batches, batched_views;   /* blend launches and views they carried */
  int64_t bytes_in_use;             /* resident device buffers               */
  double latency_p50_ms, latency_p99_ms, latency_mean_ms; /* submit to done  */
  int64_t pairs_evaluated, pairs_blended; /* blend work of the served views    */
} gs_server_stats_t;
gs_status gs_server_create(gs_server** out, size_t budget_bytes, int32_t max_slots,
                           const gs_allocator* alloc);
gs_status gs_server_add_scene(gs_server* server, gs_scene* scene, int32_t* scene_id);
/* Thread-safe.  Returns a ticket for gs_server_wait. */
gs_status gs_server_submit(gs_server* server, const gs_request* request, int64_t* ticket);
/* Blocks until the request is done (GS_OK), failed (its error), or
 * timeout_ms passed (GS_ERR_TIMEOUT; the ticket stays valid).  A finished
 * ticket is consumed. */
gs_status gs_server_wait(gs_server* server, int64_t ticket, int32_t timeout_ms);
/* Counters and latency percentiles of requests completed since the last
 * reset (reset != 0 clears them after reading). */
gs_status gs_server_stats(gs_server* server, gs_server_stats_t* out, int32_t reset);
/* Stops the worker after the work in flight; queued requests are dropped. */
gs_status gs_server_destroy(gs_server* server);

/* Diagnostics.
 * gs_kernel_launches: number of CUDA kernels this library has launched in
 *   this process (all entry points, all devices).
 * gs_profile_enable: when on, every launch of the kernel groups below is
 *   bracketed by CUDA events recorded on its own stream.
 * gs_profile_read: synchronises the recorded events of one group, returns
 *   their summed duration (ms) and count, and forgets them.  Groups:
 *   0 preprocess, 1 scan/sort/emit/ranges, 2 forward blend, 3 loss,
 *   4 backward blend, 5 preprocess backward, 6 densify/filter,
 *   7 trim contribution and pruning, 8 the vector-quantisation assignment
 *   kernel (tensor-core or CUDA-core). */
enum {
  GS_PROF_PREPROCESS = 0, GS_PROF_SORT = 1, GS_PROF_BLEND_FWD = 2, GS_PROF_LOSS = 3,
  GS_PROF_BLEND_BWD = 4, GS_PROF_PREPROCESS_BWD = 5, GS_PROF_DENSIFY = 6, GS_PROF_CONTRIB = 7,
  GS_PROF_VQ_ASSIGN = 8, GS_PROF_GROUPS = 9
};
uint64_t gs_kernel_launches(void);
gs_status gs_profile_enable(int32_t on);
gs_status gs_profile_read(int32_t group, double* total_ms, int64_t* launches);

/* Wait for `stream` with a bound: GS_ERR_TIMEOUT after timeout_ms. */
gs_status gs_sync(void* stream, int32_t timeout_ms);
const char* gs_last_error(void);
const char* gs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GS2D_H */
