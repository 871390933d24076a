/*
 * gs.h - C ABI of the tile-based differentiable Gaussian-splatting rasterizer.
 *
 * The rasterizer is the hot path of the 3D Gaussian Splatting method that
 * Mini-Splatting2 (arXiv 2411.12788) optimizes: Gaussians are projected to
 * 2-D by the local affine (EWA) approximation and coloured by spherical
 * harmonics (Sec. 3.1), depth-ordered per 16x16 tile, and alpha-blended front
 * to back (Eq. 1).  The forward pass also emits what the paper's
 * reorganisation and simplification read: the rendered index
 * i_max = argmax_i w_i and the midpoint depth d^mid_{i_max} (Eq. 2, Sec. 4.1),
 * the blended depth (Sec. 4.1), the per-Gaussian accumulated blending weight
 * I_i (Sec. 3.2; used for pruning, sampling and visibility, Sec. 4.2, 5.2)
 * and the maximum-contribution area S_i (Sec. 4.1, blur split).
 *
 * Conventions
 *  - All arrays named "device" live in GPU memory of the current device and
 *    are owned by the caller; the library never allocates or frees them.
 *    Workspaces are caller-allocated byte buffers whose sizes come from the
 *    *_workspace_size() queries; they must be 256-byte aligned.
 *  - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream) except gs_preprocess, which reads back one 8-byte
 *    count (the number of tile entries) and therefore synchronises `stream`.
 *    The read-back goes through one pinned, mapped host word per host thread
 *    (allocated on first use and kept), written by a kernel: no copy engine
 *    is involved, so large transfers on other streams do not delay it; the
 *    per-view constants are likewise passed to a kernel by value.
 *  - Every call returns a gs_status; arguments are validated on the host
 *    before any launch (GS_ERR_INVALID_ARG).  Device-side checks (entry
 *    overflow, a radix-sort look-back that exceeded its spin budget, and in
 *    the checked build, libgs_checked.so compiled with GS_CHECKED, any
 *    out-of-range index into an entry, item or output array) set a status
 *    word in the preprocess workspace that gs_device_status() reads.
 *  - Floating point is FP32 throughout.  Gaussian attributes are the
 *    activated values: linear scales, a (w,x,y,z) quaternion that need not be
 *    unit (it is normalised inside), opacity in (0,1), raw SH coefficients.
 *  - Camera space: p_c = R p + t, x right, y down, z forward; pixel (u, v)
 *    is sampled at its centre (u + 0.5, v + 0.5).
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_TILE 16          /* tile edge in pixels */
#define GS_MAX_VIEWS 64     /* views (or serving requests) per plan */
#define GS_MAX_SH_DEGREE 3

typedef enum gs_status {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1,   /* bad pointer, size, camera or degree */
  GS_ERR_CAPACITY = 2,      /* a workspace is smaller than required */
  GS_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  GS_ERR_TIMEOUT = 4,       /* a device-side wait exceeded its budget */
  GS_ERR_DEVICE_CHECK = 5   /* a device-side consistency check failed */
} gs_status;

/* Pinhole camera.  R is the row-major world->camera rotation. */
typedef struct gs_camera {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
} gs_camera;

/* Numeric conventions (defaults in brackets; gs_config_default fills them).
 *  znear     [0.2]   cull Gaussians with camera z <= znear
 *  lowpass   [0.3]   px^2 added to the diagonal of the 2-D covariance
 *  clamp     [1.3]   Jacobian evaluated at x/z, y/z clamped to +-clamp*tan(fov/2)
 *  alpha_max [0.99]  alpha = min(alpha_max, o * G)
 *  alpha_min [1/255] an entry with alpha < alpha_min is skipped
 *  t_min     [1e-4]  stop before the entry that would take T below t_min
 *  bg        [0,0,0] background, added as T_final * bg
 *  flags             GS_FLAG_* bits */
typedef struct gs_config {
  float znear, lowpass, clamp, alpha_max, alpha_min, t_min;
  float bg[3];
  uint32_t flags;
} gs_config;

/* gs_render_fwd / gs_render_bwd zero their accumulated outputs first (the
 * backward writes the attribute gradients instead of adding to them) */
#define GS_FLAG_ZERO_ACCUM 1u

/* gs_preprocess lists a Gaussian in the tiles met by the square of half-width
 * r = ceil(3 sqrt(lambda_max)) around its centre (lambda_max the larger
 * eigenvalue of the dilated 2-D covariance; a tile is met when the square
 * meets the rectangle of its pixel centres), the 3-sigma extent of the 3DGS
 * rasterizer the paper builds on (Sec. 3.1), instead of the tiles its exact
 * support q <= 2 ln(o / alpha_min) meets.  The per-pixel rule is unchanged,
 * so a pixel receives the Gaussian only inside the square's tiles: the
 * support is truncated there.  Must be the same in every call on one plan. */
#define GS_FLAG_EXTENT_3SIGMA 2u

/* gs_preprocess reads its mask as bits (see gs_preprocess): the per-view
 * visibility of many training views (Sec. 5.2) kept at one bit per
 * Gaussian. */
#define GS_FLAG_MASK_BITS 4u

/* Gaussian attributes, device, FP32, structure of arrays:
 *   means [n][3], scales [n][3], rotations [n][4] (w,x,y,z), opacities [n],
 *   sh [n][sh_coeffs][3] (band-major, m = -l..l, RGB innermost).
 * Only the first (sh_degree+1)^2 coefficients of each row are read. */
typedef struct gs_scene {
  const float* means;
  const float* scales;
  const float* rotations;
  const float* opacities;
  const float* sh;
  int64_t n;
  int32_t sh_degree;        /* 0..3 */
  int32_t sh_coeffs;        /* row length of sh, >= (sh_degree+1)^2 */
} gs_scene;

/* Host-side plan: the batch of views and the workspace layout.  Filled by
 * gs_plan_init (host only, no GPU work) and completed by gs_preprocess, which
 * stores the tile-entry count.  Items are (view, Gaussian) pairs numbered
 * item = view * n + gaussian; per-pixel outputs of view v start at
 * pixel_base[v] (row-major), the planar image of view v at 3 * pixel_base[v]. */
typedef struct gs_plan {
  int64_t n;
  int64_t n_items;
  int64_t total_pixels;
  int64_t n_entries;        /* set by gs_preprocess */
  int32_t n_views;
  int32_t total_tiles;
  int32_t sort_bits;        /* bits of the global tile id */
  int32_t n_pairs;          /* set by gs_preprocess: (item, tile row) pairs of the visible items'
                               row bands (sizes the tile-list builder of gs_bin_sort) */
  gs_camera cams[GS_MAX_VIEWS];
  int32_t tile_base[GS_MAX_VIEWS + 1];
  int64_t pixel_base[GS_MAX_VIEWS + 1];
} gs_plan;

/* Forward outputs, device.  image, final_T and n_contrib are required (the
 * backward pass reads image and n_contrib); the rest may be NULL.  The per-view
 * per-Gaussian arrays are indexed by item and ACCUMULATED (+=). */
typedef struct gs_fwd_outputs {
  float* image;             /* [3 * total_pixels] planar per view: c(x) + T bg (Eq. 1) */
  float* final_T;           /* [total_pixels] transmittance after the last blend */
  uint32_t* n_contrib;      /* [total_pixels] list position of the last blended entry + 1 */
  int32_t* imax;            /* [total_pixels] i_max (Gaussian index) or -1 (Eq. 2) */
  float* wmax;              /* [total_pixels] w_{i_max}, 0 if none */
  float* depth;             /* [total_pixels] d^mid of i_max (Eq. 2), 0 if none */
  float* depth_blend;       /* [total_pixels] sum_i w_i z_i (Sec. 4.1) */
  float* weight_sum;        /* [n_items] += sum over the view's pixels of w_i (Sec. 3.2) */
  uint32_t* max_area;       /* [n_items] += #pixels with i_max = i (S_i, Sec. 4.1) */
  uint64_t* weight_sum_fixed; /* [n_items], 8-byte aligned: += I_i in units of 2^-24.  Every
                               pixel's weight is rounded once to a multiple of 2^-24 and the
                               sums are integer, so the result does not depend on the order of
                               the atomic adds (bit-reproducible, unlike weight_sum) */
  float* depth_center;      /* [total_pixels] d^center = camera z of i_max's centre (the
                               alternative depth of Sec. 4.1), 0 if none */
  uint32_t* n_blended;      /* [total_pixels] nullable: number of entries blended at the pixel
                               (Eq. 1's terms with alpha >= alpha_min before the stop); the
                               positions before n_contrib that are not blended were skipped */
} gs_fwd_outputs;

/* Gradients, device, ACCUMULATED (+=) over views, same layouts as gs_scene;
 * d_sh has sh_coeffs columns (unused ones are left untouched).
 * d_mean2d_abs (nullable, [n]) += |dL/d mean2d| per view (3DGS densification
 * statistic).  weight_sum (nullable, [n_items]) += the accumulated blending
 * weight I_i of Sec. 3.2, the same quantity as gs_fwd_outputs.weight_sum,
 * collected during the backward pass: a training step can take I_i from here
 * and skip it in the forward pass; weight_sum_fixed likewise in fixed point
 * (bit-reproducible). */
typedef struct gs_grads {
  float* d_means;
  float* d_scales;
  float* d_rotations;
  float* d_opacities;
  float* d_sh;
  float* d_mean2d_abs;
  float* weight_sum;
  uint64_t* weight_sum_fixed; /* nullable, [n_items], 8-byte aligned: I_i collected in the
                               backward in the fixed point of gs_fwd_outputs.weight_sum_fixed */
} gs_grads;

/* ---- plan and sizes (host only) ------------------------------------- */
/* Host-side bookkeeping with no counterpart in the paper. */
void gs_config_default(gs_config* cfg);

/* Fills `plan` for n Gaussians seen by n_views cameras (host array).
 * Errors: GS_ERR_INVALID_ARG for n < 0, n_views outside 1..GS_MAX_VIEWS,
 * non-positive sizes or focal lengths, or more than 2^31 tiles or items. */
gs_status gs_plan_init(gs_plan* plan, int64_t n, const gs_camera* cams, int32_t n_views);

/* Bytes of the preprocess workspace (per-item projected state, depth sort,
 * scan, and the backward pass's per-item 2-D gradients). */
size_t gs_preprocess_workspace_size(const gs_plan* plan);

/* Bytes of the sort workspace for plan->n_entries entries (call after
 * gs_preprocess): keys and values double-buffered, tile ranges, radix
 * histograms and look-back state. */
size_t gs_bin_sort_workspace_size(const gs_plan* plan);

/* ---- the four hot-path calls ----------------------------------------- */

/* Per (view, Gaussian): cull (z <= znear, mask == 0, opacity < alpha_min),
 * covariance R(q) diag(s^2) R(q)^T, EWA projection J W Sigma W^T J^T +
 * lowpass I, conic, projected centre, SH colour max(0, sum sh Y + 0.5) in
 * the direction from the camera centre (Sec. 3.1), the midpoint-depth frame
 * (Sec. 4.1), and the exact number of touched tiles: tile T is touched iff
 * min over its pixel-centre rectangle of d^T conic d <= 2 ln(o / alpha_min)
 * (with GS_FLAG_EXTENT_3SIGMA: iff that rectangle meets the 3-sigma square).
 * Then sorts the items by the float32 depth of their centres (stable, ties
 * by item) and scans the tile counts in that order; stores the total in
 * plan->n_entries (one read-back through mapped host memory, synchronises
 * `stream`).
 * mask: device [n_items] bytes or NULL (view-dependent culling, Sec. 5.2);
 * with GS_FLAG_MASK_BITS in cfg->flags it is instead a bit mask of
 * n_views rows of ceil(n / 32) 32-bit words (4-byte aligned): Gaussian g of
 * view v is kept iff bit g % 32 of word v * ceil(n / 32) + g / 32 is set
 * (gs_pack_mask makes one from a byte mask).  cfg is read on the host. */
gs_status gs_preprocess(gs_plan* plan, const gs_scene* scene, const gs_config* cfg,
                        const uint8_t* mask, void* pre_ws, size_t pre_ws_bytes,
                        void* stream);

/* Packs a per-view visibility mask (the culling mask of Sec. 5.2) given as
 * bytes (device [n_views * n], non-zero = keep) into the bit mask
 * GS_FLAG_MASK_BITS reads: bits, device [n_views][ceil(n / 32)] 32-bit
 * words, 4-byte aligned, OVERWRITTEN (padding bits zero).  Asynchronous;
 * GS_ERR_INVALID_ARG for bad sizes or pointers. */
gs_status gs_pack_mask(const uint8_t* mask, int64_t n, int32_t n_views, uint32_t* bits, void* stream);

/* The tile binning of the rasterizer (Sec. 3.1): emits one (global tile id,
 * item) entry per touched tile in depth order, radix-sorts the entries by
 * tile id (stable, so each tile's list stays in
 * (depth, item) order) and computes each tile's [start, end) range.
 * Errors: GS_ERR_CAPACITY if sort_ws_bytes < gs_bin_sort_workspace_size. */
gs_status gs_bin_sort(const gs_plan* plan, void* pre_ws, void* sort_ws,
                      size_t sort_ws_bytes, void* stream);

/* Front-to-back alpha blending of every tile (Eq. 1) with alpha =
 * min(alpha_max, o G), skip alpha < alpha_min, stop before T (1 - alpha) <
 * t_min; writes the outputs listed in gs_fwd_outputs. */
gs_status gs_render_fwd(const gs_plan* plan, const gs_config* cfg, void* pre_ws,
                        const void* sort_ws, const gs_fwd_outputs* out, void* stream);

/* Gradients of a loss L with respect to the Gaussian attributes, given
 * dL/d image (device, [3 * total_pixels], planar like the image) and the
 * forward's image and n_contrib: for every blended entry l of a pixel,
 * dI/dc_l = w_l and dI/dalpha_l = T_l c_l - (I - F_l) / (1 - alpha_l) with
 * F_l the colour blended up to and including l (the derivative of Eq. 1),
 * then the chain rule through alpha = min(alpha_max, o G), the conic, the
 * projection and the SH colour.  The clamps pass no gradient (alpha at
 * alpha_max, colour below 0, the clamped Jacobian coordinate); the
 * thresholds are constants.  The scene must be the one passed to
 * gs_preprocess.  pre_ws is also written (its 2-D gradient scratch). */
gs_status gs_render_bwd(const gs_plan* plan, const gs_scene* scene, const gs_config* cfg,
                        void* pre_ws, const void* sort_ws, const float* dL_dimage,
                        const float* image, const uint32_t* n_contrib,
                        const gs_grads* grads, void* stream);

/* ---- allocation-free variant ------------------------------------------ */

/* No counterpart in the paper: an engineering variant of gs_bin_sort for
 * callers that cannot allocate device memory when they render (a host
 * application that owns all GPU memory and hands out fixed buffers, code
 * where an allocation could block or fail mid-frame).  It computes exactly
 * what gs_bin_sort computes, but the caller passes the outputs directly
 * (tile_ids and items: device [n_entries] uint32, 16-byte aligned; ranges:
 * device [total_tiles][2] uint32, [start, end) per tile) and the sort's scratch comes
 * from a fixed file-scope device array of GS_NOALLOC_SCRATCH_BYTES that every
 * GPU loading the library keeps until exit; nothing is allocated.
 *  - plan->n_entries above GS_NOALLOC_MAX_ENTRIES: GS_ERR_CAPACITY, nothing
 *    launched (use gs_bin_sort with a caller workspace instead).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *  - All calls share the array; each clears the parts that must start at
 *    zero, but calls that overlap on the GPU (other streams or threads) race.
 * pre_ws is the workspace of the gs_preprocess call that filled `plan`. */
#define GS_NOALLOC_MAX_ENTRIES (1 << 19)
#define GS_NOALLOC_SCRATCH_BYTES (5u << 20)
gs_status gs_bin_sort_noalloc(const gs_plan* plan, void* pre_ws, uint32_t* tile_ids,
                              uint32_t* items, uint32_t* ranges, void* stream);

/* ---- importance pruning (MSv2-D) -------------------------------------- */

/* Writable Gaussian attributes, device, same layout as gs_scene. */
typedef struct gs_scene_buf {
  float* means;
  float* scales;
  float* rotations;
  float* opacities;
  float* sh;
  int64_t n;                /* rows available */
  int32_t sh_degree;
  int32_t sh_coeffs;
} gs_scene_buf;

/* Bytes of the workspace gs_prune_select needs for n importances. */
size_t gs_prune_workspace_size(int64_t n);

/* Importance-based pruning of MSv2-D (Sec. 6.1): the importance of Gaussian
 * i is its accumulated blending weight I_i (Sec. 3.2; e.g. the weight_sum of
 * gs_render_fwd summed over views).  Writes to keep_idx (device [k]) the
 * indices of the k largest importances, ties broken towards the lower index,
 * in ascending order.  importance: device [n], non-negative floats (their bit
 * patterns are compared).  0 <= k <= n < 2^32; workspace from
 * gs_prune_workspace_size, 256-byte aligned.  Asynchronous. */
gs_status gs_prune_select(const float* importance, int64_t n, int64_t k, uint32_t* keep_idx,
                          void* ws, size_t ws_bytes, void* stream);

/* dst rows r = 0..k-1 <- src rows idx[r] of every attribute array (the
 * compaction of the pruned scene before the re-render, Sec. 6.1).
 * dst->n >= k, equal sh_coeffs. */
gs_status gs_gather_scene(const gs_scene* src, const uint32_t* idx, int64_t k,
                          const gs_scene_buf* dst, void* stream);

/* ---- identification of Gaussians (Sec. 4-5) ------------------------------ */

/* Flag bits written by gs_identify, per (view, Gaussian) item. */
#define GS_ID_BLUR 1u       /* G^blur (Sec. 4.1): S_i > theta_blur * H * W, blur-split candidate */
#define GS_ID_INTERSECT 2u  /* G^int (Sec. 4.3): S_i > 0, the i_max of at least one pixel */
#define GS_ID_VISIBLE 4u    /* V_i (Sec. 5.2): I_i above the view's keep-quantile threshold */
#define GS_ID_CRITICAL 8u   /* G^crit (Sec. 5.1): i_max of a pixel whose w_max is above the
                               view's keep-quantile threshold */

typedef struct gs_config_identify {
  float theta_blur;         /* 2e-4 (Sec. 4.1) */
  float keep_visible;       /* 0.99 keep quantile of the visibility threshold (Sec. 5.2) */
  float keep_critical;      /* 0.99 keep quantile of the critical threshold (Sec. 5.1) */
} gs_config_identify;

void gs_config_identify_default(gs_config_identify* out);

/* Bytes of the workspace gs_identify needs (256-byte aligned). */
size_t gs_identify_workspace_size(const gs_plan* plan);

/* Per-view selections of Gaussians from one forward pass over the plan's
 * views.  A keep quantile q over the M positive values of a view keeps the
 * ceil(q M) largest of them (q M formed in double), ties to the lower index;
 * the paper states the quantile only as "0.99" (Sec. 5.1, 5.2).
 *   weight_sum  device [n_items] I_i of each item (Sec. 3.2), non-negative
 *   max_area    device [n_items] S_i of each item (Sec. 4.1)
 *   imax, wmax  device [total_pixels] forward outputs of the same plan
 *   flags       device, n_items rounded up to a multiple of 4 bytes, 4-byte
 *               aligned; OVERWRITTEN with GS_ID_* bits per item
 *   visible_mask  device [n_items] or NULL: 1 where GS_ID_VISIBLE, else 0 (a
 *               mask for gs_preprocess: view-dependent culling, Sec. 5.2)
 *   counts      device [n_views][4] or NULL: per view, how many items carry
 *               BLUR, INTERSECT, VISIBLE, CRITICAL (overwritten)
 * Asynchronous; GS_ERR_INVALID_ARG for bad sizes, pointers, alignment or
 * configuration (quantiles outside [0, 1], negative theta). */
gs_status gs_identify(const gs_plan* plan, const gs_config_identify* cfg, const float* weight_sum,
                      const uint32_t* max_area, const int32_t* imax, const float* wmax,
                      uint8_t* flags, uint8_t* visible_mask, uint32_t* counts,
                      void* ws, size_t ws_bytes, void* stream);

/* Aggressive clone (Sec. 5.1): each Gaussian idx[r] (distinct indices)
 * becomes a pair at the same centre, rotation and SH with opacity
 * o' = 1 - sqrt(1 - o) and covariance o^2 (2 o' - o'^2 / sqrt(2))^-2 Sigma,
 * i.e. scales multiplied by o / (2 o' - o'^2 / sqrt(2)).  dst (rows >=
 * src->n + k, equal sh_coeffs, not overlapping src) receives src in rows
 * [0, n) with rows idx[r] replaced by the pair's first member and the second
 * member in row n + r.  Asynchronous. */
gs_status gs_clone_gaussians(const gs_scene* src, const uint32_t* idx, int64_t k,
                             const gs_scene_buf* dst, void* stream);

/* ---- sampling (Sec. 4.2, 4.3) ------------------------------------------ */

/* Bytes of the workspace gs_sample_gaussians needs for n Gaussians. */
size_t gs_sample_workspace_size(int64_t n);

/* Primitive sampling (Sec. 4.3): k Gaussians drawn without replacement with
 * probability proportional to the importance I_i (P_i = I_i / sum I), by
 * exponential clocks (Efraimidis and Spirakis): the caller draws
 * expo_i ~ Exp(1) (> 0), and the k largest keys I_i / expo_i (IEEE FP32
 * division) are kept, ties to the lower index.  Gaussians with I_i = 0 are
 * never drawn: K = min(k, #(I_i > 0)) indices are written to keep_idx
 * (device [k], ascending) and K to *k_out (device, nullable).
 *   importance, expo: device [n]; 0 <= n < 2^32; workspace 256-byte aligned.
 * Asynchronous. */
gs_status gs_sample_gaussians(const float* importance, const float* expo, int64_t n, int64_t k,
                              uint32_t* keep_idx, uint32_t* k_out, void* ws, size_t ws_bytes,
                              void* stream);

/* Bytes of the workspace gs_depth_points needs for the plan's largest view. */
size_t gs_depth_points_workspace_size(const gs_plan* plan);

/* Depth reinitialization seeds (Sec. 4.2): of the pixels of `view` that have
 * a maximum contributor (imax >= 0) and d^mid > 0, K = min(k, #such) are drawn
 * uniformly without replacement -- the K largest of the caller's uniform
 * draws u (device [H W] of that view, values in (0, 1]), ties to the lower
 * pixel index -- and reprojected: p_c = d ((x + 0.5 - cx) / fx,
 * (y + 0.5 - cy) / fy, 1), world point R^T (p_c - t), colour from the
 * target image.
 *   depth, imax: device [total_pixels], outputs of gs_render_fwd for the plan
 *   target: device planar [3][H][W] image of that view
 *   points, colours: device [k][3]; pixel_idx: device [k] (view-local pixel
 *   index y W + x, ascending); rows >= K are not written; K -> *k_out
 *   (device, nullable).
 * Asynchronous. */
gs_status gs_depth_points(const gs_plan* plan, int32_t view, const float* depth, const int32_t* imax,
                          const float* target, const float* u, int64_t k, float* points, float* colours,
                          uint32_t* pixel_idx, uint32_t* k_out, void* ws, size_t ws_bytes, void* stream);

/* ---- training-step helpers ------------------------------------------- */

/* Mean absolute error over `count` elements and its gradient (the L1 term
 * of the 3DGS photometric objective the paper trains with, Sec. 6.2):
 * *loss (device scalar) = mean |image - target|, dL_dimage = sign(image -
 * target) / count.  *loss is overwritten. */
gs_status gs_loss_l1(const float* image, const float* target, int64_t count,
                     float* loss, float* dL_dimage, void* stream);

/* Bytes of the workspace gs_loss_l1_ssim needs for the plan's views. */
size_t gs_loss_l1_ssim_workspace_size(const gs_plan* plan);

/* The 3DGS photometric objective (Sec. 6.2), fused with its gradient:
 * *loss = (1 - lambda) L1 + lambda (1 - SSIM), L1 = mean |image - target| and
 * SSIM = mean SSIM map, both over every pixel and channel of every view of the
 * plan (planar [3][H][W] per view, concatenated as gs_render_fwd writes
 * them).  SSIM per channel: 11x11 Gaussian window (sigma 1.5, normalised),
 * zero padding, C1 = 0.01^2, C2 = 0.03^2.  dL_dimage receives dL/dimage.
 * l1_out, ssim_out (device scalars, nullable) receive the two means.
 * 0 <= lambda <= 1; workspace from gs_loss_l1_ssim_workspace_size.
 * Asynchronous. */
gs_status gs_loss_l1_ssim(const gs_plan* plan, const float* image, const float* target, float lambda,
                          float* loss, float* dL_dimage, float* l1_out, float* ssim_out,
                          void* ws, size_t ws_bytes, void* stream);

/* ---- failure detection self-check ---------------------------------------- */

/* No counterpart in the paper: checks that the bounded device waits of the
 * sort and the scan give up instead of hanging.  Runs the onesweep look-back
 * and the exclusive scan's look-back for a tile whose predecessor never
 * publishes;
 * every wait runs out after its bound (about a second each), records the
 * timeout in a status word of its own, and the call returns GS_ERR_TIMEOUT
 * when both did, with the context still usable (GS_OK would mean a wait did
 * not detect the missing publisher).  scratch: device,
 * GS_SELFTEST_SCRATCH_BYTES bytes, 16-byte aligned.  Synchronous. */
#define GS_SELFTEST_SCRATCH_BYTES 4096u
gs_status gs_selftest_wait_timeout(void* scratch, size_t scratch_bytes, void* stream);

/* ---- inspection --------------------------------------------------------- */
/* Test and tooling access with no counterpart in the paper. */

/* Device pointers into a preprocess workspace after gs_preprocess, for tests
 * and tools (read-only use).  Entries of culled items (tiles == 0) are not
 * written and hold stale values. */
typedef struct gs_preprocess_view {
  const float* xy_tau_z;        /* [n_items][4] centre x, y, tau = 2 ln(o/alpha_min), z */
  const float* conic_o;         /* [n_items][4] A, B, C, opacity */
  const float* rgb;             /* [n_items][4] r, g, b, support half-extents (x, y) as two halves */
  const uint32_t* tiles;        /* [n_items] touched-tile count, 0 if culled */
  const uint32_t* rect;         /* [n_items][2] (tx0 | ty0 << 16, tx1 | ty1 << 16) */
  const uint32_t* sorted_items; /* [n_items] items in (float32 z, item) order, culled last */
  const uint32_t* offsets;      /* [n_items] exclusive scan of tiles in that order (written when
                                   gs_bin_sort sorts the entries by tile id, and by
                                   gs_bin_sort_noalloc) */
  const uint32_t* pair_offsets; /* [n_items] exclusive scan of the band sizes (tile rows ty1 - ty0
                                   + 1 of the visible items) in that order (written when
                                   gs_bin_sort builds the lists from (item, tile row) pairs) */
} gs_preprocess_view;
gs_status gs_inspect_preprocess(const gs_plan* plan, const void* pre_ws, gs_preprocess_view* out);

/* Device pointers into a sort workspace after gs_bin_sort. */
typedef struct gs_sort_view {
  const uint32_t* tile_ids;     /* [n_entries] global tile id, ascending; NULL when the lists were
                                   built from (item, tile row) pairs (the ranges give the tiles) */
  const uint32_t* items;        /* [n_entries] item of each entry */
  const uint32_t* ranges;       /* [total_tiles][2] [start, end) of each tile */
} gs_sort_view;
gs_status gs_inspect_sort(const gs_plan* plan, const void* sort_ws, gs_sort_view* out);

/* ---- timing --------------------------------------------------------------- */
/* Measurement support with no counterpart in the paper. */

/* Opt-in per-kernel timing: while enabled, every kernel launch of the library
 * is bracketed by CUDA events recorded on its launch stream (events come from
 * a pool created by the first enable; single-threaded use).  gs_timing_collect
 * waits for the recorded events, writes up to max_out per-kernel totals since
 * the previous collect (name, summed milliseconds, launches) and returns the
 * number of distinct kernels.  Names are static strings. */
typedef struct gs_kernel_time {
  const char* name;
  double ms;
  int64_t launches;
} gs_kernel_time;
gs_status gs_timing_enable(int on);
int gs_timing_collect(gs_kernel_time* out, int max_out);

/* ---- status ------------------------------------------------------------ */
/* Failure reporting with no counterpart in the paper. */

/* Reads (and clears) the device status word of a preprocess workspace;
 * synchronises `stream`.  Returns GS_OK, GS_ERR_TIMEOUT or GS_ERR_DEVICE_CHECK.
 * gs_preprocess also clears the word when it starts (and itself returns
 * GS_ERR_TIMEOUT for its own depth sort), so a frame's bin, render and
 * backward checks are read before the next gs_preprocess on the workspace. */
gs_status gs_device_status(const gs_plan* plan, void* pre_ws, void* stream);

const char* gs_status_string(gs_status s);

/* sizeof of the ABI structs, so bindings can check their layouts */
size_t gs_sizeof_plan(void);
size_t gs_sizeof_camera(void);
size_t gs_sizeof_config(void);
size_t gs_sizeof_scene(void);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
