/*
 * gsr.h -- C ABI of libgsr, the B300 (sm_103a) differentiable 3D-Gaussian
 * rasteriser behind Photo-SLAM-style photorealistic mapping
 * (arXiv 2311.16728, Sec. 3.3 "Photorealistic Mapping" and Sec. 3.4
 * "Gaussian-Pyramid-Based Learning").
 *
 * The problem every call serves (Sec. 3.3, Eq. 3 and Eq. 4): given hyper
 * primitives (position P, rotation r, scaling s, density sigma, SH colour),
 * a keyframe pose (R, t) with its intrinsics and a ground-truth image at a
 * pyramid level, compute the rendered image C(R, t), the photometric loss L
 * and dL/d(P, r, s, sigma, SH).  Poses are inputs only.
 *
 * Conventions shared by every entry point:
 *  - Every pointer named d_* or documented "device" is CUDA device memory
 *    owned by the caller.  No entry point allocates, frees or synchronises the
 *    device; scratch memory is a caller buffer sized by the matching
 *    *_workspace_size query.  The one exception is gsr_autotune, a set-up
 *    call outside the iteration: it creates and destroys CUDA events and
 *    synchronises the stream it times (never inside a stream capture).  Structs and scalars are read on the host during
 *    the call and may be freed on return.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and runs asynchronously; outputs are valid once the stream has
 *    reached that point.  Some kernels are launched with programmatic
 *    dependent launch (the mapping step's kernels after the binning): each
 *    waits (griddepcontrol.wait) for the work before it in the stream to
 *    complete before it touches memory, so stream order holds as for plain
 *    launches.  A caller's own kernel launched with programmatic stream
 *    serialization directly after one of ours may start early and must
 *    itself wait (cudaGridDependencySynchronize) before reading our
 *    outputs; plainly launched work, copies and events need nothing.
 *  - The return value is a gsr_status.  Argument errors are detected on the
 *    host before anything is enqueued (GSR_ERR_INVALID_ARG) and leave every
 *    output untouched.  GSR_ERR_CUDA means a launch failed; gsr_last_error()
 *    gives the message.  Data-dependent errors found on the device (too many
 *    (Gaussian, tile) pairs for the caller's capacity, a bounded wait that ran
 *    out) are OR-ed as bit flags (1 << code) into the caller's device status
 *    word d_status, which the caller zeroes and reads after synchronising.
 *  - Layout of the parameter store (SoA, 16-byte aligned float4 planes):
 *      mean_op  float4[n]      x, y, z, opacity logit
 *      quat     float4[n]      w, x, y, z (need not be normalised)
 *      logscale float4[n]      log s_x, log s_y, log s_z, pad (pad kept 0)
 *      sh       float4[12][n]  48 SH coefficients per Gaussian,
 *                              coefficient-major: float f of the 48 is SH
 *                              coefficient f / 3 of colour channel f % 3
 *    Gradients and Adam moments use the same layout.
 *  - Images are planar float32 C x H x W (C = 3 for colour).
 *  - Pixel (px, py) is sampled at integer coordinates; cx = W/2, cy = H/2
 *    makes pyramid intrinsics exact (level l divides fx, fy, cx, cy by 2^l).
 */
#ifndef GSR_H
#define GSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gsr_stream_t; /* binary-compatible with cudaStream_t */

typedef enum {
    GSR_OK = 0,
    GSR_ERR_INVALID_ARG = 1, /* bad pointer / size / alignment / enum     */
    GSR_ERR_CAPACITY = 2,    /* pair or workspace capacity too small       */
    GSR_ERR_CUDA = 3,        /* a CUDA launch or copy failed               */
    GSR_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up         */
    GSR_ERR_UNSUPPORTED = 5  /* a configuration this build does not serve  */
} gsr_status;

/* Read-only parameter store (layout above).  sh_degree in 0..3: only the
 * first (sh_degree + 1)^2 coefficients take part. */
typedef struct {
    const float *mean_op;
    const float *quat;
    const float *logscale;
    const float *sh;
    int64_t n;
    int32_t sh_degree;
} gsr_gaussians;

/* Writable buffers in the parameter-store layout: gradients (accumulated
 * with +=), parameters and Adam moments. */
typedef struct {
    float *mean_op;
    float *quat;
    float *logscale;
    float *sh;
} gsr_param_buffers;

/* Pinhole camera at one pyramid level.  R is the row-major world-to-camera
 * rotation and t the translation (x_cam = R x_world + t); fx, fy, cx, cy in
 * pixels of this level; width x height pixels (Sec. 3.2 pi_m projection). */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
} gsr_camera;

/* Screen tiling and the blend kernels' launch shape, all pure performance
 * choices (the autotuner's knobs): the rendered image does not depend on
 * them, since each Gaussian only reaches the pixels of its own 3-sigma pixel
 * box and the per-pixel arithmetic is the same in every shape.
 *  - tile_w x tile_h pixels per tile: tile_h even, tile_w a divisor or a
 *    multiple of 32, tile_w * tile_h a multiple of 64 and at most 1024.
 *  - batch_depth: depth-ordered records staged in shared memory per round by
 *    the blend kernels, a multiple of 32 up to 512, for the whole tile; 0 =
 *    each kernel's default: for 16 x 16 tiles every warp of the blends (one
 *    view or the batched window) stages its own 32 records a round (only
 *    those it can see; no barrier ties the warps of a tile together);
 *    elsewhere one record per thread.
 *  - bwd_threads: threads per tile of the backward blend; 0 = the default
 *    (64, four pixels a thread, for 16 x 16 tiles; tile_w * tile_h / 2
 *    otherwise), 128 for 16 x 16 tiles = two pixels a thread, else
 *    tile_w * tile_h / 2.  The forward always runs two pixels a thread. */
typedef struct {
    int32_t tile_w, tile_h;
    int32_t batch_depth;
    int32_t bwd_threads;
} gsr_tiling;

/* Per-Gaussian screen-space record written by gsr_preprocess (caller-owned,
 * n entries each, 16-byte aligned):
 *   xy_conic  float4  u, v, conic A, conic B   (Sigma'^-1 = [[A, B], [B, C]])
 *   c_op_box  float4  conic C, opacity, box x (u32 bits: x0 | x1 << 16),
 *                     box y (u32 bits: y0 | y1 << 16); inclusive pixel box
 *   rgb_depth float4  r, g, b (SH colour, clamped at 0), camera depth z
 *   ntiles    u32     tiles the box touches; 0 = culled
 *   uv_lo     float2  optional (NULL: not used): the residuals u64 - u and
 *                     v64 - v of the projected mean evaluated in FP64 (the
 *                     camera widened), so that u + uv_lo.x is the mean to
 *                     about 1e-6 pixel where the FP32 u alone is good to an
 *                     ulp of u (~1e-4 pixel at u ~ 1000).  u, v, the conic
 *                     and the box stay the FP32 decision chain's (keys and
 *                     culling are unchanged); when uv_lo is set, the blends
 *                     evaluate alpha at the FP64 position.  8-byte aligned.
 *   tile_order u32    optional (NULL: not used), one entry per tile of the
 *                     view: written by gsr_bin_sort with the tiles in
 *                     decreasing order of their pair counts (a permutation;
 *                     ties in any order), read by gsr_render_fwd,
 *                     gsr_blend_bwd and gsr_render_bwd, whose CTA b then
 *                     renders tile tile_order[b], so the longest lists start
 *                     first and the short ones fill the last wave.  The
 *                     image and gradients do not depend on it.  Entries of
 *                     tile_order must be valid tile indices (those outside
 *                     the view are skipped); set it only with buffers that
 *                     gsr_bin_sort filled for the same camera and tiling.
 *   tile_work u32     optional (NULL: not used; needs tile_order), one entry
 *                     per tile: gsr_bin_sort zeroes it and gsr_render_fwd
 *                     raises each entry to the tile's largest n_contrib (how
 *                     deep into its list the backward walks),
 *                     and gsr_blend_bwd / gsr_render_bwd first reorder
 *                     tile_order by it, deepest first, for their own launch.
 * Records of culled Gaussians (ntiles == 0) are left unwritten. */
typedef struct {
    float *xy_conic;
    float *c_op_box;
    float *rgb_depth;
    uint32_t *ntiles;
    float *uv_lo;
    uint32_t *tile_order;
    uint32_t *tile_work;
} gsr_proj;

/* Screen-space gradient buffer (caller-owned, 3 float4 per Gaussian):
 *   g0 = dL/d(u, v, A, B), g1 = dL/d(C, opacity, r, g), g2 = dL/d(b), 0, 0, 0
 * Written by gsr_render_bwd. */
typedef struct {
    float *g0, *g1, *g2;
} gsr_grad2d;

/* ---------------------------------------------------------------- */
/* Library facts                                                     */
/* ---------------------------------------------------------------- */

/* Version string, e.g. "gsr 0.1 sm_103a". */
const char *gsr_version(void);

/* Message of the last host-side error on the calling thread ("" if none). */
const char *gsr_last_error(void);

/* Copy the device status word to *h_status (synchronises `stream`). */
int32_t gsr_status_read(const int32_t *d_status, int32_t *h_status, gsr_stream_t stream);

/* Intrinsics of pyramid level `level` (Sec. 3.4, Eq. 5): fx, fy, cx, cy
 * divided by 2^level, width and height halved `level` times rounding up.
 * Host-only arithmetic on the struct; no device work. */
int32_t gsr_camera_at_level(const gsr_camera *in, int32_t level, gsr_camera *out);

/* ---------------------------------------------------------------- */
/* Hot path (Sec. 3.3): preprocess -> bin/sort -> render -> loss -> backward */
/* ---------------------------------------------------------------- */

/* EWA projection of every Gaussian (the splatting G of Eq. 3): camera-space
 * mean, near cull z > 0.2, 2D covariance J W Sigma W^T J^T + 0.3 I, its
 * inverse (conic), 3-sigma radius, clipped pixel box, tiles touched,
 * opacity = sigmoid(logit), colour = max(0, SH(view dir) + 0.5).  Cull,
 * depth, radius and box follow a fixed FP32 operation sequence so that tile
 * keys are reproducible bit for bit.  One thread per Gaussian. */
int32_t gsr_preprocess(const gsr_gaussians *g, const gsr_camera *cam, const gsr_tiling *tiling,
                       const gsr_proj *out, int32_t *d_status, gsr_stream_t stream);

/* Bytes of scratch gsr_bin_sort needs for n Gaussians, pair_capacity pairs
 * and the tiles of (cam, tiling). */
int32_t gsr_bin_sort_workspace_size(int64_t n, int64_t pair_capacity, const gsr_camera *cam,
                                    const gsr_tiling *tiling, size_t *bytes);

/* Tile binning (Sec. 3.3 "tile-based renderer").  Every visible Gaussian's
 * box tiles are candidates; a candidate survives when the Gaussian's largest
 * alpha over (tile x pixel box) reaches 0.5/255 -- half the per-pixel skip
 * threshold, so a dropped pair would never blend at any pixel and the image
 * is unchanged.  One (key, gid) pair is output per kept tile, key =
 * tile << 32 | bits(depth), sorted by key with equal keys in Gaussian order
 * (an in-house bucket sort by tile followed by a sort of each tile's segment
 * on depth and index); tile_ranges[2 t], [2 t + 1] = [begin, end) of tile t
 * (empty tiles [0, 0)).  keys/vals hold pair_capacity entries; the pair count
 * is written to *d_num_pairs.  If it exceeds pair_capacity, the
 * GSR_ERR_CAPACITY bit is set in *d_status, every range is empty and
 * *d_num_pairs is the capacity a retry needs; nothing is written out of
 * bounds.  A frame with 2^32 or more candidates sets GSR_ERR_UNSUPPORTED. */
int32_t gsr_bin_sort(const gsr_proj *proj, int64_t n, const gsr_camera *cam, const gsr_tiling *tiling,
                     uint64_t *keys, uint32_t *vals, int64_t pair_capacity, uint32_t *tile_ranges,
                     int64_t *d_num_pairs, void *workspace, size_t workspace_bytes, int32_t *d_status,
                     gsr_stream_t stream);

/* Forward render, Eq. 3 read as C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j)
 * + T_final * bg, front to back over each tile's depth-sorted list, with
 * alpha_i = min(0.99, sigma_i exp(-d^T Sigma'^-1 d / 2)), Gaussians skipped
 * where alpha < 1/255 or the pixel is outside their box, and the walk stopped
 * before a Gaussian that would take T below 1e-4.  Writes img (3 x H x W),
 * T_final (H x W) and n_contrib (H x W: 1 + position in the tile list of the
 * last Gaussian blended, 0 if none).  bg is a host array of 3 floats.
 * n_blended (H x W, may be NULL) receives the number of Gaussians blended
 * at each pixel (a work statistic; the render does not depend on it). */
int32_t gsr_render_fwd(const gsr_proj *proj, const uint32_t *vals, const uint32_t *tile_ranges,
                       const gsr_camera *cam, const gsr_tiling *tiling, const float *bg, float *img,
                       float *T_final, uint32_t *n_contrib, uint32_t *n_blended, gsr_stream_t stream);

/* Bytes of scratch gsr_loss_fwd_bwd needs for a C x H x W image. */
int32_t gsr_loss_workspace_size(int32_t C, int32_t H, int32_t W, size_t *bytes);

/* Eq. 4: L = (1 - lambda) mean|img - gt| + lambda (1 - mean SSIM(img, gt)),
 * SSIM per channel with an 11 x 11 Gaussian window (sigma 1.5), zero
 * padding, C1 = 0.01^2, C2 = 0.03^2, averaged over all pixels and channels;
 * the paper's lambda is 0.2 (Sec. 4.1).  Writes the scalar *d_loss and
 * dL_dimg (C x H x W).  The sum reductions run in a fixed order, so the
 * result is deterministic. */
int32_t gsr_loss_fwd_bwd(const float *img, const float *gt, int32_t C, int32_t H, int32_t W,
                         float lambda, float *d_loss, float *dL_dimg, void *workspace,
                         size_t workspace_bytes, gsr_stream_t stream);

/* Eq. 4 for a grayscale view (the monochrome stereo cameras of Sec. 4): the
 * loss of the render's luminance Y = 0.299 R + 0.587 G + 0.114 B (img, 3 x H
 * x W) against gt (1 x H x W), with dL_dimg (3 x H x W) = (0.299, 0.587,
 * 0.114) dL/dY.  Scratch: gsr_loss_luma_workspace_size. */
int32_t gsr_loss_luma_workspace_size(int32_t H, int32_t W, size_t *bytes);
int32_t gsr_loss_luma_fwd_bwd(const float *img, const float *gt, int32_t H, int32_t W, float lambda, float *d_loss,
                              float *dL_dimg, void *workspace, size_t workspace_bytes, gsr_stream_t stream);

/* Backward of Eq. 3 alone (the first half of gsr_render_bwd): zeroes grad2d
 * (n Gaussians) and accumulates the screen-space gradients into it. */
int32_t gsr_blend_bwd(const gsr_proj *proj, int64_t n, const uint32_t *vals, const uint32_t *tile_ranges,
                      const gsr_camera *cam, const gsr_tiling *tiling, const float *bg, const float *T_final,
                      const uint32_t *n_contrib, const float *dL_dimg, const gsr_grad2d *grad2d,
                      gsr_stream_t stream);

/* Backward of the projection alone (the second half of gsr_render_bwd):
 * chains grad2d to the parameter gradients, adding (+=) into `grads`, for
 * the Gaussians with ntiles > 0; densify statistics as in gsr_render_bwd. */
int32_t gsr_preprocess_bwd(const gsr_gaussians *g, const gsr_proj *proj, const gsr_camera *cam,
                           const gsr_tiling *tiling, const gsr_grad2d *grad2d, const gsr_param_buffers *grads,
                           float *densify_stat, float *densify_count, gsr_stream_t stream);

/* Camera pose gradient, for photometric pose refinement of a frame against
 * a fixed map (the camera (R, t) of the Eq. 3 projection as the variable).
 * From the screen-space gradients of the Gaussians with ntiles > 0 (grad2d
 * as gsr_blend_bwd leaves it), adds (+=) into d_pose (15 floats, device):
 *   d_pose[0..8]   dL/dR, row-major, R taken as a general 3 x 3 matrix;
 *   d_pose[9..11]  dL/dt;
 *   d_pose[12..14] dL/dphi for the left perturbation R <- exp([phi]x) R,
 *                  t <- exp([phi]x) t (a rotation about the camera centre);
 *                  the matching translation R, t <- R, t + rho has dL/drho =
 *                  dL/dt, so (dL/drho, dL/dphi) is the se(3) gradient.
 * The pose enters through the camera-space mean R mean + t, through the
 * R of the projected covariance J R Sigma R^T J^T and through the camera
 * centre -R^T t of the SH view direction.  The sums are FP32 atomics (their
 * order, and so the last bits, vary from run to run).  Parameter gradients
 * are not computed (gsr_preprocess_bwd does that). */
int32_t gsr_pose_bwd(const gsr_gaussians *g, const gsr_proj *proj, const gsr_camera *cam, const gsr_tiling *tiling,
                     const gsr_grad2d *grad2d, float *d_pose, gsr_stream_t stream);

/* gsr_preprocess_bwd that stores (=) instead of adding: the gradients of the
 * Gaussians with ntiles > 0 are replaced, all others are left as they are.
 * For callers whose gradients are zero before the pass (an optimiser step
 * that zeroes them, as gsr_adam_step does), it saves reading them back. */
int32_t gsr_preprocess_bwd_store(const gsr_gaussians *g, const gsr_proj *proj, const gsr_camera *cam,
                                 const gsr_tiling *tiling, const gsr_grad2d *g2d, const gsr_param_buffers *grads,
                                 float *densify_stat, float *densify_count, gsr_stream_t stream);

/* Backward of Eq. 3 then of the projection.  Replays each pixel back to
 * front from T_final and n_contrib, recovering T_i = T_{i+1} / (1 - alpha_i)
 * instead of storing per-pixel lists; per-Gaussian screen-space gradients are
 * pre-reduced across each warp with shuffles before the global atomics into
 * grad2d (zeroed by this call).  Then chains them, per Gaussian, to mean
 * (through the projection, the Jacobian and the SH view direction),
 * quaternion (through its normalisation), log-scale, opacity logit and SH,
 * ADDING (+=) into `grads` so several views accumulate.  dL_dimg is
 * 3 x H x W.  If densify_stat is not NULL, |dL/d(u, v)| of each visible
 * Gaussian, with (u, v) in normalised device coordinates (pixels scaled by
 * 2 / W, 2 / H: the 3DGS densification statistic), is added to
 * densify_stat[gid] and 1 to densify_count[gid]. */
int32_t gsr_render_bwd(const gsr_gaussians *g, const gsr_proj *proj, const uint32_t *vals,
                       const uint32_t *tile_ranges, const gsr_camera *cam, const gsr_tiling *tiling,
                       const float *bg, const float *T_final, const uint32_t *n_contrib,
                       const float *dL_dimg, const gsr_grad2d *grad2d, const gsr_param_buffers *grads,
                       float *densify_stat, float *densify_count, gsr_stream_t stream);

/* Allocation-free variant of gsr_loss_fwd_bwd, for callers that cannot
 * allocate device memory at the point where they evaluate the loss -- for
 * example code that runs while a stream is being captured in the global
 * capture mode (where cudaMalloc is an error), or a host application that
 * owns every allocation itself and hands this library only its images.
 * There is no counterpart in the paper: it is a packaging of Eq. 4.
 *
 * Computes exactly what gsr_loss_fwd_bwd computes (same kernels), but its
 * scratch lives in one fixed array in device memory that the library defines
 * (29.6 MB).  The array is allocated on a device when the library's loss
 * module is first loaded there (CUDA loads modules lazily: the first call on
 * that device of any loss entry point, this one or gsr_loss_fwd_bwd /
 * gsr_loss_luma_fwd_bwd, or the address lookup below) and is held until the
 * process exits.  Limits: C * H * W <= 2,457,600 values (a 3 x 1200 x 680
 * frame fits) and at most 16,384 blocks of 32 x 32 pixels summed over
 * channels; larger images return GSR_ERR_CAPACITY with a message and enqueue
 * nothing.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and caches it for
 * the process: make that first call, and so the module load, before any
 * stream capture, and do not use this entry point across a cudaDeviceReset
 * (or any other teardown of the device's primary context) in the same
 * process, after which the cached address is stale.  It never calls
 * cudaMalloc or cudaFree.  All calls on a device share the array and it keeps
 * the last call's contents; every entry a call reads is written earlier in
 * the same call, so nothing needs clearing between calls.  Calls whose work
 * overlaps on the GPU -- on different streams, or from different host
 * threads -- race on it and must be serialised by the caller. */
int32_t gsr_loss_fwd_bwd_static(const float *img, const float *gt, int32_t C, int32_t H, int32_t W,
                                float lambda, float *d_loss, float *dL_dimg, gsr_stream_t stream);

/* ---------------------------------------------------------------- */
/* Batched Gaussian-pyramid window (Sec. 3.4, Eq. 5)                 */
/* ---------------------------------------------------------------- */
/* Eq. 5 supervises pyramid level l with GP^l(I_gt), one level after the
 * other.  These calls evaluate the levels of a whole window of keyframes in
 * one iteration instead: views v = 0 .. nviews - 1 (nviews <= 64), each a
 * (keyframe, level) camera with its GP^l image, L = sum_v weight_v L_v and a
 * gradient equal to the sum of the single-view gradients.  Per-view records
 * are stored view-major: record r = v n + i is Gaussian i seen from view v
 * (the proj arrays hold nviews x n entries), and tiles are numbered view
 * after view. */

/* Projects every Gaussian into every view (parameters read once). */
int32_t gsr_batched_preprocess(const gsr_gaussians *g, const gsr_camera *cams, int32_t nviews,
                               const gsr_tiling *tiling, const gsr_proj *out, gsr_stream_t stream);

/* gsr_bin_sort over all views' records (n_per_view each); tile ranges for the
 * sum over views of their tiles.  Workspace: gsr_bin_sort_workspace_size with
 * n = n_per_view x nviews.  With `compact` (may be NULL; arrays of
 * n_per_view x nviews entries) the records of the visible list are first
 * gathered in index order into compact->xy_conic, c_op_box, rgb_depth (the
 * c-th visible record at position c), compact->ntiles[r] receives record r's
 * position c (for records with proj->ntiles[r] > 0), and the pairs' values are
 * these positions: the window's later passes then read records and
 * accumulate gradients in dense arrays (the order of the pairs is the same).
 * proj->tile_order (optional) receives all views' tiles (window numbering)
 * by decreasing pair count. */
int32_t gsr_batched_bin_sort(const gsr_proj *proj, int64_t n_per_view, const gsr_camera *cams, int32_t nviews,
                             const gsr_tiling *tiling, uint64_t *keys, uint32_t *vals, int64_t pair_capacity,
                             uint32_t *tile_ranges, int64_t *d_num_pairs, const gsr_proj *compact, void *workspace,
                             size_t workspace_bytes, int32_t *d_status, gsr_stream_t stream);

/* Bytes of scratch for gsr_batched_iterate over these views. */
int32_t gsr_batched_iterate_workspace_size(const gsr_camera *cams, int32_t nviews, size_t *bytes);

/* ONE persistent cooperative launch over the whole window: forward blend of
 * every (view, tile), both SSIM passes of every (view, channel, 32 x 32
 * block), the per-view losses (d_losses[v]), dL_dimg[v] = weight_v dL_v/dI_v,
 * and the backward blend of every (view, tile), accumulating into grad2d
 * (one entry per record that the pairs' values index: proj are the records
 * the binning's values refer to, the compact ones when it gathered them;
 * must be zero on entry -- gsr_batched_preprocess_bwd
 * leaves it zero).  Work is pulled from atomic queues so uneven resolutions
 * balance; the phases are separated by grid-wide barriers whose waits are
 * bounded (about a second): a wait that gives up sets GSR_ERR_TIMEOUT in
 * *d_status and the launch winds down.  img, T_final, n_contrib, gt, dL_dimg
 * are arrays of nviews device pointers (host arrays); weights (host, may be
 * NULL = all 1).  Tiles must hold 256 pixels (16 x 16, 32 x 8 or 8 x 32).
 * With proj->tile_order set (by gsr_batched_bin_sort, window numbering) the
 * blend phases take their queue items in that order, longest lists first.
 * The last 256 bytes of the workspace hold the launch's queue and barrier
 * words; its bytes 64 .. 95 receive four uint64 global-timer stamps (ns) taken
 * by block 0 at entry and after each of the three barriers (phase split). */
int32_t gsr_batched_iterate(const gsr_proj *proj, const uint32_t *vals, const uint32_t *tile_ranges,
                            const gsr_camera *cams, int32_t nviews, const gsr_tiling *tiling, const float *bg,
                            float *const *img, float *const *T_final, uint32_t *const *n_contrib,
                            const float *const *gt, float *const *dL_dimg, const float *weights, float lambda,
                            float *d_losses, const gsr_grad2d *grad2d, void *workspace, size_t workspace_bytes,
                            int32_t *d_status, gsr_stream_t stream);

/* Chains every view's screen-space gradient into `grads` (+=, atomically)
 * and zeroes grad2d again.  Views that are exact power-of-two scalings of one
 * camera (the pyramid levels of a keyframe: same pose, fx, fy, cx, cy, width
 * and height all scaled by 2^-k) are merged before the chain rule, which then
 * runs once per (Gaussian, keyframe): u, v scale by 2^-k, the dilated
 * covariance is 4^-k M + 0.3 I, and opacity and colour are shared.
 * touched (n u32, may be NULL) receives 1 for every Gaussian some view saw,
 * else 0: the flags gsr_adam_step_touched takes.  proj gives the records'
 * visibility (ntiles); with `compact` (as passed to gsr_batched_bin_sort)
 * the conics and grad2d are read at the compact positions. */
int32_t gsr_batched_preprocess_bwd(const gsr_gaussians *g, const gsr_proj *proj, const gsr_proj *compact,
                                   const gsr_camera *cams, int32_t nviews, const gsr_tiling *tiling,
                                   const gsr_grad2d *grad2d, const gsr_param_buffers *grads, uint32_t *touched,
                                   gsr_stream_t stream);

/* ---------------------------------------------------------------- */
/* Default initialisation of new primitives (Sec. 3.3.1)             */
/* ---------------------------------------------------------------- */
/* Photo-SLAM creates primitives at inactive ORB keypoints (geometry-based
 * densification, Sec. 3.3.1) without stating their initial shape.  The
 * default (3D Gaussian splatting's convention; the learned initialiser's
 * fallback) writes Gaussians offset .. offset + M - 1 of the map (n Gaussians,
 * planes of n entries):
 *   mean      = R^T (d K^-1 [u v 1]^T - t) for keypoint m = keypoints[5 m ..]
 *               = (u, v, d, log keypoint scale, angle) in camera `cam`
 *   log-scale = log sqrt(mean squared distance to the 3 nearest other map
 *               points) on all axes (floored at 1e-7 m^2; 1e-4 m^2 when the
 *               map holds no other point; every map mean takes part)
 *   rotation  = (1, 0, 0, 0), opacity logit = logit(0.1)
 *   SH        = DC (I(p) - 0.5) / Y_00 at the keypoint's nearest pixel p
 *               (half up, clamped) of img0 (planar 3 x H x W), others 0.
 * Brute-force neighbour search (M x n distances).  Scratch from the caller:
 * gsr_default_init_workspace_size. */
int32_t gsr_default_init_workspace_size(int64_t M, int64_t n, size_t *bytes);
int32_t gsr_default_init(const float *img0, int32_t W, int32_t H, const float *keypoints, int64_t M,
                         const gsr_camera *cam, const gsr_param_buffers *map, int64_t n, int64_t offset,
                         void *workspace, size_t workspace_bytes, gsr_stream_t stream);

/* ---------------------------------------------------------------- */
/* Gradient-driven densification and pruning (Sec. 3.3.1)           */
/* ---------------------------------------------------------------- */
/* Photo-SLAM splits or clones primitives with large loss gradients, as 3D
 * Gaussian splatting does, and drops nearly transparent ones.  Thresholds
 * (FP32; decisions are exact comparisons on FP32 values):
 *   grad_thr       on g_i = stat_i / count_i, the mean |dL/d(u, v)| in
 *                  normalised device coordinates that the chain rule
 *                  accumulates (densify_stat / densify_count);
 *   logit_min      prune when the opacity logit is below it;
 *   logscale_split split (not clone) when the largest log-scale is above it;
 *   shrink         log of the scale divisor of split children (log 1.6). */
typedef struct {
    float grad_thr, logit_min, logscale_split, shrink;
} gsr_densify_config;

int32_t gsr_densify_workspace_size(int64_t n, size_t *bytes);

/* One densification step of n Gaussians (params, Adam moments m, v) into a
 * second store of cap Gaussians (out_params, out_m, out_v; must not alias the
 * inputs), in input order: prune (or padding: a zero quaternion) -> nothing; keep -> a copy; clone -> a copy
 * and a second copy with zero moments; split -> two children with zero
 * moments, mean mu + R(q) (s * eps_k) (eps: n x 6 floats, two standard normal
 * 3-vectors per Gaussian, supplied by the caller), log-scale - shrink, rest
 * copied.  *d_n_out (device) receives the output count; the tail [n_out, cap)
 * becomes inert padding (all zero: a zero quaternion is never visible).  If
 * n_out > cap, GSR_ERR_CAPACITY is set in *d_status, *d_n_out holds the
 * count a retry needs and the outputs are incomplete. */
int32_t gsr_densify(const gsr_param_buffers *params, const gsr_param_buffers *m, const gsr_param_buffers *v,
                    int64_t n, const float *stat, const float *count, const float *eps,
                    const gsr_densify_config *cfg, const gsr_param_buffers *out_params,
                    const gsr_param_buffers *out_m, const gsr_param_buffers *out_v, int64_t cap, int64_t *d_n_out,
                    void *workspace, size_t workspace_bytes, int32_t *d_status, gsr_stream_t stream);

/* ---------------------------------------------------------------- */
/* Learned initialiser (tensor-core MLP)                             */
/* ---------------------------------------------------------------- */

/* BF16 GEMM on the tcgen05 tensor cores with an FP32 accumulator in tensor
 * memory: D = A B^T, A [M x K] and B [N x K] row-major BF16 with K
 * contiguous (row strides lda, ldb elements, multiples of 8, base pointers
 * 16-byte aligned); M % 128 == 0, N % 64 == 0, K % 64 == 0 (callers pad).
 * Epilogue, applied in this order to each FP32 element (n = column, m = row):
 * += bias[n] (if bias), max(., 0) (if relu), zeroed where mask[m * ldm + n]
 * (BF16) is not positive (if mask).  Outputs (any subset, at least one):
 * out_bf16[m * ldo + n] (BF16, round to nearest even), out_bf16_t[n * ldt + m]
 * (transposed BF16), out_f32[m * ldf + n] (FP32, 16-byte aligned, ldf % 4 ==
 * 0; added with atomics when atomic_f32), colsum[n] += sum over rows
 * m < valid_rows (FP32 atomics).  ksplit > 1 splits K over that many CTAs per
 * output tile and needs an atomic FP32 output and no element-wise epilogue.
 * A tensor-core wait that gives up sets the GSR_ERR_TIMEOUT bit in *d_status.
 * Used by the MLP calls below; exposed so it can be checked on its own. */
int32_t gsr_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, int32_t M, int32_t N, int32_t K,
                      const float *bias, int32_t relu, const void *mask, int32_t ldm, void *out_bf16, int32_t ldo,
                      void *out_bf16_t, int32_t ldt, float *out_f32, int32_t ldf, int32_t atomic_f32, float *colsum,
                      int64_t valid_rows, int32_t ksplit, int32_t *d_status, gsr_stream_t stream);

/* MLP weights (caller-owned device memory).  FP32 masters, row-major:
 * W1 [256 x 2368] (inputs padded from 2308 to 2368 with zero columns), b1
 * [256], W2 [256 x 256], b2 [256], W3 [64 x 256] (56 outputs + 8 zero rows),
 * b3 [64]; BF16 working copies W1h (as W1), W2h (as W2), W2hT (W2
 * transposed), W3h (as W3), W3hT (W3 transposed, [256 x 64]).  The same
 * struct holds the Adam moments, where only the FP32 pointers are used. */
typedef struct {
    float *W1, *b1, *W2, *b2, *W3, *b3;
    void *W1h, *W2h, *W2hT, *W3h, *W3hT;
} gsr_mlp_weights;

/* Bytes of scratch for a batch padded to Mpad rows (Mpad % 128 == 0). */
int32_t gsr_mlp_workspace_size(int64_t Mpad, size_t *bytes);

/* Writes the BF16 copies of the FP32 master weights (after initialising or
 * loading them). */
int32_t gsr_mlp_sync_weights(const gsr_mlp_weights *w, gsr_stream_t stream);

/* Input rows of the initialiser (the patches of Sec. 3.3.1's densification
 * keypoints): for keypoint m (keypoints[5 m ..] = u, v at level 0, depth,
 * log keypoint scale, angle) row m of x (BF16 [Mpad x 2368]) is the 16 x 16
 * RGB patch of each of the three pyramid levels around (u, v) / 2^l (nearest
 * pixel, clamped; index l * 768 + (16 row + col) * 3 + channel), then depth,
 * log scale, cos, sin of the angle, then zeros; rows >= M are zero.  Level l
 * is a planar 3 x H_l x W_l image with W_l, H_l halved l times rounding up.
 * xT (may be NULL) receives the transpose [2368 x Mpad] for training. */
int32_t gsr_patch_gather(const float *level0, const float *level1, const float *level2, int32_t W0, int32_t H0,
                         const float *keypoints, int64_t M, int64_t Mpad, void *x, void *xT, gsr_stream_t stream);

/* y [Mpad x 64] FP32 = W3 relu(W2 relu(W1 x + b1) + b2) + b3 on the tensor
 * cores (BF16 operands, FP32 accumulation; hidden activations rounded to
 * BF16). */
int32_t gsr_mlp_forward(const gsr_mlp_weights *w, const void *x, int64_t Mpad, float *y, void *workspace,
                        size_t workspace_bytes, int32_t *d_status, gsr_stream_t stream);

/* One training step on M valid rows: forward, L = sum_{m < M, j < 56}
 * out_weight[j] (y - target)^2 / M into *d_loss, backward by the five
 * tensor-core GEMMs (weight gradients split over the batch), then Adam
 * (step t = *d_step + 1, bias-corrected) on every FP32 master with m and v
 * as moments, refreshed BF16 copies, and *d_step += 1.  target is FP32
 * [Mpad x 64]; y receives the forward output. */
int32_t gsr_mlp_train_step(const gsr_mlp_weights *w, const gsr_mlp_weights *m, const gsr_mlp_weights *v,
                           const void *x, const void *xT, const float *target, const float *out_weight, int64_t M,
                           int64_t Mpad, float lr, float beta1, float beta2, float eps, int32_t *d_step,
                           float *d_loss, float *y, void *workspace, size_t workspace_bytes, int32_t *d_status,
                           gsr_stream_t stream);

/* Addresses, inside a training workspace for Mpad rows, of the FP32
 * gradients of the last gsr_mlp_train_step (valid until the next step
 * clears them): W1 [256 x 2368], b1, W2 [256 x 256], b2, W3 TRANSPOSED
 * [256 x 64], b3 [64]; the BF16 pointers are set to NULL.  Host-only. */
int32_t gsr_mlp_gradients(void *workspace, int64_t Mpad, gsr_mlp_weights *grads);

/* Training targets for keypoints whose primitive is known (gids[m]): log-scale
 * minus log(depth / fx), rotation in the camera frame (unit quaternion with
 * w >= 0), opacity logit, the 48 SH coefficients; columns 56..63 zero.  With
 * `base` (FP32 [Mpad x 64], may be NULL) the row minus base's row is written
 * (the initialiser learns a correction of a base initialisation).  Rows
 * M .. Mpad - 1 are zeroed. */
int32_t gsr_mlp_encode_targets(const gsr_gaussians *g, const uint32_t *gids, const float *keypoints, int64_t M,
                               int64_t Mpad, const gsr_camera *cam, const float *base, float *target,
                               gsr_stream_t stream);

/* Inverse of the encoding applied to y + base (base may be NULL): writes
 * Gaussians offset .. offset + M - 1 of a store of n Gaussians, the mean
 * back-projected from the keypoint at its depth (R^T (depth K^-1 [u v 1] -
 * t)). */
int32_t gsr_mlp_decode(const float *y, const float *base, const float *keypoints, int64_t M, const gsr_camera *cam,
                       const gsr_param_buffers *out, int64_t n, int64_t offset, gsr_stream_t stream);

/* ---------------------------------------------------------------- */
/* Optimiser, pyramid and metrics                                    */
/* ---------------------------------------------------------------- */

/* Learning rates per parameter group (the paper's optimiser is plain SGD
 * with a fixed rate, Sec. 4.1; this is its Adam variant). */
typedef struct {
    float lr_mean, lr_opacity, lr_quat, lr_scale, lr_sh;
    float beta1, beta2, eps;
} gsr_adam_config;

/* One fused Adam step over all n Gaussians' 60-float records (the log-scale
 * pad has zero gradient and never moves): m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 * with t = *d_step + 1 (FP32; the square root and the division use the fast
 * reciprocal square root and reciprocal, a few 1e-7 relative error on the
 * update), then zeroes the gradients and increments *d_step (device int32)
 * so that a captured graph can replay it. */
int32_t gsr_adam_step(const gsr_param_buffers *params, const gsr_param_buffers *grads,
                      const gsr_param_buffers *m, const gsr_param_buffers *v, int64_t n,
                      const gsr_adam_config *cfg, int32_t *d_step, gsr_stream_t stream);

/* gsr_adam_step for gradients that are zero wherever touched[i] == 0 (n
 * flags, device): such Gaussians' gradients are neither read nor rewritten
 * (their moments decay and their parameters move as Adam prescribes for a
 * zero gradient), which saves a quarter of the step's HBM bytes for every
 * Gaussian the iteration did not see.  A one-view iteration passes its
 * proj.ntiles (non-zero exactly for the Gaussians whose gradient it wrote);
 * the batched window passes the flags gsr_batched_preprocess_bwd writes. */
int32_t gsr_adam_step_touched(const gsr_param_buffers *params, const gsr_param_buffers *grads,
                              const gsr_param_buffers *m, const gsr_param_buffers *v, int64_t n,
                              const gsr_adam_config *cfg, const uint32_t *touched, int32_t *d_step,
                              gsr_stream_t stream);

/* ---------------------------------------------------------------- autotuner */

/* Actions of the autotuner's callback. */
enum { GSR_AUTOTUNE_SETUP = 0, GSR_AUTOTUNE_STEP = 1, GSR_AUTOTUNE_RELEASE = 2 };

/* Callback of gsr_autotune: for candidate `candidate`, SETUP builds its
 * state (and may check that it renders what the others render), STEP
 * enqueues one step of it on the stream given to gsr_autotune, RELEASE frees
 * its state.  Returns GSR_OK, or an error code that stops the tuning. */
typedef int32_t (*gsr_autotune_fn)(int32_t candidate, int32_t action, void *ctx);

/* Timing driver of the tiling autotuner (the tile shape, which fixes the
 * staging batch and the threads per tile, is a pure performance choice: the
 * image does not depend on it).  For each of ncand candidates in order:
 * SETUP, `warmup` STEPs, a synchronisation, then `steps` STEPs each
 * bracketed by CUDA events on `stream`, then RELEASE.  ms[c] (host, ncand
 * floats) = the median step time of candidate c in milliseconds; *best (host)
 * = the fastest candidate.  Unlike every other entry point this one
 * synchronises `stream` (after the warm-up and after the timed steps, to
 * read the events) and creates its own events: call it outside any stream
 * capture.  A callback error or a CUDA error stops the run
 * (after the failing candidate's RELEASE when its SETUP succeeded), is
 * returned, and leaves *best = -1. */
int32_t gsr_autotune(int32_t ncand, gsr_autotune_fn fn, void *ctx, int32_t warmup, int32_t steps,
                     gsr_stream_t stream, float *ms, int32_t *best);

/* ---------------------------------------------------------------- map order */

/* Bytes of scratch for gsr_spatial_order over n Gaussians. */
int32_t gsr_spatial_order_workspace_size(int64_t n, size_t *bytes);

/* Spatial order of the map store (maintenance, outside the iteration):
 * perm[i] (n uint32, device) = the index of the Gaussian that goes to place
 * i when the Gaussians are sorted by the 30-bit Morton code of their means
 * (each coordinate quantised to 10 bits over the box [lo, hi], host float[3],
 * clamped; the three coordinates' bits interleaved), equal codes by index.
 * With the store in this order the Gaussians a warp handles are spatial
 * neighbours, which keeps the per-Gaussian kernels' visibility decisions
 * coherent within a warp and their reads of visible Gaussians contiguous; it
 * changes no result except the order of exactly equal depths.  n < 2^32. */
int32_t gsr_spatial_order(const gsr_gaussians *g, const float *lo, const float *hi, uint32_t *perm,
                          void *workspace, size_t workspace_bytes, gsr_stream_t stream);

/* dst entry i = src entry perm[i] for every plane of n Gaussians' buffers
 * (parameters, gradients or Adam moments; all 12 SH planes); src and dst
 * must not overlap. */
int32_t gsr_permute(const gsr_param_buffers *src, const gsr_param_buffers *dst, const uint32_t *perm, int64_t n,
                    gsr_stream_t stream);

/* One Gaussian-pyramid step down (Sec. 3.4, Eq. 5 GP^l): separable binomial
 * [1 4 6 4 1]/16 blur with reflect-101 borders, keeping even pixels.
 * in is C x H x W, out is C x ceil(H/2) x ceil(W/2). */
int32_t gsr_pyramid_down(const float *in, int32_t C, int32_t H, int32_t W, float *out,
                         gsr_stream_t stream);

/* Bytes of scratch gsr_psnr needs for `count` values. */
int32_t gsr_psnr_workspace_size(int64_t count, size_t *bytes);

/* PSNR (Sec. 4.1 metric) of img clamped to [0, 1] against gt, peak 1:
 * 10 log10(1 / MSE), written to *d_psnr (device float); FP64 sum in a fixed
 * order. */
int32_t gsr_psnr(const float *img, const float *gt, int64_t count, float *d_psnr, void *workspace,
                 size_t workspace_bytes, gsr_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GSR_H */
