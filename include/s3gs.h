/*
 * s3gs.h -- C ABI of the GB300 (sm_103a) differentiable Gaussian-splatting
 * rasteriser: the data-parallel hot path of S3PO-GS.
 *
 * The renderer implements the paper's statement of the problem:
 *   render(G, K, T) -> rgb (Sec. 3.1, Eq. 2), depth (Sec. 3.2.1, Eq. 3),
 *                      accumulated alpha (1 - final transmittance of Eq. 2/3),
 *                      pointmap X^r = K^-1 [iD, jD, D] (Eq. 4/5);
 *   backward(dL/d outputs) -> dL/d(means, log-scales, quaternions, opacity
 *                      logits, colour/SH coefficients) (Sec. 3.1: "optimize all
 *                      Gaussian parameters") and dL/d(camera twist) (Sec. 3.2.2,
 *                      Eq. 11, pose linearised in se(3)).
 * The covariance is Sigma = R S S^T R^T (Eq. 1) with S = diag(exp(log_scale))
 * and R from the normalised quaternion.
 *
 * Fixed rendering rules (the paper leaves them to its 3DGS rasteriser):
 * 0.3 px^2 is added to the 2D covariance diagonal; a Gaussian reaches a pixel
 * only inside its 3-sigma ellipse (d^T Sigma'^-1 d <= 9); alpha =
 * min(0.99, opacity * exp(-q/2)); alpha < 1/255 is skipped; compositing stops
 * before the Gaussian that would take the transmittance below 1e-4. Pixel
 * (i, j) is column i, row j, centred at integer coordinates; depth is the
 * view-space z of each Gaussian's mean, blended without normalisation. A
 * Gaussian is projected into a view only if its mean has z > near_z and lies
 * in the guard cone |x/z| <= G, |y/z| <= G (G = guard_slope, default 1.5): the
 * first-order projection of the 3DGS rasteriser the paper builds on is
 * meaningless, and its gradient ill-conditioned, far off-axis just in front of
 * the camera. The cone depends on the mean's direction only, so a crop of a view
 * (shifted principal point) renders exactly that window of the view.
 * Colour: SH degree 0 uses c = k0 directly (Eq. 2); degree d >= 1 uses
 * c = max(0, k0 + sum_{l=1..d, m} Y_lm(v) k_lm) with the real orthonormal
 * spherical harmonics and v the unit vector from the camera centre to the mean.
 *
 * Conventions
 *  - All tensors are float32, C-contiguous, in DEVICE memory unless stated.
 *  - Cameras: T_cw is the 3x4 row-major world-to-camera transform [R | t]
 *    (Eq. 9 composes poses on the left). The twist tau = (rho, phi) perturbs a
 *    pose as Exp(tau) * T_cw; its gradient is taken at tau = 0.
 *  - Image outputs of a multi-view call are packed view after view; within a
 *    view they are planar [C][H][W]. View v starts at pixel offset
 *    P_v = sum_{u<v} H_u W_u (rgb and pointmap start at 3 P_v).
 *  - Ownership: the caller owns every pointer passed in; the library owns
 *    contexts, states and their scratch. Nothing here takes ownership of, or
 *    frees, caller memory.
 *  - Errors: no call aborts, traps or exits. Each returns an s3gs_status;
 *    s3gs_last_error() gives a message for the last failure on a context.
 *    CUDA errors are reported as S3GS_E_CUDA.
 *  - Streams: every GPU call takes a cudaStream_t (as void*; NULL = legacy
 *    default stream) and is asynchronous unless documented otherwise.
 */
#ifndef S3GS_H
#define S3GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    S3GS_OK = 0,
    S3GS_E_INVALID = -1,  /* bad argument: NULL where required, size out of range, NaN camera */
    S3GS_E_CAPACITY = -2, /* duplicate (Gaussian, tile) pairs exceeded the reserved capacity */
    S3GS_E_CUDA = -3,     /* a CUDA runtime call failed; see s3gs_last_error */
    S3GS_E_TIMEOUT = -4,  /* reserved: no device-side wait exists in this library */
    S3GS_E_NOMEM = -5,    /* device or host allocation failed */
    S3GS_E_STATE = -6     /* backward called on a state with no successful forward */
} s3gs_status;

#define S3GS_MAX_VIEWS 32
#define S3GS_MAX_SH_DEGREE 3
/* Largest number of (Gaussian, tile) duplicates one call can hold (unsigned
 * 32-bit offsets); larger windows must be split across calls. */
#define S3GS_MAX_DUPLICATES 4294967295LL

typedef struct s3gs_ctx s3gs_ctx;
typedef struct s3gs_state s3gs_state;

/* Gaussian set (Sec. 3.1). Device pointers, structure of arrays:
 *   means [n][3], log_scales [n][3], quats [n][4] (w, x, y, z; need not be
 *   unit), opacity_logits [n], colors [n][(sh_degree+1)^2][3]. */
typedef struct {
    int64_t n;
    int32_t sh_degree; /* 0..3 */
    const float *means;
    const float *log_scales;
    const float *quats;
    const float *opacity_logits;
    const float *colors;
} s3gs_gaussians;

/* One pinhole view (HOST struct): intrinsics K of Eq. 4 and pose T_cw. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float T_cw[12];
} s3gs_camera;

/* Options. Zero-initialised fields select the defaults shown. Tile shape and
 * batch size do not change forward results; they change only the summation
 * order of atomically accumulated gradients (and nothing in deterministic mode). */
typedef struct {
    int32_t tile_w, tile_h;  /* tile shape: 16x16 (default), 16x8, 8x8 or 32x8 */
    int32_t pixels_per_thread; /* pixels each forward-blend thread owns: 1, 2 or 4; 0 = auto
                                  (2, or 1 where a tile would not fill whole warps) */
    int32_t bwd_pixels_per_thread; /* the same for the backward blend; 0 = auto (4, else 2, else 1) */
    int32_t batch;           /* Gaussians staged per shared-memory batch: 0 = 256 */
    int32_t blocks_per_sm;   /* blend kernels: 0 = one CTA per tile; k > 0 = persistent grid of
                                k CTAs per SM pulling tiles (heaviest first) from a work counter */
    int32_t deterministic;   /* 1: gradients are bitwise reproducible run to run */
    int32_t recompute;       /* 1: do not store per-pixel blend state; the backward replays it */
    int32_t auto_grow;       /* 1: the forward synchronises once to size the duplicate buffer
                                (not capture-safe); 0: overflow is reported as S3GS_E_CAPACITY */
    float near_z;            /* cull Gaussians with view-space z <= near_z (0 = 0.2) */
    float guard_slope;       /* guard cone G (0 = 1.5; negative = no cone) */
    float bg[3];             /* background colour composited with the final transmittance */
    int32_t full_lists;      /* 0 (default): occlusion cut. Each tile's list ends after the first
                                depth bin by which the Gaussians that cover the whole tile are
                                certain, by a bound with FP32 margins, to have driven every pixel
                                of the tile below the 1e-4 transmittance stop of Eq. 2; no pixel
                                reaches a later bin, so outputs and gradients are unchanged.
                                1: list every covered (tile, Gaussian) pair. */
} s3gs_options;

/* Fill *opt with the defaults (16x16 tiles, 2 / 4 pixels per forward / backward
 * thread, batches of 256,
 * one CTA per tile, atomic gradients, stored blend state, auto_grow = 1,
 * near_z = 0.2, black background). */
void s3gs_options_default(s3gs_options *opt);

/* Create a context on CUDA device `device`. *out receives the handle. */
s3gs_status s3gs_create(int device, s3gs_ctx **out);
/* Destroy a context (NULL is a no-op). States must be destroyed first. */
void s3gs_destroy(s3gs_ctx *ctx);
/* Message of the last failed call on this context (never NULL). */
const char *s3gs_last_error(const s3gs_ctx *ctx);

/* A state holds what the backward of one forward needs: the projected
 * Gaussians, the tile-sorted duplicate list and the per-pixel blend state.
 * It stays valid until the next forward on the same state or its destruction. */
s3gs_status s3gs_state_create(s3gs_ctx *ctx, s3gs_state **out);
void s3gs_state_destroy(s3gs_state *state);

/* Pre-size a state so that forwards within these limits never allocate (as
 * CUDA-graph capture requires): n Gaussians, n_views views, total_pixels over
 * all views, total_tiles over all views at the smallest tile used (each tile
 * holds 256 depth buckets internally), and max_duplicates (Gaussian, tile)
 * pairs (16 bytes of device memory each: the emission buffer and the sorted
 * list). Synchronous. */
s3gs_status s3gs_reserve(s3gs_ctx *ctx, s3gs_state *state, int64_t n, int32_t n_views,
                         int64_t total_pixels, int64_t total_tiles, int64_t max_duplicates);

/* Forward render (Eq. 1-5) of n_views views in one batched pass.
 *   cams          HOST array of n_views cameras (sizes, intrinsics, poses).
 *   T_cw_device   optional DEVICE array [n_views][12]; when non-NULL it
 *                 replaces the poses of `cams` at kernel time (for pose loops
 *                 replayed from a CUDA graph). May be NULL.
 *   rgb [3 P], depth [P], pointmap [3 P], alpha [P] (P = total pixels), packed
 *   as described above; any output may be NULL. The Gaussian pointers are
 *   remembered by the state and must stay valid and unchanged until the
 *   matching backward has been enqueued.
 * Errors: INVALID (bad sizes, n_views outside 1..S3GS_MAX_VIEWS, sh_degree
 * outside 0..3, non-finite intrinsics), CAPACITY (only with auto_grow = 0;
 * the result is then undefined; reported by this call if already known or by
 * s3gs_state_check), NOMEM, CUDA. */
s3gs_status s3gs_render_fwd(s3gs_ctx *ctx, s3gs_state *state, const s3gs_gaussians *gaussians,
                            const s3gs_camera *cams, int32_t n_views, const float *T_cw_device,
                            const s3gs_options *opt, float *rgb, float *depth, float *pointmap,
                            float *alpha, void *stream);

/* Backward of the last forward on `state` (Eq. 11 and the Gaussian-parameter
 * gradients). Upstream gradients use the forward's packed layout; NULL = zero.
 * Outputs (NULL = not requested): d_means [n][3], d_log_scales [n][3],
 * d_quats [n][4], d_opacity_logits [n], d_colors [n][(d+1)^2][3],
 * d_twist [n_views][6] (rho then phi). accumulate = 0 overwrites the outputs,
 * 1 adds to them. A call with only d_twist is the pose-only backward of
 * tracking (Sec. 3.2.2). */
s3gs_status s3gs_render_bwd(s3gs_ctx *ctx, s3gs_state *state, const float *d_rgb,
                            const float *d_depth, const float *d_pointmap, const float *d_alpha,
                            float *d_means, float *d_log_scales, float *d_quats,
                            float *d_opacity_logits, float *d_colors, float *d_twist,
                            int32_t accumulate, void *stream);

/* Backward with the L1 mapping loss of s3gs_mapping_loss fused in (Eq. 10/15/17):
 * the same result as s3gs_mapping_loss on the forward's outputs followed by
 * s3gs_render_bwd with the gradients it writes (and d_alpha = NULL), in one pass
 * that forms each pixel's upstream gradient from its output and target instead
 * of writing and re-reading gradient images. rgb, depth, pointmap: the outputs
 * the last forward on `state` wrote (device, packed); t_rgb, t_depth,
 * t_pointmap: targets (NULL = term off); mask: per-pixel weights (NULL = 1);
 * w_*: term weights; loss_device: device float [1] out, the loss value (the
 * same terms as s3gs_mapping_loss, summed in another order; NULL = not wanted).
 * Gradient outputs, accumulate and errors as in s3gs_render_bwd; INVALID also
 * for a target without its output. */
s3gs_status s3gs_render_bwd_l1(s3gs_ctx *ctx, s3gs_state *state, const float *rgb, const float *depth,
                               const float *pointmap, const float *t_rgb, const float *t_depth,
                               const float *t_pointmap, const float *mask, float w_rgb, float w_depth, float w_geo,
                               float *loss_device, float *d_means, float *d_log_scales, float *d_quats,
                               float *d_opacity_logits, float *d_colors, float *d_twist, int32_t accumulate,
                               void *stream);

/* Synchronise with the state's last stream and report its device-side status:
 * S3GS_E_CAPACITY if the last forward overflowed. *n_duplicates (optional)
 * receives that forward's number of (Gaussian, tile) pairs, *capacity
 * (optional) the reserved capacity. */
s3gs_status s3gs_state_check(s3gs_ctx *ctx, s3gs_state *state, int64_t *n_duplicates,
                             int64_t *capacity);

/* Mapping / tracking loss of Eq. 10, 15 and 17 on packed outputs (device)
 * of the views `cams` (HOST, n_views; only their sizes are used):
 *   loss = w_rgb * mean|rgb - t_rgb| + w_depth * mean|depth - t_depth|
 *        + w_geo * mean|pointmap - t_pointmap|
 * (means over all elements of each term across all views; a NULL target drops
 * its term) and its gradient with respect to the rendered outputs (d_* NULL =
 * not wanted; the sign of a zero residual is taken as 0). mask (optional,
 * [P]) multiplies every term per pixel (the edge / invalid weighting of
 * Sec. 3.2.2). *loss_device (device, 1 float) receives the scalar. The sum is
 * taken in a fixed order. */
s3gs_status s3gs_mapping_loss(s3gs_ctx *ctx, const s3gs_camera *cams, int32_t n_views,
                              const float *rgb, const float *depth, const float *pointmap,
                              const float *t_rgb, const float *t_depth, const float *t_pointmap,
                              const float *mask, float w_rgb, float w_depth, float w_geo,
                              float *d_rgb, float *d_depth, float *d_pointmap, float *loss_device,
                              void *stream);

/* Allocation-free variant of s3gs_mapping_loss (the paper has no counterpart:
 * this is a deployment convenience). Same arguments, layout and result, but no
 * context and no allocation: it calls no cudaMalloc/cudaFree and no allocating
 * library routine. It is for callers that cannot allocate device memory --
 * code running inside a global-mode CUDA stream capture, hosts whose device
 * memory belongs to a pooling allocator or a fixed budget, and latency-bound
 * loops that must avoid the implicit synchronisation of cudaMalloc/cudaFree.
 * Its partial sums live in a fixed 8 KB static device array (64 per view, so
 * n_views <= S3GS_MAX_VIEWS); larger requests return S3GS_E_INVALID. The first
 * call on each device looks up that array's address (cudaGetSymbolAddress),
 * so make one call per device before any stream capture (a first call on a
 * capturing stream returns S3GS_E_INVALID and leaves the capture as it was);
 * the address is cached for the life of the process, so do not call this entry
 * point on a device after cudaDeviceReset. All calls share the
 * array: calls that overlap on the GPU (e.g. on two concurrent streams) race
 * and give wrong results; each call rewrites every partial it reads, so
 * nothing needs clearing between calls. err (optional, err_len bytes) receives
 * a message on failure; the status is INVALID for bad arguments or sizes and
 * CUDA for runtime failures. */
s3gs_status s3gs_mapping_loss_noalloc(const s3gs_camera *cams, int32_t n_views, const float *rgb,
                                      const float *depth, const float *pointmap, const float *t_rgb,
                                      const float *t_depth, const float *t_pointmap, const float *mask,
                                      float w_rgb, float w_depth, float w_geo, float *d_rgb,
                                      float *d_depth, float *d_pointmap, float *loss_device,
                                      void *stream, char *err, size_t err_len);

/* Diagnostics (synchronous; HOST output arrays, any may be NULL).
 * s3gs_debug_records: per record r = v * n + g of the last forward:
 *   xy [r][2], conic_opacity [r][4] (A, B, C, opacity), rgb_depth [r][4]
 *   (r, g, b, view-space z), extent [r][2] (integer half-extents rx, ry of the
 *   bounding rectangle of the tile cover, 0 = culled). n_records must equal
 *   n_views * n.
 * s3gs_debug_binning: the tile-sorted duplicate list as 64-bit keys
 *   (global tile id << 32 | float bits of z), values (Gaussian index g) and
 *   per-tile ranges [n_tiles + 1]; *n_tiles and *n_dup receive the sizes (pass
 *   NULL arrays first to query them). */
s3gs_status s3gs_debug_records(s3gs_ctx *ctx, s3gs_state *state, int64_t n_records, float *xy,
                               float *conic_opacity, float *rgb_depth, int32_t *extent);
/* s3gs_debug_cover: per record the bound q_cover of its tile cover (the record
 * is listed in a tile iff its ellipse A dx^2 + 2 B dx dy + C dy^2 <= q_cover
 * meets the box of the tile's pixel centres; 0 for culled records). */
s3gs_status s3gs_debug_cover(s3gs_ctx *ctx, s3gs_state *state, int64_t n_records, float *q_cover);
s3gs_status s3gs_debug_binning(s3gs_ctx *ctx, s3gs_state *state, uint64_t *keys,
                               uint32_t *values, int64_t *ranges, int64_t *n_tiles,
                               int64_t *n_dup);

/* Counters of the last forward and backward (synchronous): processed and
 * blended Gaussian-pixel pairs of the forward, processed pairs of the
 * backward. Counting is enabled by s3gs_set_counting(ctx, 1); it slows the
 * blend kernels and is off by default. */
s3gs_status s3gs_set_counting(s3gs_ctx *ctx, int32_t enable);
s3gs_status s3gs_read_counters(s3gs_ctx *ctx, s3gs_state *state, int64_t *fwd_processed,
                               int64_t *fwd_blended, int64_t *bwd_processed);

/* Per-stage timing with CUDA events recorded on the launch stream (also
 * inside captured CUDA graphs). Stages, in this order:
 *   0 project, 1 scan, 2 emit, 3 tile_sort, 4 tile_order, 5 blend_fwd,
 *   6 blend_bwd, 7 det_reduce, 8 project_bwd, 9 twist_reduce, 10 loss.
 * s3gs_read_timing waits for the last recorded events and writes, for each of
 * the first n stages, its duration in ms in the most recent call that ran it
 * (-1 if it has not run since timing was enabled). Synchronous. */
#define S3GS_NUM_STAGES 11
s3gs_status s3gs_set_timing(s3gs_ctx *ctx, int32_t enable);
s3gs_status s3gs_read_timing(s3gs_ctx *ctx, float *ms, int32_t n);

/* Library version string. */
const char *s3gs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* S3GS_H */
