/*
 * s3gs_slam.h -- C ABI of the S3PO-GS steps that consume the renderer's
 * outputs on the GPU: patch-based pointmap scale alignment (Sec. 3.3.1 and
 * Algorithm 1 of the supplementary material), pointmap replacement (Sec.
 * 3.3.2, Eq. 14), the remedial scale factor (supplementary material, the
 * paragraph after Algorithm 1), the pose update of photometric tracking
 * (Sec. 3.2.2, Eq. 10/11), the map optimiser step (Eq. 16/17) and keyframe
 * covisibility / window management (supplementary material, Eq. S1/S2).
 *
 * Conventions are those of s3gs.h: float32 device tensors, packed views
 * (pointmaps planar [3][H][W] per view, view v starting at 3 P_v with
 * P_v = sum_{u<v} H_u W_u; per-pixel masks [H][W] per view starting at P_v),
 * the caller owns every buffer, no call aborts, every GPU call is
 * asynchronous on the given stream and none of them allocates memory, so all
 * of them may be captured in a CUDA graph. Scratch is a caller-provided
 * workspace whose size a host-only query returns.
 *
 * Readings of the paper these calls implement:
 *  - Patches are the P x P blocks of the H x W grid from pixel (0, 0); the
 *    ragged last row/column of patches is used as it is.
 *  - A patch's mean and standard deviation are joint over all coordinate
 *    values of its points (population standard deviation).
 *  - A patch is a candidate when |mu_r - mu_p| < delta_mu mu_p and
 *    |sigma_r - sigma_p| < delta_sigma sigma_p, with X^p scaled by the
 *    current factor; a point of a candidate patch is a correct point (CP)
 *    when the Euclidean norm of the difference of its normalised 3-vectors is
 *    below eps_r.
 *  - CP is rebuilt at every iteration and the factor is
 *    sum(X^r[CP]) / sum(X^p[CP]) over all coordinates of the correct points,
 *    against the unscaled X^p; an empty CP keeps the previous factor.
 *  - Eq. 14 compares per-point Euclidean norms:
 *    keep X^r(x) iff ||X^r(x) - s X^p(x)|| <= eps_m ||s X^p(x)||.
 */
#ifndef S3GS_SLAM_H
#define S3GS_SLAM_H

#include "s3gs.h"

#ifdef __cplusplus
extern "C" {
#endif

#define S3GS_MAX_PATCH 32

/* Hyperparameters of Algorithm 1 (defaults: the supplementary material's
 * parameter table: P = 10, delta_mu = delta_sigma = 0.3, eps_r = 0.1,
 * max_iter = 3, tau = 0.01). */
typedef struct {
    int32_t patch;      /* P, 1..S3GS_MAX_PATCH */
    float delta_mu;     /* relative gate on patch means */
    float delta_sigma;  /* relative gate on patch standard deviations */
    float eps_r;        /* correct-point threshold on normalised distance */
    int32_t max_iter;   /* iterations, 1..64 */
    float tau;          /* |CP| < tau * H * W flags the view as insufficient */
} s3gs_align_params;

/* Host only: fills the defaults above. */
void s3gs_align_params_default(s3gs_align_params *params);

/* Host only: bytes of device workspace s3gs_scale_align needs for these views
 * (view_wh: host [n_views][2] = width, height) and patch size. Returns
 * S3GS_E_INVALID for sizes out of range. */
s3gs_status s3gs_scale_align_workspace(const int32_t *view_wh, int32_t n_views, int32_t patch, size_t *bytes);

/* Algorithm 1 for every view of the batch, independently.
 *   X_r, X_p      rendered and pre-trained pointmaps, packed planar (read only)
 *   sigma_init    device [n_views] starting factors, or NULL for 1 (Algorithm 1
 *                 starts from 1; the remedy re-runs one iteration from its
 *                 remedial factor). May alias sigma.
 *   sigma         device [n_views] out: the factor after max_iter iterations
 *   n_cp          device [n_views] out (optional): |CP| of the last iteration
 *   insufficient  device [n_views] out (optional): 1 if |CP| < tau H W else 0
 *   cp_mask       device uint8 per pixel out (optional): CP of the last iteration
 *   workspace     device, at least s3gs_scale_align_workspace() bytes, 16-byte
 *                 aligned; contents on entry are ignored
 * Returns S3GS_E_INVALID for NULL required pointers, n_views outside
 * 1..S3GS_MAX_VIEWS, a view larger than 65536 on a side, parameters out of
 * range or a workspace that is too small; S3GS_E_CUDA if a launch fails. */
s3gs_status s3gs_scale_align(s3gs_ctx *ctx, const int32_t *view_wh, int32_t n_views, const float *X_r,
                             const float *X_p, const s3gs_align_params *params, const float *sigma_init,
                             float *sigma, int64_t *n_cp, int32_t *insufficient, uint8_t *cp_mask,
                             void *workspace, size_t workspace_bytes, void *stream);

/* Pointmap replacement (Eq. 14) with the aligned map Xhat^p = sigma_v X^p.
 *   sigma       device [n_views] factors (e.g. from s3gs_scale_align)
 *   X_r_hat     out, packed planar; may alias X_r (each point is read before it
 *               is written by the same thread)
 *   X_p_hat     out (optional): sigma_v X^p
 *   replaced    out (optional): uint8 per pixel, 1 where X^p replaced X^r
 *   n_replaced  out (optional): device int64 [n_views] counts
 * Returns S3GS_E_INVALID for NULL required pointers, bad sizes or eps_m < 0. */
s3gs_status s3gs_pointmap_replace(s3gs_ctx *ctx, const int32_t *view_wh, int32_t n_views, const float *X_r,
                                  const float *X_p, const float *sigma, float eps_m, float *X_r_hat,
                                  float *X_p_hat, uint8_t *replaced, int64_t *n_replaced, void *stream);

/* Remedial scale factor from matched points: sigma = sum(X_ak_hat[:, a_k]) /
 * sum(X_n[:, b_k]) over all coordinates, with matches device int32
 * [n_matches][2] = (a_k, b_k), flat pixel indices into the aligned adjacent
 * keyframe map (hw_ak pixels, planar [3][hw_ak]) and the current map (hw_n
 * pixels). Matches with an index out of range are skipped; n_used (optional,
 * device int64 [1]) receives the number of matches used. With no usable match
 * sigma is set to 1. The matcher itself (a learned feature matcher in the
 * paper) is outside this library. */
s3gs_status s3gs_scale_remedy(s3gs_ctx *ctx, const float *X_ak_hat, int64_t hw_ak, const float *X_n, int64_t hw_n,
                              const int32_t *matches, int64_t n_matches, float *sigma, int64_t *n_used,
                              void *stream);

/* ---- Pose refinement (Sec. 3.2.2, Eq. 10/11) and window poses (Eq. 17) ----
 * Readings: a pose is the world-to-camera T_cw, perturbed on the left,
 * T(tau) = Exp(tau) T_cw, tau = (rho, phi), exactly as the renderer's d_twist
 * (s3gs_render_bwd) is defined. The optimiser is Adam on tau, taken from
 * tau = 0 each iteration with moments that persist, followed by the retraction
 * T_cw <- Exp(delta) T_cw; the paper names no optimiser and no step sizes, so
 * they are inputs (defaults below are this library's choice). */
typedef struct {
    float lr_rho;  /* step size of the translation part (default 1e-3) */
    float lr_phi;  /* step size of the rotation part, radians (default 1e-3) */
    float beta1;   /* default 0.9 */
    float beta2;   /* default 0.999 */
    float eps;     /* default 1e-8 */
} s3gs_pose_adam;

/* Host only: fills the defaults above. */
void s3gs_pose_adam_default(s3gs_pose_adam *hp);

/* Exp of n twists tau [n][6] = (rho, phi) into 3x4 row-major [R | V rho]
 * (E [n][12]), from the closed forms of the SE(3) exponential with Taylor
 * series where those lose FP32 accuracy. Device pointers; n = 0 is a no-op. */
s3gs_status s3gs_se3_exp(s3gs_ctx *ctx, int64_t n, const float *tau, float *E, void *stream);

/* One optimiser step per view:
 *   d_twist   device [n_views][6], dL/dtau at tau = 0 (from s3gs_render_bwd)
 *   adam_m, adam_v  device [n_views][6] moments (zero before the first step), updated
 *   step      device int32 [n_views] step counters (zero before the first step),
 *             incremented; Adam's bias correction uses the new value
 *   T_cw      device [n_views][12] poses, replaced by Exp(delta) T_cw
 *   delta     device [n_views][6] out (optional): the step taken
 *   frozen    device uint8 [n_views] (optional): nonzero keeps that view's pose,
 *             moments and counter unchanged (delta = 0)
 * The poses can be passed straight to s3gs_render_fwd as T_cw_device, so a
 * whole refinement loop (render, loss, backward, update) captures into one
 * CUDA graph. Returns S3GS_E_INVALID for NULL pointers or hyperparameters out
 * of range (lr >= 0, 0 <= beta < 1, eps > 0). */
s3gs_status s3gs_pose_update(s3gs_ctx *ctx, int32_t n_views, const float *d_twist, const s3gs_pose_adam *hp,
                             float *adam_m, float *adam_v, int32_t *step, float *T_cw, float *delta,
                             const uint8_t *frozen, void *stream);

/* ---- Map optimiser step (Eq. 17) with the isotropic regulariser (Eq. 16) ----
 * Readings: s_i = exp(log_scale_i) and s~_i = mean of its three entries;
 * L_iso = lambda_iso * sum_i ||s_i - s~_i 1||_1 summed over Gaussians as
 * printed (scale lambda_iso by 1 / (3 |G|) for a mean), with d|x|/dx = sign(x)
 * (0 at 0). The optimiser is Adam (the paper names none) with one step count,
 * a learning rate per tensor and a separate one for the SH bands l >= 1; the
 * default rates are this library's choice. The window poses take the same
 * kind of step through s3gs_pose_update. */
typedef struct {
    float lr_means;        /* default 1.6e-4 */
    float lr_log_scales;   /* default 5e-3 */
    float lr_quats;        /* default 1e-3 */
    float lr_opacity;      /* default 5e-2 */
    float lr_colors;       /* colour / SH band 0, default 2.5e-3 */
    float lr_colors_rest;  /* SH bands l >= 1, default 1.25e-4 */
    float beta1;           /* default 0.9 */
    float beta2;           /* default 0.999 */
    float eps;             /* default 1e-15 */
    float lambda_iso;      /* default 10 (supplementary material) */
} s3gs_map_adam;

/* Host only: fills the defaults above. */
void s3gs_map_adam_default(s3gs_map_adam *hp);

/* One fused Adam step over all Gaussian tensors, in place, in one launch plus
 * a one-thread counter update. params / grads / adam_m / adam_v are HOST
 * arrays of 5 DEVICE pointers in the order means [n][3], log_scales [n][3],
 * quats [n][4], opacity_logits [n], colors [n][(d+1)^2][3] (the layouts of
 * s3gs_gaussians); a NULL gradient pointer means a zero gradient for that
 * tensor (momentum still moves it, as in Adam); moments start at zero. step
 * is a device int32 counter (0 before the first step), advanced by one.
 * Returns S3GS_E_INVALID for NULL arrays or pointers, n < 0, sh_degree outside
 * 0..3 or hyperparameters out of range. */
s3gs_status s3gs_map_adam_step(s3gs_ctx *ctx, int64_t n, int32_t sh_degree, float *const params[5],
                               const float *const grads[5], float *const adam_m[5], float *const adam_v[5],
                               int32_t *step, const s3gs_map_adam *hp, void *stream);

/* ---- Keyframe covisibility and window management (supplementary material,
 * "Keyframe Management", Eq. S1/S2) ----
 * Readings: the visible set G_i^v of view i is the set of Gaussians the last
 * forward projected into view i with a non-empty pixel footprint (near plane,
 * guard cone and 3-sigma tile cover of s3gs.h); IOU and OC are 0 when their
 * denominator is 0; the median depth is the lower median (rank
 * floor((N - 1) / 2)) of the N pixels with depth > 0, 0 if there are none. */

/* Intersection counts of the visible sets of the last forward on `state`:
 * counts device int64 [V][V] out (counts[i][i] = |G_i|), iou and oc device
 * float [V][V] out (optional), V = that forward's n_views. Enqueued on
 * `stream`, which the caller orders after the forward. Returns S3GS_E_STATE
 * if the state has no forward. */
s3gs_status s3gs_covisibility(s3gs_ctx *ctx, s3gs_state *state, int64_t *counts, float *iou, float *oc,
                              void *stream);

/* Host only: workspace bytes of s3gs_median_depth for n_views views. */
s3gs_status s3gs_median_depth_workspace(int32_t n_views, size_t *bytes);

/* Median depth per view of packed depth maps (view_wh host [n_views][2]):
 * median device float [n_views] out, n_valid device int64 [n_views] out
 * (optional, the number of positive depths); workspace device, 16-byte
 * aligned. Exact (a radix select on the float bits, no rounding). */
s3gs_status s3gs_median_depth(s3gs_ctx *ctx, const int32_t *view_wh, int32_t n_views, const float *depth,
                              float *median, int64_t *n_valid, void *workspace, size_t workspace_bytes,
                              void *stream);

/* Window parameters (the supplementary material's values as defaults:
 * k_I = 0.9, k_d = 0.08, k_o = 0.3, |W| = 8). */
typedef struct {
    float k_iou;         /* a frame with IOU < k_iou against the latest keyframe becomes a keyframe */
    float k_d;           /* ... as does one that moved more than k_d times its median depth */
    float k_oc;          /* window keyframes with OC < k_oc against a new keyframe leave */
    int32_t max_window;  /* window size, the new keyframe included */
} s3gs_keyframe_params;

/* Host only: fills the defaults above. */
void s3gs_keyframe_params_default(s3gs_keyframe_params *p);

/* Host only: 1 if frame i becomes a keyframe given IOU(i, j) with the latest
 * keyframe j, the translation distance d_ij and i's median depth, else 0;
 * -1 if p is NULL. */
int32_t s3gs_keyframe_is_new(const s3gs_keyframe_params *p, float iou_ij, float d_ij, float median_depth_i);

/* Host only: the window after keyframe new_id joined. window_ids [n] are the
 * current keyframes (oldest first) and oc_with_new [n] their OC with the new
 * keyframe. Every keyframe with OC < k_oc leaves; while the window would
 * exceed max_window, the remaining one with the lowest OC leaves (the earlier
 * one on ties); new_id is appended. out_ids (capacity n + 1) and *out_n
 * receive the result. */
s3gs_status s3gs_keyframe_window_update(const s3gs_keyframe_params *p, const int32_t *window_ids,
                                        const float *oc_with_new, int32_t n, int32_t new_id, int32_t *out_ids,
                                        int32_t *out_n);

#ifdef __cplusplus
}
#endif

#endif /* S3GS_SLAM_H */
