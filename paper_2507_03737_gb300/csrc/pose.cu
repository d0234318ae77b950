// On-device pose update of photometric tracking and window optimisation
// (Sec. 3.2.2, Eq. 10 and 11; Eq. 17 for the window poses): one Adam step on
// the twist tau = (rho, phi) of every view, taken from tau = 0 with the
// gradient the backward wrote, and the retraction T_cw <- Exp(delta) T_cw
// (the left perturbation of the renderer's twist gradient). One thread per
// view; the step counter lives on the device, so a captured refinement loop
// replays without the host. C ABI in include/s3gs_slam.h.
#include <cstdio>

#include "../../include/s3gs_slam.h"
#include "s3gs_internal.cuh"

namespace s3gs {
namespace {

// Exp of tau = (rho, phi): R = I + a K + b K^2, V = I + b K + c K^2 with
// K = [phi]_x, theta = |phi|, a = sin(theta)/theta, b = (1 - cos(theta))/theta^2,
// c = (theta - sin(theta))/theta^3. b is evaluated as (sin(theta/2)/theta)^2 * 2,
// which has no cancellation; a and c use their Taylor series where the closed
// forms lose accuracy in FP32.
__device__ void se3_exp_dev(const float tau[6], float E[12]) {
    const float px = tau[3], py = tau[4], pz = tau[5];
    const float th2 = px * px + py * py + pz * pz;
    const float th = sqrtf(th2);
    float a, b, c;
    if (th < 0.5f) {
        const float t4 = th2 * th2, t6 = t4 * th2;
        a = 1.0f - th2 / 6.0f + t4 / 120.0f - t6 / 5040.0f;
        b = 0.5f - th2 / 24.0f + t4 / 720.0f - t6 / 40320.0f;
        c = 1.0f / 6.0f - th2 / 120.0f + t4 / 5040.0f - t6 / 362880.0f;
        if (th >= 1e-2f) {
            a = sinf(th) / th;
            const float h = sinf(0.5f * th) / th;
            b = 2.0f * h * h;
        }
    } else {
        const float s = sinf(th);
        a = s / th;
        const float h = sinf(0.5f * th) / th;
        b = 2.0f * h * h;
        c = (th - s) / (th2 * th);
    }
    // K and K^2
    const float K[9] = {0.f, -pz, py, pz, 0.f, -px, -py, px, 0.f};
    float K2[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float vr = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float id = i == j ? 1.f : 0.f;
            E[4 * i + j] = id + a * K[3 * i + j] + b * K2[3 * i + j];
            vr += (id + b * K[3 * i + j] + c * K2[3 * i + j]) * tau[j];
        }
        E[4 * i + 3] = vr;
    }
}

__global__ void se3_exp_kernel(const float *__restrict__ tau, float *__restrict__ E, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float t[6], e[12];
#pragma unroll
    for (int k = 0; k < 6; ++k) t[k] = tau[6 * i + k];
    se3_exp_dev(t, e);
#pragma unroll
    for (int k = 0; k < 12; ++k) E[12 * i + k] = e[k];
}

struct PoseUpdateArgs {
    const float *d_twist;
    float *m, *v;
    int *step;
    float *T;
    float *delta;
    const unsigned char *frozen;
    float lr[6];
    float beta1, beta2, eps;
    int n;
};

__global__ void pose_update_kernel(const PoseUpdateArgs a) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    if (a.frozen && a.frozen[k]) {
        if (a.delta)
            for (int i = 0; i < 6; ++i) a.delta[6 * k + i] = 0.f;
        return;
    }
    const int t = a.step[k] + 1;
    a.step[k] = t;
    const float c1 = 1.0f - powf(a.beta1, (float)t), c2 = 1.0f - powf(a.beta2, (float)t);
    float d[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float g = a.d_twist[6 * k + i];
        const float m = a.beta1 * a.m[6 * k + i] + (1.0f - a.beta1) * g;
        const float v = a.beta2 * a.v[6 * k + i] + (1.0f - a.beta2) * g * g;
        a.m[6 * k + i] = m;
        a.v[6 * k + i] = v;
        d[i] = -a.lr[i] * (m / c1) / (sqrtf(v / c2) + a.eps);
    }
    float E[12];
    se3_exp_dev(d, E);
    float T[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) T[i] = a.T[12 * k + i];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float s = E[4 * i] * T[j] + E[4 * i + 1] * T[4 + j] + E[4 * i + 2] * T[8 + j];
            if (j == 3) s += E[4 * i + 3];
            a.T[12 * k + 4 * i + j] = s;
        }
    }
    if (a.delta)
#pragma unroll
        for (int i = 0; i < 6; ++i) a.delta[6 * k + i] = d[i];
}

s3gs_status launch_error(s3gs_ctx *ctx, cudaError_t e, const char *where) {
    char msg[256];
    snprintf(msg, sizeof(msg), "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
    return ctx_error(ctx, S3GS_E_CUDA, msg);
}

bool finite_pos(float x) { return x == x && x > 0.f && x < 3.0e38f; }

}  // namespace
}  // namespace s3gs

using namespace s3gs;

extern "C" {

void s3gs_pose_adam_default(s3gs_pose_adam *p) {
    if (!p) return;
    p->lr_rho = 1e-3f;
    p->lr_phi = 1e-3f;
    p->beta1 = 0.9f;
    p->beta2 = 0.999f;
    p->eps = 1e-8f;
}

s3gs_status s3gs_se3_exp(s3gs_ctx *ctx, int64_t n, const float *tau, float *E, void *stream) {
    if (!ctx) return S3GS_E_INVALID;
    if (n < 0 || (n > 0 && (!tau || !E))) return ctx_error(ctx, S3GS_E_INVALID, "se3_exp: bad size or NULL pointer");
    if (n == 0) return S3GS_OK;
    se3_exp_kernel<<<(unsigned)((n + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(tau, E, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? S3GS_OK : launch_error(ctx, e, "se3_exp");
}

s3gs_status s3gs_pose_update(s3gs_ctx *ctx, int32_t n_views, const float *d_twist, const s3gs_pose_adam *hp,
                             float *adam_m, float *adam_v, int32_t *step, float *T_cw, float *delta,
                             const uint8_t *frozen, void *stream) {
    if (!ctx) return S3GS_E_INVALID;
    if (n_views < 1 || n_views > (1 << 24) || !d_twist || !hp || !adam_m || !adam_v || !step || !T_cw)
        return ctx_error(ctx, S3GS_E_INVALID, "pose_update: bad n_views or NULL pointer");
    if (!(hp->lr_rho >= 0.f && hp->lr_phi >= 0.f && hp->lr_rho < 1e30f && hp->lr_phi < 1e30f) ||
        !(hp->beta1 >= 0.f && hp->beta1 < 1.f) || !(hp->beta2 >= 0.f && hp->beta2 < 1.f) || !finite_pos(hp->eps))
        return ctx_error(ctx, S3GS_E_INVALID, "pose_update: learning rates >= 0, betas in [0, 1), eps > 0 required");
    PoseUpdateArgs a;
    a.d_twist = d_twist;
    a.m = adam_m;
    a.v = adam_v;
    a.step = step;
    a.T = T_cw;
    a.delta = delta;
    a.frozen = frozen;
    for (int i = 0; i < 3; ++i) {
        a.lr[i] = hp->lr_rho;
        a.lr[3 + i] = hp->lr_phi;
    }
    a.beta1 = hp->beta1;
    a.beta2 = hp->beta2;
    a.eps = hp->eps;
    a.n = n_views;
    pose_update_kernel<<<(n_views + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? S3GS_OK : launch_error(ctx, e, "pose_update");
}

}  // extern "C"
