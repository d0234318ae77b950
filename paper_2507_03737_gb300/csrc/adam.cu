// Fused map-optimiser step (Eq. 17 with the isotropic regulariser of Eq. 16):
// one Adam step over every Gaussian parameter tensor in a single launch, with
// the L_iso gradient added to the log-scale gradient on the fly. The launch's
// blocks are split into five segments (means, log-scales, quaternions,
// opacity logits, colours); each element is read once (parameter, gradient,
// two moments) and written once (parameter, two moments), so the step is one
// pass over 7 floats of traffic per parameter. The step counter lives on the
// device and a second, one-thread kernel advances it, so the step replays
// from a CUDA graph. C ABI in include/s3gs_slam.h.
#include <cstdio>
#include <cstring>

#include "../../include/s3gs_slam.h"
#include "s3gs_internal.cuh"

namespace s3gs {
namespace {

constexpr int kAdamThreads = 256;
constexpr int kSegments = 5;

struct AdamArgs {
    float *p[kSegments];
    const float *g[kSegments];
    float *m[kSegments];
    float *v[kSegments];
    long long count[kSegments];   // elements (log-scales: Gaussians)
    int block_end[kSegments];     // exclusive end of each segment's blocks
    float lr[kSegments];
    float lr_rest;                // colour coefficients 1.. (SH bands l >= 1)
    int nc;                       // colour coefficients per Gaussian
    float beta1, beta2, eps, lambda_iso;
    const int *step;
};

__device__ __forceinline__ void adam_one(float &p, float g, float &m, float &v, float lr, float b1, float b2,
                                         float eps, float c1, float c2) {
    m = b1 * m + (1.0f - b1) * g;
    v = b2 * v + (1.0f - b2) * g * g;
    p -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void __launch_bounds__(kAdamThreads) map_adam_kernel(const __grid_constant__ AdamArgs a) {
    __shared__ float s_c[2];
    if (threadIdx.x == 0) {
        const float t = (float)(*a.step + 1);
        s_c[0] = 1.0f - powf(a.beta1, t);
        s_c[1] = 1.0f - powf(a.beta2, t);
    }
    __syncthreads();
    const float c1 = s_c[0], c2 = s_c[1];
    int seg = 0;
    while (seg < kSegments - 1 && (int)blockIdx.x >= a.block_end[seg]) ++seg;
    const int b0 = seg == 0 ? 0 : a.block_end[seg - 1];
    const long long nthreads = (long long)(a.block_end[seg] - b0) * kAdamThreads;
    float *P = a.p[seg], *M = a.m[seg], *Vv = a.v[seg];
    const float *G = a.g[seg];
    const float lr = a.lr[seg];
    for (long long i = (long long)(blockIdx.x - b0) * kAdamThreads + threadIdx.x; i < a.count[seg]; i += nthreads) {
        if (seg == 1) {
            // one Gaussian's three log-scales, with the gradient of L_iso (Eq. 16)
            float ls[3], s[3], g[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ls[k] = P[3 * i + k];
                s[k] = expf(ls[k]);
                g[k] = G ? G[3 * i + k] : 0.f;
            }
            const float mean = (s[0] + s[1] + s[2]) * (1.0f / 3.0f);
            float sg[3], ssum = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float d = s[k] - mean;
                sg[k] = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                ssum += sg[k];
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float gi = g[k] + a.lambda_iso * (sg[k] - ssum * (1.0f / 3.0f)) * s[k];
                float pm = M[3 * i + k], pv = Vv[3 * i + k];
                adam_one(ls[k], gi, pm, pv, lr, a.beta1, a.beta2, a.eps, c1, c2);
                P[3 * i + k] = ls[k];
                M[3 * i + k] = pm;
                Vv[3 * i + k] = pv;
            }
        } else {
            float pp = P[i], pm = M[i], pv = Vv[i];
            const float g = G ? G[i] : 0.f;
            float r = lr;
            if (seg == 4 && ((i / 3) % a.nc) != 0) r = a.lr_rest;
            adam_one(pp, g, pm, pv, r, a.beta1, a.beta2, a.eps, c1, c2);
            P[i] = pp;
            M[i] = pm;
            Vv[i] = pv;
        }
    }
}

__global__ void step_advance_kernel(int *step) { *step += 1; }

bool finite_nonneg(float x) { return x == x && x >= 0.f && x < 3.0e38f; }

}  // namespace
}  // namespace s3gs

using namespace s3gs;

extern "C" {

void s3gs_map_adam_default(s3gs_map_adam *hp) {
    if (!hp) return;
    hp->lr_means = 1.6e-4f;
    hp->lr_log_scales = 5e-3f;
    hp->lr_quats = 1e-3f;
    hp->lr_opacity = 5e-2f;
    hp->lr_colors = 2.5e-3f;
    hp->lr_colors_rest = 2.5e-3f / 20.0f;
    hp->beta1 = 0.9f;
    hp->beta2 = 0.999f;
    hp->eps = 1e-15f;
    hp->lambda_iso = 10.0f;
}

s3gs_status s3gs_map_adam_step(s3gs_ctx *ctx, int64_t n, int32_t sh_degree, float *const params[5],
                               const float *const grads[5], float *const adam_m[5], float *const adam_v[5],
                               int32_t *step, const s3gs_map_adam *hp, void *stream) {
    if (!ctx) return S3GS_E_INVALID;
    if (!params || !grads || !adam_m || !adam_v || !step || !hp || n < 0 || sh_degree < 0 ||
        sh_degree > S3GS_MAX_SH_DEGREE)
        return ctx_error(ctx, S3GS_E_INVALID, "map_adam_step: NULL argument, n < 0 or sh_degree outside 0..3");
    for (int k = 0; k < kSegments; ++k)
        if (n > 0 && (!params[k] || !adam_m[k] || !adam_v[k]))
            return ctx_error(ctx, S3GS_E_INVALID, "map_adam_step: a parameter or moment pointer is NULL");
    const float lrs[6] = {hp->lr_means, hp->lr_log_scales, hp->lr_quats, hp->lr_opacity, hp->lr_colors,
                          hp->lr_colors_rest};
    for (float x : lrs)
        if (!finite_nonneg(x)) return ctx_error(ctx, S3GS_E_INVALID, "map_adam_step: learning rates must be >= 0");
    if (!(hp->beta1 >= 0.f && hp->beta1 < 1.f && hp->beta2 >= 0.f && hp->beta2 < 1.f && hp->eps > 0.f &&
          hp->eps < 1e30f && finite_nonneg(hp->lambda_iso)))
        return ctx_error(ctx, S3GS_E_INVALID, "map_adam_step: betas in [0, 1), eps > 0, lambda_iso >= 0 required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n > 0) {
        AdamArgs a;
        memset(&a, 0, sizeof(a));
        const int nc = (sh_degree + 1) * (sh_degree + 1);
        const long long counts[kSegments] = {3 * n, n, 4 * n, n, 3LL * nc * n};
        int dev_sms = 152;
        cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx_device(ctx));
        int blocks = 0;
        for (int k = 0; k < kSegments; ++k) {
            a.p[k] = params[k];
            a.g[k] = grads[k];
            a.m[k] = adam_m[k];
            a.v[k] = adam_v[k];
            a.count[k] = counts[k];
            a.lr[k] = lrs[k];
            // blocks in proportion to the segment's traffic, at most 8 per SM per segment
            long long want = (counts[k] * (k == 1 ? 3 : 1) + kAdamThreads * 4 - 1) / (kAdamThreads * 4);
            const long long cap = 8LL * dev_sms;
            blocks += (int)(want < 1 ? 1 : (want > cap ? cap : want));
            a.block_end[k] = blocks;
        }
        a.lr_rest = hp->lr_colors_rest;
        a.nc = nc;
        a.beta1 = hp->beta1;
        a.beta2 = hp->beta2;
        a.eps = hp->eps;
        a.lambda_iso = hp->lambda_iso;
        a.step = step;
        map_adam_kernel<<<blocks, kAdamThreads, 0, s>>>(a);
    }
    step_advance_kernel<<<1, 1, 0, s>>>(step);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "map_adam_step: %s (%s)", cudaGetErrorName(e), cudaGetErrorString(e));
        return ctx_error(ctx, S3GS_E_CUDA, msg);
    }
    return S3GS_OK;
}

}  // extern "C"
