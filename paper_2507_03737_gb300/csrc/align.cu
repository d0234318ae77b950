// Patch-based pointmap scale alignment (Sec. 3.3.1; Algorithm 1 of the
// supplementary material), pointmap replacement (Sec. 3.3.2, Eq. 14) and the
// remedial scale factor, for every view of a batch (C ABI in
// include/s3gs_slam.h).
//
// One alignment iteration is one pass over both pointmaps. A CTA stages a band
// of P rows by ppc * P columns (ppc = 128 / P patches) of X^r and X^p in shared
// memory, computes the joint mean and population standard deviation of each
// of its patches (mean first, then centred squares, both from shared memory),
// gates the patches, tests every point of the candidate patches and reduces
// the correct points' coordinate sums and count to one partial per CTA. An
// update kernel sums each view's partials in a fixed order (in double) and
// rewrites the view's factor in place, so all iterations run back to back on
// the stream with no host round trip and the result is deterministic.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/s3gs_slam.h"
#include "s3gs_internal.cuh"

namespace s3gs {
namespace {

constexpr int kAlignThreads = 128;  // small CTAs: about 7 resident per SM at P = 10
constexpr int kMaxDevices = 64;

struct AlignView {
    int w, h;
    int bands, chunks;  // patch rows of the view; CTAs per patch row
    int unit_base;      // first CTA of this view
    int pad;
    long long pix_base;  // first pixel of the view in the packed layout
};

struct AlignBatch {
    int n_views, P, ppc, total_units;
    float delta_mu, delta_sigma, eps_r, tau;
    AlignView v[S3GS_MAX_VIEWS];
};

struct AlignPartial {
    float sum_r, sum_p;  // coordinate sums of X^r and (unscaled) X^p over the CTA's correct points
    unsigned count, pad;
};

int align_ppc(int P) { return kAlignThreads / P; }

size_t align_smem_bytes(int P) {
    const int ppc = align_ppc(P), maxc = ppc * P;
    return sizeof(float) * ((size_t)6 * P * maxc + 2 * (size_t)maxc + 4 * (size_t)ppc) + sizeof(int) * ppc;
}

// 4-byte asynchronous global -> shared copy (no register staging), and the
// wait for all of this thread's outstanding copies.
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__global__ void align_init_kernel(const float *sigma_init, float *sigma, int n_views) {
    const int v = threadIdx.x;
    if (v < n_views) sigma[v] = sigma_init ? sigma_init[v] : 1.0f;
}

__global__ void __launch_bounds__(kAlignThreads)
    align_pass_kernel(const float *__restrict__ Xr, const float *__restrict__ Xp, const float *__restrict__ sigma,
                      AlignPartial *__restrict__ part, unsigned char *__restrict__ cp_mask,
                      const __grid_constant__ AlignBatch b) {
    extern __shared__ float sm[];
    __shared__ float s_red[3][kAlignThreads / 32];
    const int unit = blockIdx.x;
    int v = 0;
    while (v + 1 < b.n_views && b.v[v + 1].unit_base <= unit) ++v;
    const AlignView &vw = b.v[v];
    const int local = unit - vw.unit_base;
    const int band = local / vw.chunks, chunk = local - band * vw.chunks;
    const int P = b.P, ppc = b.ppc, maxc = ppc * P;
    const int y0 = band * P, rows = min(P, vw.h - y0);
    const int x0 = chunk * maxc, ncols = min(maxc, vw.w - x0);
    const int npatch = (ncols + P - 1) / P;
    float *s_r = sm;                     // [3][P][maxc]
    float *s_p = s_r + 3 * P * maxc;     // [3][P][maxc]
    float *s_col = s_p + 3 * P * maxc;   // [2][maxc] per-column partial sums
    float *s_mu = s_col + 2 * maxc;      // [2][ppc] patch means of X^r, s X^p
    float *s_sd = s_mu + 2 * ppc;        // [2][ppc] reciprocal standard deviations (candidates)
    int *s_cand = reinterpret_cast<int *>(s_sd + 2 * ppc);  // [ppc]

    const long long HW = (long long)vw.w * vw.h;
    const float s = sigma[v];
    const int t = threadIdx.x;
    const bool col = t < ncols;
    const int j = t / P;  // patch of this thread's column
    // Each thread copies its own column of both maps into shared memory with
    // asynchronous copies (coalesced across the warp for every channel and row;
    // all of a thread's copies are in flight at once), then sums it.
    if (col) {
        const float *rc = Xr + 3 * vw.pix_base + (long long)y0 * vw.w + x0 + t;
        const float *pc = Xp + 3 * vw.pix_base + (long long)y0 * vw.w + x0 + t;
        for (int c = 0; c < 3; ++c)
            for (int y = 0; y < rows; ++y) {
                const long long off = c * HW + (long long)y * vw.w;
                cp_async4(s_r + (c * P + y) * maxc + t, rc + off);
                cp_async4(s_p + (c * P + y) * maxc + t, pc + off);
            }
    }
    cp_async_wait_all();
    if (col) {
        float a = 0.f, q = 0.f;
        for (int c = 0; c < 3; ++c)
            for (int y = 0; y < rows; ++y) {
                a += s_r[(c * P + y) * maxc + t];
                q += s_p[(c * P + y) * maxc + t];
            }
        s_col[t] = a;
        s_col[maxc + t] = q;
    }
    __syncthreads();
    if (t < npatch) {
        const int c0 = t * P, c1 = min(c0 + P, ncols);
        float a = 0.f, q = 0.f;
        for (int x = c0; x < c1; ++x) {
            a += s_col[x];
            q += s_col[maxc + x];
        }
        const float nval = (float)(3 * rows * (c1 - c0));
        s_mu[t] = a / nval;
        s_mu[ppc + t] = s * (q / nval);
    }
    __syncthreads();
    if (col) {
        const float mr = s_mu[j], mp = s_mu[ppc + j];
        float a = 0.f, q = 0.f;
        for (int c = 0; c < 3; ++c)
            for (int y = 0; y < rows; ++y) {
                const float dr = s_r[(c * P + y) * maxc + t] - mr;
                const float dp = fmaf(s, s_p[(c * P + y) * maxc + t], -mp);
                a = fmaf(dr, dr, a);
                q = fmaf(dp, dp, q);
            }
        s_col[t] = a;
        s_col[maxc + t] = q;
    }
    __syncthreads();
    if (t < npatch) {
        const int c0 = t * P, c1 = min(c0 + P, ncols);
        float a = 0.f, q = 0.f;
        for (int x = c0; x < c1; ++x) {
            a += s_col[x];
            q += s_col[maxc + x];
        }
        const float nval = (float)(3 * rows * (c1 - c0));
        const float sd_r = sqrtf(a / nval), sd_p = sqrtf(q / nval);
        const float mr = s_mu[t], mp = s_mu[ppc + t];
        const bool cand = fabsf(mr - mp) < b.delta_mu * mp && fabsf(sd_r - sd_p) < b.delta_sigma * sd_p;
        // a candidate has sd_p > 0 and sd_r > (1 - delta_sigma) sd_p; store reciprocals
        s_sd[t] = cand ? 1.0f / sd_r : 0.f;
        s_sd[ppc + t] = cand ? 1.0f / sd_p : 0.f;
        s_cand[t] = cand;
    }
    __syncthreads();

    float acc_r = 0.f, acc_p = 0.f;
    unsigned cnt = 0;
    if (col) {
        const bool cand = s_cand[j] != 0;
        const float mr = s_mu[j], mp = s_mu[ppc + j], isr = s_sd[j], isp = s_sd[ppc + j];
        unsigned char *mrow = cp_mask ? cp_mask + vw.pix_base + (long long)y0 * vw.w + x0 + t : nullptr;
        for (int y = 0; y < rows; ++y) {
            bool cp = false;
            if (cand) {
                float d2 = 0.f, vr = 0.f, vp = 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float xr = s_r[(c * P + y) * maxc + t], xp = s_p[(c * P + y) * maxc + t];
                    const float e = (xr - mr) * isr - fmaf(s, xp, -mp) * isp;
                    d2 = fmaf(e, e, d2);
                    vr += xr;
                    vp += xp;
                }
                cp = sqrtf(d2) < b.eps_r;
                if (cp) {
                    acc_r += vr;
                    acc_p += vp;
                    ++cnt;
                }
            }
            if (mrow) mrow[(long long)y * vw.w] = cp ? 1 : 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_r += __shfl_xor_sync(0xffffffffu, acc_r, o);
        acc_p += __shfl_xor_sync(0xffffffffu, acc_p, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((t & 31) == 0) {
        s_red[0][t >> 5] = acc_r;
        s_red[1][t >> 5] = acc_p;
        s_red[2][t >> 5] = __uint_as_float(cnt);
    }
    __syncthreads();
    if (t == 0) {
        AlignPartial out;
        out.sum_r = 0.f;
        out.sum_p = 0.f;
        out.count = 0;
        out.pad = 0;
        for (int w = 0; w < kAlignThreads / 32; ++w) {
            out.sum_r += s_red[0][w];
            out.sum_p += s_red[1][w];
            out.count += __float_as_uint(s_red[2][w]);
        }
        part[unit] = out;
    }
}

// The same pass for a compile-time patch size PP (the paper's P = 10): each
// thread holds its column of both maps (3 PP values each) in registers, loaded
// all at once, so only the per-column partial sums and the patch statistics go
// through shared memory. Decisions and partials are computed by the same
// formulas as align_pass_kernel.
template <int PP>
__global__ void __launch_bounds__(kAlignThreads)
    align_pass_reg_kernel(const float *__restrict__ Xr, const float *__restrict__ Xp, const float *__restrict__ sigma,
                          AlignPartial *__restrict__ part, unsigned char *__restrict__ cp_mask,
                          const __grid_constant__ AlignBatch b) {
    constexpr int ppc = kAlignThreads / PP, maxc = ppc * PP;
    __shared__ float s_col[2][maxc];
    __shared__ float s_mu[2][ppc], s_sd[2][ppc];
    __shared__ int s_cand[ppc];
    __shared__ float s_red[3][kAlignThreads / 32];
    const int unit = blockIdx.x;
    int v = 0;
    while (v + 1 < b.n_views && b.v[v + 1].unit_base <= unit) ++v;
    const AlignView &vw = b.v[v];
    const int local = unit - vw.unit_base;
    const int band = local / vw.chunks, chunk = local - band * vw.chunks;
    const int y0 = band * PP, rows = min(PP, vw.h - y0);
    const int x0 = chunk * maxc, ncols = min(maxc, vw.w - x0);
    const int npatch = (ncols + PP - 1) / PP;
    const long long HW = (long long)vw.w * vw.h;
    const float s = sigma[v];
    const int t = threadIdx.x;
    const bool col = t < ncols;
    const int j = t / PP;
    float xr[3][PP], xp[3][PP];
    if (col) {
        const float *rc = Xr + 3 * vw.pix_base + (long long)y0 * vw.w + x0 + t;
        const float *pc = Xp + 3 * vw.pix_base + (long long)y0 * vw.w + x0 + t;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int y = 0; y < PP; ++y) {
                const bool in = y < rows;
                const long long off = c * HW + (long long)y * vw.w;
                xr[c][y] = in ? __ldg(rc + off) : 0.f;
                xp[c][y] = in ? __ldg(pc + off) : 0.f;
            }
        float a = 0.f, q = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int y = 0; y < PP; ++y)
                if (y < rows) {
                    a += xr[c][y];
                    q += xp[c][y];
                }
        s_col[0][t] = a;
        s_col[1][t] = q;
    }
    __syncthreads();
    if (t < npatch) {
        const int c0 = t * PP, c1 = min(c0 + PP, ncols);
        float a = 0.f, q = 0.f;
        for (int x = c0; x < c1; ++x) {
            a += s_col[0][x];
            q += s_col[1][x];
        }
        const float nval = (float)(3 * rows * (c1 - c0));
        s_mu[0][t] = a / nval;
        s_mu[1][t] = s * (q / nval);
    }
    __syncthreads();
    if (col) {
        const float mr = s_mu[0][j], mp = s_mu[1][j];
        float a = 0.f, q = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int y = 0; y < PP; ++y)
                if (y < rows) {
                    const float dr = xr[c][y] - mr;
                    const float dp = fmaf(s, xp[c][y], -mp);
                    a = fmaf(dr, dr, a);
                    q = fmaf(dp, dp, q);
                }
        s_col[0][t] = a;
        s_col[1][t] = q;
    }
    __syncthreads();
    if (t < npatch) {
        const int c0 = t * PP, c1 = min(c0 + PP, ncols);
        float a = 0.f, q = 0.f;
        for (int x = c0; x < c1; ++x) {
            a += s_col[0][x];
            q += s_col[1][x];
        }
        const float nval = (float)(3 * rows * (c1 - c0));
        const float sd_r = sqrtf(a / nval), sd_p = sqrtf(q / nval);
        const float mr = s_mu[0][t], mp = s_mu[1][t];
        const bool cand = fabsf(mr - mp) < b.delta_mu * mp && fabsf(sd_r - sd_p) < b.delta_sigma * sd_p;
        s_sd[0][t] = cand ? 1.0f / sd_r : 0.f;
        s_sd[1][t] = cand ? 1.0f / sd_p : 0.f;
        s_cand[t] = cand;
    }
    __syncthreads();
    float acc_r = 0.f, acc_p = 0.f;
    unsigned cnt = 0;
    if (col) {
        const bool cand = s_cand[j] != 0;
        const float mr = s_mu[0][j], mp = s_mu[1][j], isr = s_sd[0][j], isp = s_sd[1][j];
        unsigned char *mrow = cp_mask ? cp_mask + vw.pix_base + (long long)y0 * vw.w + x0 + t : nullptr;
#pragma unroll
        for (int y = 0; y < PP; ++y) {
            if (y >= rows) break;
            bool cp = false;
            if (cand) {
                float d2 = 0.f, vr = 0.f, vp = 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float e = (xr[c][y] - mr) * isr - fmaf(s, xp[c][y], -mp) * isp;
                    d2 = fmaf(e, e, d2);
                    vr += xr[c][y];
                    vp += xp[c][y];
                }
                cp = sqrtf(d2) < b.eps_r;
                if (cp) {
                    acc_r += vr;
                    acc_p += vp;
                    ++cnt;
                }
            }
            if (mrow) mrow[(long long)y * vw.w] = cp ? 1 : 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_r += __shfl_xor_sync(0xffffffffu, acc_r, o);
        acc_p += __shfl_xor_sync(0xffffffffu, acc_p, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((t & 31) == 0) {
        s_red[0][t >> 5] = acc_r;
        s_red[1][t >> 5] = acc_p;
        s_red[2][t >> 5] = __uint_as_float(cnt);
    }
    __syncthreads();
    if (t == 0) {
        AlignPartial out;
        out.sum_r = 0.f;
        out.sum_p = 0.f;
        out.count = 0;
        out.pad = 0;
        for (int w = 0; w < kAlignThreads / 32; ++w) {
            out.sum_r += s_red[0][w];
            out.sum_p += s_red[1][w];
            out.count += __float_as_uint(s_red[2][w]);
        }
        part[unit] = out;
    }
}

// One CTA per view: fixed-order double sum of the view's partials, then the
// factor update of Algorithm 1 (an empty CP keeps the previous factor).
__global__ void __launch_bounds__(kAlignThreads)
    align_update_kernel(const AlignPartial *__restrict__ part, float *__restrict__ sigma, long long *n_cp,
                        int *insufficient, const __grid_constant__ AlignBatch b) {
    __shared__ double s_a[kAlignThreads], s_q[kAlignThreads];
    __shared__ unsigned long long s_c[kAlignThreads];
    const int v = blockIdx.x;
    const AlignView &vw = b.v[v];
    const int n_units = vw.bands * vw.chunks;
    double a = 0.0, q = 0.0;
    unsigned long long c = 0;
    for (int i = threadIdx.x; i < n_units; i += kAlignThreads) {
        const AlignPartial p = part[vw.unit_base + i];
        a += (double)p.sum_r;
        q += (double)p.sum_p;
        c += p.count;
    }
    s_a[threadIdx.x] = a;
    s_q[threadIdx.x] = q;
    s_c[threadIdx.x] = c;
    __syncthreads();
    for (int h = kAlignThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s_a[threadIdx.x] += s_a[threadIdx.x + h];
            s_q[threadIdx.x] += s_q[threadIdx.x + h];
            s_c[threadIdx.x] += s_c[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long total = s_c[0];
        if (total > 0) sigma[v] = (float)(s_a[0] / s_q[0]);
        if (n_cp) n_cp[v] = (long long)total;
        if (insufficient) insufficient[v] = (double)total < (double)b.tau * (double)vw.w * (double)vw.h ? 1 : 0;
    }
}

struct ReplaceViews {
    int n_views;
    int w[S3GS_MAX_VIEWS], h[S3GS_MAX_VIEWS];
    long long pix_base[S3GS_MAX_VIEWS];
};

__global__ void __launch_bounds__(256)
    replace_kernel(const float *__restrict__ Xr, const float *__restrict__ Xp, const float *__restrict__ sigma,
                   float eps_m, float *Xr_hat, float *__restrict__ Xp_hat, unsigned char *__restrict__ replaced,
                   unsigned long long *n_replaced, const __grid_constant__ ReplaceViews rv) {
    const int v = blockIdx.y;
    const long long HW = (long long)rv.w[v] * rv.h[v];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool rep = false;
    if (i < HW) {
        const long long base = 3 * rv.pix_base[v] + i;
        const float s = sigma[v];
        float xr[3], ph[3];
        float e2 = 0.f, n2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xr[c] = Xr[base + c * HW];
            ph[c] = s * __ldg(Xp + base + c * HW);
            const float d = xr[c] - ph[c];
            e2 = fmaf(d, d, e2);
            n2 = fmaf(ph[c], ph[c], n2);
        }
        rep = sqrtf(e2) > eps_m * sqrtf(n2);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Xr_hat[base + c * HW] = rep ? ph[c] : xr[c];
            if (Xp_hat) Xp_hat[base + c * HW] = ph[c];
        }
        if (replaced) replaced[rv.pix_base[v] + i] = rep ? 1 : 0;
    }
    if (n_replaced) {
        const unsigned bal = __ballot_sync(0xffffffffu, rep);
        if ((threadIdx.x & 31) == 0 && bal) atomicAdd(n_replaced + v, (unsigned long long)__popc(bal));
    }
}

__global__ void __launch_bounds__(512)
    remedy_kernel(const float *__restrict__ A, long long hwa, const float *__restrict__ B, long long hwb,
                  const int *__restrict__ matches, long long n, float *sigma, long long *n_used) {
    __shared__ double s_a[512], s_b[512];
    __shared__ long long s_n[512];
    double a = 0.0, q = 0.0;
    long long used = 0;
    for (long long k = threadIdx.x; k < n; k += blockDim.x) {
        const int ia = matches[2 * k], ib = matches[2 * k + 1];
        if (ia < 0 || ib < 0 || ia >= hwa || ib >= hwb) continue;
        a += (double)A[ia] + (double)A[hwa + ia] + (double)A[2 * hwa + ia];
        q += (double)B[ib] + (double)B[hwb + ib] + (double)B[2 * hwb + ib];
        ++used;
    }
    s_a[threadIdx.x] = a;
    s_b[threadIdx.x] = q;
    s_n[threadIdx.x] = used;
    __syncthreads();
    for (int h = 256; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s_a[threadIdx.x] += s_a[threadIdx.x + h];
            s_b[threadIdx.x] += s_b[threadIdx.x + h];
            s_n[threadIdx.x] += s_n[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sigma[0] = s_n[0] > 0 ? (float)(s_a[0] / s_b[0]) : 1.0f;
        if (n_used) n_used[0] = s_n[0];
    }
}

bool fill_batch(const int32_t *view_wh, int n_views, int P, AlignBatch &b, const char **why) {
    if (!view_wh) { *why = "view sizes are NULL"; return false; }
    if (n_views < 1 || n_views > S3GS_MAX_VIEWS) { *why = "n_views must be in 1..S3GS_MAX_VIEWS"; return false; }
    if (P < 1 || P > S3GS_MAX_PATCH) { *why = "patch must be in 1..S3GS_MAX_PATCH"; return false; }
    memset(&b, 0, sizeof(b));
    b.n_views = n_views;
    b.P = P;
    b.ppc = align_ppc(P);
    long long units = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const int w = view_wh[2 * v], h = view_wh[2 * v + 1];
        if (w < 1 || h < 1 || w > 65536 || h > 65536) { *why = "view width/height must be in 1..65536"; return false; }
        AlignView &a = b.v[v];
        a.w = w;
        a.h = h;
        a.bands = (h + P - 1) / P;
        a.chunks = ((w + P - 1) / P + b.ppc - 1) / b.ppc;
        a.unit_base = (int)units;
        a.pix_base = pix;
        units += (long long)a.bands * a.chunks;
        pix += (long long)w * h;
    }
    if (units > (1LL << 30)) { *why = "too many patches"; return false; }
    b.total_units = (int)units;
    return true;
}

std::mutex g_attr_mu;
size_t g_attr_bytes[kMaxDevices] = {};

cudaError_t ensure_align_smem(int device, size_t bytes) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (g_attr_bytes[device] >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(align_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g_attr_bytes[device] = bytes;
    return e;
}

s3gs_status launch_error(s3gs_ctx *ctx, cudaError_t e, const char *where) {
    char msg[256];
    snprintf(msg, sizeof(msg), "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
    return ctx_error(ctx, S3GS_E_CUDA, msg);
}

bool finite_nonneg(float x) { return x == x && x >= 0.f && x < 3.0e38f; }

}  // namespace
}  // namespace s3gs

using namespace s3gs;

extern "C" {

void s3gs_align_params_default(s3gs_align_params *p) {
    if (!p) return;
    p->patch = 10;
    p->delta_mu = 0.3f;
    p->delta_sigma = 0.3f;
    p->eps_r = 0.1f;
    p->max_iter = 3;
    p->tau = 0.01f;
}

s3gs_status s3gs_scale_align_workspace(const int32_t *view_wh, int32_t n_views, int32_t patch, size_t *bytes) {
    if (!bytes) return S3GS_E_INVALID;
    AlignBatch b;
    const char *why = nullptr;
    if (!fill_batch(view_wh, n_views, patch, b, &why)) return S3GS_E_INVALID;
    *bytes = sizeof(AlignPartial) * (size_t)b.total_units;
    return S3GS_OK;
}

s3gs_status s3gs_scale_align(s3gs_ctx *ctx, const int32_t *view_wh, int32_t n_views, const float *X_r,
                             const float *X_p, const s3gs_align_params *params, const float *sigma_init,
                             float *sigma, int64_t *n_cp, int32_t *insufficient, uint8_t *cp_mask,
                             void *workspace, size_t workspace_bytes, void *stream) {
    if (!ctx) return S3GS_E_INVALID;
    if (!X_r || !X_p || !params || !sigma || !workspace)
        return ctx_error(ctx, S3GS_E_INVALID, "scale_align: NULL pointmap, params, sigma or workspace");
    AlignBatch b;
    const char *why = nullptr;
    if (!fill_batch(view_wh, n_views, params->patch, b, &why))
        return ctx_error(ctx, S3GS_E_INVALID, (std::string("scale_align: ") + why).c_str());
    if (params->max_iter < 1 || params->max_iter > 64)
        return ctx_error(ctx, S3GS_E_INVALID, "scale_align: max_iter must be in 1..64");
    if (!finite_nonneg(params->delta_mu) || !finite_nonneg(params->delta_sigma) || !finite_nonneg(params->eps_r) ||
        !finite_nonneg(params->tau))
        return ctx_error(ctx, S3GS_E_INVALID, "scale_align: thresholds must be finite and >= 0");
    if (workspace_bytes < sizeof(AlignPartial) * (size_t)b.total_units ||
        (reinterpret_cast<uintptr_t>(workspace) & 15u) != 0)
        return ctx_error(ctx, S3GS_E_INVALID, "scale_align: workspace too small or not 16-byte aligned");
    b.delta_mu = params->delta_mu;
    b.delta_sigma = params->delta_sigma;
    b.eps_r = params->eps_r;
    b.tau = params->tau;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t smem = align_smem_bytes(b.P);
    cudaError_t e = ensure_align_smem(ctx_device(ctx), smem);
    if (e != cudaSuccess) return launch_error(ctx, e, "scale_align: shared-memory attribute");
    AlignPartial *part = static_cast<AlignPartial *>(workspace);
    align_init_kernel<<<1, S3GS_MAX_VIEWS, 0, s>>>(sigma_init, sigma, n_views);
    for (int it = 0; it < params->max_iter; ++it) {
        const bool last = it + 1 == params->max_iter;
        if (b.P == 10)
            align_pass_reg_kernel<10><<<b.total_units, kAlignThreads, 0, s>>>(X_r, X_p, sigma, part,
                                                                             last ? cp_mask : nullptr, b);
        else
            align_pass_kernel<<<b.total_units, kAlignThreads, smem, s>>>(X_r, X_p, sigma, part,
                                                                         last ? cp_mask : nullptr, b);
        align_update_kernel<<<n_views, kAlignThreads, 0, s>>>(part, sigma, last ? reinterpret_cast<long long *>(n_cp)
                                                                                : nullptr,
                                                              last ? insufficient : nullptr, b);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return launch_error(ctx, e, "scale_align");
    return S3GS_OK;
}

s3gs_status s3gs_pointmap_replace(s3gs_ctx *ctx, const int32_t *view_wh, int32_t n_views, const float *X_r,
                                  const float *X_p, const float *sigma, float eps_m, float *X_r_hat,
                                  float *X_p_hat, uint8_t *replaced, int64_t *n_replaced, void *stream) {
    if (!ctx) return S3GS_E_INVALID;
    if (!X_r || !X_p || !sigma || !X_r_hat || !view_wh)
        return ctx_error(ctx, S3GS_E_INVALID, "pointmap_replace: NULL pointmap, sigma, output or view sizes");
    if (n_views < 1 || n_views > S3GS_MAX_VIEWS)
        return ctx_error(ctx, S3GS_E_INVALID, "pointmap_replace: n_views must be in 1..S3GS_MAX_VIEWS");
    if (!finite_nonneg(eps_m)) return ctx_error(ctx, S3GS_E_INVALID, "pointmap_replace: eps_m must be finite and >= 0");
    ReplaceViews rv;
    memset(&rv, 0, sizeof(rv));
    rv.n_views = n_views;
    long long pix = 0, max_hw = 0;
    for (int v = 0; v < n_views; ++v) {
        const int w = view_wh[2 * v], h = view_wh[2 * v + 1];
        if (w < 1 || h < 1 || w > 65536 || h > 65536)
            return ctx_error(ctx, S3GS_E_INVALID, "pointmap_replace: view width/height must be in 1..65536");
        rv.w[v] = w;
        rv.h[v] = h;
        rv.pix_base[v] = pix;
        pix += (long long)w * h;
        max_hw = (long long)w * h > max_hw ? (long long)w * h : max_hw;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_replaced) {
        cudaError_t e = cudaMemsetAsync(n_replaced, 0, sizeof(int64_t) * n_views, s);
        if (e != cudaSuccess) return launch_error(ctx, e, "pointmap_replace: clear counts");
    }
    dim3 grid((unsigned)((max_hw + 255) / 256), (unsigned)n_views);
    replace_kernel<<<grid, 256, 0, s>>>(X_r, X_p, sigma, eps_m, X_r_hat, X_p_hat, replaced,
                                        reinterpret_cast<unsigned long long *>(n_replaced), rv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return launch_error(ctx, e, "pointmap_replace");
    return S3GS_OK;
}

s3gs_status s3gs_scale_remedy(s3gs_ctx *ctx, const float *X_ak_hat, int64_t hw_ak, const float *X_n, int64_t hw_n,
                              const int32_t *matches, int64_t n_matches, float *sigma, int64_t *n_used,
                              void *stream) {
    if (!ctx) return S3GS_E_INVALID;
    if (!X_ak_hat || !X_n || !sigma || (n_matches > 0 && !matches))
        return ctx_error(ctx, S3GS_E_INVALID, "scale_remedy: NULL pointmap, matches or sigma");
    if (hw_ak < 1 || hw_n < 1 || hw_ak > (1LL << 31) - 1 || hw_n > (1LL << 31) - 1 || n_matches < 0)
        return ctx_error(ctx, S3GS_E_INVALID, "scale_remedy: sizes out of range");
    remedy_kernel<<<1, 512, 0, static_cast<cudaStream_t>(stream)>>>(X_ak_hat, hw_ak, X_n, hw_n, matches, n_matches,
                                                                    sigma, reinterpret_cast<long long *>(n_used));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return launch_error(ctx, e, "scale_remedy");
    return S3GS_OK;
}

}  // extern "C"
