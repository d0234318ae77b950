// Keyframe covisibility and window management (supplementary material,
// "Keyframe Management": Eq. S1/S2 and the selection rules after them).
//
// covis_kernel: pairwise intersection counts |G_i & G_j| of the views' visible
// Gaussian sets, from the per-Gaussian view bitmask the projection writes.
// Each warp takes 32 Gaussians at a time; one ballot per view turns the 32
// masks into the view's 32-bit membership word, and every lane counts its
// share of the V (V + 1) / 2 view pairs with popc(word_i & word_j). Counts are
// integers, so the result does not depend on the order of the atomic sums.
//
// median kernels: lower median of the positive depths of each view by a
// three-level radix select on the float bits (positive floats order like their
// bit patterns): 11 + 11 + 9 bits, one histogram pass and one select step per
// level, all views of a batch at once.
//
// The window rules are host logic on a handful of numbers per keyframe.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../include/s3gs_slam.h"
#include "s3gs_internal.cuh"

namespace s3gs {
namespace {

constexpr int kCovisThreads = 256;
constexpr int kMaxPairs = S3GS_MAX_VIEWS * (S3GS_MAX_VIEWS + 1) / 2;  // 528
constexpr int kPairSlots = (kMaxPairs + 31) / 32;                      // 17 per lane

struct CovisArgs {
    const unsigned *vis;
    long long n;
    int V, n_pairs;
    unsigned long long *counts;  // [V][V], upper triangle accumulated
    unsigned char pi[kMaxPairs], pj[kMaxPairs];
};

__global__ void __launch_bounds__(kCovisThreads) covis_kernel(const __grid_constant__ CovisArgs a) {
    __shared__ unsigned s_b[kCovisThreads / 32][S3GS_MAX_VIEWS];
    __shared__ unsigned s_acc[kMaxPairs];
    __shared__ unsigned char s_pi[kMaxPairs], s_pj[kMaxPairs];  // lane-varying indices: keep them out of the
                                                                 // constant bank, which serialises them
    for (int p = threadIdx.x; p < a.n_pairs; p += kCovisThreads) {
        s_acc[p] = 0u;
        s_pi[p] = a.pi[p];
        s_pj[p] = a.pj[p];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned cnt[kPairSlots];
#pragma unroll
    for (int k = 0; k < kPairSlots; ++k) cnt[k] = 0u;
    const long long stride = (long long)gridDim.x * (kCovisThreads / 32) * 32;
    for (long long base = ((long long)blockIdx.x * (kCovisThreads / 32) + warp) * 32; base < a.n; base += stride) {
        const long long g = base + lane;
        const unsigned m = g < a.n ? a.vis[g] : 0u;
        for (int i = 0; i < a.V; ++i) {
            const unsigned word = __ballot_sync(0xffffffffu, (m >> i) & 1u);
            if (lane == i) s_b[warp][i] = word;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < kPairSlots; ++k) {
            const int p = lane + 32 * k;
            if (p < a.n_pairs) cnt[k] += __popc(s_b[warp][s_pi[p]] & s_b[warp][s_pj[p]]);
        }
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < kPairSlots; ++k) {
        const int p = lane + 32 * k;
        if (p < a.n_pairs && cnt[k]) atomicAdd(&s_acc[p], cnt[k]);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < a.n_pairs; p += kCovisThreads)
        if (s_acc[p]) atomicAdd(&a.counts[s_pi[p] * a.V + s_pj[p]], (unsigned long long)s_acc[p]);
}

// Mirror the upper triangle and form IOU (Eq. S1) and OC (Eq. S2).
__global__ void covis_final_kernel(unsigned long long *counts, int V, float *iou, float *oc) {
    for (int e = threadIdx.x; e < V * V; e += blockDim.x) {
        const int i = e / V, j = e % V;
        const int lo = i < j ? i : j, hi = i < j ? j : i;
        const unsigned long long c = counts[lo * V + hi];
        const unsigned long long ci = counts[i * V + i], cj = counts[j * V + j];
        const unsigned long long uni = ci + cj - c, small = ci < cj ? ci : cj;
        if (iou) iou[e] = uni > 0 ? (float)((double)c / (double)uni) : 0.f;
        if (oc) oc[e] = small > 0 ? (float)((double)c / (double)small) : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < V * V; e += blockDim.x) {
        const int i = e / V, j = e % V;
        if (i > j) counts[e] = counts[j * V + i];
    }
}

// ---- median depth: radix select over the positive float bit patterns ----
constexpr int kMedThreads = 256;
constexpr int kMedBlocksPerView = 64;
constexpr int kMedBins = 2048;

struct MedianView {
    long long pix_base, hw;
};
struct MedianBatch {
    int n_views;
    MedianView v[S3GS_MAX_VIEWS];
};
struct MedianState {
    unsigned prefix;     // bits fixed so far
    unsigned long long rank;  // rank still to find inside the current bin
    unsigned long long n_valid;
    unsigned pad;
};

// level 0: bits 30..20, level 1: bits 19..9, level 2: bits 8..0
__device__ __forceinline__ void level_bits(int level, int &shift, unsigned &mask_hi) {
    shift = level == 0 ? 20 : (level == 1 ? 9 : 0);
    mask_hi = level == 0 ? 0u : (level == 1 ? 0x7ff00000u : 0x7ffffe00u);
}

__global__ void __launch_bounds__(kMedThreads)
    median_hist_kernel(const float *__restrict__ depth, unsigned *__restrict__ hist, const MedianState *st,
                       int level, const __grid_constant__ MedianBatch b) {
    __shared__ unsigned s_h[kMedBins];
    const int v = blockIdx.y;
    for (int i = threadIdx.x; i < kMedBins; i += kMedThreads) s_h[i] = 0u;
    __syncthreads();
    int shift;
    unsigned mask_hi;
    level_bits(level, shift, mask_hi);
    const unsigned prefix = level == 0 ? 0u : st[v].prefix;
    const unsigned nbins_mask = level == 2 ? 0x1ffu : 0x7ffu;
    const float *d = depth + b.v[v].pix_base;
    for (long long i = (long long)blockIdx.x * kMedThreads + threadIdx.x; i < b.v[v].hw;
         i += (long long)gridDim.x * kMedThreads) {
        const float x = d[i];
        if (!(x > 0.f)) continue;
        const unsigned u = __float_as_uint(x);
        if ((u & mask_hi) != prefix) continue;
        atomicAdd(&s_h[(u >> shift) & nbins_mask], 1u);
    }
    __syncthreads();
    unsigned *h = hist + (long long)v * kMedBins;
    for (int i = threadIdx.x; i < kMedBins; i += kMedThreads)
        if (s_h[i]) atomicAdd(&h[i], s_h[i]);
}

// One CTA per view: find the bin holding the wanted rank, fix its bits and clear
// the histogram for the next level. At level 0 the wanted rank is set from the
// number of positive depths.
__global__ void __launch_bounds__(kMedThreads)
    median_select_kernel(unsigned *__restrict__ hist, MedianState *st, int level, float *median,
                         long long *n_valid) {
    __shared__ unsigned long long s_sum[kMedThreads];
    const int v = blockIdx.x;
    unsigned *h = hist + (long long)v * kMedBins;
    constexpr int per = kMedBins / kMedThreads;  // 8 consecutive bins per thread
    unsigned long long local = 0;
    for (int k = 0; k < per; ++k) local += h[threadIdx.x * per + k];
    s_sum[threadIdx.x] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        MedianState s = st[v];
        if (level == 0) {
            unsigned long long tot = 0;
            for (int t = 0; t < kMedThreads; ++t) tot += s_sum[t];
            s.n_valid = tot;
            s.rank = tot > 0 ? (tot - 1) / 2 : 0;
            s.prefix = 0u;
        }
        int shift;
        unsigned mask_hi;
        level_bits(level, shift, mask_hi);
        if (s.n_valid > 0) {
            unsigned long long before = 0;
            int t = 0;
            while (t < kMedThreads - 1 && before + s_sum[t] <= s.rank) before += s_sum[t++];
            int bin = t * per;
            while (bin < t * per + per - 1 && before + h[bin] <= s.rank) before += h[bin++];
            s.rank -= before;
            s.prefix |= (unsigned)bin << shift;
        }
        st[v] = s;
        if (level == 2) {
            if (median) median[v] = s.n_valid > 0 ? __uint_as_float(s.prefix) : 0.f;
            if (n_valid) n_valid[v] = (long long)s.n_valid;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kMedBins; i += kMedThreads) h[i] = 0u;
}

s3gs_status launch_error(s3gs_ctx *ctx, cudaError_t e, const char *where) {
    char msg[256];
    snprintf(msg, sizeof(msg), "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
    return ctx_error(ctx, S3GS_E_CUDA, msg);
}

size_t median_ws_bytes(int n_views) {
    return (size_t)n_views * (kMedBins * sizeof(unsigned) + sizeof(MedianState));
}

}  // namespace

cudaError_t launch_covis(const unsigned *vis, long long n, int V, unsigned long long *counts, float *iou, float *oc,
                         int num_sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * V * V, s);
    if (e != cudaSuccess) return e;
    CovisArgs a;
    memset(&a, 0, sizeof(a));
    a.vis = vis;
    a.n = n;
    a.V = V;
    a.counts = counts;
    int p = 0;
    for (int i = 0; i < V; ++i)
        for (int j = i; j < V; ++j) {
            a.pi[p] = (unsigned char)i;
            a.pj[p] = (unsigned char)j;
            ++p;
        }
    a.n_pairs = p;
    if (n > 0) {
        long long want = (n + kCovisThreads - 1) / kCovisThreads;
        const long long cap = 4LL * (num_sms > 0 ? num_sms : 152);
        const int grid = (int)(want < cap ? want : cap);
        covis_kernel<<<grid, kCovisThreads, 0, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    covis_final_kernel<<<1, 1024, 0, s>>>(counts, V, iou, oc);
    return cudaGetLastError();
}

}  // namespace s3gs

using namespace s3gs;

extern "C" {

s3gs_status s3gs_median_depth_workspace(int32_t n_views, size_t *bytes) {
    if (!bytes || n_views < 1 || n_views > S3GS_MAX_VIEWS) return S3GS_E_INVALID;
    *bytes = median_ws_bytes(n_views);
    return S3GS_OK;
}

s3gs_status s3gs_median_depth(s3gs_ctx *ctx, const int32_t *view_wh, int32_t n_views, const float *depth,
                              float *median, int64_t *n_valid, void *workspace, size_t workspace_bytes,
                              void *stream) {
    if (!ctx) return S3GS_E_INVALID;
    if (!view_wh || !depth || !median || !workspace || n_views < 1 || n_views > S3GS_MAX_VIEWS)
        return ctx_error(ctx, S3GS_E_INVALID, "median_depth: NULL pointer or n_views outside 1..S3GS_MAX_VIEWS");
    if (workspace_bytes < median_ws_bytes(n_views) || (reinterpret_cast<uintptr_t>(workspace) & 15u) != 0)
        return ctx_error(ctx, S3GS_E_INVALID, "median_depth: workspace too small or not 16-byte aligned");
    MedianBatch b;
    memset(&b, 0, sizeof(b));
    b.n_views = n_views;
    long long pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const int w = view_wh[2 * v], h = view_wh[2 * v + 1];
        if (w < 1 || h < 1 || w > 65536 || h > 65536)
            return ctx_error(ctx, S3GS_E_INVALID, "median_depth: view width/height must be in 1..65536");
        b.v[v].pix_base = pix;
        b.v[v].hw = (long long)w * h;
        pix += (long long)w * h;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned *hist = static_cast<unsigned *>(workspace);
    MedianState *st = reinterpret_cast<MedianState *>(hist + (size_t)n_views * kMedBins);
    cudaError_t e = cudaMemsetAsync(workspace, 0, median_ws_bytes(n_views), s);
    if (e != cudaSuccess) return launch_error(ctx, e, "median_depth: clear");
    for (int level = 0; level < 3; ++level) {
        median_hist_kernel<<<dim3(kMedBlocksPerView, n_views), kMedThreads, 0, s>>>(depth, hist, st, level, b);
        median_select_kernel<<<n_views, kMedThreads, 0, s>>>(hist, st, level, median,
                                                             reinterpret_cast<long long *>(n_valid));
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? S3GS_OK : launch_error(ctx, e, "median_depth");
}

void s3gs_keyframe_params_default(s3gs_keyframe_params *p) {
    if (!p) return;
    p->k_iou = 0.9f;
    p->k_d = 0.08f;
    p->k_oc = 0.3f;
    p->max_window = 8;
}

int32_t s3gs_keyframe_is_new(const s3gs_keyframe_params *p, float iou_ij, float d_ij, float median_depth_i) {
    if (!p) return -1;
    return (iou_ij < p->k_iou || d_ij > p->k_d * median_depth_i) ? 1 : 0;
}

s3gs_status s3gs_keyframe_window_update(const s3gs_keyframe_params *p, const int32_t *window_ids,
                                        const float *oc_with_new, int32_t n, int32_t new_id, int32_t *out_ids,
                                        int32_t *out_n) {
    if (!p || !out_ids || !out_n || n < 0 || (n > 0 && (!window_ids || !oc_with_new)) || p->max_window < 1)
        return S3GS_E_INVALID;
    // keep[k] = position in the input window of the k-th survivor
    int32_t *keep = static_cast<int32_t *>(malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1)));
    if (!keep) return S3GS_E_NOMEM;
    int m = 0;
    for (int k = 0; k < n; ++k)
        if (!(oc_with_new[k] < p->k_oc)) keep[m++] = k;
    while (m + 1 > p->max_window && m > 0) {
        int worst = 0;
        for (int t = 1; t < m; ++t)
            if (oc_with_new[keep[t]] < oc_with_new[keep[worst]]) worst = t;  // earlier one on ties
        for (int t = worst; t + 1 < m; ++t) keep[t] = keep[t + 1];
        --m;
    }
    for (int t = 0; t < m; ++t) out_ids[t] = window_ids[keep[t]];
    out_ids[m] = new_id;
    *out_n = m + 1;
    free(keep);
    return S3GS_OK;
}

}  // extern "C"
