// Fixed-order reductions: the per-view camera twist (Eq. 11), the
// deterministic per-record sum of per-tile gradient partials, and the L1
// mapping/tracking loss (Eq. 10, 15, 17) with its gradient.
#include "s3gs_internal.cuh"

namespace s3gs {
namespace {

// One block per view: sum of the per-block twist partials in a fixed order.
__global__ void __launch_bounds__(256) twist_reduce_kernel(const TwistReduceArgs a) {
    __shared__ float s[8][6];
    const int v = blockIdx.x;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int p = threadIdx.x; p < a.n_parts; p += blockDim.x) {
        const float *src = a.twist_partial + ((long long)p * a.n_views + v) * 6;
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += src[c];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        float x = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s[warp][c] = x;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float x = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += s[w][threadIdx.x];
        float *dst = a.d_twist + v * 6 + threadIdx.x;
        *dst = a.accumulate ? *dst + x : x;
    }
}

// Deterministic mode: each visible record gathers its per-tile partials, tile
// by tile in row-major order over the tiles its cover lists it in; its position
// inside each tile's list is found by binary search of its unique (depth bits,
// index) key.
__global__ void __launch_bounds__(256) det_reduce_kernel(const DetReduceArgs a, const __grid_constant__ ViewBatch vb) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long total = (long long)vb.n_views * a.n;
    if (r >= total) return;
    int2 ext = a.ext[r];
    if (ext.x <= 0) return;
    int v = (int)(r / a.n);
    unsigned g = (unsigned)(r - (long long)v * a.n);
    const ViewInfo &vi = vb.v[v];
    float4 ra = a.rec[r].a;
    float z = a.rec[r].b.z;
    float x0 = ceilf(__fsub_rn(ra.x, (float)ext.x)), x1 = floorf(__fadd_rn(ra.x, (float)ext.x));
    float y0 = ceilf(__fsub_rn(ra.y, (float)ext.y)), y1 = floorf(__fadd_rn(ra.y, (float)ext.y));
    int tx0 = tile_of(x0 > 0.f ? (int)x0 : 0, vb.tile_w);
    int tx1 = tile_of(x1 < (float)(vi.w - 1) ? (int)x1 : vi.w - 1, vb.tile_w);
    int ty0 = tile_of(y0 > 0.f ? (int)y0 : 0, vb.tile_h);
    int ty1 = tile_of(y1 < (float)(vi.h - 1) ? (int)y1 : vi.h - 1, vb.tile_h);
    const unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | g;
    const int bin = depth_bin(z);
    float acc[kGrad2d];
#pragma unroll
    for (int q = 0; q < kGrad2d; ++q) acc[q] = 0.f;
    const CoverEllipse ell = cover_ellipse(ra.x, ra.y, ra.z, ra.w, a.rec[r].b.x, a.rec[r].c.w);
    const float inv_tw = __frcp_rn((float)vb.tile_w);
    for (int ty = ty0; ty <= ty1; ++ty) {
        const int py0 = ty * vb.tile_h, py1 = min(py0 + vb.tile_h - 1, vi.h - 1);
        const int2 span = row_span(ell, py0, py1, tx0, tx1, inv_tw);  // the tiles the record is listed in
        for (int tx = span.x; tx <= span.y; ++tx) {
            int t = vi.tile_base + ty * vi.tiles_x + tx;
            if (a.cut && bin > (int)a.cut[t]) continue;  // behind the tile's occlusion cut: not listed
            unsigned lo = a.tile_start[t * kDepthBins], hi = a.tile_start[(t + 1) * kDepthBins];
            while (lo < hi) {
                unsigned mid = lo + ((hi - lo) >> 1);
                if (a.keys[mid] < key) lo = mid + 1; else hi = mid;
            }
            const float *src = a.det_partial + (long long)lo * kGrad2d;
#pragma unroll
            for (int q = 0; q < kGrad2d; ++q) acc[q] += src[q];
        }
    }
    float *dst = a.grad2d + r * kGrad2d;
#pragma unroll
    for (int q = 0; q < kGrad2d; ++q) dst[q] = acc[q];
}

constexpr int kLossThreads = 256;

__device__ __forceinline__ float sgn(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// One pixel-group of the L1 terms: W consecutive pixels of one view (W = 4 with
// 16-byte vector loads when every plane is 16-byte aligned, else W = 1).
template <int W>
struct Lanes {
    float x[W];
};

template <int W>
__device__ __forceinline__ Lanes<W> ldv(const float *p) {
    Lanes<W> r;
    if (W == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        r.x[0] = q.x; r.x[1] = q.y; r.x[2] = q.z; r.x[3] = q.w;
    } else {
#pragma unroll
        for (int k = 0; k < W; ++k) r.x[k] = p[k];
    }
    return r;
}

template <int W>
__device__ __forceinline__ void stv(float *p, const Lanes<W> &v) {
    if (W == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v.x[0], v.x[1], v.x[2], v.x[3]);
    } else {
#pragma unroll
        for (int k = 0; k < W; ++k) p[k] = v.x[k];
    }
}

// L1 term over W pixels: adds sum c_k |x_k - t_k| to acc, writes c_k sign(x_k - t_k).
template <int W>
__device__ __forceinline__ void l1_group(const float *x, const float *t, float *d, long long i, const Lanes<W> &c,
                                         float &acc) {
    const Lanes<W> xv = ldv<W>(x + i), tv = ldv<W>(t + i);
    Lanes<W> dv;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const float r = xv.x[k] - tv.x[k];
        dv.x[k] = c.x[k] * sgn(r);
        acc += c.x[k] * fabsf(r);
    }
    if (d) stv<W>(d + i, dv);
}

template <int W>
__device__ __forceinline__ void zero_group(float *d, long long i) {
    Lanes<W> z;
#pragma unroll
    for (int k = 0; k < W; ++k) z.x[k] = 0.f;
    stv<W>(d + i, z);
}

// grid.y = view; every thread handles whole pixel groups (all channels of each
// term), so each term's gradient is written by the thread that read its inputs.
template <int W>
__global__ void __launch_bounds__(kLossThreads) loss_kernel(const LossArgs a, const __grid_constant__ ViewBatch vb) {
    __shared__ float s[kLossThreads / 32];
    const int v = blockIdx.y;
    const ViewInfo &vi = vb.v[v];
    const long long HW = (long long)vi.w * vi.h;
    const long long p1 = vi.pix_base, p3 = 3 * vi.pix_base;
    const float P = (float)vb.total_pixels;
    const float kr = a.w_rgb / (3.f * P), kd = a.w_depth / P, kg = a.w_geo / (3.f * P);
    float acc = 0.f;
    const long long groups = HW / W;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < groups;
         q += (long long)gridDim.x * blockDim.x) {
        const long long p = q * W;
        Lanes<W> m;
        if (a.mask) {
            m = ldv<W>(a.mask + p1 + p);
        } else {
#pragma unroll
            for (int k = 0; k < W; ++k) m.x[k] = 1.f;
        }
        Lanes<W> cr, cd, cg;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            cr.x[k] = m.x[k] * kr;
            cd.x[k] = m.x[k] * kd;
            cg.x[k] = m.x[k] * kg;
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const long long i = p3 + ch * HW + p;
            if (a.t_rgb) l1_group<W>(a.rgb, a.t_rgb, a.d_rgb, i, cr, acc);
            else if (a.d_rgb) zero_group<W>(a.d_rgb, i);
            if (a.t_pointmap) l1_group<W>(a.pointmap, a.t_pointmap, a.d_pointmap, i, cg, acc);
            else if (a.d_pointmap) zero_group<W>(a.d_pointmap, i);
        }
        if (a.t_depth) l1_group<W>(a.depth, a.t_depth, a.d_depth, p1 + p, cd, acc);
        else if (a.d_depth) zero_group<W>(a.d_depth, p1 + p);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float x = 0.f;
        for (int w = 0; w < kLossThreads / 32; ++w) x += s[w];
        a.partial[(long long)v * gridDim.x + blockIdx.x] = x;
    }
}

// One block: fixed-order sum of the loss partials, four independent loads in
// flight per thread so that a long partial list is not latency-bound.
constexpr int kFinalThreads = 1024;
__global__ void __launch_bounds__(kFinalThreads) loss_final_kernel(const float *partial, int n, float *loss) {
    __shared__ float s[kFinalThreads / 32];
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int i = threadIdx.x;
    for (; i + 3 * kFinalThreads < n; i += 4 * kFinalThreads) {
        a0 += partial[i];
        a1 += partial[i + kFinalThreads];
        a2 += partial[i + 2 * kFinalThreads];
        a3 += partial[i + 3 * kFinalThreads];
    }
    for (; i < n; i += kFinalThreads) a0 += partial[i];
    float acc = (a0 + a1) + (a2 + a3);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float x = 0.f;
        for (int w = 0; w < kFinalThreads / 32; ++w) x += s[w];
        *loss = x;
    }
}

}  // namespace

cudaError_t launch_twist_reduce(const TwistReduceArgs &a, cudaStream_t s) {
    if (a.n_views <= 0) return cudaSuccess;
    twist_reduce_kernel<<<a.n_views, 256, 0, s>>>(a);
    return cudaGetLastError();
}

int loss_blocks_per_view() { return 64; }

cudaError_t launch_loss(const LossArgs &a, const ViewBatch &vb, cudaStream_t s) {
    dim3 grid(loss_blocks_per_view(), vb.n_views);
    // 4-pixel vector groups when every plane of every view starts on a 16-byte boundary
    bool vec = true;
    for (int v = 0; v < vb.n_views; ++v)
        vec = vec && ((long long)vb.v[v].w * vb.v[v].h) % 4 == 0 && vb.v[v].pix_base % 4 == 0;
    const void *ptrs[] = {a.rgb, a.depth, a.pointmap, a.t_rgb, a.t_depth, a.t_pointmap, a.mask,
                          a.d_rgb, a.d_depth, a.d_pointmap};
    for (const void *q : ptrs) vec = vec && (reinterpret_cast<uintptr_t>(q) & 15u) == 0;
    if (vec) loss_kernel<4><<<grid, kLossThreads, 0, s>>>(a, vb);
    else loss_kernel<1><<<grid, kLossThreads, 0, s>>>(a, vb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    loss_final_kernel<<<1, kFinalThreads, 0, s>>>(a.partial, loss_blocks_per_view() * vb.n_views, a.loss);
    return cudaGetLastError();
}

cudaError_t launch_loss_final(const float *partial, int n, float *loss, cudaStream_t s) {
    loss_final_kernel<<<1, kFinalThreads, 0, s>>>(partial, n, loss);
    return cudaGetLastError();
}

cudaError_t launch_det_reduce(const DetReduceArgs &a, const ViewBatch &vb, cudaStream_t s) {
    long long total = (long long)vb.n_views * a.n;
    if (total == 0) return cudaSuccess;
    det_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a, vb);
    return cudaGetLastError();
}

}  // namespace s3gs
