// EWA projection of 3D Gaussians (Sec. 3.1, Eq. 1) and its backward (Sec. 3.2.2,
// Eq. 11), as structure-of-arrays passes with one thread per Gaussian looping
// over all views of the call, so each Gaussian's parameters are read once per
// call however many views there are.
#include "s3gs_internal.cuh"

namespace s3gs {
namespace {

// Real orthonormal spherical harmonics (no Condon-Shortley phase), l = 1..3,
// at a unit direction; coefficient k = l^2 + l + m. Constants are
// sqrt((2l+1)/(4 pi) * (l-|m|)!/(l+|m|)!) times the polynomial normalisation.
constexpr float kSH1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
constexpr float kSH2a = 1.09254843059207907f;  // 0.5 sqrt(15 / pi)
constexpr float kSH2b = 0.31539156525252001f;  // 0.25 sqrt(5 / pi)
constexpr float kSH2c = 0.54627421529603954f;  // 0.25 sqrt(15 / pi)
constexpr float kSH3a = 0.59004358992664352f;  // 0.25 sqrt(35 / (2 pi))
constexpr float kSH3b = 2.89061144264055406f;  // 0.5 sqrt(105 / pi)
constexpr float kSH3c = 0.45704579946446573f;  // 0.25 sqrt(21 / (2 pi))
constexpr float kSH3d = 0.37317633259011540f;  // 0.25 sqrt(7 / pi)
constexpr float kSH3e = 1.44530572132027703f;  // 0.25 sqrt(105 / pi)

template <int D>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
    Y[0] = 1.0f;  // the DC coefficient is used directly (Eq. 2 colour)
    if (D >= 1) {
        Y[1] = kSH1 * y;
        Y[2] = kSH1 * z;
        Y[3] = kSH1 * x;
    }
    if (D >= 2) {
        Y[4] = kSH2a * x * y;
        Y[5] = kSH2a * y * z;
        Y[6] = kSH2b * (3.0f * z * z - 1.0f);
        Y[7] = kSH2a * x * z;
        Y[8] = kSH2c * (x * x - y * y);
    }
    if (D >= 3) {
        Y[9] = kSH3a * y * (3.0f * x * x - y * y);
        Y[10] = kSH3b * x * y * z;
        Y[11] = kSH3c * y * (5.0f * z * z - 1.0f);
        Y[12] = kSH3d * z * (5.0f * z * z - 3.0f);
        Y[13] = kSH3c * x * (5.0f * z * z - 1.0f);
        Y[14] = kSH3e * z * (x * x - y * y);
        Y[15] = kSH3a * x * (x * x - 3.0f * y * y);
    }
}

// sum_k w[k] * grad Y_k (gradient of the polynomials above in x, y, z)
template <int D>
__device__ __forceinline__ float3 sh_weighted_grad(float x, float y, float z, const float w[16]) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (D >= 1) {
        gy += kSH1 * w[1];
        gz += kSH1 * w[2];
        gx += kSH1 * w[3];
    }
    if (D >= 2) {
        gx += kSH2a * y * w[4];  gy += kSH2a * x * w[4];
        gy += kSH2a * z * w[5];  gz += kSH2a * y * w[5];
        gz += kSH2b * 6.0f * z * w[6];
        gx += kSH2a * z * w[7];  gz += kSH2a * x * w[7];
        gx += kSH2c * 2.0f * x * w[8];  gy -= kSH2c * 2.0f * y * w[8];
    }
    if (D >= 3) {
        gx += kSH3a * 6.0f * x * y * w[9];
        gy += kSH3a * (3.0f * x * x - 3.0f * y * y) * w[9];
        gx += kSH3b * y * z * w[10]; gy += kSH3b * x * z * w[10]; gz += kSH3b * x * y * w[10];
        gy += kSH3c * (5.0f * z * z - 1.0f) * w[11]; gz += kSH3c * 10.0f * y * z * w[11];
        gz += kSH3d * (15.0f * z * z - 3.0f) * w[12];
        gx += kSH3c * (5.0f * z * z - 1.0f) * w[13]; gz += kSH3c * 10.0f * x * z * w[13];
        gx += kSH3e * 2.0f * x * z * w[14]; gy -= kSH3e * 2.0f * y * z * w[14];
        gz += kSH3e * (x * x - y * y) * w[14];
        gx += kSH3a * (3.0f * x * x - 3.0f * y * y) * w[15];
        gy -= kSH3a * 6.0f * x * y * w[15];
    }
    return make_float3(gx, gy, gz);
}

struct Activated {
    float s[3];
    float qn[4];
    float qinv;   // 1 / |q|
    float R[9];
    float Sig[6]; // world covariance: xx, xy, xz, yy, yz, zz
    float opacity;
};

__device__ __forceinline__ bool activate(const float *ls, const float *q, float ol, Activated &A) {
    A.s[0] = expf(ls[0]);
    A.s[1] = expf(ls[1]);
    A.s[2] = expf(ls[2]);
    float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(qq > 0.f)) return false;
    float nrm = sqrtf(qq);
    A.qinv = 1.0f / nrm;
    float w = q[0] * A.qinv, x = q[1] * A.qinv, y = q[2] * A.qinv, z = q[3] * A.qinv;
    A.qn[0] = w; A.qn[1] = x; A.qn[2] = y; A.qn[3] = z;
    float *R = A.R;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
    // Sigma = (R S)(R S)^T
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * A.s[j];
    A.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    A.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    A.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    A.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    A.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    A.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    A.opacity = 1.0f / (1.0f + expf(-ol));
    return true;
}

__device__ __forceinline__ void sym_full(const float s[6], float F[9]) {
    F[0] = s[0]; F[1] = s[1]; F[2] = s[2];
    F[3] = s[1]; F[4] = s[3]; F[5] = s[4];
    F[6] = s[2]; F[7] = s[4]; F[8] = s[5];
}

// Camera-frame covariance Sc = W Sig W^T (full 3x3).
__device__ __forceinline__ void cam_cov(const float T[12], const float Sig[6], float Sc[9]) {
    float S[9], WS[9];
    sym_full(Sig, S);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            WS[3 * i + j] = T[4 * i] * S[j] + T[4 * i + 1] * S[3 + j] + T[4 * i + 2] * S[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Sc[3 * i + j] = WS[3 * i] * T[4 * j] + WS[3 * i + 1] * T[4 * j + 1] + WS[3 * i + 2] * T[4 * j + 2];
}

__device__ __forceinline__ void cam_centre(const float T[12], float c[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) c[i] = -(T[i] * T[3] + T[4 + i] * T[7] + T[8 + i] * T[11]);
}

// One coordinate of the view transform, r . m + t, to about one rounding of the
// result. A mean tens of metres from the world origin seen by a camera a metre
// away makes the terms cancel: plain FP32 leaves an error near ulp(|m|), which
// the projection magnifies by f / z (milli-pixels for near Gaussians on a long
// trajectory, enough to flip a 1/255-skip decision against the FP64 reference).
// Each product is split exactly with an FMA (p + e = r m) and the sum is a
// chain of error-free two-sums whose errors are accumulated and added once
// (compensated dot product, Ogita, Rump and Oishi 2005, "Dot2").
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float view_coord(const float *r, const float m[3], float t) {
    const float p0 = __fmul_rn(r[0], m[0]), e0 = __fmaf_rn(r[0], m[0], -p0);
    const float p1 = __fmul_rn(r[1], m[1]), e1 = __fmaf_rn(r[1], m[1], -p1);
    const float p2 = __fmul_rn(r[2], m[2]), e2 = __fmaf_rn(r[2], m[2], -p2);
    float s, e, c;
    two_sum(p0, p1, s, e);
    c = __fadd_rn(__fadd_rn(e0, e1), e);
    two_sum(s, p2, s, e);
    c = __fadd_rn(c, __fadd_rn(e2, e));
    two_sum(s, t, s, e);
    c = __fadd_rn(c, e);
    return __fadd_rn(s, c);
}

// Counts the (tile, depth bin) buckets of the 32 records a warp has just made
// for one view, in two levels. Level 1: a warp scan numbers the tile rows of the
// records' bounding rectangles; in each round every lane takes one (record, row),
// fetches the record's cover ellipse with shuffles and computes the row's span of
// covered tile columns (row_span). Level 2: a second scan numbers the round's
// covered tiles, and in each sub-round every lane counts one. All lanes stay busy
// whatever the mix of record sizes, and only covered tiles cost a count (a round
// whose rows are all at most 16 tiles long skips level 2: each lane counts its own
// row). With the occlusion cut on, the bucket counts are made later (after the cut) and this pass
// takes only the records that can hold a whole tile: each of their pairs adds its
// optical depth bound over the tile to the bucket (occl_units).
__device__ __forceinline__ void count_cover_warp(const ProjectArgs &a, const ViewBatch &vb, const ViewInfo &vi,
                                                 bool has, const CoverEllipse &ell, int tx0, int ty0, int ntx, int nty,
                                                 int bin, const OcclGauss &og) {
    __shared__ float4 s_og0[8][32], s_og1[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (a.occl) {
        s_og0[warp][lane] = make_float4(og.u, og.v, og.a, og.b);
        s_og1[warp][lane] = make_float4(og.c, og.thr, og.lo2, og.w);
        __syncwarp();
    }
    const unsigned nrows = (has && (!a.occl || og.w > 0.f)) ? (unsigned)nty : 0u;
    const unsigned incl = warp_incl_scan(nrows);
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    const unsigned excl = incl - nrows;
    const unsigned t0 = (unsigned)tx0 | ((unsigned)ty0 << 16);
    const float inv_tw = __frcp_rn((float)vb.tile_w);  // exact: the tile width is a power of two
    for (unsigned base = 0; base < total; base += 32) {
        const unsigned j = base + lane;
        const int src = warp_find(incl, j);
        const CoverEllipse e = shfl_ellipse(ell, src);
        const unsigned s_excl = __shfl_sync(0xffffffffu, excl, src);
        const unsigned s_t0 = __shfl_sync(0xffffffffu, t0, src);
        const int s_ntx = __shfl_sync(0xffffffffu, ntx, src);
        const int s_bin = __shfl_sync(0xffffffffu, bin, src);
        int c0 = 0;
        unsigned len = 0, rowbase = 0, rinfo = 0;
        if (j < total) {
            const int ty = (int)(s_t0 >> 16) + (int)(j - s_excl);
            rinfo = (unsigned)src | ((unsigned)ty << 8);
            const int py0 = ty * vb.tile_h, py1 = min(py0 + vb.tile_h - 1, vi.h - 1);
            const int cx0 = (int)(s_t0 & 0xffffu);
            int2 span;
            if (a.occl) {
                // only tiles inside the ellipse where alpha >= kOcclAlpha can add
                const float4 g0 = s_og0[warp][src], g1 = s_og1[warp][src];
                const OcclGauss g = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
                span = strong_span(g, fmaxf(g.thr, kOcclLog2Alpha - g.lo2), py0, py1, cx0, cx0 + s_ntx - 1,
                                   vb.tile_w, vi.w);
            } else {
                span = row_span(e, py0, py1, cx0, cx0 + s_ntx - 1, inv_tw);
            }
            c0 = span.x;
            len = span.y >= span.x ? (unsigned)(span.y - span.x + 1) : 0u;
            rowbase = (unsigned)(vi.tile_base + ty * vi.tiles_x) * kDepthBins + (unsigned)s_bin;
        }
        if (!a.occl && __reduce_max_sync(0xffffffffu, len) <= 16u) {
            // short rows (small Gaussians): each lane counts its own row's tiles
            for (unsigned q = 0; q < len; ++q) atomicAdd(a.tile_count + rowbase + (size_t)(c0 + (int)q) * kDepthBins, 1u);
            continue;
        }
        const unsigned incl2 = warp_incl_scan(len);
        const unsigned tot2 = __shfl_sync(0xffffffffu, incl2, 31);
        const unsigned excl2 = incl2 - len;
        for (unsigned b2 = 0; b2 < tot2; b2 += 32) {
            const unsigned j2 = b2 + lane;
            const int src2 = warp_find(incl2, j2);
            const int h0 = __shfl_sync(0xffffffffu, c0, src2);
            const unsigned he = __shfl_sync(0xffffffffu, excl2, src2);
            const unsigned hb = __shfl_sync(0xffffffffu, rowbase, src2);
            const unsigned ri = __shfl_sync(0xffffffffu, rinfo, src2);
            if (j2 < tot2) {
                const int tx = h0 + (int)(j2 - he);
                const size_t bucket = hb + (size_t)tx * kDepthBins;
                if (!a.occl) {
                    atomicAdd(a.tile_count + bucket, 1u);
                } else if ((bucket & (kDepthBins - 1)) <= a.cut_hint[bucket / kDepthBins] + kHintSlack) {
                    const float4 g0 = s_og0[warp][ri & 31u], g1 = s_og1[warp][ri & 31u];
                    const OcclGauss g = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
                    const int ty = (int)(ri >> 8);
                    const int x0 = tx * vb.tile_w, y0 = ty * vb.tile_h;
                    const unsigned q = occl_units(g, (float)x0, (float)min(x0 + vb.tile_w - 1, vi.w - 1),
                                                  (float)y0, (float)min(y0 + vb.tile_h - 1, vi.h - 1));
                    if (q) atomicAdd(a.occl + bucket, q);
                }
            }
        }
    }
}

constexpr int kShStride = 257;  // shared-memory row of one SH coefficient over a CTA's 256 Gaussians

template <int D>
__global__ void __launch_bounds__(256) project_kernel(const ProjectArgs a, const __grid_constant__ ViewBatch vb) {
    // every lane stays to the end: the tile counting below is warp-cooperative
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = gid < a.n;
    const long long g = live ? gid : 0;
    constexpr int NC = (D + 1) * (D + 1);
    float m[3] = {a.means[3 * g], a.means[3 * g + 1], a.means[3 * g + 2]};
    float ls[3] = {a.log_scales[3 * g], a.log_scales[3 * g + 1], a.log_scales[3 * g + 2]};
    float4 q4 = reinterpret_cast<const float4 *>(a.quats)[g];
    float q[4] = {q4.x, q4.y, q4.z, q4.w};
    Activated A;
    bool ok = activate(ls, q, a.opacity_logits[g], A) && live;
    const float lo2 = log2f(A.opacity);  // per Gaussian, staged with every visible record
    // Degree 0 keeps its colour in registers. Higher degrees stage the CTA's SH
    // coefficients in shared memory once (a coalesced copy of one contiguous block),
    // and each view that sees a Gaussian reads them there: coefficient k of thread t
    // sits at k * kShStride + t, so a warp's reads of one coefficient hit 32 banks.
    const float *cp = a.colors + (long long)g * NC * 3;
    float k0[3] = {cp[0], cp[1], cp[2]};
    extern __shared__ float s_sh[];
    if (D > 0) {
        const long long g0 = (long long)blockIdx.x * blockDim.x;
        const long long ng = a.n - g0 < (long long)blockDim.x ? a.n - g0 : (long long)blockDim.x;
        const float *src = a.colors + g0 * NC * 3;
        for (int e = threadIdx.x; e < (int)ng * NC * 3; e += blockDim.x) {
            const int lt = e / (NC * 3), k = e - lt * (NC * 3);
            s_sh[k * kShStride + lt] = __ldg(src + e);
        }
        __syncthreads();
    }

    unsigned mask = 0;
    for (int v = 0; v < vb.n_views; ++v) {
        const ViewInfo &vi = vb.v[v];
        long long r = (long long)v * a.n + g;
        int2 ext = make_int2(0, 0);
        bool has = false;
        CoverEllipse ell;
        ell.u = ell.v = ell.B = ell.iA = ell.Aqc = ell.det = ell.yL = ell.mq = 0.f;
        ell.ym = -1.0f;
        int ctx0 = 0, cty0 = 0, cntx = 0, cnty = 0, cbin = 0;
        OcclGauss og = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float T[12];
        load_pose(vi, a.Tdev, v, T);
        float px = view_coord(T, m, T[3]);
        float py = view_coord(T + 4, m, T[7]);
        float pz = view_coord(T + 8, m, T[11]);
        const bool in_cone = a.guard <= 0.f || (fabsf(px) <= a.guard * pz && fabsf(py) <= a.guard * pz);
        if (ok && pz > a.near_z && in_cone) {
            float Sc[9];
            cam_cov(T, A.Sig, Sc);
            float iz = 1.0f / pz;
            float j00 = vi.fx * iz, j02 = -vi.fx * px * iz * iz;
            float j11 = vi.fy * iz, j12 = -vi.fy * py * iz * iz;
            // cov2 = J Sc J^T + 0.3 I, J = [[j00, 0, j02], [0, j11, j12]]
            float ca = j00 * (j00 * Sc[0] + j02 * Sc[2]) + j02 * (j00 * Sc[6] + j02 * Sc[8]) + kDilation;
            float cb = j11 * (j00 * Sc[1] + j02 * Sc[7]) + j12 * (j00 * Sc[2] + j02 * Sc[8]);
            float cc = j11 * (j11 * Sc[4] + j12 * Sc[5]) + j12 * (j11 * Sc[7] + j12 * Sc[8]) + kDilation;
            float det = ca * cc - cb * cb;
            float u = vi.fx * px * iz + vi.cx;
            float vv = vi.fy * py * iz + vi.cy;
            if (det > 0.f && isfinite(u) && isfinite(vv)) {
                float idet = 1.0f / det;
                // Integer half-extents of the 3-sigma ellipse's bounding box, widened
                // by a margin that covers FP32 rounding of the conic: its error grows
                // with the condition number of the 2D covariance.
                const float mid = 0.5f * (ca + cc);
                const float disc = sqrtf(fmaxf(mid * mid - det, 0.0f));
                const float kappa = (mid + disc) / fmaxf(mid - disc, 1e-6f);
                const float widen = 1.0f + 1e-5f + 4e-7f * kappa;
                float ex = ceilf(3.0f * sqrtf(ca) * widen + 0.01f), ey = ceilf(3.0f * sqrtf(cc) * widen + 0.01f);
                int rx = ex < (float)kExtentMax ? (int)ex : kExtentMax;
                int ry = ey < (float)kExtentMax ? (int)ey : kExtentMax;
                float x0 = ceilf(__fsub_rn(u, (float)rx)), x1 = floorf(__fadd_rn(u, (float)rx));
                float y0 = ceilf(__fsub_rn(vv, (float)ry)), y1 = floorf(__fadd_rn(vv, (float)ry));
                if (x1 >= 0.f && x0 <= (float)(vi.w - 1) && y1 >= 0.f && y0 <= (float)(vi.h - 1) && x0 <= x1 && y0 <= y1) {
                    int tx0 = tile_of(x0 > 0.f ? (int)x0 : 0, vb.tile_w);
                    int tx1 = tile_of(x1 < (float)(vi.w - 1) ? (int)x1 : vi.w - 1, vb.tile_w);
                    int ty0 = tile_of(y0 > 0.f ? (int)y0 : 0, vb.tile_h);
                    int ty1 = tile_of(y1 < (float)(vi.h - 1) ? (int)y1 : vi.h - 1, vb.tile_h);
                    // colour (Eq. 2; SH for degree >= 1)
                    float col[3];
                    if (D == 0) {
                        col[0] = k0[0]; col[1] = k0[1]; col[2] = k0[2];
                    } else {
                        float C[3];
                        cam_centre(T, C);
                        float dx = m[0] - C[0], dy = m[1] - C[1], dz = m[2] - C[2];
                        float in = rsqrtf(dx * dx + dy * dy + dz * dz);
                        float Y[16];
                        sh_basis<D>(dx * in, dy * in, dz * in, Y);
                        float c3[3] = {k0[0], k0[1], k0[2]};
#pragma unroll
                        for (int i = 1; i < NC; ++i) {
#pragma unroll
                            for (int ch = 0; ch < 3; ++ch) c3[ch] += Y[i] * s_sh[(3 * i + ch) * kShStride + threadIdx.x];
                        }
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) col[ch] = fmaxf(c3[ch], 0.0f);
                    }
                    Record R;
                    const float qc = fminf(kCutoffQ, 2.0f * kLn2 * (lo2 - kSkipL)) * (1.0f + 2e-5f + 8e-7f * kappa);
                    R.a = make_float4(u, vv, cc * idet, -cb * idet);
                    R.b = make_float4(ca * idet, A.opacity, pz, lo2);
                    R.c = make_float4(col[0], col[1], col[2], qc);
                    a.rec[r] = R;
                    ext = make_int2(rx, ry);
                    mask |= 1u << v;
                    has = true;
                    ell = cover_ellipse(u, vv, R.a.z, R.a.w, R.b.x, qc);
                    ctx0 = tx0; cty0 = ty0; cntx = tx1 - tx0 + 1; cnty = ty1 - ty0 + 1;
                    cbin = depth_bin(pz);
                    if (a.occl) {
                        // the blend's staged values (stage_record), and whether the
                        // ellipse on which alpha falls to kOcclAlpha (q = 2 ln(o / kOcclAlpha),
                        // within the cover bound) has an inscribed disc wide enough for a tile
                        const StagedGauss sg = stage_record(R);
                        og = {sg.u, sg.v, sg.a, sg.b, sg.c, sg.thr, sg.lo2, 0.f};
                        const float ha = 0.5f * (R.a.z - R.b.x);
                        const float lmax = 0.5f * (R.a.z + R.b.x) + sqrtf(ha * ha + R.a.w * R.a.w);
                        const float qa = fminf(qc, 2.0f * kLn2 * (lo2 - kOcclLog2Alpha) * 1.001f);
                        og.w = qa > 0.f && qa >= lmax * (float)a.tile_fit &&
                                       (unsigned)cbin <= min(a.view_hint[v], 255u) + kHintSlack ? 1.f : 0.f;
                    }
                }
            }
        }
        count_cover_warp(a, vb, vi, has, ell, ctx0, cty0, cntx, cnty, cbin, og);
        if (live) a.ext[r] = ext;
    }
    if (live) a.vis_mask[g] = mask;
}

// Backward of the projection for every view of one Gaussian, accumulating
// the parameter gradients in registers and writing each once.
template <int D>
__global__ void __launch_bounds__(256, 2) project_bwd_kernel(const ProjectBwdArgs a, const __grid_constant__ ViewBatch vb) {
    constexpr int NC = (D + 1) * (D + 1);
    __shared__ float s_tw[8][S3GS_MAX_VIEWS][6];
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool live = g < a.n;
    long long gg = live ? g : 0;

    float m[3] = {a.means[3 * gg], a.means[3 * gg + 1], a.means[3 * gg + 2]};
    float ls[3] = {a.log_scales[3 * gg], a.log_scales[3 * gg + 1], a.log_scales[3 * gg + 2]};
    float4 q4 = reinterpret_cast<const float4 *>(a.quats)[gg];
    float q[4] = {q4.x, q4.y, q4.z, q4.w};
    Activated A;
    bool ok = activate(ls, q, a.opacity_logits[gg], A) && live;
    // Colour coefficients and their gradient: degree 0 in registers; higher degrees
    // in shared memory (coefficient e of thread t at e * kShStride + t), staged and
    // written back by the CTA as one contiguous block, so that 2 x 3 (D + 1)^2
    // values per thread do not limit the kernel's occupancy.
    extern __shared__ float s_dyn[];
    float *s_k = s_dyn, *s_dk = s_dyn + NC * 3 * kShStride;
    float k0[3] = {0.f, 0.f, 0.f}, dk0[3] = {0.f, 0.f, 0.f};
    const long long g0 = (long long)blockIdx.x * blockDim.x;
    const int ng = (int)(a.n - g0 < (long long)blockDim.x ? a.n - g0 : (long long)blockDim.x);
    if (D == 0) {
        const float *cp = a.colors + gg * 3;
        k0[0] = cp[0]; k0[1] = cp[1]; k0[2] = cp[2];
    } else {
        const float *src = a.colors + g0 * NC * 3;
        for (int e = threadIdx.x; e < ng * NC * 3; e += blockDim.x) {
            const int lt = e / (NC * 3), kk = e - lt * (NC * 3);
            s_k[kk * kShStride + lt] = __ldg(src + e);
        }
#pragma unroll
        for (int i = 0; i < NC * 3; ++i) s_dk[i * kShStride + threadIdx.x] = 0.f;
    }

    float dmu[3] = {0.f, 0.f, 0.f};
    float dSig[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // gradient w.r.t. the world covariance
    float dO = 0.f;

    // Views are processed in chunks whose 2D-gradient rows are all requested
    // before any is used, so their latencies overlap; the visibility mask says
    // which rows exist without reading the per-record extents.
    const unsigned vis = ok ? a.vis_mask[gg] : 0u;
    // Every seen view's row is requested into L2 up front, so the chunked loads
    // below wait on L2 rather than on DRAM (the prefetch holds no registers).
    for (int v = 0; v < vb.n_views; ++v)
        if ((vis >> v) & 1u) {
            const char *row = reinterpret_cast<const char *>(a.grad2d + ((long long)v * a.n + gg) * kGrad2d);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(row));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(row + 32));
        }
    for (int i = threadIdx.x; i < 8 * S3GS_MAX_VIEWS * 6; i += blockDim.x) (&s_tw[0][0][0])[i] = 0.f;
    __syncthreads();
    constexpr int CH = D >= 2 ? 2 : 4;
    for (int v0 = 0; v0 < vb.n_views; v0 += CH) {
        const unsigned chunk_any = __any_sync(0xffffffffu, (vis >> v0) & ((1u << CH) - 1u));
        if (!chunk_any) continue;  // no Gaussian of this warp is seen by these views
        float gr4[CH][kGrad2d];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const bool seen = (v0 + u < vb.n_views) && ((vis >> (v0 + u)) & 1u);
            const float2 *src = reinterpret_cast<const float2 *>(a.grad2d + ((long long)(v0 + u) * a.n + gg) * kGrad2d);
#pragma unroll
            for (int i = 0; i < kGrad2d / 2; ++i) {
                const float2 x = seen ? src[i] : make_float2(0.f, 0.f);
                gr4[u][2 * i] = x.x;
                gr4[u][2 * i + 1] = x.y;
            }
        }
#pragma unroll
        for (int u = 0; u < CH; ++u)
            if ((v0 + u < vb.n_views) && ((vis >> (v0 + u)) & 1u)) {  // leave the accumulator clean
                float2 *dst = reinterpret_cast<float2 *>(a.grad2d + ((long long)(v0 + u) * a.n + gg) * kGrad2d);
#pragma unroll
                for (int i = 0; i < kGrad2d / 2; ++i) dst[i] = make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int v = v0 + u;
            if (v >= vb.n_views) break;
            const ViewInfo &vi = vb.v[v];
            const bool seen = (vis >> v) & 1u;
            if (!__any_sync(0xffffffffu, seen)) continue;
            float tw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (seen) {
                const float *gr = gr4[u];
                float T[12];
                load_pose(vi, a.Tdev, v, T);
                float px = view_coord(T, m, T[3]);
                float py = view_coord(T + 4, m, T[7]);
                float pz = view_coord(T + 8, m, T[11]);
                float Sc[9];
                cam_cov(T, A.Sig, Sc);
                float iz = 1.0f / pz, iz2 = iz * iz;
                float fx = vi.fx, fy = vi.fy;
                float j00 = fx * iz, j02 = -fx * px * iz2, j11 = fy * iz, j12 = -fy * py * iz2;
                float ca = j00 * (j00 * Sc[0] + j02 * Sc[2]) + j02 * (j00 * Sc[6] + j02 * Sc[8]) + kDilation;
                float cb = j11 * (j00 * Sc[1] + j02 * Sc[7]) + j12 * (j00 * Sc[2] + j02 * Sc[8]);
                float cc = j11 * (j11 * Sc[4] + j12 * Sc[5]) + j12 * (j11 * Sc[7] + j12 * Sc[8]) + kDilation;
                float idet = 1.0f / (ca * cc - cb * cb);
                float cA = cc * idet, cB = -cb * idet, cC = ca * idet;
                // the blend's moments of g = dL/dalpha * alpha -> gradients of the centre
                // (u, v) and of the conic [[A, B], [B, C]] (alpha = o exp(-(A dx^2 + 2 B dx dy
                // + C dy^2) / 2), dx = i - u)
                const float gU = cA * gr[kGU] + cB * gr[kGV];
                const float gV = cB * gr[kGU] + cC * gr[kGV];
                const float gA = -0.5f * gr[kGA], gC = -0.5f * gr[kGC];
                // conic -> 2D covariance: G2 = -Sinv Ginv Sinv, Ginv = [[gA, gB/2], [gB/2, gC]]
                float hB = -0.5f * gr[kGB];
                float t00 = cA * gA + cB * hB, t01 = cA * hB + cB * gC;
                float t10 = cB * gA + cC * hB, t11 = cB * hB + cC * gC;
                float g00 = -(t00 * cA + t01 * cB);
                float g01 = -(t00 * cB + t01 * cC);
                float g11 = -(t10 * cB + t11 * cC);
                // cov2 = J Sc J^T: dSc = J^T G2 J, dJ = 2 G2 J Sc
                float P0[3] = {g00 * j00, g01 * j11, g00 * j02 + g01 * j12};  // row 0 of G2 J
                float P1[3] = {g01 * j00, g11 * j11, g01 * j02 + g11 * j12};  // row 1 of G2 J
                float Gc[9];
                const float J0[3] = {j00, 0.f, j02}, J1[3] = {0.f, j11, j12};
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) Gc[3 * i + j] = J0[i] * P0[j] + J1[i] * P1[j];
                float dJ00 = 2.f * (P0[0] * Sc[0] + P0[1] * Sc[3] + P0[2] * Sc[6]);
                float dJ02 = 2.f * (P0[0] * Sc[2] + P0[1] * Sc[5] + P0[2] * Sc[8]);
                float dJ11 = 2.f * (P1[0] * Sc[1] + P1[1] * Sc[4] + P1[2] * Sc[7]);
                float dJ12 = 2.f * (P1[0] * Sc[2] + P1[1] * Sc[5] + P1[2] * Sc[8]);
                // Sc = W Sig W^T: dSig += W^T Gc W
                float GW[9];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        GW[3 * i + j] = Gc[3 * i] * T[j] + Gc[3 * i + 1] * T[4 + j] + Gc[3 * i + 2] * T[8 + j];
                {
                    float WG[9];
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            WG[3 * i + j] = T[i] * GW[j] + T[4 + i] * GW[3 + j] + T[8 + i] * GW[6 + j];
                    dSig[0] += WG[0]; dSig[1] += WG[1]; dSig[2] += WG[2];
                    dSig[3] += WG[4]; dSig[4] += WG[5]; dSig[5] += WG[8];
                }
                // camera-frame mean
                float dp0 = gU * fx * iz - dJ02 * fx * iz2;
                float dp1 = gV * fy * iz - dJ12 * fy * iz2;
                float dp2 = -gU * fx * px * iz2 - gV * fy * py * iz2 + gr[kGZ] - dJ00 * fx * iz2 +
                            2.f * dJ02 * fx * px * iz2 * iz - dJ11 * fy * iz2 + 2.f * dJ12 * fy * py * iz2 * iz;
                dmu[0] += T[0] * dp0 + T[4] * dp1 + T[8] * dp2;
                dmu[1] += T[1] * dp0 + T[5] * dp1 + T[9] * dp2;
                dmu[2] += T[2] * dp0 + T[6] * dp1 + T[10] * dp2;
                // twist: dp = rho + phi x p; dSc = [phi]x Sc - Sc [phi]x
                tw[0] = dp0; tw[1] = dp1; tw[2] = dp2;
                tw[3] = py * dp2 - pz * dp1;
                tw[4] = pz * dp0 - px * dp2;
                tw[5] = px * dp1 - py * dp0;
                // Q = Sc Gc - Gc Sc; dphi += 2 (Q12, Q20, Q01)
                float Q12 = 0.f, Q20 = 0.f, Q01 = 0.f;
#pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
                    Q12 += Sc[3 + kk] * Gc[3 * kk + 2] - Gc[3 + kk] * Sc[3 * kk + 2];
                    Q20 += Sc[6 + kk] * Gc[3 * kk + 0] - Gc[6 + kk] * Sc[3 * kk + 0];
                    Q01 += Sc[0 + kk] * Gc[3 * kk + 1] - Gc[0 + kk] * Sc[3 * kk + 1];
                }
                tw[3] += 2.f * Q12; tw[4] += 2.f * Q20; tw[5] += 2.f * Q01;
                dO += gr[kGO];
                // colour
                if (D == 0) {
                    dk0[0] += gr[kGR]; dk0[1] += gr[kGG]; dk0[2] += gr[kGBl];
                } else {
                    float C[3];
                    cam_centre(T, C);
                    float ddx = m[0] - C[0], ddy = m[1] - C[1], ddz = m[2] - C[2];
                    float in = rsqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
                    float hx = ddx * in, hy = ddy * in, hz = ddz * in;
                    float Y[16];
                    sh_basis<D>(hx, hy, hz, Y);
                    float gcol[3] = {gr[kGR], gr[kGG], gr[kGBl]};
                    const float *kt = s_k + threadIdx.x;
                    float *dkt = s_dk + threadIdx.x;
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        float c = kt[ch * kShStride];
#pragma unroll
                        for (int i = 1; i < NC; ++i) c += Y[i] * kt[(3 * i + ch) * kShStride];
                        if (!(c > 0.f)) gcol[ch] = 0.f;  // clamped at zero
                    }
                    float w[16];
#pragma unroll
                    for (int i = 0; i < NC; ++i) {
                        dkt[(3 * i) * kShStride] += Y[i] * gcol[0];
                        dkt[(3 * i + 1) * kShStride] += Y[i] * gcol[1];
                        dkt[(3 * i + 2) * kShStride] += Y[i] * gcol[2];
                        w[i] = gcol[0] * kt[(3 * i) * kShStride] + gcol[1] * kt[(3 * i + 1) * kShStride] +
                               gcol[2] * kt[(3 * i + 2) * kShStride];
                    }
                    float3 gh = sh_weighted_grad<D>(hx, hy, hz, w);
                    float dd = gh.x * hx + gh.y * hy + gh.z * hz;
                    float dx_ = (gh.x - hx * dd) * in, dy_ = (gh.y - hy * dd) * in, dz_ = (gh.z - hz * dd) * in;
                    dmu[0] += dx_; dmu[1] += dy_; dmu[2] += dz_;
                    // the camera centre moves by -W^T rho: d rho += W ddir
                    tw[0] += T[0] * dx_ + T[1] * dy_ + T[2] * dz_;
                    tw[1] += T[4] * dx_ + T[5] * dy_ + T[6] * dz_;
                    tw[2] += T[8] * dx_ + T[9] * dy_ + T[10] * dz_;
                }
            }
            // warp reduce the twist contributions of this view (fixed order)
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                float x = tw[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) s_tw[warp][v][i] = x;
            }
        }
    }

    if (ok) {
        // Sig = M M^T with M = R diag(s): dM = 2 dSig M
        float S[9];
        sym_full(dSig, S);
        float M[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) M[3 * i + j] = A.R[3 * i + j] * A.s[j];
        float dR[9], ds[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float dMij = 2.f * (S[3 * i] * M[j] + S[3 * i + 1] * M[3 + j] + S[3 * i + 2] * M[6 + j]);
                ds[j] += dMij * A.R[3 * i + j];
                dR[3 * i + j] = dMij * A.s[j];
            }
        float w = A.qn[0], x = A.qn[1], y = A.qn[2], z = A.qn[3];
        float dq[4];
        dq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
        dq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                       2.f * x * dR[8]);
        dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                       2.f * y * dR[8]);
        dq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                       x * dR[6] + y * dR[7]);
        float dot = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
        float dqq[4] = {(dq[0] - w * dot) * A.qinv, (dq[1] - x * dot) * A.qinv, (dq[2] - y * dot) * A.qinv,
                        (dq[3] - z * dot) * A.qinv};
        float dls[3] = {ds[0] * A.s[0], ds[1] * A.s[1], ds[2] * A.s[2]};
        // alpha = o 2^p: d alpha / d logit = alpha (1 - o), applied once to the sum of g
        float dol = (1.0f - A.opacity) * dO;
        const bool acc = a.accumulate != 0;
        if (a.d_means) {
            float *o = a.d_means + 3 * g;
#pragma unroll
            for (int i = 0; i < 3; ++i) o[i] = acc ? o[i] + dmu[i] : dmu[i];
        }
        if (a.d_log_scales) {
            float *o = a.d_log_scales + 3 * g;
#pragma unroll
            for (int i = 0; i < 3; ++i) o[i] = acc ? o[i] + dls[i] : dls[i];
        }
        if (a.d_quats) {
            float4 *o = reinterpret_cast<float4 *>(a.d_quats) + g;
            float4 val = make_float4(dqq[0], dqq[1], dqq[2], dqq[3]);
            if (acc) {
                float4 old = *o;
                val.x += old.x; val.y += old.y; val.z += old.z; val.w += old.w;
            }
            *o = val;
        }
        if (a.d_opacity_logits) a.d_opacity_logits[g] = acc ? a.d_opacity_logits[g] + dol : dol;
        if (a.d_colors && D == 0) {
            float *o = a.d_colors + g * 3;
#pragma unroll
            for (int i = 0; i < 3; ++i) o[i] = acc ? o[i] + dk0[i] : dk0[i];
        }
    } else if (live) {
        // invalid quaternion: the Gaussian is never rendered, its gradient is zero
        const bool acc = a.accumulate != 0;
        if (!acc) {
            if (a.d_means) for (int i = 0; i < 3; ++i) a.d_means[3 * g + i] = 0.f;
            if (a.d_log_scales) for (int i = 0; i < 3; ++i) a.d_log_scales[3 * g + i] = 0.f;
            if (a.d_quats) for (int i = 0; i < 4; ++i) a.d_quats[4 * g + i] = 0.f;
            if (a.d_opacity_logits) a.d_opacity_logits[g] = 0.f;
            if (a.d_colors && D == 0) for (int i = 0; i < 3; ++i) a.d_colors[g * 3 + i] = 0.f;
        }
    }

    __syncthreads();
    if (D > 0 && a.d_colors) {
        // the CTA's colour gradients, one coalesced block; a Gaussian with an invalid
        // quaternion gets zeros, or keeps its accumulated value
        __shared__ unsigned char s_ok[256];
        s_ok[threadIdx.x] = ok ? 1 : 0;
        __syncthreads();
        const bool acc = a.accumulate != 0;
        float *dst = a.d_colors + g0 * NC * 3;
        for (int e = threadIdx.x; e < ng * NC * 3; e += blockDim.x) {
            const int lt = e / (NC * 3), kk = e - lt * (NC * 3);
            if (acc && !s_ok[lt]) continue;
            const float x = s_dk[kk * kShStride + lt];
            dst[e] = acc ? dst[e] + x : x;
        }
    }
    // block partial of the twist, summed over warps in a fixed order
    for (int i = threadIdx.x; i < vb.n_views * 6; i += blockDim.x) {
        int v = i / 6, c = i % 6;
        float s = 0.f;
        for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += s_tw[wv][v][c];
        a.twist_partial[((long long)blockIdx.x * vb.n_views + v) * 6 + c] = s;
    }
}

}  // namespace

// shared memory of the staged SH coefficients of degree D (none for degree 0)
constexpr size_t sh_smem(int D) { return D == 0 ? 0 : (size_t)(D + 1) * (D + 1) * 3 * kShStride * sizeof(float); }

template <int D>
cudaError_t launch_project_d(const ProjectArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    static SmemOptIn st;
    cudaError_t e = opt_in_smem(project_kernel<D>, sh_smem(D), st);
    if (e != cudaSuccess) return e;
    project_kernel<D><<<grid, 256, sh_smem(D), s>>>(a, vb);
    return cudaGetLastError();
}

// the backward holds the coefficients and their gradients
template <int D>
cudaError_t launch_project_bwd_d(const ProjectBwdArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    static SmemOptIn st;
    cudaError_t e = opt_in_smem(project_bwd_kernel<D>, 2 * sh_smem(D), st);
    if (e != cudaSuccess) return e;
    project_bwd_kernel<D><<<grid, 256, 2 * sh_smem(D), s>>>(a, vb);
    return cudaGetLastError();
}

cudaError_t launch_project(const ProjectArgs &a, const ViewBatch &vb, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    int grid = (int)((a.n + 255) / 256);
    switch (a.sh_degree) {
    case 0: return launch_project_d<0>(a, vb, grid, s);
    case 1: return launch_project_d<1>(a, vb, grid, s);
    case 2: return launch_project_d<2>(a, vb, grid, s);
    default: return launch_project_d<3>(a, vb, grid, s);
    }
}

int project_bwd_grid(long long n) { return (int)((n + 255) / 256); }

cudaError_t launch_project_bwd(const ProjectBwdArgs &a, const ViewBatch &vb, int *grid_out, cudaStream_t s) {
    int grid = project_bwd_grid(a.n);
    if (grid_out) *grid_out = grid;
    if (a.n == 0) return cudaSuccess;
    switch (a.sh_degree) {
    case 0: return launch_project_bwd_d<0>(a, vb, grid, s);
    case 1: return launch_project_bwd_d<1>(a, vb, grid, s);
    case 2: return launch_project_bwd_d<2>(a, vb, grid, s);
    default: return launch_project_bwd_d<3>(a, vb, grid, s);
    }
}

}  // namespace s3gs
