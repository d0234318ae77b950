// Internal declarations of the sm_103a Gaussian-splatting library.
//
// Pipeline of one forward (all views of a call in one pass per stage):
//   project_kernel      EWA projection + colour of every (view, Gaussian) record
//                       and per-tile duplicate counts              (Eq. 1, Sec. 3.1)
//   scan_*              exclusive scan of the tile counts -> tile ranges, total K
//   emit_kernel         bucket (depth, index) keys into their tiles
//   tile_sort_kernel    per-tile sort of the keys by (depth, index)  (Eq. 3 order)
//   blend_fwd_kernel    front-to-back compositing per tile          (Eq. 2-5)
// and of one backward:
//   blend_bwd_kernel    back-to-front per tile, warp-reduced gradients   (Eq. 11)
//   det_reduce_kernel   (deterministic mode) fixed-order sum of per-tile partials
//   project_bwd_kernel  chain to Gaussian parameters and per-view twist partials
//   twist_reduce_kernel fixed-order sum of the twist partials
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/s3gs.h"

namespace s3gs {

// Rendering constants (the 3DGS rules the paper inherits; see s3gs.h).
constexpr float kDilation = 0.3f;
constexpr float kCutoffQ = 9.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr int kExtentMax = 1 << 24;  // clamp of the integer half-extent of a tile cover
constexpr int kGrad2d = 10;          // per-record 2D gradient slots

// Duplicates are bucketed by (tile, coarse depth bin). The bin is the exponent
// and the top 4 mantissa bits of the float depth (16 bins per octave), offset so
// that z = 0.2 falls in bin 0; 256 bins cover 0.2 m to about 13 km and deeper
// keys share the last bin. The bin is monotone in depth, so a tile's buckets,
// each sorted, concatenate to the tile's list in (depth, index) order; bucket b
// of tile t has id t * 256 + b.
constexpr int kDepthBins = 256;

// q = floor(x / d) and r = x - q d for x < 2^24, d >= 1, without an integer
// division: both roundings toward zero make the float estimate a lower bound,
// off by less than 4 / d, and the loop adds what it is short of.
__device__ __forceinline__ unsigned div_small(unsigned x, unsigned d, unsigned &r) {
    unsigned q = __float2uint_rz(__fmul_rz(__uint2float_rz(x), __frcp_rz(__uint2float_rz(d))));
    r = x - q * d;
    while (r >= d) {
        ++q;
        r -= d;
    }
    return q;
}
// Tile index of a non-negative pixel coordinate. Every supported tile side (8,
// 16 or 32) is a power of two, so the quotient is a shift.
__device__ __forceinline__ int tile_of(int x, int side) { return x >> (__ffs(side) - 1); }
__device__ __forceinline__ int depth_bin(float z) {
    const int b = (int)(__float_as_uint(z) >> 19) - 1993;
    return b < 0 ? 0 : (b > kDepthBins - 1 ? kDepthBins - 1 : b);
}

// 2D gradient row of a record, as the backward blend accumulates it over the
// pixels, with g = dL/dalpha * alpha per (pixel, Gaussian) pair and (dx, dy) the
// pixel's offset from the centre: kGU = sum g dx, kGV = sum g dy, kGA = sum g dx^2,
// kGB = sum g dx dy, kGC = sum g dy^2, kGO = sum g (moments, turned into the
// gradients of the centre, conic and opacity logit by the projection backward),
// then dL/d(r, g, b) and dL/dz directly.
enum { kGU = 0, kGV, kGA, kGB, kGC, kGO, kGR, kGG, kGBl, kGZ };

struct ViewInfo {
    int w, h;
    float fx, fy, cx, cy;
    float T[12];   // world-to-camera, row-major 3x4
    int tiles_x, tiles_y;
    int tile_base;  // first global tile id of this view
    int pad;
    long long pix_base;  // first pixel of this view in the packed outputs
};

struct ViewBatch {
    int n_views;
    int tile_w, tile_h;
    int total_tiles;
    long long total_pixels;
    ViewInfo v[S3GS_MAX_VIEWS];
};

// One projected (view, Gaussian) record: 48 bytes, read as three float4.
struct __align__(16) Record {
    float4 a;  // u, v, A, B  (conic = [[A, B], [B, C]])
    float4 b;  // C, opacity, z, log2(opacity)
    float4 c;  // r, g, b, q_cover (the tile-cover bound on q, see row_span)
};

// Tile cover. A record is listed in a tile only if its ellipse q(d) <= q_cover,
// q(d) = A dx^2 + 2 B dx dy + C dy^2, meets the box spanned by the centres of
// the tile's pixels inside the image. q_cover is the largest q at which the
// blend can accept a pair -- min(9, 2 ln 2 (log2 opacity - log2(1/255))), the
// 3-sigma cutoff or the 1/255 skip -- widened for FP32 rounding of the conic
// (relative 2e-5 plus 8e-7 times its condition number).
//
// The cover is taken one tile row at a time. The part of the ellipse inside the
// row's band of pixel-centre rows dy in [lo, hi] is convex, so its x-extent is an
// interval, and a tile of the row meets the ellipse iff its columns of pixel
// centres meet that interval. For fixed dy the ellipse spans
// dx = (-B dy -/+ sqrt(A q_cover - det dy^2)) / A (det = A C - B^2); its leftmost
// point lies at dy_L = B sqrt(q_cover / (C det)) and its rightmost at -dy_L, so
// the band's interval runs from the left boundary at dy_L clamped to the band to
// the right boundary at -dy_L clamped to the band, and the band is empty beyond
// |dy| > sqrt(A q_cover / det). The interval is widened by 1e-5 of its terms,
// by 7e-4 sqrt(q_cover / A) (the square root's sensitivity where the span
// narrows to a point) and by 1e-3 px, so that it contains every column at which
// the FP32 blend can pass; a tile listed needlessly only costs evaluations. The
// tile range is rounded outwards and clamped to the record's bounding
// rectangle. Every operation is an explicit round-to-nearest intrinsic (or an
// exact min/max/ceil/floor), so the projection's counts, the emission and the
// deterministic reduce list identical tiles, and the integer referee can repeat
// the arithmetic in plain C.
struct CoverEllipse {
    float u, v, B, iA;
    float Aqc, det, ym, yL;  // A q_cover, A C - B^2, the band limit sqrt(A q_cover / det), dy_L
    float mq;                // absolute widening (px): 7e-4 sqrt(q_cover / A) + 1e-3
};

__device__ __forceinline__ CoverEllipse cover_ellipse(float u, float v, float A, float B, float C, float qc) {
    CoverEllipse e;
    e.u = u;
    e.v = v;
    e.B = B;
    e.iA = __fdiv_rn(1.0f, A);
    e.Aqc = __fmul_rn(A, qc);
    e.det = __fmaf_rn(A, C, -__fmul_rn(B, B));
    if (!(qc >= 0.f)) {
        e.ym = -1.0f;  // q_cover < 0: the record reaches no pixel
        e.yL = 0.f;
        e.mq = 0.f;
        return e;
    }
    const float g = e.det > 0.f ? __fdiv_rn(qc, e.det) : 0.f;
    e.ym = e.det > 0.f ? __fmaf_rn(__fsqrt_rn(__fmul_rn(A, g)), 1.00001f, 1e-3f) : 3.0e38f;
    e.yL = e.det > 0.f ? __fmul_rn(B, __fsqrt_rn(__fdiv_rn(g, C))) : 0.f;
    e.mq = __fmaf_rn(7e-4f, __fsqrt_rn(__fmul_rn(qc, e.iA)), 1e-3f);
    return e;
}

// Tile columns [c.x, c.y] (empty when c.y < c.x) of the tile row whose pixel-centre
// rows are [py0, py1] that meet the record's ellipse, within the rectangle's columns
// [tx0, tx1]; inv_tw = 1 / tile width (a power of two, so the product is exact).
__device__ __forceinline__ int2 row_span(const CoverEllipse &e, int py0, int py1, int tx0, int tx1, float inv_tw) {
    const float lo = fmaxf(__fsub_rn((float)py0, e.v), -e.ym);
    const float hi = fminf(__fsub_rn((float)py1, e.v), e.ym);
    if (!(lo <= hi)) return make_int2(1, 0);
    if (!(e.det > 0.f)) return make_int2(tx0, tx1);  // degenerate conic: the whole rectangle row
    const float yl = fminf(fmaxf(e.yL, lo), hi), yr = fminf(fmaxf(-e.yL, lo), hi);
    const float sl = __fsqrt_rn(fmaxf(__fmaf_rn(-e.det, __fmul_rn(yl, yl), e.Aqc), 0.f));
    const float sr = __fsqrt_rn(fmaxf(__fmaf_rn(-e.det, __fmul_rn(yr, yr), e.Aqc), 0.f));
    const float byl = __fmul_rn(e.B, yl), byr = __fmul_rn(e.B, yr);
    const float xl = __fmul_rn(__fsub_rn(-byl, sl), e.iA);
    const float xr = __fmul_rn(__fadd_rn(-byr, sr), e.iA);
    const float ml = __fmaf_rn(1e-5f, __fmul_rn(__fadd_rn(fabsf(byl), sl), e.iA), e.mq);
    const float mr = __fmaf_rn(1e-5f, __fmul_rn(__fadd_rn(fabsf(byr), sr), e.iA), e.mq);
    const float a = __fsub_rn(__fadd_rn(e.u, xl), ml), b = __fadd_rn(__fadd_rn(e.u, xr), mr);
    // tile c holds centre columns [c tw, c tw + tw - 1]: it meets [a, b] iff
    // c >= ceil((a + 1) / tw) - 1 and c <= floor(b / tw)
    const float c0 = fminf(fmaxf(__fsub_rn(ceilf(__fmul_rn(__fadd_rn(a, 1.0f), inv_tw)), 1.0f), (float)tx0),
                           (float)(tx1 + 1));
    const float c1 = fmaxf(fminf(floorf(__fmul_rn(b, inv_tw)), (float)tx1), (float)(tx0 - 1));
    return make_int2((int)c0, (int)c1);
}

// Warp helpers of the two-level cover enumeration: an inclusive scan of one
// count per lane, and the lane whose interval [incl - count, incl) holds j (a
// 5-step search over the scan; every lane must take part).
__device__ __forceinline__ unsigned warp_incl_scan(unsigned v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

__device__ __forceinline__ int warp_find(unsigned incl, unsigned j) {
    int src = 0;
#pragma unroll
    for (int b = 16; b > 0; b >>= 1)
        if (__shfl_sync(0xffffffffu, incl, src + b - 1) <= j) src += b;
    return src > 31 ? 31 : src;
}

__device__ __forceinline__ CoverEllipse shfl_ellipse(const CoverEllipse &e, int src) {
    CoverEllipse r;
    r.u = __shfl_sync(0xffffffffu, e.u, src);
    r.v = __shfl_sync(0xffffffffu, e.v, src);
    r.B = __shfl_sync(0xffffffffu, e.B, src);
    r.iA = __shfl_sync(0xffffffffu, e.iA, src);
    r.Aqc = __shfl_sync(0xffffffffu, e.Aqc, src);
    r.det = __shfl_sync(0xffffffffu, e.det, src);
    r.ym = __shfl_sync(0xffffffffu, e.ym, src);
    r.yL = __shfl_sync(0xffffffffu, e.yL, src);
    r.mq = __shfl_sync(0xffffffffu, e.mq, src);
    return r;
}

struct DevCounters {
    unsigned long long n_dup;     // total (Gaussian, tile) pairs K of the last forward
    unsigned int overflow;        // 1 if K exceeded the key capacity
    unsigned int work_fwd;        // persistent-grid work counters
    unsigned int work_bwd;
    unsigned int pad;
    unsigned long long fwd_processed, fwd_blended, bwd_processed;
};

// Read a view's pose: the device override if given, else the camera's.
__device__ __forceinline__ void load_pose(const ViewInfo &vi, const float *Tdev, int v, float T[12]) {
    if (Tdev) {
#pragma unroll
        for (int k = 0; k < 12; ++k) T[k] = __ldg(Tdev + 12 * v + k);
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) T[k] = vi.T[k];
    }
}

__device__ __forceinline__ int view_of_tile(const ViewBatch &vb, int t) {
    int v = 0;
    for (int k = 1; k < vb.n_views; ++k)
        if (t >= vb.v[k].tile_base) v = k;
    return v;
}

// Per-pair evaluation shared by the forward, the recompute replay and the
// backward. A staged Gaussian carries its conic pre-scaled into the log2 domain
// (a = -log2(e)/2 A, b = -log2(e) B, c = -log2(e)/2 C) and log2 of its opacity,
// so that p = a dx^2 + b dx dy + c dy^2 = -log2(e) q / 2 and
// alpha = opacity * exp(-q/2) = 2^(p + log2 opacity). The 3-sigma cutoff
// (q <= 9), the 1/255 skip and the 0.99 clamp are all decided on these
// exponents, before any exponential is evaluated. Explicit round-to-nearest
// intrinsics make the three callers bit-identical, so the backward takes
// exactly the forward's cutoff/skip/stop decisions.
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kCutP = -6.4921276840003355f;   // -4.5 log2(e): q <= 9
constexpr float kSkipL = -7.9943534368588578f;  // log2(1/255)
constexpr float kClampL = -0.0144995696951151f; // log2(0.99)

struct StagedGauss {
    float u, v, a, b;      // centre, scaled conic (xx, 2 xy)
    float c, lo2, thr, z;  // scaled conic (yy), log2 opacity, pass threshold on p, depth
};

__device__ __forceinline__ StagedGauss stage_record(const Record &r) {
    StagedGauss g;
    g.u = r.a.x;
    g.v = r.a.y;
    g.a = __fmul_rn(-0.5f * kLog2e, r.a.z);
    g.b = __fmul_rn(-kLog2e, r.a.w);
    g.c = __fmul_rn(-0.5f * kLog2e, r.b.x);
    g.z = r.b.z;
    g.lo2 = r.b.w;
    // a pair passes when p >= kCutP (inside the 3-sigma ellipse) and p + log2 o >=
    // log2(1/255) (alpha not skipped): one compare against the larger bound
    g.thr = fmaxf(kCutP, __fsub_rn(kSkipL, g.lo2));
    return g;
}

struct PairEval {
    float dx, dy;
    float l;       // p + log2(opacity): alpha = 2^l before the clamp
    bool pass;     // inside the 3-sigma ellipse and alpha >= 1/255
    bool clamped;  // alpha hit the 0.99 clamp
};

// The terms of p that depend on the column only: p = a dx^2 + b dx dy + c dy^2 is
// evaluated as (a dx) dx + dy (b dx + c dy), so a thread whose pixels share a
// column forms A0 = (a dx) dx and B0 = b dx once per Gaussian.
struct ColTerms {
    float dx, A0, B0;
};

__device__ __forceinline__ ColTerms col_terms(float px, float u, float a, float b) {
    ColTerms t;
    t.dx = __fsub_rn(px, u);
    t.A0 = __fmul_rn(__fmul_rn(a, t.dx), t.dx);
    t.B0 = __fmul_rn(b, t.dx);
    return t;
}

__device__ __forceinline__ PairEval eval_pair(float px, float py, float u, float v, float a, float b, float c,
                                              float lo2, float thr) {
    const ColTerms ct = col_terms(px, u, a, b);
    PairEval e;
    e.dx = ct.dx;
    e.dy = __fsub_rn(py, v);
    const float p = __fmaf_rn(e.dy, __fmaf_rn(c, e.dy, ct.B0), ct.A0);
    e.l = __fadd_rn(p, lo2);
    e.pass = p >= thr;
    e.clamped = e.l >= kClampL;
    return e;
}

// The same evaluation for two pixels of one column (rows py.x and py.y) in packed
// FP32 (Blackwell's paired FP32 instructions): every lane of __ffma2_rn /
// __fadd2_rn rounds as the scalar intrinsic does, so each lane equals eval_pair
// bit for bit (a - b is formed as a + (-b), which rounds identically).
__device__ __forceinline__ float2 bcast2(float x) { return make_float2(x, x); }

__device__ __forceinline__ void eval_pair2(const ColTerms &ct, float2 py, float v, float c, float lo2, float2 &dy,
                                           float2 &p, float2 &l) {
    dy = __fadd2_rn(py, bcast2(-v));
    p = __ffma2_rn(dy, __ffma2_rn(bcast2(c), dy, bcast2(ct.B0)), bcast2(ct.A0));
    l = __fadd2_rn(p, bcast2(lo2));
}

// 2^x with the hardware approximation (relative error below 2^-22); every
// exponent reaching it lies in [log2(1/255), log2(0.99)] (to within the rounding
// of the pass threshold), far from denormals.
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// alpha of a passing pair
__device__ __forceinline__ float pair_alpha(const PairEval &e) { return e.clamped ? kAlphaMax : fast_exp2(e.l); }

__device__ __forceinline__ float next_T(float T, float alpha) { return __fmul_rn(T, __fsub_rn(1.0f, alpha)); }

// ---- occlusion cut ----
// Eq. 2 composites a pixel front to back and stops at the first Gaussian that
// would take the transmittance below 1e-4. If the Gaussians of a tile's depth bins
// 0..b are certain to drive every pixel of the tile below that level, no pixel
// reaches bin b + 1, and the tile's list can end after bin b without changing any
// output or gradient. The certainty comes from Gaussians that cover the whole tile:
// for such a Gaussian the alpha of every pixel is at least alpha_min (below), so
// every pixel's transmittance after bins 0..b is at most exp(-sum of -ln(1 -
// alpha_min)). Each covered (Gaussian, tile) pair adds its optical depth -ln(1 -
// alpha_min), rounded down in fixed point, to its (tile, depth bin) bucket; the cut
// is the first bin at which the tile's running sum reaches ln(1e4) plus a margin.
constexpr float kOcclScale = 65536.0f;  // fixed-point units per nat
constexpr unsigned kHintSlack = 4;      // depth bins (a quarter octave) beyond a cut hint
// Pairs whose alpha bound is below this add nothing: leaving out part of the sum can
// only move a cut later, and on scenes of large Gaussians these faint tile covers are
// most of the pairs but little of the optical depth.
constexpr float kOcclAlpha = 0.05f;
constexpr float kOcclLog2Alpha = -4.3219280948873623f;  // log2(0.05)
// ln(1e4) + 1e-3 in units: exp(-(ln(1e4) + 1e-3)) is below the FP32 constant 1e-4f
constexpr unsigned kOcclThreshold = 603675u;

struct OcclGauss {
    float u, v, a, b;      // centre and scaled conic as staged by the blend (see stage_record)
    float c, thr, lo2, w;  // w > 0: the ellipse can hold a whole tile
};

// Optical depth lower bound of one Gaussian over the pixel centres [x0, x1] x [y0, y1]
// of a tile, in fixed-point units (0 if some pixel may cut or skip it). The blend
// computes p = a dx^2 + b dx dy + c dy^2 in FP32; in exact arithmetic p is concave
// (the conic is positive definite), so over the rectangle its minimum is at a corner.
// The FP32 error of the blend's evaluation at any pixel and of the evaluation here
// at the corners is below 20 ulp of M = |a| dx^2 + |b dx dy| + |c| dy^2 taken at the
// farthest extents; p is lowered by M 2^-18. The exponent l of alpha = 2^l is lowered
// by 1e-5 and alpha (ex2.approx, relative error below 2^-22) by a factor 1 - 1e-5;
// -log2(1 - alpha) (lg2.approx:
// absolute error below 2^-22 on [0.5, 2], 2 ulp elsewhere; the rounding of 1 - alpha
// moves it by less than 1e-5 for alpha <= 0.99) is lowered by 2e-5 and a factor
// 1 - 1e-5. The rounding of each transmittance product (a factor of at most
// (1 + 2^-24)^2 per blended Gaussian) is covered by one unit taken off each pair.
// Tile columns of [tx0, tx1] whose pixel centres, on both edge rows py0 and py1 of
// a tile row, lie where p >= T (a filter for occl_units, widened by a pixel: a tile
// is inside the convex region exactly when its four corners are).
__device__ __forceinline__ int2 strong_span(const OcclGauss &g, float T, int py0, int py1, int tx0, int tx1, int tw,
                                            int w) {
    float lo = -3.0e38f, hi = 3.0e38f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float dy = (float)(k ? py1 : py0) - g.v;
        const float B = g.b * dy, C = g.c * dy * dy - T;
        const float disc = B * B - 4.0f * g.a * C;  // a < 0: p >= T between the roots
        if (!(disc >= 0.f)) return make_int2(1, 0);
        const float sq = sqrtf(disc), i2a = 0.5f / g.a;
        const float r1 = (sq - B) * i2a, r2 = (-sq - B) * i2a;
        lo = fmaxf(lo, g.u + fminf(r1, r2));
        hi = fminf(hi, g.u + fmaxf(r1, r2));
    }
    lo -= 1.0f;
    hi += 1.0f;
    if (!(hi >= lo)) return make_int2(1, 0);
    const float ftw = (float)tw;
    const int first = max(tx0, (int)ceilf(fmaxf(lo, -1.0f) / ftw));
    const int last = hi >= (float)(w - 1) ? tx1 : min(tx1, (int)floorf((hi - (float)(tw - 1)) / ftw));
    return make_int2(first, last);
}

__device__ __forceinline__ unsigned occl_units(const OcclGauss &g, float x0, float x1, float y0, float y1) {
    const float dx0 = __fsub_rn(x0, g.u), dx1 = __fsub_rn(x1, g.u);
    const float dy0 = __fsub_rn(y0, g.v), dy1 = __fsub_rn(y1, g.v);
    const float ax0 = g.a * dx0 * dx0, ax1 = g.a * dx1 * dx1;
    const float cy0 = g.c * dy0 * dy0, cy1 = g.c * dy1 * dy1;
    const float bx0 = g.b * dx0, bx1 = g.b * dx1;
    const float pmin = fminf(fminf(fmaf(bx0, dy0, ax0 + cy0), fmaf(bx1, dy0, ax1 + cy0)),
                             fminf(fmaf(bx0, dy1, ax0 + cy1), fmaf(bx1, dy1, ax1 + cy1)));
    const float mx = fmaxf(fabsf(dx0), fabsf(dx1)), my = fmaxf(fabsf(dy0), fabsf(dy1));
    const float M = fabsf(g.a) * mx * mx + fabsf(g.b) * mx * my + fabsf(g.c) * my * my;
    const float plo = pmin - M * 3.814697265625e-6f - 1e-6f;  // 2^-18
    if (!(plo >= g.thr)) return 0u;
    const float l = plo + g.lo2 - 1e-5f;
    const float alpha = (l >= kClampL ? kAlphaMax : fast_exp2(l)) * (1.0f - 1e-5f);
    if (alpha < kOcclAlpha) return 0u;
    const float od2 = (-__log2f(1.0f - alpha) - 2e-5f) * (1.0f - 1e-5f);  // log2 units
    const float q = od2 * (kLn2 * kOcclScale);
    if (!(q >= 2.0f)) return 0u;
    return (unsigned)q - 1u;  // truncation rounds down
    return q > 0u ? q - 1u : 0u;
}

// ---- dynamic shared memory above the default limit ----
// A kernel needs cudaFuncAttributeMaxDynamicSharedMemorySize raised, per device, before
// it is launched with more than 48 KB of dynamic shared memory. Each launcher keeps one
// SmemOptIn per kernel; the attribute is raised only when a larger size than before is
// first needed on the current device, so steady-state calls (and stream capture) issue
// nothing but the launch.
struct SmemOptIn {
    std::mutex mu;
    size_t bytes[64] = {};
};

template <class K>
cudaError_t opt_in_smem(K kernel, size_t bytes, SmemOptIn &st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(st.mu);
    if (st.bytes[dev] >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) st.bytes[dev] = bytes;
    return e;
}

// ---- launch wrappers (one per translation unit) ----
struct ProjectArgs {
    const float *means, *log_scales, *quats, *opacity_logits, *colors;
    long long n;
    int sh_degree;
    float near_z;
    float guard;  // guard-cone slope; <= 0: no cone
    const float *Tdev;
    Record *rec;
    int2 *ext;
    unsigned *vis_mask;  // [n]: bit v set if the Gaussian is projected into view v
    unsigned *tile_count;
    unsigned *occl;      // per bucket optical depth lower bound (see occl_units); null: no cut
    int tile_fit;        // (min(tile_w, tile_h) - 1)^2 / 4: squared inradius a tile needs
    // Hints: the previous forward's cut per tile and its largest value per view (all 255
    // when there is none). Pairs behind the hint add no optical depth. Whatever the hint,
    // the sums of the bins up to it are complete, so a tile whose sum reaches the threshold
    // there gets the same cut as without a hint, and one whose sum does not keeps its
    // whole list (the cut search then finds no bin): the hint can only lose culling.
    const unsigned char *cut_hint;
    const unsigned *view_hint;
    // (pairs up to kHintSlack bins behind the hint still add, so that a cut that moves
    // back a little between two forwards is still found)
};
cudaError_t launch_project(const ProjectArgs &a, const ViewBatch &vb, cudaStream_t s);

// Per tile: the last depth bin its list keeps (255: all); per tile row and per view
// the largest of these.
struct CutArgs {
    const unsigned *occl;
    unsigned char *cut;
    unsigned *row_max;   // [tiles], at each row's first tile; zeroed before
    unsigned *view_max;  // [views]; zeroed before
    long long n_tiles;
};
cudaError_t launch_cut(const CutArgs &a, const ViewBatch &vb, cudaStream_t s);

struct ScanArgs {
    const unsigned *tile_count;  // per bucket
    unsigned *tile_start;  // [buckets + 1]
    unsigned *cursor;      // [buckets]
    unsigned *partials;    // [ceil(buckets / 4096) + 1]
    DevCounters *ctr;
    long long n_tiles;     // number of buckets (tiles * kDepthBins)
    unsigned long long key_capacity;
};
cudaError_t launch_scan(const ScanArgs &a, cudaStream_t s);

struct EmitArgs {
    const Record *rec;
    const int2 *ext;
    long long n;
    unsigned *cursor;
    unsigned long long *keys;
    unsigned long long key_capacity;
    const DevCounters *ctr;
    const unsigned char *cut;  // per tile last kept depth bin; null: keep all
    const unsigned *row_max, *view_max;  // the cut's maxima (see CutArgs)
    unsigned *tile_count;      // the count mode's bucket counts
};
cudaError_t launch_emit(const EmitArgs &a, const ViewBatch &vb, cudaStream_t s);
// The same enumeration counting the pairs in front of their tile's cut (a.cut set).
cudaError_t launch_count(const EmitArgs &a, const ViewBatch &vb, cudaStream_t s);

struct SortArgs {
    const unsigned *tile_start;  // bucket starts
    const unsigned long long *keys_in;  // keys in emission order (bucketed by tile and depth bin)
    unsigned long long *keys;           // the same keys sorted within each tile
    long long n_tiles;
    const DevCounters *ctr;
};
cudaError_t launch_tile_sort(const SortArgs &a, cudaStream_t s);

struct OrderArgs {
    const unsigned *tile_start;  // bucket starts
    unsigned *order;       // [T] tiles, heaviest first (approximate, by log2 bucket)
    unsigned *bucket_cnt;  // [33] scratch
    long long n_tiles;
};
cudaError_t launch_tile_order(const OrderArgs &a, cudaStream_t s);

struct BlendArgs {
    const Record *rec;
    const unsigned long long *keys;
    const unsigned *tile_start;  // bucket starts: tile t spans buckets [t * 256, (t + 1) * 256)
    const unsigned *order;  // may be NULL: natural tile order
    long long n;
    float bg[3];
    // forward outputs
    float *rgb, *depth, *pointmap, *alpha;
    float *T_final;     // per-pixel state (NULL in recompute mode)
    unsigned *n_last;   // per-pixel state (NULL in recompute mode)
    // backward inputs / outputs
    const float *d_rgb, *d_depth, *d_pointmap, *d_alpha;
    float *grad2d;      // [records][10] atomic accumulation
    float *det_partial; // [K][10] deterministic mode, else NULL
    DevCounters *ctr;
    int persistent;     // 0: one CTA per tile
    int batch;
    int ppt;            // pixels per thread (1, 2 or 4)
    int counting;
    int geom_only;      // backward: only the geometry slots (u, v, conic, z) are needed
    // backward with the L1 mapping loss fused in (l1 != 0): the upstream gradients
    // are formed per pixel from the forward's outputs and the targets instead of
    // being read, and the loss of each tile goes to loss_partial[tile]
    int l1;
    const float *o_rgb, *o_depth, *o_pointmap;  // the forward's outputs
    const float *t_rgb, *t_depth, *t_pointmap, *mask;
    float kr, kd, kg;                           // w_rgb / (3 P), w_depth / P, w_geo / (3 P)
    float *loss_partial;                        // [total tiles]: the loss of each tile
};
cudaError_t launch_blend_fwd(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s);
cudaError_t launch_blend_bwd(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s);

struct DetReduceArgs {
    const Record *rec;
    const int2 *ext;
    const unsigned long long *keys;
    const unsigned *tile_start;
    const float *det_partial;
    float *grad2d;
    long long n;
    const unsigned char *cut;  // per tile last kept depth bin; null: keep all
};
cudaError_t launch_det_reduce(const DetReduceArgs &a, const ViewBatch &vb, cudaStream_t s);

struct ProjectBwdArgs {
    const float *means, *log_scales, *quats, *opacity_logits, *colors;
    long long n;
    int sh_degree;
    const float *Tdev;
    const unsigned *vis_mask;
    float *grad2d;  // read, then cleared to zero for the next backward
    float *d_means, *d_log_scales, *d_quats, *d_opacity_logits, *d_colors;
    int accumulate;
    float *twist_partial;  // [gridDim.x][n_views][6]
};
cudaError_t launch_project_bwd(const ProjectBwdArgs &a, const ViewBatch &vb, int *grid_out,
                               cudaStream_t s);
int project_bwd_grid(long long n);

struct TwistReduceArgs {
    const float *twist_partial;
    int n_parts;
    int n_views;
    float *d_twist;
    int accumulate;
};
cudaError_t launch_twist_reduce(const TwistReduceArgs &a, cudaStream_t s);

struct LossArgs {
    const float *rgb, *depth, *pointmap, *t_rgb, *t_depth, *t_pointmap, *mask;
    float w_rgb, w_depth, w_geo;
    float *d_rgb, *d_depth, *d_pointmap;
    float *partial;  // [loss_blocks_per_view() * n_views]
    float *loss;
};
int loss_blocks_per_view();
cudaError_t launch_loss(const LossArgs &a, const ViewBatch &vb, cudaStream_t s);
// Fixed-order sum of n loss partials into *loss (one block).
cudaError_t launch_loss_final(const float *partial, int n, float *loss, cudaStream_t s);

// Context access for entry points defined outside api.cu: record an error
// message on the context and return the status; the context's device.
s3gs_status ctx_error(s3gs_ctx *ctx, s3gs_status st, const char *msg);
int ctx_device(const s3gs_ctx *ctx);

// Pairwise visible-set intersection counts of V views from the per-Gaussian
// view bitmask (counts [V][V], zeroed here), and IOU / OC when non-NULL.
cudaError_t launch_covis(const unsigned *vis, long long n, int V, unsigned long long *counts, float *iou, float *oc,
                         int num_sms, cudaStream_t s);

}  // namespace s3gs
