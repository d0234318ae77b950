// Per-tile front-to-back compositing (Sec. 3.1 Eq. 2, Sec. 3.2.1 Eq. 3-5) and its
// back-to-front backward (Sec. 3.2.2, Eq. 11).
//
// One CTA owns one tile; each thread owns P pixels of it (the same column, P
// adjacent rows), so that staged-Gaussian loads, loop control and - in the
// backward - the warp reduction of the per-Gaussian gradient are shared by P
// pixels. Projected Gaussians of the tile's depth-sorted list are staged in
// shared memory in batches; a batch load is skipped once every pixel of the
// tile has stopped (block-wide vote). With a persistent grid the CTAs pull
// tiles, heaviest first, from a work counter, which removes the tail of
// heavy-tailed tile loads.
#include "s3gs_internal.cuh"

namespace s3gs {
namespace {

// Pixel p of a thread: one column, P adjacent rows. Where the tile allows it (TW a
// multiple of 8 and TH / P a multiple of 4) each warp covers a compact block of
// 8 columns x 4P rows (lane & 7 the column, lane >> 3 the row group), so that fewer
// warps meet each Gaussian than with bands of full tile rows: fewer warps evaluate
// pairs outside the ellipse and fewer reduce a Gaussian's gradient in the backward.
// Otherwise thread t takes column t % TW and rows (t / TW) P + p.
template <int TW, int TH, int P>
struct TileCoord {
    int v;
    int i, j[P];
    bool inside[P];
    long long pix[P];  // packed pixel index within view v
    int HW;
};

template <int TW, int TH, int P>
__device__ __forceinline__ TileCoord<TW, TH, P> tile_coord(const ViewBatch &vb, int t) {
    static_assert(TH % P == 0 && (TW * TH / P) % 32 == 0, "tile rows must split evenly into whole warps");
    TileCoord<TW, TH, P> c;
    c.v = view_of_tile(vb, t);
    const ViewInfo &vi = vb.v[c.v];
    const int tl = t - vi.tile_base;
    const int ty = tl / vi.tiles_x, tx = tl - ty * vi.tiles_x;
    constexpr bool kBlocks = TW % 8 == 0 && (TH / P) % 4 == 0;
    int col, trow;
    if (kBlocks) {
        constexpr int WX = TW / 8;  // warps across the tile
        const int lane = (int)(threadIdx.x & 31u), w = (int)(threadIdx.x >> 5);
        col = (w % WX) * 8 + (lane & 7);
        trow = (w / WX) * 4 + (lane >> 3);
    } else {
        col = (int)(threadIdx.x % TW);
        trow = (int)(threadIdx.x / TW);
    }
    c.i = tx * TW + col;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        c.j[p] = ty * TH + trow * P + p;
        c.inside[p] = c.i < vi.w && c.j[p] < vi.h;
        c.pix[p] = (long long)c.j[p] * vi.w + c.i;
    }
    c.HW = vi.w * vi.h;
    return c;
}

// Next tile for this CTA (uniform across the block), or -1 when done.
__device__ __forceinline__ int next_tile(const BlendArgs &a, const ViewBatch &vb, unsigned *counter, int iter,
                                         int *s_tile) {
    if (!a.persistent) return iter == 0 ? (int)blockIdx.x : -1;
    __syncthreads();
    if (threadIdx.x == 0) *s_tile = (int)atomicAdd(counter, 1u);
    __syncthreads();
    int w = *s_tile;
    if (w >= vb.total_tiles) return -1;
    return a.order ? (int)a.order[w] : w;
}

// Stage list entries [b, b + cnt) of a tile into shared memory.
__device__ __forceinline__ void stage(const BlendArgs &a, long long rbase, unsigned b, unsigned cnt, float4 *s_p0,
                                      float4 *s_p1, float4 *s_col, unsigned *s_g) {
    for (unsigned k = threadIdx.x; k < cnt; k += blockDim.x) {
        const unsigned g = (unsigned)a.keys[b + k];
        const Record r = a.rec[rbase + g];
        const StagedGauss sg = stage_record(r);
        s_p0[k] = make_float4(sg.u, sg.v, sg.a, sg.b);
        s_p1[k] = make_float4(sg.c, sg.lo2, sg.thr, sg.z);
        if (s_col) s_col[k] = r.c;
        if (s_g) s_g[k] = g;
    }
}

// Warp sum of 10 per-lane values as a reduce-scatter: each butterfly level
// halves the number of values a lane carries (10 -> 5 -> 3 -> 2 -> 1 -> 1), so
// the whole reduction takes 12 shuffles instead of 50. Afterwards the even
// lanes (lane & 1 == 0) whose code below is >= 0 own one distinct slot each;
// the return value is that slot (or -1) and *sum its warp total.
__device__ __forceinline__ int warp_reduce_scatter10(const float v[kGrad2d], float *sum) {
    const unsigned lane = threadIdx.x & 31u;
    const bool b4 = lane & 16u, b3 = lane & 8u, b2 = lane & 4u, b1 = lane & 2u;
    float a5[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float send = b4 ? v[i] : v[i + 5];
        const float keep = b4 ? v[i + 5] : v[i];
        a5[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float c3[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float hi = j < 2 ? a5[3 + j] : 0.f;
        const float send = b3 ? a5[j] : hi;
        const float keep = b3 ? hi : a5[j];
        c3[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float d2[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float hi = j == 0 ? c3[2] : 0.f;
        const float send = b2 ? c3[j] : hi;
        const float keep = b2 ? hi : c3[j];
        d2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    float e = (b1 ? d2[1] : d2[0]) + __shfl_xor_sync(0xffffffffu, b1 ? d2[0] : d2[1], 2);
    e += __shfl_xor_sync(0xffffffffu, e, 1);
    *sum = e;
    int slot;
    if (!b3) slot = b2 ? (b1 ? -1 : 2) : (b1 ? 1 : 0);
    else slot = b2 ? -1 : (b1 ? 4 : 3);
    if ((lane & 1u) || slot < 0) return -1;
    return slot + (b4 ? 5 : 0);
}

// The same for the six geometry slots (the moments X, Y, XX, XY, YY and z) of a geometry-only
// backward: 3 + 2 + 1 shuffles halve the lanes' values, two more finish the sums;
// lanes with lane & 3 == 0 own one slot each (compact index 0..5, or -1).
__device__ __forceinline__ int warp_reduce_scatter6(const float v[6], float *sum) {
    const unsigned lane = threadIdx.x & 31u;
    const bool b4 = lane & 16u, b3 = lane & 8u, b2 = lane & 4u;
    float a3[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float send = b4 ? v[i] : v[i + 3];
        const float keep = b4 ? v[i + 3] : v[i];
        a3[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float c2[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float hi = j == 0 ? a3[2] : 0.f;
        const float send = b3 ? a3[j] : hi;
        const float keep = b3 ? hi : a3[j];
        c2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float e = (b2 ? c2[1] : c2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? c2[0] : c2[1], 4);
    e += __shfl_xor_sync(0xffffffffu, e, 2);
    e += __shfl_xor_sync(0xffffffffu, e, 1);
    *sum = e;
    const int slot = b3 ? (b2 ? -1 : 2) : (b2 ? 1 : 0);
    if ((lane & 3u) || slot < 0) return -1;
    return slot + (b4 ? 3 : 0);
}

template <int TW, int TH, int P, bool COUNT>
__global__ void __launch_bounds__(TW *TH / P) blend_fwd_kernel(const BlendArgs a, const __grid_constant__ ViewBatch vb) {
    constexpr int NT = TW * TH / P;
    extern __shared__ float4 smem[];
    __shared__ int s_tile;
    const unsigned B = (unsigned)a.batch;
    float4 *s_p0 = smem;
    float4 *s_p1 = smem + B;
    float4 *s_col = smem + 2 * B;
    if (a.ctr->overflow) return;
    unsigned long long n_proc = 0, n_blend = 0;
    for (int iter = 0;; ++iter) {
        const int t = next_tile(a, vb, &a.ctr->work_fwd, iter, &s_tile);
        if (t < 0) break;
        const TileCoord<TW, TH, P> c = tile_coord<TW, TH, P>(vb, t);
        const ViewInfo &vi = vb.v[c.v];
        const long long rbase = (long long)c.v * a.n;
        const float px = (float)c.i;
        const unsigned s = a.tile_start[t * kDepthBins], e = a.tile_start[(t + 1) * kDepthBins];
        float T[P], C0[P], C1[P], C2[P], D[P], py[P];
        unsigned last[P];
        bool done[P];
        bool all_done = true;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            T[p] = 1.f; C0[p] = C1[p] = C2[p] = D[p] = 0.f; last[p] = 0;
            py[p] = (float)c.j[p];
            done[p] = !c.inside[p];
            all_done = all_done && done[p];
        }
        for (unsigned b = s; b < e; b += B) {
            if (__syncthreads_count(all_done) == NT) break;
            const unsigned cnt = min(B, e - b);
            stage(a, rbase, b, cnt, s_p0, s_p1, s_col, nullptr);
            __syncthreads();
            for (unsigned k = 0; k < cnt && !all_done; ++k) {
                const float4 p0 = s_p0[k], p1 = s_p1[k], col = s_col[k];
                const unsigned idx = b - s + k + 1;
                if constexpr (P % 2 == 0) {
                    // the quadratic form of two pixels of the column at once (packed FP32,
                    // each lane rounding as eval_pair does); the rest per pixel
                    const ColTerms ct = col_terms(px, p0.x, p0.z, p0.w);
#pragma unroll
                    for (int h = 0; h < P / 2; ++h) {
                        if (done[2 * h] && done[2 * h + 1]) continue;
                        float2 dy, pp, ll;
                        eval_pair2(ct, make_float2(py[2 * h], py[2 * h + 1]), p0.y, p1.x, p1.y, dy, pp, ll);
#pragma unroll
                        for (int e2 = 0; e2 < 2; ++e2) {
                            const int p = 2 * h + e2;
                            if (done[p]) continue;
                            if (COUNT) ++n_proc;
                            const float pe = e2 ? pp.y : pp.x, le = e2 ? ll.y : ll.x;
                            if (!(pe >= p1.z)) continue;  // outside the 3-sigma ellipse or below 1/255
                            const float al = le >= kClampL ? kAlphaMax : fast_exp2(le);
                            const float Tn = next_T(T[p], al);
                            if (Tn < kTMin) {
                                done[p] = true;
                                continue;
                            }
                            const float w = al * T[p];
                            C0[p] = fmaf(col.x, w, C0[p]);
                            C1[p] = fmaf(col.y, w, C1[p]);
                            C2[p] = fmaf(col.z, w, C2[p]);
                            D[p] = fmaf(p1.w, w, D[p]);
                            T[p] = Tn;
                            last[p] = idx;
                            if (COUNT) ++n_blend;
                        }
                    }
                } else {
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        if (done[p]) continue;
                        const PairEval pe = eval_pair(px, py[p], p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z);
                        if (COUNT) ++n_proc;
                        if (!pe.pass) continue;
                        const float al = pair_alpha(pe);
                        const float Tn = next_T(T[p], al);
                        if (Tn < kTMin) {
                            done[p] = true;
                            continue;
                        }
                        const float w = al * T[p];
                        C0[p] = fmaf(col.x, w, C0[p]);
                        C1[p] = fmaf(col.y, w, C1[p]);
                        C2[p] = fmaf(col.z, w, C2[p]);
                        D[p] = fmaf(p1.w, w, D[p]);
                        T[p] = Tn;
                        last[p] = idx;
                        if (COUNT) ++n_blend;
                    }
                }
                all_done = true;
#pragma unroll
                for (int p = 0; p < P; ++p) all_done = all_done && done[p];
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (!c.inside[p]) continue;
            const long long q1 = vi.pix_base + c.pix[p];
            const long long q3 = 3 * vi.pix_base + c.pix[p];
            if (a.rgb) {
                a.rgb[q3] = C0[p] + T[p] * a.bg[0];
                a.rgb[q3 + c.HW] = C1[p] + T[p] * a.bg[1];
                a.rgb[q3 + 2 * c.HW] = C2[p] + T[p] * a.bg[2];
            }
            if (a.depth) a.depth[q1] = D[p];
            if (a.alpha) a.alpha[q1] = 1.f - T[p];
            if (a.pointmap) {
                // Eq. 5: X^r = ((i - cx) D / fx, (j - cy) D / fy, D)
                a.pointmap[q3] = (px - vi.cx) / vi.fx * D[p];
                a.pointmap[q3 + c.HW] = ((float)c.j[p] - vi.cy) / vi.fy * D[p];
                a.pointmap[q3 + 2 * c.HW] = D[p];
            }
            if (a.T_final) {
                a.T_final[q1] = T[p];
                a.n_last[q1] = last[p];
            }
        }
    }
    if (COUNT) {
        atomicAdd(&a.ctr->fwd_processed, n_proc);
        atomicAdd(&a.ctr->fwd_blended, n_blend);
    }
}

__device__ __forceinline__ float l1_sign(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

template <int TW, int TH, int P, bool RECOMPUTE, bool DET, bool COUNT, bool GEOM = false>
__global__ void __launch_bounds__(TW *TH / P) blend_bwd_kernel(const BlendArgs a, const __grid_constant__ ViewBatch vb) {
    constexpr int NT = TW * TH / P;
    constexpr int NW = NT / 32;
    extern __shared__ float4 smem[];
    __shared__ int s_tile;
    __shared__ unsigned s_maxlast;
    __shared__ float s_loss[NW];
    const unsigned B = (unsigned)a.batch;
    float4 *s_p0 = smem;
    float4 *s_p1 = smem + B;
    float4 *s_col = smem + 2 * B;
    unsigned *s_g = reinterpret_cast<unsigned *>(smem + 3 * B);
    float *s_part = reinterpret_cast<float *>(s_g + B);  // DET: [NW][B][10]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (a.ctr->overflow) return;
    unsigned long long n_proc = 0;
    float loss_acc = 0.f;  // fused L1 loss of this thread's pixels in the current tile
    for (int iter = 0;; ++iter) {
        const int t = next_tile(a, vb, &a.ctr->work_bwd, iter, &s_tile);
        if (t < 0) break;
        const TileCoord<TW, TH, P> c = tile_coord<TW, TH, P>(vb, t);
        const ViewInfo &vi = vb.v[c.v];
        const long long rbase = (long long)c.v * a.n;
        const float px = (float)c.i;
        const unsigned s = a.tile_start[t * kDepthBins], e = a.tile_start[(t + 1) * kDepthBins];

        // per-pixel blend state: stored by the forward, or replayed here
        float T[P], py[P];
        unsigned last[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            T[p] = 1.f;
            last[p] = 0;
            py[p] = (float)c.j[p];
        }
        if (RECOMPUTE) {
            bool done[P];
            bool all_done = true;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                done[p] = !c.inside[p];
                all_done = all_done && done[p];
            }
            for (unsigned b = s; b < e; b += B) {
                if (__syncthreads_count(all_done) == NT) break;
                const unsigned cnt = min(B, e - b);
                stage(a, rbase, b, cnt, s_p0, s_p1, nullptr, nullptr);
                __syncthreads();
                for (unsigned k = 0; k < cnt && !all_done; ++k) {
                    const float4 p0 = s_p0[k], q1 = s_p1[k];
                    const unsigned idx = b - s + k + 1;
                    if constexpr (P % 2 == 0) {
                        // the forward's evaluation (packed quadratic form, per-pixel decisions),
                        // T and the last index only
                        const ColTerms ct = col_terms(px, p0.x, p0.z, p0.w);
#pragma unroll
                        for (int h = 0; h < P / 2; ++h) {
                            if (done[2 * h] && done[2 * h + 1]) continue;
                            float2 dy, pp, ll;
                            eval_pair2(ct, make_float2(py[2 * h], py[2 * h + 1]), p0.y, q1.x, q1.y, dy, pp, ll);
#pragma unroll
                            for (int e2 = 0; e2 < 2; ++e2) {
                                const int p = 2 * h + e2;
                                if (done[p]) continue;
                                const float pe = e2 ? pp.y : pp.x, le = e2 ? ll.y : ll.x;
                                if (!(pe >= q1.z)) continue;
                                const float Tn = next_T(T[p], le >= kClampL ? kAlphaMax : fast_exp2(le));
                                if (Tn < kTMin) {
                                    done[p] = true;
                                    continue;
                                }
                                T[p] = Tn;
                                last[p] = idx;
                            }
                        }
                    } else {
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            if (done[p]) continue;
                            const PairEval pe = eval_pair(px, py[p], p0.x, p0.y, p0.z, p0.w, q1.x, q1.y, q1.z);
                            if (!pe.pass) continue;
                            const float Tn = next_T(T[p], pair_alpha(pe));
                            if (Tn < kTMin) {
                                done[p] = true;
                                continue;
                            }
                            T[p] = Tn;
                            last[p] = idx;
                        }
                    }
                    all_done = true;
#pragma unroll
                    for (int p = 0; p < P; ++p) all_done = all_done && done[p];
                }
            }
            __syncthreads();
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p)
                if (c.inside[p]) {
                    T[p] = a.T_final[vi.pix_base + c.pix[p]];
                    last[p] = a.n_last[vi.pix_base + c.pix[p]];
                }
        }

        // upstream gradients; the pointmap (Eq. 5) is linear in D
        float gC0[P], gC1[P], gC2[P], gD[P], Bacc[P];
        unsigned mylast = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            gC0[p] = gC1[p] = gC2[p] = gD[p] = 0.f;
            float gT = 0.f;
            if (c.inside[p] && a.l1) {
                // L1 mapping loss (Eq. 10/15/17) on this pixel: the same terms and the same
                // FP32 operations as the separate loss kernel, so the gradients match it
                const long long q1 = vi.pix_base + c.pix[p];
                const long long q3 = 3 * vi.pix_base + c.pix[p];
                const float m = a.mask ? a.mask[q1] : 1.f;
                const float cr = m * a.kr, cd = m * a.kd, cg = m * a.kg;
                float dpm[3] = {0.f, 0.f, 0.f};
                if (a.t_rgb) {
                    const float r0 = a.o_rgb[q3] - a.t_rgb[q3];
                    const float r1 = a.o_rgb[q3 + c.HW] - a.t_rgb[q3 + c.HW];
                    const float r2 = a.o_rgb[q3 + 2 * c.HW] - a.t_rgb[q3 + 2 * c.HW];
                    gC0[p] = cr * l1_sign(r0);
                    gC1[p] = cr * l1_sign(r1);
                    gC2[p] = cr * l1_sign(r2);
                    loss_acc += cr * fabsf(r0);
                    loss_acc += cr * fabsf(r1);
                    loss_acc += cr * fabsf(r2);
                }
                if (a.t_pointmap)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        const float r = a.o_pointmap[q3 + ch * c.HW] - a.t_pointmap[q3 + ch * c.HW];
                        dpm[ch] = cg * l1_sign(r);
                        loss_acc += cg * fabsf(r);
                    }
                if (a.t_depth) {
                    const float r = a.o_depth[q1] - a.t_depth[q1];
                    gD[p] = cd * l1_sign(r);
                    loss_acc += cd * fabsf(r);
                }
                if (a.t_pointmap)
                    gD[p] += (px - vi.cx) / vi.fx * dpm[0] + ((float)c.j[p] - vi.cy) / vi.fy * dpm[1] + dpm[2];
                gT = a.bg[0] * gC0[p] + a.bg[1] * gC1[p] + a.bg[2] * gC2[p];
            } else if (c.inside[p]) {
                const long long q1 = vi.pix_base + c.pix[p];
                const long long q3 = 3 * vi.pix_base + c.pix[p];
                if (a.d_rgb) {
                    gC0[p] = a.d_rgb[q3];
                    gC1[p] = a.d_rgb[q3 + c.HW];
                    gC2[p] = a.d_rgb[q3 + 2 * c.HW];
                }
                if (a.d_depth) gD[p] = a.d_depth[q1];
                if (a.d_pointmap) {
                    gD[p] += (px - vi.cx) / vi.fx * a.d_pointmap[q3] +
                             ((float)c.j[p] - vi.cy) / vi.fy * a.d_pointmap[q3 + c.HW] + a.d_pointmap[q3 + 2 * c.HW];
                }
                gT = a.bg[0] * gC0[p] + a.bg[1] * gC1[p] + a.bg[2] * gC2[p];
                if (a.d_alpha) gT -= a.d_alpha[q1];
            } else {
                last[p] = 0;
            }
            Bacc[p] = gT;  // gradient-weighted value of everything behind the current Gaussian
            mylast = max(mylast, last[p]);
        }

        if (threadIdx.x == 0) s_maxlast = 0;
        if (a.l1) {
            // this tile's loss: warps summed in a fixed order, one partial per tile, so
            // the loss does not depend on which CTA of a persistent grid took the tile
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
            if (lane == 0) s_loss[warp] = loss_acc;
            loss_acc = 0.f;
        }
        __syncthreads();
        if (mylast) atomicMax(&s_maxlast, mylast);
        if (a.l1 && threadIdx.x == 0) {
            float x = 0.f;
            for (int w = 0; w < NW; ++w) x += s_loss[w];
            a.loss_partial[t] = x;
        }
        __syncthreads();
        const unsigned maxlast = s_maxlast;
        const unsigned wmaxlast = __reduce_max_sync(0xffffffffu, mylast);  // this warp's last list entry
        if (DET) {
            // duplicates never reached by any pixel carry a zero partial
            for (unsigned k = s + maxlast + threadIdx.x; k < e; k += NT)
#pragma unroll
                for (int q = 0; q < kGrad2d; ++q) a.det_partial[(long long)k * kGrad2d + q] = 0.f;
        }

        for (unsigned bend = s + maxlast; bend > s;) {
            const unsigned bstart = (bend - s > B) ? bend - B : s;
            const unsigned cnt = bend - bstart;
            __syncthreads();
            stage(a, rbase, bstart, cnt, s_p0, s_p1, s_col, s_g);
            __syncthreads();
            for (int k = (int)cnt - 1; k >= 0; --k) {
                const unsigned pos = bstart - s + (unsigned)k;
                if (pos >= wmaxlast) {
                    // no pixel of this warp reaches the entry: its partial is zero
                    if (DET && lane < kGrad2d) s_part[((size_t)warp * B + k) * kGrad2d + lane] = 0.f;
                    continue;
                }
                float vals[kGrad2d];
#pragma unroll
                for (int q = 0; q < kGrad2d; ++q) vals[q] = 0.f;
                bool contrib = false;
                const float4 p0 = s_p0[k], q1 = s_p1[k];
                if constexpr (P % 2 == 0) {
                    // pixels in pairs of adjacent rows, branch-free in packed FP32: a pixel
                    // the Gaussian does not reach (beyond its last contributor, outside the
                    // cutoff or skipped) takes the arithmetic with alpha = 0, which leaves its
                    // T, its behind-value and every sum exactly unchanged; the quadratic form
                    // and the decisions round as the scalar path below does. The pair sums
                    // are per lane (even rows, odd rows) and added before the warp reduction.
                    // A thread's pixels share their column, hence dx: the moments carrying
                    // dx are sum g dx = dx S, sum g dx^2 = dx (dx S) and sum g dx dy = dx Y
                    // (S = sum g, Y = sum g dy), so per pair only S, Y and sum g dy^2 are
                    // accumulated.
                    const float4 col = s_col[k];
                    const ColTerms ct = col_terms(px, p0.x, p0.z, p0.w);
                    const float dx = ct.dx;
                    float2 v2[kGrad2d];
#pragma unroll
                    for (int q = 0; q < kGrad2d; ++q) v2[q] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int h = 0; h < P / 2; ++h) {
                        const int r0 = 2 * h, r1 = 2 * h + 1;
                        if (pos >= last[r0] && pos >= last[r1]) continue;
                        float2 dy, pp, ll;
                        eval_pair2(ct, make_float2(py[r0], py[r1]), p0.y, q1.x, q1.y, dy, pp, ll);
                        const bool c0 = pos < last[r0] && pp.x >= q1.z, c1 = pos < last[r1] && pp.y >= q1.z;
                        if (COUNT) n_proc += (unsigned long long)(pos < last[r0]) + (unsigned long long)(pos < last[r1]);
                        if (!(c0 || c1)) continue;  // neither pixel passes the cutoff and skip
                        contrib = true;
                        const bool k0 = ll.x >= kClampL, k1 = ll.y >= kClampL;
                        const float a0 = c0 ? (k0 ? kAlphaMax : fast_exp2(ll.x)) : 0.f;
                        const float a1 = c1 ? (k1 ? kAlphaMax : fast_exp2(ll.y)) : 0.f;
                        const float2 al = make_float2(a0, a1);
                        const float2 om = __fadd2_rn(bcast2(1.f), make_float2(-a0, -a1));
                        const float2 Tp = make_float2(T[r0], T[r1]);
                        // T in front of this Gaussian (alpha = 0: T / 1)
                        const float2 Tk = make_float2(c0 ? __fdividef(Tp.x, om.x) : Tp.x, c1 ? __fdividef(Tp.y, om.y) : Tp.y);
                        const float2 w = __fmul2_rn(al, Tk);
                        const float2 g0 = make_float2(gC0[r0], gC0[r1]), g1 = make_float2(gC1[r0], gC1[r1]);
                        const float2 g2 = make_float2(gC2[r0], gC2[r1]), gd = make_float2(gD[r0], gD[r1]);
                        const float2 f = __ffma2_rn(bcast2(col.x), g0, __ffma2_rn(bcast2(col.y), g1,
                                                    __ffma2_rn(bcast2(col.z), g2, __fmul2_rn(bcast2(q1.w), gd))));
                        const float2 Bp = make_float2(Bacc[r0], Bacc[r1]);
                        const float2 fb = __fadd2_rn(f, make_float2(-Bp.x, -Bp.y));  // f - B
                        const float2 da = __fmul2_rn(Tk, fb);
                        // the value behind the next Gaussian: alpha f + (1 - alpha) B = B + alpha (f - B)
                        const float2 Bn = __ffma2_rn(al, fb, Bp);
                        Bacc[r0] = Bn.x; Bacc[r1] = Bn.y;
                        T[r0] = Tk.x; T[r1] = Tk.y;
                        if (!GEOM) {
                            v2[kGR] = __ffma2_rn(w, g0, v2[kGR]);
                            v2[kGG] = __ffma2_rn(w, g1, v2[kGG]);
                            v2[kGBl] = __ffma2_rn(w, g2, v2[kGBl]);
                        }
                        v2[kGZ] = __ffma2_rn(w, gd, v2[kGZ]);
                        // g = dL/dalpha * alpha (zero where alpha is clamped): S, Y, sum g dy^2
                        const float2 g = __fmul2_rn(da, make_float2(k0 ? 0.f : a0, k1 ? 0.f : a1));
                        const float2 gy = __fmul2_rn(g, dy);
                        v2[kGO] = __fadd2_rn(v2[kGO], g);
                        v2[kGV] = __fadd2_rn(v2[kGV], gy);
                        v2[kGC] = __ffma2_rn(gy, dy, v2[kGC]);
                    }
                    const float S = __fadd_rn(v2[kGO].x, v2[kGO].y);
                    const float Y = __fadd_rn(v2[kGV].x, v2[kGV].y);
                    if (!GEOM) {
                        vals[kGR] = __fadd_rn(v2[kGR].x, v2[kGR].y);
                        vals[kGG] = __fadd_rn(v2[kGG].x, v2[kGG].y);
                        vals[kGBl] = __fadd_rn(v2[kGBl].x, v2[kGBl].y);
                        vals[kGO] = S;
                    }
                    vals[kGZ] = __fadd_rn(v2[kGZ].x, v2[kGZ].y);
                    vals[kGC] = __fadd_rn(v2[kGC].x, v2[kGC].y);
                    vals[kGV] = Y;
                    vals[kGU] = __fmul_rn(dx, S);
                    vals[kGA] = __fmul_rn(dx, vals[kGU]);
                    vals[kGB] = __fmul_rn(dx, Y);
                } else {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if (pos >= last[p]) continue;
                    const PairEval pe = eval_pair(px, py[p], p0.x, p0.y, p0.z, p0.w, q1.x, q1.y, q1.z);
                    if (COUNT) ++n_proc;
                    if (!pe.pass) continue;
                    contrib = true;
                    // Gradient terms of one pair, with explicit rounding so that every
                    // instantiation (stored or recomputed state, any schedule) computes
                    // the same bits and deterministic mode is reproducible across them.
                    const float al = pair_alpha(pe);
                    const float om = __fsub_rn(1.f, al);
                    const float Tk = __fdividef(T[p], om);  // T in front of this Gaussian
                    const float w = __fmul_rn(al, Tk);
                    const float4 col = s_col[k];
                    const float f = __fmaf_rn(col.x, gC0[p], __fmaf_rn(col.y, gC1[p],
                                              __fmaf_rn(col.z, gC2[p], __fmul_rn(q1.w, gD[p]))));
                    const float da = __fmul_rn(Tk, __fsub_rn(f, Bacc[p]));
                    Bacc[p] = __fmaf_rn(f, al, __fmul_rn(om, Bacc[p]));
                    T[p] = Tk;
                    if (!GEOM) {
                        vals[kGR] = __fmaf_rn(w, gC0[p], vals[kGR]);
                        vals[kGG] = __fmaf_rn(w, gC1[p], vals[kGG]);
                        vals[kGBl] = __fmaf_rn(w, gC2[p], vals[kGBl]);
                    }
                    vals[kGZ] = __fmaf_rn(w, gD[p], vals[kGZ]);
                    if (!pe.clamped) {
                        // alpha = o exp(-q/2), q = A dx^2 + 2 B dx dy + C dy^2, dx = i - u: with
                        // g = dL/dalpha * alpha, the pair adds g (A dx + B dy) to dL/du,
                        // g (B dx + C dy) to dL/dv, -g dx^2 / 2, -g dx dy, -g dy^2 / 2 to dL/d(A, B, C)
                        // and g (1 - o) to dL/dlogit. The conic and o are fixed per Gaussian, so
                        // only the moments of g are summed here (slot order of the record's
                        // gradient row: X, Y, XX, XY, YY, S with X = sum g dx, XY = sum g dx dy,
                        // S = sum g); the projection backward applies the per-Gaussian factors.
                        const float g = __fmul_rn(da, al);
                        const float gx = __fmul_rn(g, pe.dx);
                        const float gy = __fmul_rn(g, pe.dy);
                        if (!GEOM) vals[kGO] = __fadd_rn(vals[kGO], g);
                        vals[kGA] = __fmaf_rn(gx, pe.dx, vals[kGA]);
                        vals[kGB] = __fmaf_rn(gx, pe.dy, vals[kGB]);
                        vals[kGC] = __fmaf_rn(gy, pe.dy, vals[kGC]);
                        vals[kGU] = __fadd_rn(vals[kGU], gx);
                        vals[kGV] = __fadd_rn(vals[kGV], gy);
                    }
                }
                }
                if (DET) {
                    float sum;
                    const int slot = warp_reduce_scatter10(vals, &sum);
                    if (slot >= 0) s_part[((size_t)warp * B + k) * kGrad2d + slot] = sum;
                } else if (GEOM) {
                    if (__any_sync(0xffffffffu, contrib)) {
                        const float gv[6] = {vals[kGU], vals[kGV], vals[kGA], vals[kGB], vals[kGC], vals[kGZ]};
                        float sum;
                        const int c = warp_reduce_scatter6(gv, &sum);
                        if (c >= 0) atomicAdd(a.grad2d + (rbase + s_g[k]) * kGrad2d + (c == 5 ? kGZ : c), sum);
                    }
                } else if (__any_sync(0xffffffffu, contrib)) {
                    float sum;
                    const int slot = warp_reduce_scatter10(vals, &sum);
                    if (slot >= 0) atomicAdd(a.grad2d + (rbase + s_g[k]) * kGrad2d + slot, sum);
                }
            }
            if (DET) {
                __syncthreads();
                // per-duplicate partial: warps summed in a fixed order
                for (unsigned idx = threadIdx.x; idx < cnt * kGrad2d; idx += NT) {
                    const unsigned k = idx / kGrad2d, q = idx % kGrad2d;
                    float x = 0.f;
#pragma unroll
                    for (int wv = 0; wv < NW; ++wv) x += s_part[((size_t)wv * B + k) * kGrad2d + q];
                    a.det_partial[(long long)(bstart + k) * kGrad2d + q] = x;
                }
            }
            bend = bstart;
        }
    }
    if (COUNT) atomicAdd(&a.ctr->bwd_processed, n_proc);
}

size_t fwd_smem(int batch) { return (size_t)batch * (3 * sizeof(float4)); }

size_t bwd_smem(int batch, int n_warps, bool det) {
    size_t s = (size_t)batch * (3 * sizeof(float4) + sizeof(unsigned));
    if (det) s += (size_t)n_warps * batch * kGrad2d * sizeof(float);
    return s;
}

template <int TW, int TH, int P, bool C>
cudaError_t fwd_impl3(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    static SmemOptIn st;
    const size_t sm = fwd_smem(a.batch);
    auto k = blend_fwd_kernel<TW, TH, P, C>;
    cudaError_t e = opt_in_smem(k, sm, st);
    if (e != cudaSuccess) return e;
    k<<<grid, TW * TH / P, sm, s>>>(a, vb);
    return cudaGetLastError();
}

template <int TW, int TH, int P>
cudaError_t fwd_impl2(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    return a.counting ? fwd_impl3<TW, TH, P, true>(a, vb, grid, s) : fwd_impl3<TW, TH, P, false>(a, vb, grid, s);
}

template <int TW, int TH, int P, bool R, bool D, bool C, bool G = false>
cudaError_t bwd_impl4(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    static SmemOptIn st;
    const size_t sm = bwd_smem(a.batch, TW * TH / P / 32, D);
    auto k = blend_bwd_kernel<TW, TH, P, R, D, C, G>;
    cudaError_t e = opt_in_smem(k, sm, st);
    if (e != cudaSuccess) return e;
    k<<<grid, TW * TH / P, sm, s>>>(a, vb);
    return cudaGetLastError();
}

template <int TW, int TH, int P, bool R, bool D>
cudaError_t bwd_impl3(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    if (a.counting) return bwd_impl4<TW, TH, P, R, D, true>(a, vb, grid, s);
    if constexpr (!D)
        if (a.geom_only) return bwd_impl4<TW, TH, P, R, D, false, true>(a, vb, grid, s);
    return bwd_impl4<TW, TH, P, R, D, false>(a, vb, grid, s);
}

template <int TW, int TH, int P>
cudaError_t bwd_impl2(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    const bool R = a.T_final == nullptr, D = a.det_partial != nullptr;
    if (R && D) return bwd_impl3<TW, TH, P, true, true>(a, vb, grid, s);
    if (R) return bwd_impl3<TW, TH, P, true, false>(a, vb, grid, s);
    if (D) return bwd_impl3<TW, TH, P, false, true>(a, vb, grid, s);
    return bwd_impl3<TW, TH, P, false, false>(a, vb, grid, s);
}

// Tile shape x pixels per thread, for the forward (F = true) or the backward.
template <bool F, int TW, int TH>
cudaError_t by_ppt(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    switch (a.ppt) {
    case 1: return F ? fwd_impl2<TW, TH, 1>(a, vb, grid, s) : bwd_impl2<TW, TH, 1>(a, vb, grid, s);
    case 2: return F ? fwd_impl2<TW, TH, 2>(a, vb, grid, s) : bwd_impl2<TW, TH, 2>(a, vb, grid, s);
    case 4:
        if constexpr ((TW * TH / 4) % 32 == 0)
            return F ? fwd_impl2<TW, TH, 4>(a, vb, grid, s) : bwd_impl2<TW, TH, 4>(a, vb, grid, s);
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <bool F>
cudaError_t dispatch(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    const int tw = vb.tile_w, th = vb.tile_h;
    if (tw == 16 && th == 16) return by_ppt<F, 16, 16>(a, vb, grid, s);
    if (tw == 16 && th == 8) return by_ppt<F, 16, 8>(a, vb, grid, s);
    if (tw == 8 && th == 8) return by_ppt<F, 8, 8>(a, vb, grid, s);
    if (tw == 32 && th == 8) return by_ppt<F, 32, 8>(a, vb, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_blend_fwd(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    return dispatch<true>(a, vb, grid, s);
}

cudaError_t launch_blend_bwd(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    return dispatch<false>(a, vb, grid, s);
}

}  // namespace s3gs
