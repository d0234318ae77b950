// Per-tile front-to-back compositing (Sec. 3.1 Eq. 2, Sec. 3.2.1 Eq. 3-5) and its
// back-to-front backward (Sec. 3.2.2, Eq. 11).
//
// One CTA owns one tile (one thread per pixel). Projected Gaussians of the
// tile's depth-sorted list are staged in shared memory in batches; a batch
// load is skipped once every pixel of the tile has stopped (block-wide vote).
// With a persistent grid the CTAs pull tiles, heaviest first, from a work
// counter, which removes the tail of heavy-tailed tile loads.
#include "s3gs_internal.cuh"

namespace s3gs {
namespace {

struct TileCoord {
    int v;
    int i, j;
    bool inside;
    long long pix;  // packed pixel index of (i, j) within view v
    int HW;
};

template <int TW, int TH>
__device__ __forceinline__ TileCoord tile_coord(const ViewBatch &vb, int t) {
    TileCoord c;
    c.v = view_of_tile(vb, t);
    const ViewInfo &vi = vb.v[c.v];
    int tl = t - vi.tile_base;
    int ty = tl / vi.tiles_x, tx = tl - ty * vi.tiles_x;
    c.i = tx * TW + (int)(threadIdx.x % TW);
    c.j = ty * TH + (int)(threadIdx.x / TW);
    c.inside = c.i < vi.w && c.j < vi.h;
    c.HW = vi.w * vi.h;
    c.pix = (long long)c.j * vi.w + c.i;
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

__device__ __forceinline__ void stage(const BlendArgs &a, long long rbase, unsigned b, unsigned cnt, float2 *s_xy,
                                      float4 *s_con, float4 *s_col, unsigned *s_g) {
    for (unsigned k = threadIdx.x; k < cnt; k += blockDim.x) {
        unsigned g = (unsigned)a.keys[b + k];
        const Record *r = a.rec + rbase + g;
        float4 ra = r->a, rb = r->b, rc = r->c;
        s_xy[k] = make_float2(ra.x, ra.y);
        s_con[k] = make_float4(ra.z, ra.w, rb.x, rb.y);
        if (s_col) s_col[k] = make_float4(rc.x, rc.y, rc.z, rb.z);
        if (s_g) s_g[k] = g;
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) blend_fwd_kernel(const BlendArgs a, const __grid_constant__ ViewBatch vb) {
    constexpr int NT = TW * TH;
    extern __shared__ float4 smem[];
    __shared__ int s_tile;
    const unsigned B = (unsigned)a.batch;
    float4 *s_con = smem;
    float4 *s_col = smem + B;
    float2 *s_xy = reinterpret_cast<float2 *>(smem + 2 * B);
    if (a.ctr->overflow) return;
    unsigned long long n_proc = 0, n_blend = 0;
    for (int iter = 0;; ++iter) {
        int t = next_tile(a, vb, &a.ctr->work_fwd, iter, &s_tile);
        if (t < 0) break;
        TileCoord c = tile_coord<TW, TH>(vb, t);
        const ViewInfo &vi = vb.v[c.v];
        const long long rbase = (long long)c.v * a.n;
        const float px = (float)c.i, py = (float)c.j;
        const unsigned s = a.tile_start[t], e = a.tile_start[t + 1];
        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
        unsigned last = 0;
        bool done = !c.inside;
        for (unsigned b = s; b < e; b += B) {
            if (__syncthreads_count(done) == NT) break;
            unsigned cnt = min(B, e - b);
            stage(a, rbase, b, cnt, s_xy, s_con, s_col, nullptr);
            __syncthreads();
            if (!done) {
                for (unsigned k = 0; k < cnt; ++k) {
                    float2 xy = s_xy[k];
                    float4 cn = s_con[k];
                    PairEval pe = eval_pair(px, py, xy.x, xy.y, cn.x, cn.y, cn.z, cn.w);
                    if (a.counting) ++n_proc;
                    if (!pe.pass) continue;
                    float Tn = next_T(T, pe.alpha);
                    if (Tn < kTMin) {
                        done = true;
                        break;
                    }
                    float w = pe.alpha * T;
                    float4 cz = s_col[k];
                    C0 = fmaf(cz.x, w, C0);
                    C1 = fmaf(cz.y, w, C1);
                    C2 = fmaf(cz.z, w, C2);
                    D = fmaf(cz.w, w, D);
                    T = Tn;
                    last = b - s + k + 1;
                    if (a.counting) ++n_blend;
                }
            }
        }
        if (c.inside) {
            const long long p1 = vi.pix_base + c.pix;
            const long long p3 = 3 * vi.pix_base + c.pix;
            if (a.rgb) {
                a.rgb[p3] = C0 + T * a.bg[0];
                a.rgb[p3 + c.HW] = C1 + T * a.bg[1];
                a.rgb[p3 + 2 * c.HW] = C2 + T * a.bg[2];
            }
            if (a.depth) a.depth[p1] = D;
            if (a.alpha) a.alpha[p1] = 1.f - T;
            if (a.pointmap) {
                // Eq. 5: X^r = ((i - cx) D / fx, (j - cy) D / fy, D)
                a.pointmap[p3] = (px - vi.cx) / vi.fx * D;
                a.pointmap[p3 + c.HW] = (py - vi.cy) / vi.fy * D;
                a.pointmap[p3 + 2 * c.HW] = D;
            }
            if (a.T_final) {
                a.T_final[p1] = T;
                a.n_last[p1] = last;
            }
        }
    }
    if (a.counting) {
        atomicAdd(&a.ctr->fwd_processed, n_proc);
        atomicAdd(&a.ctr->fwd_blended, n_blend);
    }
}

template <int TW, int TH, bool RECOMPUTE, bool DET>
__global__ void __launch_bounds__(TW *TH) blend_bwd_kernel(const BlendArgs a, const __grid_constant__ ViewBatch vb) {
    constexpr int NT = TW * TH;
    constexpr int NW = NT / 32;
    extern __shared__ float4 smem[];
    __shared__ int s_tile;
    __shared__ unsigned s_maxlast;
    const unsigned B = (unsigned)a.batch;
    float4 *s_con = smem;
    float4 *s_col = smem + B;
    float2 *s_xy = reinterpret_cast<float2 *>(smem + 2 * B);
    unsigned *s_g = reinterpret_cast<unsigned *>(s_xy + B);
    float *s_part = reinterpret_cast<float *>(s_g + B);  // DET: [NW][B][10]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (a.ctr->overflow) return;
    unsigned long long n_proc = 0;
    for (int iter = 0;; ++iter) {
        int t = next_tile(a, vb, &a.ctr->work_bwd, iter, &s_tile);
        if (t < 0) break;
        TileCoord c = tile_coord<TW, TH>(vb, t);
        const ViewInfo &vi = vb.v[c.v];
        const long long rbase = (long long)c.v * a.n;
        const float px = (float)c.i, py = (float)c.j;
        const unsigned s = a.tile_start[t], e = a.tile_start[t + 1];
        const long long p1 = vi.pix_base + c.pix;
        const long long p3 = 3 * vi.pix_base + c.pix;

        // per-pixel blend state: stored by the forward, or replayed here
        float T = 1.f;
        unsigned last = 0;
        if (RECOMPUTE) {
            bool done = !c.inside;
            for (unsigned b = s; b < e; b += B) {
                if (__syncthreads_count(done) == NT) break;
                unsigned cnt = min(B, e - b);
                stage(a, rbase, b, cnt, s_xy, s_con, nullptr, nullptr);
                __syncthreads();
                if (!done) {
                    for (unsigned k = 0; k < cnt; ++k) {
                        float2 xy = s_xy[k];
                        float4 cn = s_con[k];
                        PairEval pe = eval_pair(px, py, xy.x, xy.y, cn.x, cn.y, cn.z, cn.w);
                        if (!pe.pass) continue;
                        float Tn = next_T(T, pe.alpha);
                        if (Tn < kTMin) {
                            done = true;
                            break;
                        }
                        T = Tn;
                        last = b - s + k + 1;
                    }
                }
            }
            __syncthreads();
        } else if (c.inside) {
            T = a.T_final[p1];
            last = a.n_last[p1];
        }

        // upstream gradients; the pointmap (Eq. 5) is linear in D
        float gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gT = 0.f;
        if (c.inside) {
            if (a.d_rgb) {
                gC0 = a.d_rgb[p3];
                gC1 = a.d_rgb[p3 + c.HW];
                gC2 = a.d_rgb[p3 + 2 * c.HW];
            }
            if (a.d_depth) gD = a.d_depth[p1];
            if (a.d_pointmap) {
                gD += (px - vi.cx) / vi.fx * a.d_pointmap[p3] + (py - vi.cy) / vi.fy * a.d_pointmap[p3 + c.HW] +
                      a.d_pointmap[p3 + 2 * c.HW];
            }
            gT = a.bg[0] * gC0 + a.bg[1] * gC1 + a.bg[2] * gC2;
            if (a.d_alpha) gT -= a.d_alpha[p1];
        } else {
            last = 0;
        }

        if (threadIdx.x == 0) s_maxlast = 0;
        __syncthreads();
        if (last) atomicMax(&s_maxlast, last);
        __syncthreads();
        const unsigned maxlast = s_maxlast;
        if (DET) {
            // duplicates never reached by any pixel carry a zero partial
            for (unsigned k = s + maxlast + threadIdx.x; k < e; k += NT)
#pragma unroll
                for (int q = 0; q < kGrad2d; ++q) a.det_partial[(long long)k * kGrad2d + q] = 0.f;
        }

        float Bacc = gT;  // gradient-weighted value of everything behind the current Gaussian
        for (unsigned bend = s + maxlast; bend > s;) {
            unsigned bstart = (bend - s > B) ? bend - B : s;
            unsigned cnt = bend - bstart;
            __syncthreads();
            stage(a, rbase, bstart, cnt, s_xy, s_con, s_col, s_g);
            __syncthreads();
            for (int k = (int)cnt - 1; k >= 0; --k) {
                unsigned pos = bstart - s + (unsigned)k;
                float vals[kGrad2d];
#pragma unroll
                for (int q = 0; q < kGrad2d; ++q) vals[q] = 0.f;
                bool contrib = false;
                if (pos < last) {
                    float2 xy = s_xy[k];
                    float4 cn = s_con[k];
                    PairEval pe = eval_pair(px, py, xy.x, xy.y, cn.x, cn.y, cn.z, cn.w);
                    if (a.counting) ++n_proc;
                    if (pe.pass) {
                        contrib = true;
                        const float al = pe.alpha;
                        const float Tk = __fdiv_rn(T, __fsub_rn(1.f, al));  // T before this Gaussian
                        const float w = al * Tk;
                        const float4 cz = s_col[k];
                        const float f = cz.x * gC0 + cz.y * gC1 + cz.z * gC2 + cz.w * gD;
                        const float da = Tk * (f - Bacc);
                        Bacc = f * al + (1.f - al) * Bacc;
                        T = Tk;
                        vals[kGR] = w * gC0;
                        vals[kGG] = w * gC1;
                        vals[kGBl] = w * gC2;
                        vals[kGZ] = w * gD;
                        if (!pe.clamped) {
                            // alpha = o exp(-q/2): d/do = G, d/dq = -alpha/2
                            vals[kGO] = da * pe.G;
                            const float dq = -0.5f * da * al;
                            vals[kGA] = dq * pe.dx * pe.dx;
                            vals[kGB] = 2.f * dq * pe.dx * pe.dy;
                            vals[kGC] = dq * pe.dy * pe.dy;
                            // dx = i - u, dy = j - v
                            vals[kGU] = -2.f * dq * (cn.x * pe.dx + cn.y * pe.dy);
                            vals[kGV] = -2.f * dq * (cn.y * pe.dx + cn.z * pe.dy);
                        }
                    }
                }
                if (DET) {
#pragma unroll
                    for (int q = 0; q < kGrad2d; ++q) {
                        float x = vals[q];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                        vals[q] = x;
                    }
                    if (lane == 0) {
                        float *dst = s_part + ((size_t)warp * B + k) * kGrad2d;
#pragma unroll
                        for (int q = 0; q < kGrad2d; ++q) dst[q] = vals[q];
                    }
                } else if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
                    for (int q = 0; q < kGrad2d; ++q) {
                        float x = vals[q];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                        vals[q] = x;
                    }
                    if (lane == 0) {
                        float *dst = a.grad2d + (rbase + s_g[k]) * kGrad2d;
#pragma unroll
                        for (int q = 0; q < kGrad2d; ++q) atomicAdd(dst + q, vals[q]);
                    }
                }
            }
            if (DET) {
                __syncthreads();
                // per-duplicate partial: warps summed in a fixed order
                for (unsigned idx = threadIdx.x; idx < cnt * kGrad2d; idx += NT) {
                    unsigned k = idx / kGrad2d, q = idx % kGrad2d;
                    float x = 0.f;
#pragma unroll
                    for (int wv = 0; wv < NW; ++wv) x += s_part[((size_t)wv * B + k) * kGrad2d + q];
                    a.det_partial[(long long)(bstart + k) * kGrad2d + q] = x;
                }
            }
            bend = bstart;
        }
    }
    if (a.counting) atomicAdd(&a.ctr->bwd_processed, n_proc);
}

template <int TW, int TH>
size_t fwd_smem(int batch) { return (size_t)batch * (2 * sizeof(float4) + sizeof(float2)); }

template <int TW, int TH, bool DET>
size_t bwd_smem(int batch) {
    size_t s = (size_t)batch * (2 * sizeof(float4) + sizeof(float2) + sizeof(unsigned));
    if (DET) s += (size_t)(TW * TH / 32) * batch * kGrad2d * sizeof(float);
    return s;
}

// Raise a kernel's dynamic shared-memory limit only when a larger size is first
// needed, so that steady-state calls (and stream capture) issue nothing but launches.
template <class K>
cudaError_t ensure_smem(K kernel, size_t bytes, int *cached) {
    if ((int)bytes <= *cached) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) *cached = (int)bytes;
    return e;
}

template <int TW, int TH>
cudaError_t fwd_impl(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    static int cached = 48 * 1024;
    size_t sm = fwd_smem<TW, TH>(a.batch);
    auto k = blend_fwd_kernel<TW, TH>;
    cudaError_t e = ensure_smem(k, sm, &cached);
    if (e != cudaSuccess) return e;
    k<<<grid, TW * TH, sm, s>>>(a, vb);
    return cudaGetLastError();
}

template <int TW, int TH, bool R, bool D>
cudaError_t bwd_impl2(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    static int cached = 48 * 1024;
    size_t sm = bwd_smem<TW, TH, D>(a.batch);
    auto k = blend_bwd_kernel<TW, TH, R, D>;
    cudaError_t e = ensure_smem(k, sm, &cached);
    if (e != cudaSuccess) return e;
    k<<<grid, TW * TH, sm, s>>>(a, vb);
    return cudaGetLastError();
}

template <int TW, int TH>
cudaError_t bwd_impl(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    const bool R = a.T_final == nullptr, D = a.det_partial != nullptr;
    if (R && D) return bwd_impl2<TW, TH, true, true>(a, vb, grid, s);
    if (R) return bwd_impl2<TW, TH, true, false>(a, vb, grid, s);
    if (D) return bwd_impl2<TW, TH, false, true>(a, vb, grid, s);
    return bwd_impl2<TW, TH, false, false>(a, vb, grid, s);
}

}  // namespace

cudaError_t launch_blend_fwd(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    const int tw = vb.tile_w, th = vb.tile_h;
    if (tw == 16 && th == 16) return fwd_impl<16, 16>(a, vb, grid, s);
    if (tw == 16 && th == 8) return fwd_impl<16, 8>(a, vb, grid, s);
    if (tw == 8 && th == 8) return fwd_impl<8, 8>(a, vb, grid, s);
    if (tw == 32 && th == 8) return fwd_impl<32, 8>(a, vb, grid, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_blend_bwd(const BlendArgs &a, const ViewBatch &vb, int grid, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    const int tw = vb.tile_w, th = vb.tile_h;
    if (tw == 16 && th == 16) return bwd_impl<16, 16>(a, vb, grid, s);
    if (tw == 16 && th == 8) return bwd_impl<16, 8>(a, vb, grid, s);
    if (tw == 8 && th == 8) return bwd_impl<8, 8>(a, vb, grid, s);
    if (tw == 32 && th == 8) return bwd_impl<32, 8>(a, vb, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace s3gs
