// C ABI of the library (declared in include/s3gs.h): contexts, states, argument
// checking, buffer planning and the launch sequence of the forward and backward.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "s3gs_internal.cuh"

using namespace s3gs;

enum Stage {
    kStProject = 0, kStScan, kStEmit, kStSort, kStOrder, kStBlendFwd, kStBlendBwd, kStDetReduce,
    kStProjectBwd, kStTwist, kStLoss, kNumStages
};
static_assert(kNumStages == S3GS_NUM_STAGES, "stage list");

struct s3gs_ctx {
    int device = 0;
    int num_sms = 0;
    int counting = 0;
    int timing = 0;
    bool events_made = false;
    cudaEvent_t ev[kNumStages][2];
    bool ev_used[kNumStages] = {};
    float *loss_partial = nullptr;  // [loss_blocks_per_view() * S3GS_MAX_VIEWS]
    std::string err;
};

bool capturing(cudaStream_t s);

// Records a start/stop event pair around one stage when timing is on. Inside a
// stream capture the records become event nodes of the graph (external
// records), so replays of the graph are timed too. A failed record disables
// timing and clears the runtime's error state rather than leaving it pending.
struct StageTimer {
    s3gs_ctx *ctx;
    int stage;
    cudaStream_t s;
    static void record(s3gs_ctx *c, cudaEvent_t ev, cudaStream_t str) {
        cudaError_t e = capturing(str) ? cudaEventRecordWithFlags(ev, str, cudaEventRecordExternal)
                                       : cudaEventRecord(ev, str);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            c->timing = 0;
        }
    }
    StageTimer(s3gs_ctx *c, int st, cudaStream_t str) : ctx(c), stage(st), s(str) {
        if (ctx->timing) record(ctx, ctx->ev[stage][0], s);
    }
    ~StageTimer() {
        if (ctx->timing) {
            record(ctx, ctx->ev[stage][1], s);
            if (ctx->timing) ctx->ev_used[stage] = true;
        }
    }
};

// A device buffer and its capacity in elements.
template <class T>
struct DevBuf {
    T *p = nullptr;
    long long cap = 0;
};

struct s3gs_state {
    s3gs_ctx *ctx = nullptr;
    DevBuf<Record> rec;
    DevBuf<int2> ext;
    DevBuf<unsigned> vis_mask;
    DevBuf<float> grad2d;
    DevBuf<unsigned> tile_count, tile_start, cursor, order, scan_part;
    DevBuf<unsigned> occl;        // per bucket optical depth lower bound (occlusion cut)
    DevBuf<unsigned char> cut;    // per tile last listed depth bin
    DevBuf<unsigned> cut_max;     // [tiles] row maxima of the cut (at row starts)
    DevBuf<unsigned> cut_view;    // [32] view maxima of the cut; the next forward's hint
    const void *cut_hint_for = nullptr;  // cut buffer whose contents are a valid hint ...
    long long cut_hint_tiles = -1;       // ... for a view batch of this many tiles
    DevBuf<unsigned long long> keys;       // tile-sorted duplicate list
    DevBuf<unsigned long long> keys_emit;  // emission order, read by the tile sort
    DevBuf<float> det_partial;
    DevBuf<float> T_final;
    DevBuf<unsigned> n_last;
    DevBuf<float> twist_part;
    DevBuf<float> loss_part;  // fused-loss backward: one partial per tile
    unsigned *bucket = nullptr;
    DevCounters *ctr = nullptr;
    DevCounters *ctr_host = nullptr;  // pinned
    // last forward
    bool valid = false;
    bool grad_clean = true;
    ViewBatch vb;
    s3gs_gaussians g;
    s3gs_options opt;
    const float *Tdev = nullptr;
    cudaStream_t stream = nullptr;
};

namespace {

const char *kVersion = "s3gs 1.0 (sm_103a)";

s3gs_status fail(s3gs_ctx *ctx, s3gs_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

s3gs_status cuda_fail(s3gs_ctx *ctx, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return fail(ctx, S3GS_E_NOMEM, m);
    return fail(ctx, S3GS_E_CUDA, m);
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

}  // namespace

namespace s3gs {
s3gs_status ctx_error(s3gs_ctx *ctx, s3gs_status st, const char *msg) {
    if (ctx) ctx->err = msg;
    return st;
}
int ctx_device(const s3gs_ctx *ctx) { return ctx ? ctx->device : 0; }
}  // namespace s3gs

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

namespace {

// Grow a device buffer to at least `need` elements (contents are not kept).
template <class T>
s3gs_status grow(s3gs_ctx *ctx, DevBuf<T> &b, long long need, cudaStream_t s, const char *name, bool zero = false) {
    if (need < 1) need = 1;
    if (need <= b.cap && b.p) return S3GS_OK;
    if (capturing(s))
        return fail(ctx, S3GS_E_INVALID, std::string("buffer '") + name +
                                             "' must grow during stream capture; call s3gs_reserve first");
    if (b.p) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, name);
        e = cudaFree(b.p);
        if (e != cudaSuccess) return cuda_fail(ctx, e, name);
        b.p = nullptr;
        b.cap = 0;
    }
    cudaError_t e = cudaMalloc((void **)&b.p, (size_t)need * sizeof(T));
    if (e != cudaSuccess) {
        b.p = nullptr;
        return cuda_fail(ctx, e, name);
    }
    if (zero) {
        e = cudaMemset(b.p, 0, (size_t)need * sizeof(T));
        if (e != cudaSuccess) return cuda_fail(ctx, e, name);
    }
    b.cap = need;
    return S3GS_OK;
}

// The duplicate list lives in two buffers of one capacity: the emission writes
// its buckets into keys_emit, the tile sort reads them and writes the sorted
// list into keys.
s3gs_status grow_keys(s3gs_ctx *ctx, s3gs_state *st, long long need, cudaStream_t s) {
    s3gs_status r = grow(ctx, st->keys, need, s, "keys");
    if (r != S3GS_OK) return r;
    return grow(ctx, st->keys_emit, st->keys.cap, s, "keys_emit");
}

bool finite_cam(const s3gs_camera &c) {
    if (!(std::isfinite(c.fx) && std::isfinite(c.fy) && std::isfinite(c.cx) && std::isfinite(c.cy))) return false;
    if (c.fx == 0.f || c.fy == 0.f) return false;
    for (int k = 0; k < 12; ++k)
        if (!std::isfinite(c.T_cw[k])) return false;
    return true;
}

bool valid_tile(int tw, int th) {
    return (tw == 16 && th == 16) || (tw == 16 && th == 8) || (tw == 8 && th == 8) || (tw == 32 && th == 8);
}

void fill_options(const s3gs_options *in, s3gs_options &o) {
    if (in) o = *in; else s3gs_options_default(&o);
    if (o.tile_w == 0 && o.tile_h == 0) { o.tile_w = 16; o.tile_h = 16; }
    // automatic pixels per thread: the preferred value if the tile still fills whole warps
    const int px = o.tile_w * o.tile_h;
    if (o.pixels_per_thread == 0) o.pixels_per_thread = (px / 2) % 32 == 0 ? 2 : 1;
    if (o.bwd_pixels_per_thread == 0)
        o.bwd_pixels_per_thread = (px / 4) % 32 == 0 ? 4 : ((px / 2) % 32 == 0 ? 2 : 1);
    if (o.batch <= 0) o.batch = 256;
    if (o.near_z == 0.f) o.near_z = 0.2f;
    if (o.guard_slope == 0.f) o.guard_slope = 1.5f;
}

s3gs_status plan_views(s3gs_ctx *ctx, const s3gs_camera *cams, int n_views, int tw, int th, ViewBatch &vb) {
    memset(&vb, 0, sizeof(vb));
    vb.n_views = n_views;
    vb.tile_w = tw;
    vb.tile_h = th;
    long long tiles = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const s3gs_camera &c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > (1 << 16) || c.height > (1 << 16))
            return fail(ctx, S3GS_E_INVALID, "camera " + std::to_string(v) + ": width/height out of range");
        if (!finite_cam(c))
            return fail(ctx, S3GS_E_INVALID, "camera " + std::to_string(v) + ": non-finite or zero intrinsics/pose");
        ViewInfo &vi = vb.v[v];
        vi.w = c.width; vi.h = c.height;
        vi.fx = c.fx; vi.fy = c.fy; vi.cx = c.cx; vi.cy = c.cy;
        memcpy(vi.T, c.T_cw, sizeof(vi.T));
        vi.tiles_x = (c.width + tw - 1) / tw;
        vi.tiles_y = (c.height + th - 1) / th;
        vi.tile_base = (int)tiles;
        vi.pix_base = pix;
        tiles += (long long)vi.tiles_x * vi.tiles_y;
        pix += (long long)c.width * c.height;
        if (tiles > (1LL << 30)) return fail(ctx, S3GS_E_INVALID, "too many tiles in one call");
    }
    vb.total_tiles = (int)tiles;
    vb.total_pixels = pix;
    return S3GS_OK;
}

s3gs_status ensure_forward_buffers(s3gs_ctx *ctx, s3gs_state *st, long long n_rec, long long n_pix,
                                   long long n_tiles, long long n_views, long long n, bool store, cudaStream_t s) {
    s3gs_status r;
    if ((r = grow(ctx, st->rec, n_rec, s, "records")) != S3GS_OK) return r;
    if ((r = grow(ctx, st->ext, n_rec, s, "extents")) != S3GS_OK) return r;
    if ((r = grow(ctx, st->vis_mask, n, s, "visibility")) != S3GS_OK) return r;
    if (n_rec * kGrad2d > st->grad2d.cap || !st->grad2d.p) {
        if ((r = grow(ctx, st->grad2d, n_rec * kGrad2d, s, "grad2d", true)) != S3GS_OK) return r;
        st->grad_clean = true;
    }
    const long long n_buckets = n_tiles * kDepthBins;
    if ((r = grow(ctx, st->tile_count, n_buckets + 1, s, "bucket_count")) != S3GS_OK) return r;
    if ((r = grow(ctx, st->tile_start, n_buckets + 1, s, "bucket_start")) != S3GS_OK) return r;
    if ((r = grow(ctx, st->cursor, n_buckets + 1, s, "cursor")) != S3GS_OK) return r;
    if ((r = grow(ctx, st->order, n_tiles + 1, s, "order")) != S3GS_OK) return r;
    if ((r = grow(ctx, st->scan_part, (n_buckets + 4095) / 4096 + 2, s, "scan_part")) != S3GS_OK) return r;
    if ((r = grow(ctx, st->occl, n_buckets + 1, s, "occlusion")) != S3GS_OK) return r;
    if ((r = grow(ctx, st->cut, n_tiles + 16, s, "cut")) != S3GS_OK) return r;
    if ((r = grow(ctx, st->cut_max, n_tiles + 16, s, "cut_max")) != S3GS_OK) return r;
    if ((r = grow(ctx, st->cut_view, S3GS_MAX_VIEWS, s, "cut_view")) != S3GS_OK) return r;
    if (store) {
        if ((r = grow(ctx, st->T_final, n_pix, s, "T_final")) != S3GS_OK) return r;
        if ((r = grow(ctx, st->n_last, n_pix, s, "n_last")) != S3GS_OK) return r;
    }
    long long need_twp = (long long)project_bwd_grid(n > 0 ? n : 1) * n_views * 6;
    if ((r = grow(ctx, st->twist_part, need_twp, s, "twist_partials")) != S3GS_OK) return r;
    if ((r = grow(ctx, st->loss_part, n_tiles + 1, s, "loss_partials")) != S3GS_OK) return r;
    return S3GS_OK;
}

// Inputs of the backward with the L1 mapping loss fused in.
struct L1Fused {
    const float *rgb, *depth, *pointmap, *t_rgb, *t_depth, *t_pointmap, *mask;
    float w_rgb, w_depth, w_geo;
};

s3gs_status render_bwd_impl(s3gs_ctx *ctx, s3gs_state *st, const float *d_rgb, const float *d_depth,
                            const float *d_pointmap, const float *d_alpha, const L1Fused *l1, float *loss_device,
                            float *d_means, float *d_log_scales, float *d_quats, float *d_opacity_logits,
                            float *d_colors, float *d_twist, int32_t accumulate, void *stream_);

}  // namespace

extern "C" {

void s3gs_options_default(s3gs_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->tile_w = 16;
    opt->tile_h = 16;
    opt->pixels_per_thread = 0;
    opt->bwd_pixels_per_thread = 0;
    opt->batch = 256;
    opt->blocks_per_sm = 0;
    opt->deterministic = 0;
    opt->recompute = 0;
    opt->auto_grow = 1;
    opt->near_z = 0.2f;
    opt->guard_slope = 1.5f;
}

const char *s3gs_version(void) { return kVersion; }

s3gs_status s3gs_create(int device, s3gs_ctx **out) {
    if (!out) return S3GS_E_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return S3GS_E_INVALID;
    s3gs_ctx *ctx = new (std::nothrow) s3gs_ctx();
    if (!ctx) return S3GS_E_NOMEM;
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc((void **)&ctx->loss_partial, sizeof(float) * loss_blocks_per_view() * S3GS_MAX_VIEWS) !=
            cudaSuccess) {
        delete ctx;
        return S3GS_E_CUDA;
    }
    *out = ctx;
    return S3GS_OK;
}

void s3gs_destroy(s3gs_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->loss_partial) cudaFree(ctx->loss_partial);
    if (ctx->events_made)
        for (int i = 0; i < kNumStages; ++i) {
            cudaEventDestroy(ctx->ev[i][0]);
            cudaEventDestroy(ctx->ev[i][1]);
        }
    delete ctx;
}

s3gs_status s3gs_set_timing(s3gs_ctx *ctx, int32_t enable) {
    if (!ctx) return S3GS_E_INVALID;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (enable && !ctx->events_made) {
        for (int i = 0; i < kNumStages; ++i) {
            CK(cudaEventCreate(&ctx->ev[i][0]), "cudaEventCreate");
            CK(cudaEventCreate(&ctx->ev[i][1]), "cudaEventCreate");
        }
        ctx->events_made = true;
    }
    for (int i = 0; i < kNumStages; ++i) ctx->ev_used[i] = false;
    ctx->timing = enable ? 1 : 0;
    return S3GS_OK;
}

s3gs_status s3gs_read_timing(s3gs_ctx *ctx, float *ms, int32_t n) {
    if (!ctx || !ms || n < 0) return fail(ctx, S3GS_E_INVALID, "read_timing: bad argument");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    for (int i = 0; i < n; ++i) {
        ms[i] = -1.f;
        if (i >= kNumStages || !ctx->events_made || !ctx->ev_used[i]) continue;
        CK(cudaEventSynchronize(ctx->ev[i][1]), "cudaEventSynchronize");
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ctx->ev[i][0], ctx->ev[i][1]), "cudaEventElapsedTime");
        ms[i] = t;
    }
    return S3GS_OK;
}

const char *s3gs_last_error(const s3gs_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

s3gs_status s3gs_state_create(s3gs_ctx *ctx, s3gs_state **out) {
    if (!ctx || !out) return fail(ctx, S3GS_E_INVALID, "state_create: null argument");
    *out = nullptr;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    s3gs_state *st = new (std::nothrow) s3gs_state();
    if (!st) return fail(ctx, S3GS_E_NOMEM, "state_create: host allocation");
    st->ctx = ctx;
    cudaError_t e = cudaMalloc((void **)&st->ctr, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMemset(st->ctr, 0, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMalloc((void **)&st->bucket, 33 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&st->ctr_host, sizeof(DevCounters));
    if (e != cudaSuccess) {
        s3gs_state_destroy(st);
        return cuda_fail(ctx, e, "state_create");
    }
    memset(st->ctr_host, 0, sizeof(DevCounters));
    *out = st;
    return S3GS_OK;
}

void s3gs_state_destroy(s3gs_state *st) {
    if (!st) return;
    if (st->ctx) cudaSetDevice(st->ctx->device);
    cudaDeviceSynchronize();
    void *bufs[] = {st->rec.p,       st->ext.p,       st->vis_mask.p,  st->grad2d.p,      st->tile_count.p,
                    st->tile_start.p, st->cursor.p,    st->order.p,     st->scan_part.p,   st->bucket,
                    st->keys.p,      st->keys_emit.p, st->det_partial.p, st->T_final.p,   st->n_last.p,
                    st->twist_part.p, st->loss_part.p, st->occl.p,   st->cut.p,       st->cut_max.p,
                    st->cut_view.p,  st->ctr};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (st->ctr_host) cudaFreeHost(st->ctr_host);
    delete st;
}

s3gs_status s3gs_reserve(s3gs_ctx *ctx, s3gs_state *st, int64_t n, int32_t n_views, int64_t total_pixels,
                         int64_t total_tiles, int64_t max_duplicates) {
    if (!ctx || !st || n < 0 || n_views < 1 || n_views > S3GS_MAX_VIEWS || total_pixels < 0 || total_tiles < 0 ||
        max_duplicates < 0 || max_duplicates > S3GS_MAX_DUPLICATES)
        return fail(ctx, S3GS_E_INVALID, "reserve: argument out of range");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    s3gs_status r = ensure_forward_buffers(ctx, st, (long long)n * n_views, total_pixels, total_tiles, n_views, n,
                                           true, nullptr);
    if (r != S3GS_OK) return r;
    if ((r = grow_keys(ctx, st, max_duplicates, nullptr)) != S3GS_OK) return r;
    CK(cudaDeviceSynchronize(), "reserve");
    return S3GS_OK;
}

s3gs_status s3gs_render_fwd(s3gs_ctx *ctx, s3gs_state *st, const s3gs_gaussians *g, const s3gs_camera *cams,
                            int32_t n_views, const float *T_cw_device, const s3gs_options *opt_in, float *rgb,
                            float *depth, float *pointmap, float *alpha, void *stream_) {
    if (!ctx) return S3GS_E_INVALID;
    if (!st || !g || !cams) return fail(ctx, S3GS_E_INVALID, "render_fwd: null state, gaussians or cameras");
    if (st->ctx != ctx) return fail(ctx, S3GS_E_INVALID, "render_fwd: state belongs to another context");
    st->valid = false;
    if (n_views < 1 || n_views > S3GS_MAX_VIEWS)
        return fail(ctx, S3GS_E_INVALID, "render_fwd: n_views must be in 1.." + std::to_string(S3GS_MAX_VIEWS));
    if (g->n < 0 || g->n > (1LL << 31) - 1) return fail(ctx, S3GS_E_INVALID, "render_fwd: n out of range");
    if (g->sh_degree < 0 || g->sh_degree > S3GS_MAX_SH_DEGREE)
        return fail(ctx, S3GS_E_INVALID, "render_fwd: sh_degree must be in 0..3");
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->colors))
        return fail(ctx, S3GS_E_INVALID, "render_fwd: null Gaussian parameter pointer");
    if (g->n > 0 && ((uintptr_t)g->quats & 15u))
        return fail(ctx, S3GS_E_INVALID, "render_fwd: quats must be 16-byte aligned");
    s3gs_options opt;
    fill_options(opt_in, opt);
    if (!valid_tile(opt.tile_w, opt.tile_h))
        return fail(ctx, S3GS_E_INVALID, "render_fwd: tile shape must be 16x16, 16x8, 8x8 or 32x8");
    if (opt.batch > 1024) return fail(ctx, S3GS_E_INVALID, "render_fwd: batch must be <= 1024");
    if (opt.pixels_per_thread != 1 && opt.pixels_per_thread != 2 && opt.pixels_per_thread != 4)
        return fail(ctx, S3GS_E_INVALID, "render_fwd: pixels_per_thread must be 1, 2 or 4");
    if (opt.bwd_pixels_per_thread != 1 && opt.bwd_pixels_per_thread != 2 && opt.bwd_pixels_per_thread != 4)
        return fail(ctx, S3GS_E_INVALID, "render_fwd: bwd_pixels_per_thread must be 1, 2 or 4");
    if ((opt.tile_w * opt.tile_h / opt.pixels_per_thread) % 32 != 0 ||
        (opt.tile_w * opt.tile_h / opt.bwd_pixels_per_thread) % 32 != 0)
        return fail(ctx, S3GS_E_INVALID, "render_fwd: tile_w * tile_h / pixels per thread must be a multiple of 32");
    if (opt.blocks_per_sm < 0 || opt.blocks_per_sm > 64)
        return fail(ctx, S3GS_E_INVALID, "render_fwd: blocks_per_sm must be in 0..64");
    if (!(opt.near_z > 0.f) || !std::isfinite(opt.near_z))
        return fail(ctx, S3GS_E_INVALID, "render_fwd: near_z must be positive");
    if (!std::isfinite(opt.guard_slope))
        return fail(ctx, S3GS_E_INVALID, "render_fwd: guard_slope must be finite");
    cudaStream_t s = (cudaStream_t)stream_;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    ViewBatch vb;
    s3gs_status r = plan_views(ctx, cams, n_views, opt.tile_w, opt.tile_h, vb);
    if (r != S3GS_OK) return r;
    const long long n = g->n;
    const long long n_rec = n * n_views;
    const bool store = !opt.recompute;
    r = ensure_forward_buffers(ctx, st, n_rec, vb.total_pixels, vb.total_tiles, n_views, n, store, s);
    if (r != S3GS_OK) return r;
    if (!st->keys.p) {
        if ((r = grow_keys(ctx, st, 1 << 16, s)) != S3GS_OK) return r;
    }
    const long long T = vb.total_tiles;
    const long long NBK = T * kDepthBins;  // (tile, depth bin) buckets

    CK(cudaMemsetAsync(st->tile_count.p, 0, (size_t)(NBK + 1) * sizeof(unsigned), s), "memset bucket counts");
    CK(cudaMemsetAsync(st->ctr, 0, sizeof(DevCounters), s), "memset counters");
    const bool cut = !opt.full_lists;
    if (cut) {
        CK(cudaMemsetAsync(st->occl.p, 0, (size_t)NBK * sizeof(unsigned), s), "memset occlusion");
        CK(cudaMemsetAsync(st->cut_max.p, 0, (size_t)T * sizeof(unsigned), s), "memset cut row maxima");
        if (st->cut_hint_for != (const void *)st->cut.p || st->cut_hint_tiles != T) {
            // no previous cut of this layout: hints that exclude nothing
            CK(cudaMemsetAsync(st->cut.p, 0xff, (size_t)T, s), "init cut hint");
            CK(cudaMemsetAsync(st->cut_view.p, 0xff, S3GS_MAX_VIEWS * sizeof(unsigned), s), "init view hint");
            st->cut_hint_for = st->cut.p;
            st->cut_hint_tiles = T;
        }
    }

    ProjectArgs pa;
    pa.means = g->means; pa.log_scales = g->log_scales; pa.quats = g->quats;
    pa.opacity_logits = g->opacity_logits; pa.colors = g->colors;
    pa.n = n; pa.sh_degree = g->sh_degree; pa.near_z = opt.near_z; pa.guard = opt.guard_slope;
    pa.Tdev = T_cw_device;
    pa.rec = st->rec.p; pa.ext = st->ext.p; pa.vis_mask = st->vis_mask.p; pa.tile_count = st->tile_count.p;
    pa.occl = cut ? st->occl.p : nullptr;
    pa.cut_hint = st->cut.p; pa.view_hint = st->cut_view.p;
    {
        const int m = (opt.tile_w < opt.tile_h ? opt.tile_w : opt.tile_h) - 1;
        pa.tile_fit = m * m / 4;
    }
    EmitArgs ea;
    ea.rec = st->rec.p; ea.ext = st->ext.p; ea.n = n; ea.cursor = st->cursor.p; ea.keys = nullptr;
    ea.key_capacity = 0; ea.ctr = st->ctr; ea.tile_count = st->tile_count.p;
    ea.cut = cut ? st->cut.p : nullptr;
    ea.row_max = st->cut_max.p; ea.view_max = st->cut_view.p;
    {
        // with the cut: projection and optical depths, the cut, then the bucket counts
        StageTimer tm(ctx, kStProject, s);
        CK(launch_project(pa, vb, s), "project");
        if (cut) {
            // the projection has read the hints; the cut kernel now overwrites them
            CK(cudaMemsetAsync(st->cut_view.p, 0, S3GS_MAX_VIEWS * sizeof(unsigned), s), "memset cut view maxima");
            CutArgs ca;
            ca.occl = st->occl.p; ca.cut = st->cut.p; ca.n_tiles = T;
            ca.row_max = st->cut_max.p; ca.view_max = st->cut_view.p;
            CK(launch_cut(ca, vb, s), "cut");
            CK(launch_count(ea, vb, s), "count");
        }
    }

    ScanArgs sa;
    sa.tile_count = st->tile_count.p; sa.tile_start = st->tile_start.p; sa.cursor = st->cursor.p;
    sa.partials = st->scan_part.p; sa.ctr = st->ctr; sa.n_tiles = NBK; sa.key_capacity = (unsigned long long)st->keys.cap;
    {
        StageTimer tm(ctx, kStScan, s);
        CK(launch_scan(sa, s), "scan");
    }

    if (opt.auto_grow && !capturing(s)) {
        CK(cudaMemcpyAsync(st->ctr_host, st->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s), "read K");
        CK(cudaStreamSynchronize(s), "sync K");
        long long K = (long long)st->ctr_host->n_dup;
        if (K > S3GS_MAX_DUPLICATES)
            return fail(ctx, S3GS_E_CAPACITY, "render_fwd: " + std::to_string(K) + " duplicates exceed the 32-bit limit");
        if (K > st->keys.cap) {
            long long want = K + K / 4 + 1024;
            if (want > S3GS_MAX_DUPLICATES) want = S3GS_MAX_DUPLICATES;
            if ((r = grow_keys(ctx, st, want, s)) != S3GS_OK) return r;
            CK(cudaMemsetAsync(&st->ctr->overflow, 0, sizeof(unsigned), s), "clear overflow");
        }
    }
    if (opt.deterministic) {
        if ((r = grow(ctx, st->det_partial, st->keys.cap * kGrad2d, s, "det_partial")) != S3GS_OK) return r;
    }

    ea.keys = st->keys_emit.p;  // the duplicate buffers may have grown since the count
    ea.key_capacity = (unsigned long long)st->keys.cap;
    {
        StageTimer tm(ctx, kStEmit, s);
        CK(launch_emit(ea, vb, s), "emit");
    }

    SortArgs so;
    so.tile_start = st->tile_start.p; so.keys_in = st->keys_emit.p; so.keys = st->keys.p; so.n_tiles = T; so.ctr = st->ctr;
    {
        StageTimer tm(ctx, kStSort, s);
        CK(launch_tile_sort(so, s), "tile_sort");
    }

    const bool persistent = opt.blocks_per_sm > 0;
    if (persistent) {
        OrderArgs oa;
        oa.tile_start = st->tile_start.p; oa.order = st->order.p; oa.bucket_cnt = st->bucket; oa.n_tiles = T;
        StageTimer tm(ctx, kStOrder, s);
        CK(launch_tile_order(oa, s), "tile_order");
    }

    BlendArgs ba;
    memset(&ba, 0, sizeof(ba));
    ba.rec = st->rec.p; ba.keys = st->keys.p; ba.tile_start = st->tile_start.p;
    ba.order = persistent ? st->order.p : nullptr;
    ba.n = n;
    ba.bg[0] = opt.bg[0]; ba.bg[1] = opt.bg[1]; ba.bg[2] = opt.bg[2];
    ba.rgb = rgb; ba.depth = depth; ba.pointmap = pointmap; ba.alpha = alpha;
    ba.T_final = store ? st->T_final.p : nullptr;
    ba.n_last = store ? st->n_last.p : nullptr;
    ba.ctr = st->ctr;
    ba.persistent = persistent;
    ba.batch = opt.batch;
    ba.ppt = opt.pixels_per_thread;
    ba.counting = ctx->counting;
    long long grid = persistent ? std::min<long long>(T, (long long)ctx->num_sms * opt.blocks_per_sm) : T;
    {
        StageTimer tm(ctx, kStBlendFwd, s);
        CK(launch_blend_fwd(ba, vb, (int)grid, s), "blend_fwd");
    }

    st->vb = vb;
    st->g = *g;
    st->opt = opt;
    st->Tdev = T_cw_device;
    st->stream = s;
    st->valid = true;
    return S3GS_OK;
}

s3gs_status s3gs_render_bwd(s3gs_ctx *ctx, s3gs_state *st, const float *d_rgb, const float *d_depth,
                            const float *d_pointmap, const float *d_alpha, float *d_means, float *d_log_scales,
                            float *d_quats, float *d_opacity_logits, float *d_colors, float *d_twist,
                            int32_t accumulate, void *stream_) {
    return render_bwd_impl(ctx, st, d_rgb, d_depth, d_pointmap, d_alpha, nullptr, nullptr, d_means, d_log_scales,
                           d_quats, d_opacity_logits, d_colors, d_twist, accumulate, stream_);
}

s3gs_status s3gs_render_bwd_l1(s3gs_ctx *ctx, s3gs_state *st, const float *rgb, const float *depth,
                               const float *pointmap, const float *t_rgb, const float *t_depth,
                               const float *t_pointmap, const float *mask, float w_rgb, float w_depth, float w_geo,
                               float *loss_device, float *d_means, float *d_log_scales, float *d_quats,
                               float *d_opacity_logits, float *d_colors, float *d_twist, int32_t accumulate,
                               void *stream_) {
    if (!ctx) return S3GS_E_INVALID;
    if ((t_rgb && !rgb) || (t_depth && !depth) || (t_pointmap && !pointmap))
        return fail(ctx, S3GS_E_INVALID, "render_bwd_l1: a target is given without its rendered output");
    L1Fused l1;
    l1.rgb = rgb; l1.depth = depth; l1.pointmap = pointmap;
    l1.t_rgb = t_rgb; l1.t_depth = t_depth; l1.t_pointmap = t_pointmap; l1.mask = mask;
    l1.w_rgb = w_rgb; l1.w_depth = w_depth; l1.w_geo = w_geo;
    return render_bwd_impl(ctx, st, nullptr, nullptr, nullptr, nullptr, &l1, loss_device, d_means, d_log_scales,
                           d_quats, d_opacity_logits, d_colors, d_twist, accumulate, stream_);
}

}  // extern "C"

namespace {

s3gs_status render_bwd_impl(s3gs_ctx *ctx, s3gs_state *st, const float *d_rgb, const float *d_depth,
                            const float *d_pointmap, const float *d_alpha, const L1Fused *l1, float *loss_device,
                            float *d_means, float *d_log_scales, float *d_quats, float *d_opacity_logits,
                            float *d_colors, float *d_twist, int32_t accumulate, void *stream_) {
    if (!ctx) return S3GS_E_INVALID;
    if (!st) return fail(ctx, S3GS_E_INVALID, "render_bwd: null state");
    if (!st->valid) return fail(ctx, S3GS_E_STATE, "render_bwd: no successful forward on this state");
    if (d_quats && ((uintptr_t)d_quats & 15u))
        return fail(ctx, S3GS_E_INVALID, "render_bwd: d_quats must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream_;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const ViewBatch &vb = st->vb;
    const long long n = st->g.n;
    const long long n_rec = n * vb.n_views;
    const bool persistent = st->opt.blocks_per_sm > 0;
    const bool det = st->opt.deterministic != 0;

    if (!st->grad_clean) CK(cudaMemsetAsync(st->grad2d.p, 0, (size_t)n_rec * kGrad2d * sizeof(float), s), "memset grad2d");
    st->grad_clean = false;
    CK(cudaMemsetAsync(&st->ctr->work_bwd, 0, sizeof(unsigned), s), "memset work_bwd");
    CK(cudaMemsetAsync(&st->ctr->bwd_processed, 0, sizeof(unsigned long long), s), "memset counter");

    BlendArgs ba;
    memset(&ba, 0, sizeof(ba));
    ba.rec = st->rec.p; ba.keys = st->keys.p; ba.tile_start = st->tile_start.p;
    ba.order = persistent ? st->order.p : nullptr;
    ba.n = n;
    ba.bg[0] = st->opt.bg[0]; ba.bg[1] = st->opt.bg[1]; ba.bg[2] = st->opt.bg[2];
    ba.T_final = st->opt.recompute ? nullptr : st->T_final.p;
    ba.n_last = st->opt.recompute ? nullptr : st->n_last.p;
    ba.d_rgb = d_rgb; ba.d_depth = d_depth; ba.d_pointmap = d_pointmap; ba.d_alpha = d_alpha;
    ba.grad2d = st->grad2d.p;
    ba.det_partial = det ? st->det_partial.p : nullptr;
    ba.ctr = st->ctr;
    ba.persistent = persistent;
    ba.batch = st->opt.batch;
    ba.ppt = st->opt.bwd_pixels_per_thread;
    ba.counting = ctx->counting;
    // Colour and opacity gradients feed only d_colors and d_opacity_logits, and (for
    // SH degree >= 1) the twist through the view direction; without them the blend
    // accumulates only the geometry slots.
    ba.geom_only = !det && !d_colors && !d_opacity_logits && st->g.sh_degree == 0;
    if (l1) {
        const float Ptot = (float)vb.total_pixels;
        ba.l1 = 1;
        ba.o_rgb = l1->rgb; ba.o_depth = l1->depth; ba.o_pointmap = l1->pointmap;
        ba.t_rgb = l1->t_rgb; ba.t_depth = l1->t_depth; ba.t_pointmap = l1->t_pointmap; ba.mask = l1->mask;
        ba.kr = l1->w_rgb / (3.f * Ptot); ba.kd = l1->w_depth / Ptot; ba.kg = l1->w_geo / (3.f * Ptot);
        ba.loss_partial = st->loss_part.p;
    }
    const long long T = vb.total_tiles;
    long long grid = persistent ? std::min<long long>(T, (long long)ctx->num_sms * st->opt.blocks_per_sm) : T;
    {
        StageTimer tm(ctx, kStBlendBwd, s);
        CK(launch_blend_bwd(ba, vb, (int)grid, s), "blend_bwd");
    }
    if (l1 && loss_device) {
        StageTimer tm(ctx, kStLoss, s);
        CK(launch_loss_final(st->loss_part.p, (int)T, loss_device, s), "loss_final");
    }

    if (det) {
        DetReduceArgs da;
        da.rec = st->rec.p; da.ext = st->ext.p; da.keys = st->keys.p; da.tile_start = st->tile_start.p;
        da.det_partial = st->det_partial.p; da.grad2d = st->grad2d.p; da.n = n;
        da.cut = st->opt.full_lists ? nullptr : st->cut.p;
        StageTimer tm(ctx, kStDetReduce, s);
        CK(launch_det_reduce(da, vb, s), "det_reduce");
    }

    ProjectBwdArgs pb;
    pb.means = st->g.means; pb.log_scales = st->g.log_scales; pb.quats = st->g.quats;
    pb.opacity_logits = st->g.opacity_logits; pb.colors = st->g.colors;
    pb.n = n; pb.sh_degree = st->g.sh_degree; pb.Tdev = st->Tdev; pb.vis_mask = st->vis_mask.p;
    pb.grad2d = st->grad2d.p;
    pb.d_means = d_means; pb.d_log_scales = d_log_scales; pb.d_quats = d_quats;
    pb.d_opacity_logits = d_opacity_logits; pb.d_colors = d_colors;
    pb.accumulate = accumulate;
    pb.twist_partial = st->twist_part.p;
    int parts = 0;
    {
        StageTimer tm(ctx, kStProjectBwd, s);
        CK(launch_project_bwd(pb, vb, &parts, s), "project_bwd");
    }
    st->grad_clean = true;

    if (d_twist) {
        if (n == 0) {
            if (!accumulate) CK(cudaMemsetAsync(d_twist, 0, (size_t)vb.n_views * 6 * sizeof(float), s), "memset twist");
        } else {
            TwistReduceArgs ta;
            ta.twist_partial = st->twist_part.p; ta.n_parts = parts; ta.n_views = vb.n_views;
            ta.d_twist = d_twist; ta.accumulate = accumulate;
            StageTimer tm(ctx, kStTwist, s);
            CK(launch_twist_reduce(ta, s), "twist_reduce");
        }
    }
    st->stream = s;
    return S3GS_OK;
}

}  // namespace

extern "C" {

s3gs_status s3gs_state_check(s3gs_ctx *ctx, s3gs_state *st, int64_t *n_duplicates, int64_t *capacity) {
    if (!ctx || !st) return fail(ctx, S3GS_E_INVALID, "state_check: null argument");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(st->ctr_host, st->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st->stream), "read counters");
    CK(cudaStreamSynchronize(st->stream), "sync");
    if (n_duplicates) *n_duplicates = (int64_t)st->ctr_host->n_dup;
    if (capacity) *capacity = st->keys.cap;
    if (st->ctr_host->overflow)
        return fail(ctx, S3GS_E_CAPACITY, "last forward produced " + std::to_string(st->ctr_host->n_dup) +
                                              " duplicates, capacity " + std::to_string(st->keys.cap));
    return S3GS_OK;
}

s3gs_status s3gs_mapping_loss(s3gs_ctx *ctx, const s3gs_camera *cams, int32_t n_views, const float *rgb,
                              const float *depth, const float *pointmap, const float *t_rgb, const float *t_depth,
                              const float *t_pointmap, const float *mask, float w_rgb, float w_depth, float w_geo,
                              float *d_rgb, float *d_depth, float *d_pointmap, float *loss_device, void *stream_) {
    if (!ctx) return S3GS_E_INVALID;
    if (!cams || n_views < 1 || n_views > S3GS_MAX_VIEWS || !loss_device)
        return fail(ctx, S3GS_E_INVALID, "mapping_loss: bad cameras or null loss pointer");
    if ((t_rgb && !rgb) || (t_depth && !depth) || (t_pointmap && !pointmap))
        return fail(ctx, S3GS_E_INVALID, "mapping_loss: a target is given without its rendered output");
    cudaStream_t s = (cudaStream_t)stream_;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    ViewBatch vb;
    s3gs_status r = plan_views(ctx, cams, n_views, 16, 16, vb);
    if (r != S3GS_OK) return r;
    LossArgs la;
    la.rgb = rgb; la.depth = depth; la.pointmap = pointmap;
    la.t_rgb = t_rgb; la.t_depth = t_depth; la.t_pointmap = t_pointmap; la.mask = mask;
    la.w_rgb = w_rgb; la.w_depth = w_depth; la.w_geo = w_geo;
    la.d_rgb = d_rgb; la.d_depth = d_depth; la.d_pointmap = d_pointmap;
    la.partial = ctx->loss_partial; la.loss = loss_device;
    {
        StageTimer tm(ctx, kStLoss, s);
        CK(launch_loss(la, vb, s), "loss");
    }
    return S3GS_OK;
}

s3gs_status s3gs_debug_records(s3gs_ctx *ctx, s3gs_state *st, int64_t n_records, float *xy, float *conic_opacity,
                               float *rgb_depth, int32_t *extent) {
    if (!ctx || !st || !st->valid) return fail(ctx, S3GS_E_STATE, "debug_records: no forward on this state");
    long long nr = st->g.n * st->vb.n_views;
    if (n_records != nr) return fail(ctx, S3GS_E_INVALID, "debug_records: n_records must be n_views * n");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(st->stream), "sync");
    if (nr == 0) return S3GS_OK;
    Record *h = (Record *)malloc(sizeof(Record) * nr);
    int2 *e = (int2 *)malloc(sizeof(int2) * nr);
    if (!h || !e) { free(h); free(e); return fail(ctx, S3GS_E_NOMEM, "debug_records: host allocation"); }
    cudaError_t err = cudaMemcpy(h, st->rec.p, sizeof(Record) * nr, cudaMemcpyDeviceToHost);
    if (err == cudaSuccess) err = cudaMemcpy(e, st->ext.p, sizeof(int2) * nr, cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) { free(h); free(e); return cuda_fail(ctx, err, "debug_records"); }
    for (long long r = 0; r < nr; ++r) {
        bool vis = e[r].x > 0;
        if (xy) { xy[2 * r] = vis ? h[r].a.x : 0.f; xy[2 * r + 1] = vis ? h[r].a.y : 0.f; }
        if (conic_opacity) {
            conic_opacity[4 * r] = vis ? h[r].a.z : 0.f; conic_opacity[4 * r + 1] = vis ? h[r].a.w : 0.f;
            conic_opacity[4 * r + 2] = vis ? h[r].b.x : 0.f; conic_opacity[4 * r + 3] = vis ? h[r].b.y : 0.f;
        }
        if (rgb_depth) {
            rgb_depth[4 * r] = vis ? h[r].c.x : 0.f; rgb_depth[4 * r + 1] = vis ? h[r].c.y : 0.f;
            rgb_depth[4 * r + 2] = vis ? h[r].c.z : 0.f; rgb_depth[4 * r + 3] = vis ? h[r].b.z : 0.f;
        }
        if (extent) { extent[2 * r] = e[r].x; extent[2 * r + 1] = e[r].y; }
    }
    free(h);
    free(e);
    return S3GS_OK;
}

s3gs_status s3gs_debug_cover(s3gs_ctx *ctx, s3gs_state *st, int64_t n_records, float *q_cover) {
    if (!ctx || !st || !st->valid) return fail(ctx, S3GS_E_STATE, "debug_cover: no forward on this state");
    long long nr = st->g.n * st->vb.n_views;
    if (n_records != nr || !q_cover) return fail(ctx, S3GS_E_INVALID, "debug_cover: n_records must be n_views * n");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(st->stream), "sync");
    if (nr == 0) return S3GS_OK;
    // the bound is the fourth float of each record's third float4 (stride 12 floats)
    CK(cudaMemcpy2D(q_cover, sizeof(float), reinterpret_cast<const char *>(st->rec.p) + 11 * sizeof(float),
                    sizeof(Record), sizeof(float), (size_t)nr, cudaMemcpyDeviceToHost),
       "debug_cover");
    int2 *e = (int2 *)malloc(sizeof(int2) * nr);
    if (!e) return fail(ctx, S3GS_E_NOMEM, "debug_cover: host allocation");
    cudaError_t err = cudaMemcpy(e, st->ext.p, sizeof(int2) * nr, cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) { free(e); return cuda_fail(ctx, err, "debug_cover"); }
    for (long long r = 0; r < nr; ++r)
        if (e[r].x <= 0) q_cover[r] = 0.f;
    free(e);
    return S3GS_OK;
}

s3gs_status s3gs_debug_binning(s3gs_ctx *ctx, s3gs_state *st, uint64_t *keys, uint32_t *values, int64_t *ranges,
                               int64_t *n_tiles, int64_t *n_dup) {
    if (!ctx || !st || !st->valid) return fail(ctx, S3GS_E_STATE, "debug_binning: no forward on this state");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(st->ctr_host, st->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st->stream), "read counters");
    CK(cudaStreamSynchronize(st->stream), "sync");
    if (st->ctr_host->overflow) return fail(ctx, S3GS_E_CAPACITY, "debug_binning: last forward overflowed");
    const long long T = st->vb.total_tiles, K = (long long)st->ctr_host->n_dup;
    if (n_tiles) *n_tiles = T;
    if (n_dup) *n_dup = K;
    if (!keys && !values && !ranges) return S3GS_OK;
    const long long NBK = T * kDepthBins;
    unsigned *bsrt = (unsigned *)malloc(sizeof(unsigned) * (NBK + 1));
    unsigned *ts = (unsigned *)malloc(sizeof(unsigned) * (T + 1));
    unsigned long long *k = (unsigned long long *)malloc(sizeof(unsigned long long) * (K > 0 ? K : 1));
    if (!ts || !k || !bsrt) {
        free(ts); free(k); free(bsrt);
        return fail(ctx, S3GS_E_NOMEM, "debug_binning: host allocation");
    }
    cudaError_t err = cudaMemcpy(bsrt, st->tile_start.p, sizeof(unsigned) * (NBK + 1), cudaMemcpyDeviceToHost);
    for (long long t = 0; t <= T; ++t) ts[t] = bsrt[t * kDepthBins];
    free(bsrt);
    if (err == cudaSuccess && K > 0) err = cudaMemcpy(k, st->keys.p, sizeof(unsigned long long) * K, cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) { free(ts); free(k); return cuda_fail(ctx, err, "debug_binning"); }
    for (long long t = 0; t < T; ++t)
        for (unsigned p = ts[t]; p < ts[t + 1]; ++p) {
            if (keys) keys[p] = ((unsigned long long)t << 32) | (k[p] >> 32);
            if (values) values[p] = (uint32_t)(k[p] & 0xffffffffull);
        }
    if (ranges)
        for (long long t = 0; t <= T; ++t) ranges[t] = ts[t];
    free(ts);
    free(k);
    return S3GS_OK;
}

s3gs_status s3gs_covisibility(s3gs_ctx *ctx, s3gs_state *st, int64_t *counts, float *iou, float *oc,
                              void *stream) {
    if (!ctx) return S3GS_E_INVALID;
    if (!st || !st->valid) return fail(ctx, S3GS_E_STATE, "covisibility: no forward on this state");
    if (!counts) return fail(ctx, S3GS_E_INVALID, "covisibility: counts is NULL");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(launch_covis(st->vis_mask.p, st->g.n, st->vb.n_views, reinterpret_cast<unsigned long long *>(counts), iou, oc,
                    ctx->num_sms, static_cast<cudaStream_t>(stream)),
       "covisibility");
    return S3GS_OK;
}

s3gs_status s3gs_set_counting(s3gs_ctx *ctx, int32_t enable) {
    if (!ctx) return S3GS_E_INVALID;
    ctx->counting = enable ? 1 : 0;
    return S3GS_OK;
}

s3gs_status s3gs_read_counters(s3gs_ctx *ctx, s3gs_state *st, int64_t *fwd_processed, int64_t *fwd_blended,
                               int64_t *bwd_processed) {
    if (!ctx || !st) return fail(ctx, S3GS_E_INVALID, "read_counters: null argument");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(st->ctr_host, st->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st->stream), "read counters");
    CK(cudaStreamSynchronize(st->stream), "sync");
    if (fwd_processed) *fwd_processed = (int64_t)st->ctr_host->fwd_processed;
    if (fwd_blended) *fwd_blended = (int64_t)st->ctr_host->fwd_blended;
    if (bwd_processed) *bwd_processed = (int64_t)st->ctr_host->bwd_processed;
    return S3GS_OK;
}

}  // extern "C"
