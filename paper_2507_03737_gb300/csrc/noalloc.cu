// An allocation-free variant of the mapping loss (s3gs_mapping_loss_noalloc).
//
// The regular s3gs_mapping_loss keeps its per-block partial sums in a buffer
// that s3gs_create allocates with cudaMalloc. Some callers cannot allocate
// device memory at all: code that runs while a stream is being captured into a
// CUDA graph in the default (global) capture mode, where cudaMalloc is not
// allowed; hosts whose device memory is owned entirely by a pooling allocator
// or a fixed budget, where an extra allocation by a library may fail or
// fragment memory; and latency-critical tracking loops that cannot accept the
// implicit device synchronisation that cudaMalloc/cudaFree may cause. For them
// the partial sums live in the fixed array below instead.
//
// The array is a file-scope static device variable: every GPU that loads this
// library holds its 8 KB until the process exits. Host code must never pass
// the array's name to a kernel (on the host it is only a stand-in for the
// symbol); its device address is obtained once per device with
// cudaGetSymbolAddress and cached for the life of the process. A cached address is
// valid only while the device's context lives: after cudaDeviceReset the module may
// load at another address, so a caller that resets a device must not call this entry
// point on it again.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "s3gs_internal.cuh"

namespace {

// Capacity of the static scratch: 64 partial sums per view for up to
// S3GS_MAX_VIEWS views.
constexpr int kNoAllocMaxPartials = 64 * S3GS_MAX_VIEWS;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) float g_loss_partials[kNoAllocMaxPartials];

std::mutex g_setup_mu;
float *g_partials_ptr[kNoAllocMaxDevices] = {};

void put_error(char *buf, size_t len, const char *msg) {
    if (buf && len > 0) snprintf(buf, len, "%s", msg);
}

// Device address of g_loss_partials on the current device (set-up on first use). The
// set-up may load the module, which must not happen inside a stream capture: a first call
// on a capturing stream is refused (*capturing = true) and leaves the capture untouched.
cudaError_t partials_address(int device, cudaStream_t stream, float **out, bool *capturing) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    *capturing = false;
    if (!g_partials_ptr[device]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t ce = cudaStreamIsCapturing(stream, &cs);
        if (ce != cudaSuccess) return ce;
        if (cs != cudaStreamCaptureStatusNone) {
            *capturing = true;
            return cudaSuccess;
        }
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_loss_partials);
        if (e != cudaSuccess) return e;
        g_partials_ptr[device] = static_cast<float *>(p);
    }
    *out = g_partials_ptr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" s3gs_status s3gs_mapping_loss_noalloc(const s3gs_camera *cams, int32_t n_views, const float *rgb,
                                                 const float *depth, const float *pointmap, const float *t_rgb,
                                                 const float *t_depth, const float *t_pointmap, const float *mask,
                                                 float w_rgb, float w_depth, float w_geo, float *d_rgb,
                                                 float *d_depth, float *d_pointmap, float *loss_device,
                                                 void *stream, char *err, size_t err_len) {
    using namespace s3gs;
    if (!cams || !loss_device) {
        put_error(err, err_len, "mapping_loss_noalloc: null cameras or loss pointer");
        return S3GS_E_INVALID;
    }
    if (n_views < 1) {
        put_error(err, err_len, "mapping_loss_noalloc: n_views must be at least 1");
        return S3GS_E_INVALID;
    }
    const long long needed = (long long)loss_blocks_per_view() * n_views;
    if (n_views > S3GS_MAX_VIEWS || needed > kNoAllocMaxPartials) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "mapping_loss_noalloc: %d views need %lld partial sums; the static scratch holds %d "
                 "(at most %d views)", (int)n_views, needed, kNoAllocMaxPartials, S3GS_MAX_VIEWS);
        put_error(err, err_len, msg);
        return S3GS_E_INVALID;
    }
    if ((t_rgb && !rgb) || (t_depth && !depth) || (t_pointmap && !pointmap)) {
        put_error(err, err_len, "mapping_loss_noalloc: a target is given without its rendered output");
        return S3GS_E_INVALID;
    }
    ViewBatch vb;
    memset(&vb, 0, sizeof(vb));
    vb.n_views = n_views;
    long long pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const s3gs_camera &c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > (1 << 16) || c.height > (1 << 16)) {
            put_error(err, err_len, "mapping_loss_noalloc: camera width/height out of range");
            return S3GS_E_INVALID;
        }
        vb.v[v].w = c.width;
        vb.v[v].h = c.height;
        vb.v[v].pix_base = pix;
        pix += (long long)c.width * c.height;
    }
    vb.total_pixels = pix;

    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess && (device < 0 || device >= kNoAllocMaxDevices)) {
        put_error(err, err_len, "mapping_loss_noalloc: device index beyond the supported range");
        return S3GS_E_INVALID;
    }
    float *partials = nullptr;
    bool capturing = false;
    if (e == cudaSuccess) e = partials_address(device, static_cast<cudaStream_t>(stream), &partials, &capturing);
    if (e == cudaSuccess && capturing) {
        put_error(err, err_len, "mapping_loss_noalloc: the first call on a device sets up the scratch address and "
                                "must not be made while its stream is being captured; call it once before capture");
        return S3GS_E_INVALID;
    }
    if (e == cudaSuccess) {
        LossArgs la;
        la.rgb = rgb; la.depth = depth; la.pointmap = pointmap;
        la.t_rgb = t_rgb; la.t_depth = t_depth; la.t_pointmap = t_pointmap; la.mask = mask;
        la.w_rgb = w_rgb; la.w_depth = w_depth; la.w_geo = w_geo;
        la.d_rgb = d_rgb; la.d_depth = d_depth; la.d_pointmap = d_pointmap;
        la.partial = partials;  // every partial is written before the final sum reads it
        la.loss = loss_device;
        e = launch_loss(la, vb, static_cast<cudaStream_t>(stream));
    }
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "mapping_loss_noalloc: %s (%s)", cudaGetErrorName(e), cudaGetErrorString(e));
        put_error(err, err_len, msg);
        return S3GS_E_CUDA;
    }
    return S3GS_OK;
}
