// api.cu -- host-side library facts, argument validation and error text.
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "tma.cuh"

namespace gsr {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

int32_t check_launch(const char *what) {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return GSR_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return GSR_ERR_CUDA;
}

int32_t validate_gaussians(const gsr_gaussians *g) {
    if (!g || g->n < 0 || (g->n > 0 && (!g->mean_op || !g->quat || !g->logscale || !g->sh))) {
        set_error("gaussians: NULL pointer or negative count");
        return GSR_ERR_INVALID_ARG;
    }
    if (g->sh_degree < 0 || g->sh_degree > 3) {
        set_error("gaussians: sh_degree must be 0..3 (got %d)", g->sh_degree);
        return GSR_ERR_INVALID_ARG;
    }
    if (!aligned16(g->mean_op) || !aligned16(g->quat) || !aligned16(g->logscale) || !aligned16(g->sh)) {
        set_error("gaussians: parameter planes must be 16-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    if (g->n > 0x7fffffffLL) {
        set_error("gaussians: more than 2^31 - 1 Gaussians");
        return GSR_ERR_UNSUPPORTED;
    }
    return GSR_OK;
}

int32_t validate_camera(const gsr_camera *c) {
    if (!c || c->width <= 0 || c->height <= 0 || c->width > 65535 || c->height > 65535 || !(c->fx > 0.f) ||
        !(c->fy > 0.f)) {
        set_error("camera: need 0 < width, height <= 65535 and fx, fy > 0");
        return GSR_ERR_INVALID_ARG;
    }
    return GSR_OK;
}

int32_t validate_tiling(const gsr_tiling *t) {
    // two pixels per thread (rows 2k, 2k + 1) and whole thread rows per warp
    if (!t || t->tile_w <= 0 || t->tile_h <= 0 || t->tile_w * t->tile_h > 1024 || (t->tile_w * t->tile_h) % 64 != 0 ||
        t->tile_h % 2 != 0 || (t->tile_w % 32 != 0 && 32 % t->tile_w != 0)) {
        set_error("tiling: need tile_h even, tile_w dividing 32 or a multiple of 32, and tile_w * tile_h a multiple "
                  "of 64, at most 1024");
        return GSR_ERR_INVALID_ARG;
    }
    if (t->batch_depth < 0 || t->batch_depth > 512 || t->batch_depth % 32 != 0) {
        set_error("tiling: batch_depth must be 0 or a multiple of 32 up to 512");
        return GSR_ERR_INVALID_ARG;
    }
    const int half = t->tile_w * t->tile_h / 2;
    const bool q16 = t->tile_w == 16 && t->tile_h == 16;
    if (!(t->bwd_threads == 0 || t->bwd_threads == half || (q16 && t->bwd_threads == 64))) {
        set_error("tiling: bwd_threads must be 0, tile_w * tile_h / 2, or 64 for 16 x 16 tiles");
        return GSR_ERR_INVALID_ARG;
    }
    return GSR_OK;
}

}  // namespace gsr

using namespace gsr;

extern "C" const char *gsr_version(void) { return "gsr 0.1 sm_103a"; }

extern "C" const char *gsr_last_error(void) { return g_err; }

extern "C" int32_t gsr_status_read(const int32_t *d_status, int32_t *h_status, gsr_stream_t stream) {
    if (!d_status || !h_status) {
        set_error("gsr_status_read: NULL pointer");
        return GSR_ERR_INVALID_ARG;
    }
    cudaStream_t st = as_cuda(stream);
    if (cudaMemcpyAsync(h_status, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return check_launch("gsr_status_read");
    return GSR_OK;
}

extern "C" int32_t gsr_camera_at_level(const gsr_camera *in, int32_t level, gsr_camera *out) {
    if (!in || !out || level < 0 || level > 15) {
        set_error("gsr_camera_at_level: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    gsr_camera c = *in;
    const float s = (float)(1 << level);
    c.fx = in->fx / s;
    c.fy = in->fy / s;
    c.cx = in->cx / s;
    c.cy = in->cy / s;
    for (int l = 0; l < level; ++l) {
        c.width = (c.width + 1) / 2;
        c.height = (c.height + 1) / 2;
    }
    *out = c;
    return GSR_OK;
}
