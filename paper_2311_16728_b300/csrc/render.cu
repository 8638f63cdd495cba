// render.cu -- forward blend (K5) and its backward (K7) for the tile-based
// renderer of Photo-SLAM (arXiv 2311.16728) Sec. 3.3, Eq. 3:
//   C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j)      (+ T_final * bg)
// with the printed product index read as j.
//
// One CTA per screen tile; each thread owns two vertically adjacent pixels
// (same column, so the x terms of the exponent are shared); the backward of
// 16 x 16 tiles gives each thread four (render_q4.cuh).  The tile's
// depth-sorted Gaussians are staged through shared memory one record per
// thread per batch; while staging, each record gets a bit mask of the warps
// whose pixel rectangle can see it at all (pixel box intersected with the
// bounding box of its alpha >= 1/255 ellipse, conservatively widened), and
// each warp then visits only its set bits.  For 16 x 16 tiles at the default
// staging depth (0) every warp stages for itself instead (render_warp.cuh:
// no block-wide barrier between the warps of a tile).  The per-pixel decisions (box,
// exponent sign, 1/255 skip, 0.99 clamp, 1e-4 stop) are evaluated with the
// same instructions in both kernels, so the backward replays exactly the
// forward's choices.
#include "render_impl.cuh"
#include "render_q4.cuh"
#include "render_warp.cuh"

namespace gsr {

// kCount: also write the per-pixel number of blended Gaussians (a work
// counter); without it the counting is compiled out
// kQuad: 16 x 16 tiles (quadrant warps, box tests from staged lane masks)
// The tile CTA b renders: order[b] when the binning wrote the heavy-first
// tile order (gsr_proj.tile_order), else b; -1 for an entry outside the view.
__device__ __forceinline__ int cta_tile(const uint32_t *__restrict__ order) {
    if (!order) return (int)blockIdx.x;
    const uint32_t t = __ldg(order + blockIdx.x);
    return t < gridDim.x ? (int)t : -1;
}

template <bool kCount, bool kQuad>
__global__ void __launch_bounds__(512) render_fwd_kernel(RenderArgs a, const uint32_t *__restrict__ order,
                                                         float *__restrict__ img, float *__restrict__ T_final,
                                                         uint32_t *__restrict__ n_contrib,
                                                         uint32_t *__restrict__ n_blended,
                                                         uint32_t *__restrict__ tile_work) {
    extern __shared__ float4 smem[];
    const int tile = cta_tile(order);
    if (tile < 0) return;
    render_fwd_tile<kQuad>(a, tile, img, T_final, n_contrib, kCount ? n_blended : nullptr, smem, tile_work);
}

// The backward's tile order: tiles by decreasing tile_work (the depth of
// list each walks), a counting sort on 8-entry classes by one CTA.
constexpr int kWorkOrderThreads = 1024, kWorkClasses = 128;
__global__ void __launch_bounds__(kWorkOrderThreads) work_order_kernel(const uint32_t *__restrict__ work, uint32_t T,
                                                                       uint32_t *__restrict__ order) {
    chain_enter();
    constexpr uint32_t kPer = 4;  // tiles a thread keeps in registers between the two passes
    __shared__ uint32_t s_cls[kWorkClasses];
    for (int c = threadIdx.x; c < kWorkClasses; c += kWorkOrderThreads) s_cls[c] = 0u;
    __syncthreads();
    const bool regs = T <= kWorkOrderThreads * kPer;
    uint32_t cls[kPer];
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
        const uint32_t t = threadIdx.x + k * kWorkOrderThreads;
        cls[k] = t < T ? min((__ldg(work + t) + 7u) >> 3, (uint32_t)kWorkClasses - 1u) : 0u;
    }
    if (regs) {
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k)
            if (threadIdx.x + k * kWorkOrderThreads < T) atomicAdd(&s_cls[cls[k]], 1u);
    } else {
        for (uint32_t t = threadIdx.x; t < T; t += kWorkOrderThreads)
            atomicAdd(&s_cls[min((work[t] + 7u) >> 3, (uint32_t)kWorkClasses - 1u)], 1u);
    }
    __syncthreads();
    desc_class_bases<kWorkClasses>(s_cls);
    __syncthreads();
    if (regs) {
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k) {
            const uint32_t t = threadIdx.x + k * kWorkOrderThreads;
            if (t < T) order[atomicAdd(&s_cls[cls[k]], 1u)] = t;
        }
        return;
    }
    for (uint32_t t = threadIdx.x; t < T; t += kWorkOrderThreads)
        order[atomicAdd(&s_cls[min((work[t] + 7u) >> 3, (uint32_t)kWorkClasses - 1u)], 1u)] = t;
}

template <bool kQuad>
__global__ void __maxnreg__(80) render_bwd_kernel(RenderArgs a, const uint32_t *__restrict__ order,
                                                  const float *__restrict__ T_final,
                                                  const uint32_t *__restrict__ n_contrib,
                                                  const float *__restrict__ dL_dimg, float *__restrict__ g0,
                                                  float *__restrict__ g1, float *__restrict__ g2) {
    extern __shared__ float4 smem[];
    const int tile = cta_tile(order);
    if (tile < 0) return;
    render_bwd_tile<kQuad>(a, tile, T_final, n_contrib, dL_dimg, g0, g1, g2, smem);
}

// 16 x 16 tiles: the backward with four pixels per thread (render_q4.cuh)
__global__ void __launch_bounds__(kQ4Threads) render_bwd_q4_kernel(RenderArgs a, const uint32_t *__restrict__ order,
                                                                   const float *__restrict__ T_final,
                                                                   const uint32_t *__restrict__ n_contrib,
                                                                   const float *__restrict__ dL_dimg,
                                                                   float *__restrict__ g0, float *__restrict__ g1,
                                                                   float *__restrict__ g2) {
    extern __shared__ float4 smem[];
    const int tile = cta_tile(order);
    if (tile < 0) return;
    render_bwd_tile_q4<false, true>(a, tile, T_final, n_contrib, dL_dimg, g0, g1, g2, smem);
}

// 16 x 16 tiles with warp-private staging (render_warp.cuh), one warp per
// CTA: CTA b renders warp part b % P of tile order[b / P] (P = 4 quadrants
// forward, 2 halves backward), so the parts of the heaviest tiles start first.
__device__ __forceinline__ int cta_tile_part(const uint32_t *__restrict__ order, int parts, int &part) {
    const int b = (int)blockIdx.x / parts, nt = (int)gridDim.x / parts;
    part = (int)blockIdx.x - b * parts;
    if (!order) return b;
    const uint32_t t = __ldg(order + b);
    return t < (uint32_t)nt ? (int)t : -1;
}

template <bool kCount>
__global__ void __launch_bounds__(32) render_fwd_warp_kernel(RenderArgs a, const uint32_t *__restrict__ order,
                                                             float *__restrict__ img, float *__restrict__ T_final,
                                                             uint32_t *__restrict__ n_contrib,
                                                             uint32_t *__restrict__ n_blended,
                                                             uint32_t *__restrict__ tile_work) {
    chain_enter();
    __shared__ Staged s_buf[32];
    int part;
    const int tile = cta_tile_part(order, 4, part);
    if (tile < 0) return;
    render_fwd_quadrant<kCount>(a, tile, part, img, T_final, n_contrib, n_blended, s_buf, tile_work);
}

__global__ void __launch_bounds__(32) render_bwd_warp_kernel(RenderArgs a, const uint32_t *__restrict__ order,
                                                             const float *__restrict__ T_final,
                                                             const uint32_t *__restrict__ n_contrib,
                                                             const float *__restrict__ dL_dimg,
                                                             float *__restrict__ g0, float *__restrict__ g1,
                                                             float *__restrict__ g2) {
    chain_enter();
    __shared__ Staged s_buf[32];
    int part;
    const int tile = cta_tile_part(order, 2, part);
    if (tile < 0) return;
    render_bwd_tile_warp(a, tile, part, T_final, n_contrib, dL_dimg, g0, g1, g2, s_buf);
}

static RenderArgs make_args(const gsr_proj *proj, const uint32_t *vals, const uint32_t *ranges,
                            const gsr_camera *cam, const gsr_tiling *t, const float *bg) {
    RenderArgs a;
    a.xy_conic = reinterpret_cast<const float4 *>(proj->xy_conic);
    a.c_op_box = reinterpret_cast<const float4 *>(proj->c_op_box);
    a.rgb_depth = reinterpret_cast<const float4 *>(proj->rgb_depth);
    a.uv_lo = reinterpret_cast<const float2 *>(proj->uv_lo);
    a.vals = vals;
    a.ranges = reinterpret_cast<const uint2 *>(ranges);
    a.W = cam->width;
    a.H = cam->height;
    a.tw = t->tile_w;
    a.th = t->tile_h;
    a.gx = grid_x(cam, t);
    a.tile_off = 0;
    a.depth = t->batch_depth;
    a.bg0 = bg ? bg[0] : 0.f;
    a.bg1 = bg ? bg[1] : 0.f;
    a.bg2 = bg ? bg[2] : 0.f;
    return a;
}

}  // namespace gsr

using namespace gsr;

extern "C" int32_t gsr_render_fwd(const gsr_proj *proj, const uint32_t *vals, const uint32_t *tile_ranges,
                                  const gsr_camera *cam, const gsr_tiling *tiling, const float *bg, float *img,
                                  float *T_final, uint32_t *n_contrib, uint32_t *n_blended, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_camera(cam)) || (rc = validate_tiling(tiling))) return rc;
    if (!proj || !proj->xy_conic || !proj->c_op_box || !proj->rgb_depth || !tile_ranges || !img || !T_final ||
        !n_contrib) {
        set_error("gsr_render_fwd: NULL pointer");
        return GSR_ERR_INVALID_ARG;
    }
    const RenderArgs a = make_args(proj, vals, tile_ranges, cam, tiling, bg);
    const int nthr = tiling->tile_w * tiling->tile_h / 2;
    const int depth = a.depth > 0 ? a.depth : nthr;
    const int tiles = grid_x(cam, tiling) * grid_y(cam, tiling);
    const bool quad = tiling->tile_w == 16 && tiling->tile_h == 16;
    if (quad && a.depth == 0) {  // warp-private staging (the default for 16 x 16 tiles)
        auto wk = n_blended ? render_fwd_warp_kernel<true> : render_fwd_warp_kernel<false>;
        launch_chained(wk, dim3(4 * tiles), dim3(32), 0, as_cuda(stream), a, proj->tile_order, img, T_final,
                       n_contrib, n_blended, proj->tile_order ? proj->tile_work : nullptr);
        return check_launch("render_fwd_warp_kernel");
    }
    auto kernel = n_blended ? (quad ? render_fwd_kernel<true, true> : render_fwd_kernel<true, false>)
                            : (quad ? render_fwd_kernel<false, true> : render_fwd_kernel<false, false>);
    // (per device and cheap, not a stream operation: fine during capture)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)render_fwd_smem(depth));
    kernel<<<tiles, nthr, render_fwd_smem(depth), as_cuda(stream)>>>(
        a, proj->tile_order, img, T_final, n_contrib, n_blended, proj->tile_order ? proj->tile_work : nullptr);
    return check_launch("render_fwd_kernel");
}

extern "C" int32_t gsr_blend_bwd(const gsr_proj *proj, int64_t n, const uint32_t *vals, const uint32_t *tile_ranges,
                                 const gsr_camera *cam, const gsr_tiling *tiling, const float *bg,
                                 const float *T_final, const uint32_t *n_contrib, const float *dL_dimg,
                                 const gsr_grad2d *grad2d, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_camera(cam)) || (rc = validate_tiling(tiling))) return rc;
    if (n < 0 || !proj || (n > 0 && (!proj->xy_conic || !proj->c_op_box || !proj->rgb_depth)) || !tile_ranges ||
        !T_final || !n_contrib || !dL_dimg || !grad2d || !grad2d->g0 || !grad2d->g1 || !grad2d->g2) {
        set_error("gsr_blend_bwd: NULL pointer or negative count");
        return GSR_ERR_INVALID_ARG;
    }
    if (!aligned16(grad2d->g0) || !aligned16(grad2d->g1) || !aligned16(grad2d->g2)) {
        set_error("gsr_blend_bwd: screen-space gradient planes must be 16-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    cudaStream_t st = as_cuda(stream);
    const size_t g2bytes = sizeof(float4) * (size_t)n;
    const char *b0 = reinterpret_cast<const char *>(grad2d->g0);
    if (n > 0 && reinterpret_cast<const char *>(grad2d->g1) == b0 + g2bytes &&
        reinterpret_cast<const char *>(grad2d->g2) == b0 + 2 * g2bytes) {  // one contiguous block: one memset
        if (cudaMemsetAsync(grad2d->g0, 0, 3 * g2bytes, st) != cudaSuccess) return check_launch("memset grad2d");
    } else if (n > 0) {
        if (cudaMemsetAsync(grad2d->g0, 0, g2bytes, st) != cudaSuccess ||
            cudaMemsetAsync(grad2d->g1, 0, g2bytes, st) != cudaSuccess ||
            cudaMemsetAsync(grad2d->g2, 0, g2bytes, st) != cudaSuccess)
            return check_launch("memset grad2d");
    }
    const RenderArgs a = make_args(proj, vals, tile_ranges, cam, tiling, bg);
    const int nthr = tiling->tile_w * tiling->tile_h / 2;
    const int tiles = grid_x(cam, tiling) * grid_y(cam, tiling);
    const bool quad = tiling->tile_w == 16 && tiling->tile_h == 16;
    if (proj->tile_order && proj->tile_work) {  // deepest lists first (what the forward measured)
        launch_chained(work_order_kernel, dim3(1), dim3(kWorkOrderThreads), 0, st, proj->tile_work, (uint32_t)tiles,
                       proj->tile_order);
        if ((rc = check_launch("work_order_kernel"))) return rc;
    }
    if (quad && tiling->bwd_threads != nthr && a.depth == 0) {  // warp-private staging, four pixels a thread
        launch_chained(render_bwd_warp_kernel, dim3(2 * tiles), dim3(32), 0, st, a, proj->tile_order, T_final,
                       n_contrib, dL_dimg, grad2d->g0, grad2d->g1, grad2d->g2);
        return check_launch("render_bwd_warp_kernel");
    }
    if (quad && tiling->bwd_threads != nthr) {  // 64 threads, four pixels each, block-staged batches
        const int depth = a.depth;
        cudaFuncSetAttribute(render_bwd_q4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)render_q4_smem(depth));
        render_bwd_q4_kernel<<<tiles, kQ4Threads, render_q4_smem(depth), st>>>(
            a, proj->tile_order, T_final, n_contrib, dL_dimg, grad2d->g0, grad2d->g1, grad2d->g2);
        return check_launch("render_bwd_q4_kernel");
    }
    const int depth = a.depth > 0 ? a.depth : nthr;
    auto kernel = quad ? render_bwd_kernel<true> : render_bwd_kernel<false>;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)render_bwd_smem(depth));
    kernel<<<tiles, nthr, render_bwd_smem(depth), st>>>(a, proj->tile_order, T_final, n_contrib, dL_dimg, grad2d->g0,
                                                        grad2d->g1, grad2d->g2);
    return check_launch("render_bwd_kernel");
}

extern "C" int32_t gsr_render_bwd(const gsr_gaussians *g, const gsr_proj *proj, const uint32_t *vals,
                                  const uint32_t *tile_ranges, const gsr_camera *cam, const gsr_tiling *tiling,
                                  const float *bg, const float *T_final, const uint32_t *n_contrib,
                                  const float *dL_dimg, const gsr_grad2d *grad2d, const gsr_param_buffers *grads,
                                  float *densify_stat, float *densify_count, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_gaussians(g))) return rc;
    if ((rc = gsr_blend_bwd(proj, g->n, vals, tile_ranges, cam, tiling, bg, T_final, n_contrib, dL_dimg, grad2d,
                            stream)))
        return rc;
    return gsr_preprocess_bwd(g, proj, cam, tiling, grad2d, grads, densify_stat, densify_count, stream);
}
