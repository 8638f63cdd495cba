// render.cu -- forward blend (K5) and its backward (K7) for the tile-based
// renderer of Photo-SLAM (arXiv 2311.16728) Sec. 3.3, Eq. 3:
//   C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j)      (+ T_final * bg)
// with the printed product index read as j.  One CTA per screen tile, one
// thread per pixel; the tile's depth-sorted Gaussians are staged through
// shared memory in batches of one record per thread.
#include "gsr_internal.cuh"

namespace gsr {

struct RenderArgs {
    const float4 *xy_conic, *c_op_box, *rgb_depth;
    const uint32_t *vals;
    const uint2 *ranges;
    int W, H, tw, th, gx;
    float bg0, bg1, bg2;
};

__device__ __forceinline__ void tile_pixel(const RenderArgs &a, int &px, int &py) {
    const int tile = blockIdx.x;
    const int tx = tile % a.gx, ty = tile / a.gx;
    px = tx * a.tw + (int)threadIdx.x % a.tw;
    py = ty * a.th + (int)threadIdx.x / a.tw;
}

// ---------------------------------------------------------------- K5
__global__ void __launch_bounds__(1024) render_fwd_kernel(RenderArgs a, float *__restrict__ img,
                                                          float *__restrict__ T_final,
                                                          uint32_t *__restrict__ n_contrib) {
    extern __shared__ float4 smem[];
    const int nthr = blockDim.x;
    float4 *s_xy = smem, *s_cb = smem + nthr, *s_rgb = smem + 2 * nthr;
    int px, py;
    tile_pixel(a, px, py);
    const bool inside = px < a.W && py < a.H;
    const uint2 rg = a.ranges[blockIdx.x];
    const int begin = (int)rg.x, end = (int)rg.y;
    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    for (int base = begin; base < end; base += nthr) {
        // stop the whole tile once every pixel has terminated
        if (__syncthreads_count(done) == nthr) break;
        const int idx = base + (int)threadIdx.x;
        if (idx < end) {
            const uint32_t gid = a.vals[idx];
            s_xy[threadIdx.x] = __ldg(a.xy_conic + gid);
            s_cb[threadIdx.x] = __ldg(a.c_op_box + gid);
            s_rgb[threadIdx.x] = __ldg(a.rgb_depth + gid);
        }
        __syncthreads();
        const int cnt = min(nthr, end - base);
        for (int j = 0; j < cnt; ++j) {
            // warp-ballot early termination: the warp leaves the batch as soon
            // as none of its pixels is still accumulating
            if (!__any_sync(0xffffffffu, !done)) break;
            if (done) continue;
            const float4 g = s_xy[j], cb = s_cb[j];
            if (!in_box(__float_as_uint(cb.z), __float_as_uint(cb.w), px, py)) continue;
            const float dx = (float)px - g.x, dy = (float)py - g.y;
            const float power = splat_power(g.z, g.w, cb.x, dx, dy);
            if (power > 0.0f) continue;
            const float alpha = fminf(kAlphaMax, FM(cb.y, splat_gauss(power)));
            if (alpha < kAlphaMin) continue;
            const float tn = FM(T, FS(1.0f, alpha));
            if (tn < kTMin) {
                done = true;
                continue;
            }
            const float4 c = s_rgb[j];
            const float w = alpha * T;
            C0 += c.x * w;
            C1 += c.y * w;
            C2 += c.z * w;
            T = tn;
            last = (uint32_t)(base - begin + j + 1);
        }
    }
    if (inside) {
        const int64_t pix = (int64_t)py * a.W + px, plane = (int64_t)a.W * a.H;
        img[pix] = C0 + T * a.bg0;
        img[plane + pix] = C1 + T * a.bg1;
        img[2 * plane + pix] = C2 + T * a.bg2;
        T_final[pix] = T;
        n_contrib[pix] = last;
    }
}

// ---------------------------------------------------------------- K7
// Back to front from the pixel's last contributor.  T_i = T_{i+1} / (1 -
// alpha_i) recovers the transmittance in front of each Gaussian; the colour
// behind it, normalised by T_{i+1}, follows acc <- acc (1 - alpha) + c alpha.
//   dL/dc_i     = dL/dC alpha_i T_i
//   dL/dalpha_i = T_i sum_ch dL/dC_ch (c_i,ch - acc_ch)
// then through alpha = opacity exp(power) (zero where the 0.99 clamp holds).
// The nine per-Gaussian values are summed across the warp with shuffles and
// one lane issues the atomics.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(1024) render_bwd_kernel(RenderArgs a, const float *__restrict__ T_final,
                                                          const uint32_t *__restrict__ n_contrib,
                                                          const float *__restrict__ dL_dimg,
                                                          float4 *__restrict__ g0, float4 *__restrict__ g1,
                                                          float *__restrict__ g2) {
    extern __shared__ float4 smem[];
    const int nthr = blockDim.x;
    float4 *s_xy = smem, *s_cb = smem + nthr, *s_rgb = smem + 2 * nthr;
    uint32_t *s_gid = reinterpret_cast<uint32_t *>(smem + 3 * nthr);
    __shared__ uint32_t s_max[32];
    int px, py;
    tile_pixel(a, px, py);
    const bool inside = px < a.W && py < a.H;
    const uint2 rg = a.ranges[blockIdx.x];
    const int begin = (int)rg.x;
    const int64_t pix = (int64_t)py * a.W + px, plane = (int64_t)a.W * a.H;
    float T = inside ? T_final[pix] : 0.0f;
    const uint32_t last = inside ? n_contrib[pix] : 0u;
    float dC0 = 0.f, dC1 = 0.f, dC2 = 0.f;
    if (inside) {
        dC0 = dL_dimg[pix];
        dC1 = dL_dimg[plane + pix];
        dC2 = dL_dimg[2 * plane + pix];
    }
    float acc0 = a.bg0, acc1 = a.bg1, acc2 = a.bg2;
    // block-wide max of n_contrib: positions at or beyond it are never used
    uint32_t m = __reduce_max_sync(0xffffffffu, last);
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < (unsigned)(nthr >> 5) ? s_max[threadIdx.x] : 0u;
        v = __reduce_max_sync(0xffffffffu, v);
        if (threadIdx.x == 0) s_max[0] = v;
    }
    __syncthreads();
    // never past the tile's own list, whatever n_contrib holds
    const int stop = min(begin + (int)s_max[0], (int)rg.y);
    const int lane = threadIdx.x & 31;
    for (int bend = stop; bend > begin; bend -= nthr) {
        const int bstart = max(begin, bend - nthr);
        __syncthreads();
        const int idx = bstart + (int)threadIdx.x;
        if (idx < bend) {
            const uint32_t gid = a.vals[idx];
            s_gid[threadIdx.x] = gid;
            s_xy[threadIdx.x] = __ldg(a.xy_conic + gid);
            s_cb[threadIdx.x] = __ldg(a.c_op_box + gid);
            s_rgb[threadIdx.x] = __ldg(a.rgb_depth + gid);
        }
        __syncthreads();
        for (int j = bend - 1 - bstart; j >= 0; --j) {
            const int pos = bstart + j - begin;  // 0-based position in the tile list
            float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool contrib = false;
            if (pos < (int)last) {
                const float4 g = s_xy[j], cb = s_cb[j];
                if (in_box(__float_as_uint(cb.z), __float_as_uint(cb.w), px, py)) {
                    const float dx = (float)px - g.x, dy = (float)py - g.y;
                    const float power = splat_power(g.z, g.w, cb.x, dx, dy);
                    if (power <= 0.0f) {
                        const float G = splat_gauss(power);
                        const float raw = FM(cb.y, G);
                        const float alpha = fminf(kAlphaMax, raw);
                        if (alpha >= kAlphaMin) {
                            contrib = true;
                            const float one_m = 1.0f - alpha;
                            T = __fdividef(T, one_m);  // T_i, transmittance in front of this Gaussian
                            const float4 c = s_rgb[j];
                            const float aT = alpha * T;
                            v[6] = dC0 * aT;
                            v[7] = dC1 * aT;
                            v[8] = dC2 * aT;
                            const float dalpha = T * (dC0 * (c.x - acc0) + dC1 * (c.y - acc1) + dC2 * (c.z - acc2));
                            acc0 = acc0 * one_m + c.x * alpha;
                            acc1 = acc1 * one_m + c.y * alpha;
                            acc2 = acc2 * one_m + c.z * alpha;
                            if (raw <= kAlphaMax) {
                                const float dpow = dalpha * alpha;
                                v[5] = dalpha * G;
                                v[0] = dpow * (g.z * dx + g.w * dy);
                                v[1] = dpow * (cb.x * dy + g.w * dx);
                                v[2] = -0.5f * dx * dx * dpow;
                                v[3] = -dx * dy * dpow;
                                v[4] = -0.5f * dy * dy * dpow;
                            }
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
                for (int k = 0; k < 9; ++k) v[k] = warp_sum(v[k]);
                if (lane == 0) {
                    const uint32_t gid = s_gid[j];
                    atomicAdd(g0 + gid, make_float4(v[0], v[1], v[2], v[3]));
                    atomicAdd(g1 + gid, make_float4(v[4], v[5], v[6], v[7]));
                    atomicAdd(g2 + 4 * (int64_t)gid, v[8]);
                }
            }
        }
    }
}

static RenderArgs make_args(const gsr_proj *proj, const uint32_t *vals, const uint32_t *ranges,
                            const gsr_camera *cam, const gsr_tiling *t, const float *bg) {
    RenderArgs a;
    a.xy_conic = reinterpret_cast<const float4 *>(proj->xy_conic);
    a.c_op_box = reinterpret_cast<const float4 *>(proj->c_op_box);
    a.rgb_depth = reinterpret_cast<const float4 *>(proj->rgb_depth);
    a.vals = vals;
    a.ranges = reinterpret_cast<const uint2 *>(ranges);
    a.W = cam->width;
    a.H = cam->height;
    a.tw = t->tile_w;
    a.th = t->tile_h;
    a.gx = grid_x(cam, t);
    a.bg0 = bg ? bg[0] : 0.f;
    a.bg1 = bg ? bg[1] : 0.f;
    a.bg2 = bg ? bg[2] : 0.f;
    return a;
}

int32_t launch_preprocess_bwd(const gsr_gaussians *g, const gsr_proj *proj, const gsr_camera *cam,
                              const gsr_tiling *tiling, const gsr_grad2d *g2d, const gsr_param_buffers *grads,
                              float *dstat, float *dcount, cudaStream_t stream);

}  // namespace gsr

using namespace gsr;

extern "C" int32_t gsr_render_fwd(const gsr_proj *proj, const uint32_t *vals, const uint32_t *tile_ranges,
                                  const gsr_camera *cam, const gsr_tiling *tiling, const float *bg, float *img,
                                  float *T_final, uint32_t *n_contrib, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_camera(cam)) || (rc = validate_tiling(tiling))) return rc;
    if (!proj || !proj->xy_conic || !proj->c_op_box || !proj->rgb_depth || !tile_ranges || !img || !T_final ||
        !n_contrib) {
        set_error("gsr_render_fwd: NULL pointer");
        return GSR_ERR_INVALID_ARG;
    }
    const RenderArgs a = make_args(proj, vals, tile_ranges, cam, tiling, bg);
    const int nthr = tiling->tile_w * tiling->tile_h;
    const int tiles = grid_x(cam, tiling) * grid_y(cam, tiling);
    const size_t shm = 3 * sizeof(float4) * (size_t)nthr;
    if (shm > 48 * 1024) cudaFuncSetAttribute(render_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    render_fwd_kernel<<<tiles, nthr, shm, as_cuda(stream)>>>(a, img, T_final, n_contrib);
    return check_launch("render_fwd_kernel");
}

extern "C" int32_t gsr_render_bwd(const gsr_gaussians *g, const gsr_proj *proj, const uint32_t *vals,
                                  const uint32_t *tile_ranges, const gsr_camera *cam, const gsr_tiling *tiling,
                                  const float *bg, const float *T_final, const uint32_t *n_contrib,
                                  const float *dL_dimg, const gsr_grad2d *grad2d, const gsr_param_buffers *grads,
                                  float *densify_stat, float *densify_count, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_gaussians(g)) || (rc = validate_camera(cam)) || (rc = validate_tiling(tiling))) return rc;
    if (!proj || !proj->xy_conic || !proj->c_op_box || !proj->rgb_depth || !proj->ntiles || !tile_ranges ||
        !T_final || !n_contrib || !dL_dimg || !grad2d || !grad2d->g0 || !grad2d->g1 || !grad2d->g2 || !grads ||
        !grads->mean_op || !grads->quat || !grads->logscale || !grads->sh ||
        (densify_stat != nullptr) != (densify_count != nullptr)) {
        set_error("gsr_render_bwd: NULL pointer");
        return GSR_ERR_INVALID_ARG;
    }
    if (!aligned16(grad2d->g0) || !aligned16(grad2d->g1) || !aligned16(grad2d->g2) || !aligned16(grads->mean_op) ||
        !aligned16(grads->quat) || !aligned16(grads->logscale) || !aligned16(grads->sh)) {
        set_error("gsr_render_bwd: gradient buffers must be 16-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    cudaStream_t st = as_cuda(stream);
    const size_t g2bytes = sizeof(float4) * (size_t)g->n;
    if (g->n > 0) {
        if (cudaMemsetAsync(grad2d->g0, 0, g2bytes, st) != cudaSuccess ||
            cudaMemsetAsync(grad2d->g1, 0, g2bytes, st) != cudaSuccess ||
            cudaMemsetAsync(grad2d->g2, 0, g2bytes, st) != cudaSuccess)
            return check_launch("memset grad2d");
    }
    const RenderArgs a = make_args(proj, vals, tile_ranges, cam, tiling, bg);
    const int nthr = tiling->tile_w * tiling->tile_h;
    const int tiles = grid_x(cam, tiling) * grid_y(cam, tiling);
    const size_t shm = 3 * sizeof(float4) * (size_t)nthr + sizeof(uint32_t) * (size_t)nthr;
    if (shm > 48 * 1024) cudaFuncSetAttribute(render_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    render_bwd_kernel<<<tiles, nthr, shm, st>>>(a, T_final, n_contrib, dL_dimg, reinterpret_cast<float4 *>(grad2d->g0),
                                                reinterpret_cast<float4 *>(grad2d->g1), grad2d->g2);
    if ((rc = check_launch("render_bwd_kernel"))) return rc;
    return launch_preprocess_bwd(g, proj, cam, tiling, grad2d, grads, densify_stat, densify_count, st);
}
