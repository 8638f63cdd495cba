// preprocess.cu -- EWA projection of every Gaussian (forward, K1) and the
// chain rule from screen-space gradients back to the 59 parameters (K8).
//
// Photo-SLAM (arXiv 2311.16728) Sec. 3.3, Eq. 3: alpha_i = sigma_i G(R, t,
// P_i, r_i, s_i) with G the 3D Gaussian splatting footprint, c_i the colour
// of the SH coefficients (Sec. 3.1).  Both kernels run one thread per
// Gaussian over the SoA float4 parameter planes, so every load of a warp is
// one contiguous 512-byte segment per plane.
#include "chain_impl.cuh"

namespace gsr {

__global__ void __launch_bounds__(256, 3) preprocess_fwd_kernel(GaussK g, CamK cam, float4 *__restrict__ xy_conic,
                                                             float4 *__restrict__ c_op_box,
                                                             float4 *__restrict__ rgb_depth,
                                                             uint32_t *__restrict__ ntiles,
                                                             float2 *__restrict__ uv_lo) {
    chain_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < g.n;
    Chain c;
    bool vis = false;
    Splat s{};
    if (active) {
        const float4 mo = __ldg(g.mean_op + i), q = __ldg(g.quat + i), ls = __ldg(g.logscale + i);
        vis = decide_chain(mo, q, ls, cam, c);
        if (vis) {
            if (uv_lo) uv_lo[i] = uv_residual(mo, cam, c.u, c.v);
            float A, B, C, op;
            chain_conic_opacity(c, mo.w, A, B, C, op);
            // colour: SH at the unit view direction (mean - camera centre)
            const float3 cc = cam_center(cam);
            float dx = mo.x - cc.x, dy = mo.y - cc.y, dz = mo.z - cc.z;
            const float inv_len = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= inv_len; dy *= inv_len; dz *= inv_len;
            float sh[48];
            load_sh(g.sh, g.n, i, g.deg, sh);
            float Y[16];
            sh_basis(dx, dy, dz, g.deg, Y, nullptr);
            const int nc = (g.deg + 1) * (g.deg + 1);
            float rgb[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float acc = 0.5f;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < nc) acc += sh[3 * k + ch] * Y[k];
                rgb[ch] = fmaxf(acc, 0.0f);
            }
            const uint32_t bx = (uint32_t)c.x0 | ((uint32_t)c.x1 << 16), by = (uint32_t)c.y0 | ((uint32_t)c.y1 << 16);
            xy_conic[i] = make_float4(c.u, c.v, A, B);
            c_op_box[i] = make_float4(C, op, __uint_as_float(bx), __uint_as_float(by));
            rgb_depth[i] = make_float4(rgb[0], rgb[1], rgb[2], c.zc);
            s = Splat{c.u, c.v, A, B, C, op, c.x0, c.x1, c.y0, c.y1};
        }
    }
    // tiles the pixel box touches (the tile cull runs during pair expansion)
    const uint32_t cnt =
        vis ? (uint32_t)((s.x1 / cam.tw - s.x0 / cam.tw + 1) * (s.y1 / cam.th - s.y0 / cam.th + 1)) : 0u;
    if (active) ntiles[i] = vis ? cnt : 0u;
}

template <bool kStore>
__global__ void __launch_bounds__(kBwdThreads) preprocess_bwd_kernel(GaussK g, CamK cam, const uint32_t *__restrict__ ntiles,
                                                                     const float4 *__restrict__ g0,
                                                                     const float4 *__restrict__ g1,
                                                                     const float4 *__restrict__ g2,
                                                                     float4 *__restrict__ d_mo, float4 *__restrict__ d_q,
                                                                     float4 *__restrict__ d_ls, float4 *__restrict__ d_sh,
                                                                     float *__restrict__ dstat,
                                                                     float *__restrict__ dcount) {
    chain_enter();
    __shared__ uint32_t s_idx[kBwdChunk];
    __shared__ uint32_t s_cnt;
    if (threadIdx.x == 0) s_cnt = 0u;
    __syncthreads();
    compact_visible(ntiles, g.n, s_idx, &s_cnt);
    __syncthreads();
    const uint32_t cnt = s_cnt;
    for (uint32_t k = threadIdx.x; k < cnt; k += kBwdThreads)
        chain_one_gaussian(g, cam, chunk_index(s_idx[k]), g0, g1, g2, d_mo, d_q, d_ls, d_sh, dstat, dcount, kStore);
}

// Camera pose gradient: the chain of every visible Gaussian with its
// parameter gradients discarded and its pose part summed -- per thread, then
// per warp (shuffles), per CTA (shared memory) and one atomic per value and
// CTA into d_pose.
__global__ void __launch_bounds__(kBwdThreads) pose_bwd_kernel(GaussK g, CamK cam, const uint32_t *__restrict__ ntiles,
                                                               const float4 *__restrict__ g0,
                                                               const float4 *__restrict__ g1,
                                                               const float4 *__restrict__ g2,
                                                               float *__restrict__ d_pose) {
    __shared__ uint32_t s_idx[kBwdChunk];
    __shared__ uint32_t s_cnt;
    __shared__ float s_pose[kBwdThreads / 32][kPoseGrad];
    if (threadIdx.x == 0) s_cnt = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    compact_visible(ntiles, g.n, s_idx, &s_cnt);
    __syncthreads();
    const uint32_t cnt = s_cnt;
    float pose[kPoseGrad];
#pragma unroll
    for (int k = 0; k < kPoseGrad; ++k) pose[k] = 0.f;
    NullSink sink;
    for (uint32_t k = threadIdx.x; k < cnt; k += kBwdThreads) {
        const int64_t i = chunk_index(s_idx[k]);
        const float4 mo = __ldg(g.mean_op + i), q = __ldg(g.quat + i), ls = __ldg(g.logscale + i);
        const float4 G0 = g0[i], G1 = g1[i], G2 = g2[i];
        float4 shp[kShPlanes];
        load_sh_planes(g, i, shp);
        Chain c;
        if (!decide_chain(mo, q, ls, cam, c)) continue;  // cannot happen for a visible Gaussian
        float A, B, C, sig;
        chain_conic_opacity(c, mo.w, A, B, C, sig);
        ScreenGrad sg;
        sg.du = G0.x;
        sg.dv = G0.y;
        conic_grad_to_cov(A, B, C, G0.z, G0.w, G1.x, sg.Gs00, sg.Gs01, sg.Gs11);
        sg.dop = G1.y;
        sg.dr = G1.z;
        sg.dg = G1.w;
        sg.db = G2.x;
        chain_core_to<NullSink, true>(g, cam, i, mo, c, sg, sink, pose, shp);
    }
#pragma unroll
    for (int k = 0; k < kPoseGrad; ++k) {
        float v = pose[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_pose[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kPoseGrad && cnt > 0u) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < kBwdThreads / 32; ++w) v += s_pose[w][threadIdx.x];
        atomicAdd(d_pose + threadIdx.x, v);
    }
}

}  // namespace gsr

using namespace gsr;

extern "C" int32_t gsr_preprocess(const gsr_gaussians *g, const gsr_camera *cam, const gsr_tiling *tiling,
                                  const gsr_proj *out, int32_t *d_status, gsr_stream_t stream) {
    (void)d_status;
    int32_t rc;
    if ((rc = validate_gaussians(g)) || (rc = validate_camera(cam)) || (rc = validate_tiling(tiling))) return rc;
    if (g->n == 0) return GSR_OK;
    if (!out || !out->xy_conic || !out->c_op_box || !out->rgb_depth || !out->ntiles || !aligned16(out->xy_conic) ||
        !aligned16(out->c_op_box) || !aligned16(out->rgb_depth)) {
        set_error("gsr_preprocess: output record pointers must be non-NULL and 16-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    if (out->uv_lo && (reinterpret_cast<uintptr_t>(out->uv_lo) & 7u)) {
        set_error("gsr_preprocess: uv_lo must be 8-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    const CamK ck = make_camk(cam, tiling);
    const int threads = 256;
    const int64_t blocks = (g->n + threads - 1) / threads;
    launch_chained(preprocess_fwd_kernel, dim3((unsigned)blocks), dim3(threads), 0, as_cuda(stream),
        make_gk(g), ck, reinterpret_cast<float4 *>(out->xy_conic), reinterpret_cast<float4 *>(out->c_op_box),
        reinterpret_cast<float4 *>(out->rgb_depth), out->ntiles, reinterpret_cast<float2 *>(out->uv_lo));
    return check_launch("preprocess_fwd_kernel");
}

static int32_t preprocess_bwd(const gsr_gaussians *g, const gsr_proj *proj, const gsr_camera *cam,
                              const gsr_tiling *tiling, const gsr_grad2d *g2d, const gsr_param_buffers *grads,
                              float *densify_stat, float *densify_count, bool store, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_gaussians(g)) || (rc = validate_camera(cam)) || (rc = validate_tiling(tiling))) return rc;
    if (g->n == 0) return GSR_OK;
    if (!proj || !proj->ntiles || !g2d || !g2d->g0 || !g2d->g1 || !g2d->g2 || !grads || !grads->mean_op ||
        !grads->quat || !grads->logscale || !grads->sh || (densify_stat != nullptr) != (densify_count != nullptr)) {
        set_error("preprocess_bwd: NULL pointer");
        return GSR_ERR_INVALID_ARG;
    }
    if (!aligned16(g2d->g0) || !aligned16(g2d->g1) || !aligned16(g2d->g2) || !aligned16(grads->mean_op) ||
        !aligned16(grads->quat) || !aligned16(grads->logscale) || !aligned16(grads->sh)) {
        set_error("preprocess_bwd: gradient buffers must be 16-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    const CamK ck = make_camk(cam, tiling);
    const int64_t blocks = (g->n + kBwdChunk - 1) / kBwdChunk;
    auto kernel = store ? preprocess_bwd_kernel<true> : preprocess_bwd_kernel<false>;
    launch_chained(kernel, dim3((unsigned)blocks), dim3(kBwdThreads), 0, as_cuda(stream),
        make_gk(g), ck, proj->ntiles, reinterpret_cast<const float4 *>(g2d->g0),
        reinterpret_cast<const float4 *>(g2d->g1), reinterpret_cast<const float4 *>(g2d->g2),
        reinterpret_cast<float4 *>(grads->mean_op), reinterpret_cast<float4 *>(grads->quat),
        reinterpret_cast<float4 *>(grads->logscale), reinterpret_cast<float4 *>(grads->sh), densify_stat,
        densify_count);
    return check_launch("preprocess_bwd_kernel");
}

extern "C" int32_t gsr_preprocess_bwd(const gsr_gaussians *g, const gsr_proj *proj, const gsr_camera *cam,
                                      const gsr_tiling *tiling, const gsr_grad2d *g2d,
                                      const gsr_param_buffers *grads, float *densify_stat, float *densify_count,
                                      gsr_stream_t stream) {
    return preprocess_bwd(g, proj, cam, tiling, g2d, grads, densify_stat, densify_count, false, stream);
}

extern "C" int32_t gsr_preprocess_bwd_store(const gsr_gaussians *g, const gsr_proj *proj, const gsr_camera *cam,
                                            const gsr_tiling *tiling, const gsr_grad2d *g2d,
                                            const gsr_param_buffers *grads, float *densify_stat,
                                            float *densify_count, gsr_stream_t stream) {
    return preprocess_bwd(g, proj, cam, tiling, g2d, grads, densify_stat, densify_count, true, stream);
}

extern "C" int32_t gsr_pose_bwd(const gsr_gaussians *g, const gsr_proj *proj, const gsr_camera *cam,
                                const gsr_tiling *tiling, const gsr_grad2d *g2d, float *d_pose,
                                gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_gaussians(g)) || (rc = validate_camera(cam)) || (rc = validate_tiling(tiling))) return rc;
    if (!d_pose) {
        set_error("gsr_pose_bwd: NULL d_pose");
        return GSR_ERR_INVALID_ARG;
    }
    if (g->n == 0) return GSR_OK;
    if (!proj || !proj->ntiles || !g2d || !g2d->g0 || !g2d->g1 || !g2d->g2) {
        set_error("gsr_pose_bwd: NULL pointer");
        return GSR_ERR_INVALID_ARG;
    }
    if (!aligned16(g2d->g0) || !aligned16(g2d->g1) || !aligned16(g2d->g2)) {
        set_error("gsr_pose_bwd: screen-space gradient buffers must be 16-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    const CamK ck = make_camk(cam, tiling);
    const int64_t blocks = (g->n + kBwdChunk - 1) / kBwdChunk;
    pose_bwd_kernel<<<(unsigned)blocks, kBwdThreads, 0, as_cuda(stream)>>>(
        make_gk(g), ck, proj->ntiles, reinterpret_cast<const float4 *>(g2d->g0),
        reinterpret_cast<const float4 *>(g2d->g1), reinterpret_cast<const float4 *>(g2d->g2), d_pose);
    return check_launch("pose_bwd_kernel");
}
