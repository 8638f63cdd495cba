// adam.cu -- fused optimiser step (K9) and the Gaussian-pyramid step (K10).
//
// Photo-SLAM (arXiv 2311.16728) Sec. 4.1 optimises the photorealistic map
// with plain SGD at a fixed learning rate; this is the Adam variant with one
// learning rate per parameter group.  Sec. 3.4, Eq. 5 supervises level l with
// GP^l(I_gt), built by repeated Gaussian smoothing and 2x down-sampling.
#include <math.h>

#include "gsr_internal.cuh"

namespace gsr {

struct AdamK {
    float4 *p[4];
    float4 *g[4];
    float4 *m[4];
    float4 *v[4];
    int64_t n;
    float lr_mean, lr_opacity, lr_quat, lr_scale, lr_sh;
    float b1, b2, eps;
};

// One thread per float4 of the 15 planes (mean_op, quat, logscale, sh x 12).
// With `touched` (n flags), a Gaussian whose flag is 0 has a zero gradient
// by contract: its gradient is neither read nor rewritten (a quarter of the
// step's bytes for every Gaussian no view saw).
__global__ void __launch_bounds__(256) adam_kernel(AdamK a, const int32_t *__restrict__ d_step,
                                                   const uint32_t *__restrict__ touched) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 15 * a.n) return;
    const int plane = (int)(e / a.n);
    const int64_t i = e - (int64_t)plane * a.n;
    const int which = plane < 3 ? plane : 3;
    const int64_t off = plane < 3 ? i : (int64_t)(plane - 3) * a.n + i;
    float4 lr;
    if (which == 0) lr = make_float4(a.lr_mean, a.lr_mean, a.lr_mean, a.lr_opacity);
    else if (which == 1) lr = make_float4(a.lr_quat, a.lr_quat, a.lr_quat, a.lr_quat);
    else if (which == 2) lr = make_float4(a.lr_scale, a.lr_scale, a.lr_scale, a.lr_scale);
    else lr = make_float4(a.lr_sh, a.lr_sh, a.lr_sh, a.lr_sh);
    const int t = *d_step + 1;
    // 1 - b^t = -expm1(t log1p(b - 1)): no cancellation for b near 1 (b - 1 is exact)
    const float bc1 = -expm1f((float)t * log1pf(a.b1 - 1.0f));
    const float bc2 = -expm1f((float)t * log1pf(a.b2 - 1.0f));
    const float ibc1 = 1.0f / bc1, ibc2 = 1.0f / bc2;
    float4 *pp = a.p[which] + off, *gp = a.g[which] + off, *mp = a.m[which] + off, *vp = a.v[which] + off;
    const bool live = touched == nullptr || __ldg(touched + i) != 0u;
    float4 p = *pp, m = *mp, v = *vp;
    const float4 g = live ? *gp : make_float4(0.f, 0.f, 0.f, 0.f);
#define ADAM_LANE(c)                                                       \
    m.c = a.b1 * m.c + (1.0f - a.b1) * g.c;                                \
    v.c = a.b2 * v.c + (1.0f - a.b2) * g.c * g.c;                          \
    p.c -= lr.c * (m.c * ibc1) / (sqrtf(v.c * ibc2) + a.eps);
    ADAM_LANE(x)
    ADAM_LANE(y)
    ADAM_LANE(z)
    ADAM_LANE(w)
#undef ADAM_LANE
    *pp = p;
    *mp = m;
    *vp = v;
    if (live) *gp = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void step_advance_kernel(int32_t *d_step) { *d_step += 1; }

__device__ __forceinline__ int reflect101(int i, int n) {
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * (n - 1) - i;
    }
    return i;
}

__global__ void __launch_bounds__(256) pyramid_down_kernel(const float *__restrict__ in, int C, int H, int W,
                                                           float *__restrict__ out) {
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)C * Ho * Wo) return;
    const int c = (int)(e / ((int64_t)Ho * Wo));
    const int rem = (int)(e - (int64_t)c * Ho * Wo);
    const int i = rem / Wo, j = rem % Wo;
    const float k[5] = {1.f / 16.f, 4.f / 16.f, 6.f / 16.f, 4.f / 16.f, 1.f / 16.f};
    const float *src = in + (int64_t)c * H * W;
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        const int ii = reflect101(2 * i + a - 2, H);
        float r = 0.f;
#pragma unroll
        for (int b = 0; b < 5; ++b) r += k[b] * src[(int64_t)ii * W + reflect101(2 * j + b - 2, W)];
        s += k[a] * r;
    }
    out[e] = s;
}

}  // namespace gsr

using namespace gsr;

static int32_t adam_step(const gsr_param_buffers *params, const gsr_param_buffers *grads,
                         const gsr_param_buffers *m, const gsr_param_buffers *v, int64_t n,
                         const gsr_adam_config *cfg, const uint32_t *touched, int32_t *d_step, gsr_stream_t stream) {
    const gsr_param_buffers *bufs[4] = {params, grads, m, v};
    if (!cfg || !d_step || n < 0) {
        set_error("gsr_adam_step: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    for (const gsr_param_buffers *b : bufs) {
        if (!b || !b->mean_op || !b->quat || !b->logscale || !b->sh || !aligned16(b->mean_op) || !aligned16(b->quat) ||
            !aligned16(b->logscale) || !aligned16(b->sh)) {
            set_error("gsr_adam_step: every buffer must be non-NULL and 16-byte aligned");
            return GSR_ERR_INVALID_ARG;
        }
    }
    if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps >= 0.f)) {
        set_error("gsr_adam_step: betas must lie in [0, 1) and eps >= 0");
        return GSR_ERR_INVALID_ARG;
    }
    cudaStream_t st = as_cuda(stream);
    if (n > 0) {
        AdamK a;
        float4 **dst[4] = {a.p, a.g, a.m, a.v};
        for (int k = 0; k < 4; ++k) {
            dst[k][0] = reinterpret_cast<float4 *>(bufs[k]->mean_op);
            dst[k][1] = reinterpret_cast<float4 *>(bufs[k]->quat);
            dst[k][2] = reinterpret_cast<float4 *>(bufs[k]->logscale);
            dst[k][3] = reinterpret_cast<float4 *>(bufs[k]->sh);
        }
        a.n = n;
        a.lr_mean = cfg->lr_mean; a.lr_opacity = cfg->lr_opacity; a.lr_quat = cfg->lr_quat;
        a.lr_scale = cfg->lr_scale; a.lr_sh = cfg->lr_sh;
        a.b1 = cfg->beta1; a.b2 = cfg->beta2; a.eps = cfg->eps;
        const int64_t total = 15 * n;
        adam_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a, d_step, touched);
    }
    step_advance_kernel<<<1, 1, 0, st>>>(d_step);
    return check_launch("adam_kernel");
}

extern "C" int32_t gsr_adam_step(const gsr_param_buffers *params, const gsr_param_buffers *grads,
                                 const gsr_param_buffers *m, const gsr_param_buffers *v, int64_t n,
                                 const gsr_adam_config *cfg, int32_t *d_step, gsr_stream_t stream) {
    return adam_step(params, grads, m, v, n, cfg, nullptr, d_step, stream);
}

extern "C" int32_t gsr_adam_step_touched(const gsr_param_buffers *params, const gsr_param_buffers *grads,
                                         const gsr_param_buffers *m, const gsr_param_buffers *v, int64_t n,
                                         const gsr_adam_config *cfg, const uint32_t *touched, int32_t *d_step,
                                         gsr_stream_t stream) {
    if (!touched && n > 0) {
        set_error("gsr_adam_step_touched: NULL flags");
        return GSR_ERR_INVALID_ARG;
    }
    return adam_step(params, grads, m, v, n, cfg, touched, d_step, stream);
}

extern "C" int32_t gsr_pyramid_down(const float *in, int32_t C, int32_t H, int32_t W, float *out,
                                    gsr_stream_t stream) {
    if (!in || !out || C <= 0 || H <= 0 || W <= 0) {
        set_error("gsr_pyramid_down: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    const int64_t total = (int64_t)C * ((H + 1) / 2) * ((W + 1) / 2);
    pyramid_down_kernel<<<(unsigned)((total + 255) / 256), 256, 0, as_cuda(stream)>>>(in, C, H, W, out);
    return check_launch("pyramid_down_kernel");
}
