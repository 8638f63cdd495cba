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

// blockIdx.y is the plane (mean_op, quat, logscale, sh x 12); each thread
// updates the float4 of two Gaussians (i and i + 256), loading both before
// computing.  The bias corrections are computed once per block.  With
// `touched` (n flags), a Gaussian whose flag is 0 has a zero gradient by
// contract: its gradient is neither read nor rewritten (a quarter of the
// step's bytes for every Gaussian no view saw).
constexpr int kAdamThreads = 256;
constexpr int kAdamPer = 2;

__device__ __forceinline__ float adam_delta(float lr, float m, float v, float ibc1, float ibc2, float eps) {
    // lr m_hat / (sqrt(v_hat) + eps), with sqrt(x) = x rsqrt(x) (x > 0) and a
    // fast reciprocal: relative error a few 1e-7 on the update
    const float vh = v * ibc2;
    const float root = vh > 0.0f ? vh * rsqrtf(vh) : 0.0f;
    return __fdividef(lr * (m * ibc1), root + eps);
}

__global__ void __launch_bounds__(kAdamThreads) adam_kernel(AdamK a, const int32_t *__restrict__ d_step,
                                                            const uint32_t *__restrict__ touched) {
    chain_enter();
    __shared__ float s_bc[2];
    if (threadIdx.x == 0) {
        const int t = *d_step + 1;
        // 1 - b^t = -expm1(t log1p(b - 1)): no cancellation for b near 1 (b - 1 is exact)
        s_bc[0] = 1.0f / -expm1f((float)t * log1pf(a.b1 - 1.0f));
        s_bc[1] = 1.0f / -expm1f((float)t * log1pf(a.b2 - 1.0f));
    }
    __syncthreads();
    const int plane = (int)blockIdx.y;
    const int which = plane < 3 ? plane : 3;
    float4 lr;
    if (which == 0) lr = make_float4(a.lr_mean, a.lr_mean, a.lr_mean, a.lr_opacity);
    else if (which == 1) lr = make_float4(a.lr_quat, a.lr_quat, a.lr_quat, a.lr_quat);
    else if (which == 2) lr = make_float4(a.lr_scale, a.lr_scale, a.lr_scale, a.lr_scale);
    else lr = make_float4(a.lr_sh, a.lr_sh, a.lr_sh, a.lr_sh);
    const float ibc1 = s_bc[0], ibc2 = s_bc[1], b1 = a.b1, b2 = a.b2, eps = a.eps;
    const int64_t plane_off = plane < 3 ? 0 : (int64_t)(plane - 3) * a.n;
    float4 *const P = a.p[which] + plane_off, *const G = a.g[which] + plane_off, *const M = a.m[which] + plane_off,
                  *const V = a.v[which] + plane_off;
    const int64_t i0 = (int64_t)blockIdx.x * (kAdamThreads * kAdamPer) + threadIdx.x;
    float4 p[kAdamPer], g[kAdamPer], m[kAdamPer], v[kAdamPer];
    bool in[kAdamPer], live[kAdamPer];
#pragma unroll
    for (int r = 0; r < kAdamPer; ++r) {
        const int64_t i = i0 + r * kAdamThreads;
        in[r] = i < a.n;
        live[r] = in[r] && (touched == nullptr || __ldg(touched + i) != 0u);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        p[r] = in[r] ? P[i] : z;
        m[r] = in[r] ? M[i] : z;
        v[r] = in[r] ? V[i] : z;
        g[r] = live[r] ? G[i] : z;
    }
#pragma unroll
    for (int r = 0; r < kAdamPer; ++r) {
        if (!in[r]) continue;
        const int64_t i = i0 + r * kAdamThreads;
#define ADAM_LANE(c)                                             \
    m[r].c = b1 * m[r].c + (1.0f - b1) * g[r].c;                 \
    v[r].c = b2 * v[r].c + (1.0f - b2) * g[r].c * g[r].c;        \
    p[r].c -= adam_delta(lr.c, m[r].c, v[r].c, ibc1, ibc2, eps);
        ADAM_LANE(x)
        ADAM_LANE(y)
        ADAM_LANE(z)
        ADAM_LANE(w)
#undef ADAM_LANE
        P[i] = p[r];
        M[i] = m[r];
        V[i] = v[r];
        if (live[r]) G[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void step_advance_kernel(int32_t *d_step) {
    chain_enter();
    *d_step += 1;
}

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
        launch_chained(adam_kernel, dim3((unsigned)((n + kAdamThreads * kAdamPer - 1) / (kAdamThreads * kAdamPer)), 15),
                       dim3(kAdamThreads), 0, st, a, d_step, touched);
    }
    launch_chained(step_advance_kernel, dim3(1), dim3(1), 0, st, d_step);
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
