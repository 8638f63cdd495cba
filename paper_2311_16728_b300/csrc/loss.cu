// loss.cu -- Eq. 4 photometric loss of Photo-SLAM (arXiv 2311.16728,
// Sec. 3.3) with its gradient (K6), and the PSNR metric (Sec. 4.1, K15).
//
//   L = (1 - lambda) mean|x - y| + lambda (1 - mean SSIM(x, y))
// SSIM per channel (Wang et al. 2004): 11 x 11 Gaussian window, sigma 1.5,
// zero padding, C1 = 0.01^2, C2 = 0.03^2.  With S(p) the SSIM map and
// mx, E[x^2], E[xy] the windowed moments,
//   d sum_p S(p) / d x_q = (G * a)(q) + 2 x_q (G * b)(q) + y_q (G * c)(q)
// where a = dS/dmx - 2 mx dS/dsxx - my dS/dsxy, b = dS/dsxx, c = dS/dsxy
// (the window is symmetric, so the adjoint blur is the blur itself).
// Pass 1 computes the moments and (a, b, c) per pixel plus per-CTA partial
// sums; pass 2 blurs (a, b, c) and writes dL/dx; its first CTA reduces the
// partial sums in a fixed order.
#include <math.h>

#include <mutex>

#include "gsr_internal.cuh"

namespace gsr {

constexpr int kLTW = 32, kLTH = 8, kLR = 5;
constexpr int kRW = kLTW + 2 * kLR, kRH = kLTH + 2 * kLR;

struct Win {
    float w[11];
};

static Win ssim_window() {
    Win k;
    double s = 0, v[11];
    for (int i = 0; i < 11; ++i) {
        v[i] = exp(-((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
        s += v[i];
    }
    for (int i = 0; i < 11; ++i) k.w[i] = (float)(v[i] / s);
    return k;
}

__device__ __forceinline__ float block_sum_256(float v, float *s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = 0.f;
    if (threadIdx.x < 32) {
        r = threadIdx.x < 8 ? s_red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

__global__ void __launch_bounds__(256) ssim_pass1_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                                         int H, int W, Win win, float *__restrict__ mapA,
                                                         float *__restrict__ mapB, float *__restrict__ mapC,
                                                         float *__restrict__ partials) {
    __shared__ float sX[kRH][kRW], sY[kRH][kRW];
    __shared__ float sH[5][kRH][kLTW];
    __shared__ float s_red[8];
    const int c = blockIdx.z, ox = blockIdx.x * kLTW, oy = blockIdx.y * kLTH, t = threadIdx.x;
    const int64_t plane = (int64_t)H * W, cb = (int64_t)c * plane;
    for (int idx = t; idx < kRH * kRW; idx += 256) {
        const int r = idx / kRW, q = idx % kRW;
        const int gy = oy - kLR + r, gx = ox - kLR + q;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        sX[r][q] = in ? x[cb + (int64_t)gy * W + gx] : 0.f;
        sY[r][q] = in ? y[cb + (int64_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    for (int idx = t; idx < kRH * kLTW; idx += 256) {
        const int r = idx / kLTW, j = idx % kLTW;
        float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float a = sX[r][j + k], b = sY[r][j + k], w = win.w[k];
            mx += w * a;
            my += w * b;
            xx += w * a * a;
            yy += w * b * b;
            xy += w * a * b;
        }
        sH[0][r][j] = mx; sH[1][r][j] = my; sH[2][r][j] = xx; sH[3][r][j] = yy; sH[4][r][j] = xy;
    }
    __syncthreads();
    const int tx = t % kLTW, ty = t / kLTW;
    float mx = 0.f, my = 0.f, ex2 = 0.f, ey2 = 0.f, exy = 0.f;
#pragma unroll
    for (int k = 0; k < 11; ++k) {
        const float w = win.w[k];
        mx += w * sH[0][ty + k][tx];
        my += w * sH[1][ty + k][tx];
        ex2 += w * sH[2][ty + k][tx];
        ey2 += w * sH[3][ty + k][tx];
        exy += w * sH[4][ty + k][tx];
    }
    const int gx = ox + tx, gy = oy + ty;
    float l1 = 0.f, ssim = 0.f;
    if (gx < W && gy < H) {
        const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
        const float sxx = ex2 - mx * mx, syy = ey2 - my * my, sxy = exy - mx * my;
        const float A1 = 2.f * mx * my + C1, A2 = 2.f * sxy + C2;
        const float B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
        const float iB = 1.0f / (B1 * B2);
        const float S = A1 * A2 * iB;
        const float dS_dmx = 2.f * my * A2 * iB - S * 2.f * mx / B1;
        const float dS_dsxx = -S / B2;
        const float dS_dsxy = 2.f * A1 * iB;
        const int64_t o = cb + (int64_t)gy * W + gx;
        mapA[o] = dS_dmx - 2.f * mx * dS_dsxx - my * dS_dsxy;
        mapB[o] = dS_dsxx;
        mapC[o] = dS_dsxy;
        l1 = fabsf(sX[ty + kLR][tx + kLR] - sY[ty + kLR][tx + kLR]);
        ssim = S;
    }
    const float s1 = block_sum_256(l1, s_red);
    const float s2 = block_sum_256(ssim, s_red);
    if (t == 0) {
        const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[2 * b] = s1;
        partials[2 * b + 1] = s2;
    }
}

__global__ void __launch_bounds__(256) ssim_pass2_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                                         int H, int W, Win win, const float *__restrict__ mapA,
                                                         const float *__restrict__ mapB,
                                                         const float *__restrict__ mapC,
                                                         const float *__restrict__ partials, int64_t npartials,
                                                         float lambda, float *__restrict__ d_loss,
                                                         float *__restrict__ dx_out) {
    __shared__ float sM[3][kRH][kRW];
    __shared__ float sH[3][kRH][kLTW];
    const int c = blockIdx.z, ox = blockIdx.x * kLTW, oy = blockIdx.y * kLTH, t = threadIdx.x;
    const int64_t plane = (int64_t)H * W, cb = (int64_t)c * plane;
    const float inv_n = (float)(1.0 / ((double)gridDim.z * (double)plane));  // 1 / (C H W)
    for (int idx = t; idx < kRH * kRW; idx += 256) {
        const int r = idx / kRW, q = idx % kRW;
        const int gy = oy - kLR + r, gx = ox - kLR + q;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const int64_t o = cb + (int64_t)gy * W + gx;
        sM[0][r][q] = in ? mapA[o] : 0.f;
        sM[1][r][q] = in ? mapB[o] : 0.f;
        sM[2][r][q] = in ? mapC[o] : 0.f;
    }
    __syncthreads();
    for (int idx = t; idx < kRH * kLTW; idx += 256) {
        const int r = idx / kLTW, j = idx % kLTW;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float w = win.w[k];
            s0 += w * sM[0][r][j + k];
            s1 += w * sM[1][r][j + k];
            s2 += w * sM[2][r][j + k];
        }
        sH[0][r][j] = s0; sH[1][r][j] = s1; sH[2][r][j] = s2;
    }
    __syncthreads();
    const int tx = t % kLTW, ty = t / kLTW;
    const int gx = ox + tx, gy = oy + ty;
    if (gx < W && gy < H) {
        float ga = 0.f, gb = 0.f, gc = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float w = win.w[k];
            ga += w * sH[0][ty + k][tx];
            gb += w * sH[1][ty + k][tx];
            gc += w * sH[2][ty + k][tx];
        }
        const int64_t o = cb + (int64_t)gy * W + gx;
        const float xv = x[o], yv = y[o];
        const float d = xv - yv;
        const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        dx_out[o] = ((1.f - lambda) * sg - lambda * (ga + 2.f * xv * gb + yv * gc)) * inv_n;
    }
    // the first CTA folds the per-CTA partial sums, always in the same order
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
        __shared__ double s_l1[256], s_ss[256];
        double a = 0.0, b = 0.0;
        for (int64_t k = t; k < npartials; k += 256) {
            a += (double)partials[2 * k];
            b += (double)partials[2 * k + 1];
        }
        s_l1[t] = a;
        s_ss[t] = b;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (t < o) {
                s_l1[t] += s_l1[t + o];
                s_ss[t] += s_ss[t + o];
            }
            __syncthreads();
        }
        if (t == 0) {
            const double cnt = (double)gridDim.z * (double)plane;
            *d_loss = (float)((1.0 - lambda) * s_l1[0] / cnt + lambda * (1.0 - s_ss[0] / cnt));
        }
    }
}

// ---------------------------------------------------------------- PSNR
__global__ void __launch_bounds__(256) psnr_partial_kernel(const float *__restrict__ img, const float *__restrict__ gt,
                                                           int64_t count, double *__restrict__ partials) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x; k < count; k += (int64_t)gridDim.x * 256) {
        const float a = fminf(fmaxf(img[k], 0.f), 1.f);
        const double d = (double)a - (double)gt[k];
        acc += d * d;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(256) psnr_final_kernel(const double *__restrict__ partials, int nparts,
                                                         int64_t count, float *__restrict__ out) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int k = threadIdx.x; k < nparts; k += 256) acc += partials[k];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)(10.0 * log10((double)count / s[0]));
}

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct LossLayout {
    size_t a, b, c, partials, total;
    int64_t nblocks;
};

static LossLayout loss_layout(int C, int H, int W) {
    LossLayout L;
    const size_t px = (size_t)C * H * W;
    L.nblocks = (int64_t)((W + kLTW - 1) / kLTW) * ((H + kLTH - 1) / kLTH) * C;
    size_t off = 0;
    L.a = off; off += al256(sizeof(float) * px);
    L.b = off; off += al256(sizeof(float) * px);
    L.c = off; off += al256(sizeof(float) * px);
    L.partials = off; off += al256(sizeof(float) * 2 * (size_t)L.nblocks);
    L.total = off;
    return L;
}

constexpr int kPsnrBlocks = 592;  // 4 x 148 SMs

}  // namespace gsr

using namespace gsr;

extern "C" int32_t gsr_loss_workspace_size(int32_t C, int32_t H, int32_t W, size_t *bytes) {
    if (C <= 0 || H <= 0 || W <= 0 || !bytes) {
        set_error("gsr_loss_workspace_size: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    *bytes = loss_layout(C, H, W).total;
    return GSR_OK;
}

extern "C" int32_t gsr_loss_fwd_bwd(const float *img, const float *gt, int32_t C, int32_t H, int32_t W, float lambda,
                                    float *d_loss, float *dL_dimg, void *workspace, size_t workspace_bytes,
                                    gsr_stream_t stream) {
    if (!img || !gt || !d_loss || !dL_dimg || C <= 0 || H <= 0 || W <= 0 || !(lambda >= 0.f && lambda <= 1.f)) {
        set_error("gsr_loss_fwd_bwd: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    const LossLayout L = loss_layout(C, H, W);
    if (!workspace || workspace_bytes < L.total) {
        set_error("gsr_loss_fwd_bwd: workspace of %zu bytes needed, %zu given", L.total, workspace_bytes);
        return GSR_ERR_CAPACITY;
    }
    char *ws = static_cast<char *>(workspace);
    float *mA = reinterpret_cast<float *>(ws + L.a), *mB = reinterpret_cast<float *>(ws + L.b);
    float *mC = reinterpret_cast<float *>(ws + L.c), *part = reinterpret_cast<float *>(ws + L.partials);
    const Win win = ssim_window();
    const dim3 grid((W + kLTW - 1) / kLTW, (H + kLTH - 1) / kLTH, C);
    cudaStream_t st = as_cuda(stream);
    ssim_pass1_kernel<<<grid, 256, 0, st>>>(img, gt, H, W, win, mA, mB, mC, part);
    ssim_pass2_kernel<<<grid, 256, 0, st>>>(img, gt, H, W, win, mA, mB, mC, part, L.nblocks, lambda, d_loss, dL_dimg);
    return check_launch("ssim kernels");
}

extern "C" int32_t gsr_psnr_workspace_size(int64_t count, size_t *bytes) {
    if (count < 0 || !bytes) {
        set_error("gsr_psnr_workspace_size: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    *bytes = sizeof(double) * kPsnrBlocks;
    return GSR_OK;
}

extern "C" int32_t gsr_psnr(const float *img, const float *gt, int64_t count, float *d_psnr, void *workspace,
                            size_t workspace_bytes, gsr_stream_t stream) {
    if (!img || !gt || !d_psnr || count <= 0) {
        set_error("gsr_psnr: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    if (!workspace || workspace_bytes < sizeof(double) * kPsnrBlocks) {
        set_error("gsr_psnr: workspace of %zu bytes needed", sizeof(double) * kPsnrBlocks);
        return GSR_ERR_CAPACITY;
    }
    cudaStream_t st = as_cuda(stream);
    double *part = static_cast<double *>(workspace);
    psnr_partial_kernel<<<kPsnrBlocks, 256, 0, st>>>(img, gt, count, part);
    psnr_final_kernel<<<1, 256, 0, st>>>(part, kPsnrBlocks, count, d_psnr);
    return check_launch("psnr kernels");
}

// ---------------------------------------------------------------- allocation-free loss
// gsr_loss_fwd_bwd_static: the same two kernels as gsr_loss_fwd_bwd, with the
// scratch (the three SSIM partial-derivative maps and the per-CTA partial
// sums) taken from a fixed array in device memory instead of a caller buffer.
// The array is defined at file scope, so every GPU that loads this library
// holds it (about 29.6 MB) until the process exits.
namespace gsr {

constexpr int64_t kStaticLossMaxElems = 2457600;  // C x H x W, e.g. 3 x 1200 x 680 (Replica frame) fits
constexpr int64_t kStaticLossMaxBlocks = 16384;   // CTAs of 32 x 8 pixels per channel, summed over channels

static __device__ __align__(256) float g_loss_scratch[3 * kStaticLossMaxElems + 2 * kStaticLossMaxBlocks];

// Device address of g_loss_scratch, looked up once per device.  In host code
// the symbol names a host-side stand-in, not device memory, so it is never
// passed to a kernel directly.
constexpr int kMaxDevices = 64;
static float *g_loss_scratch_ptr[kMaxDevices];
static std::mutex g_loss_scratch_mu;

static int32_t static_loss_scratch(float **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_error("gsr_loss_fwd_bwd_static: no usable current device");
        return GSR_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_loss_scratch_mu);
    if (!g_loss_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_loss_scratch);
        if (e != cudaSuccess || !p) {
            set_error("gsr_loss_fwd_bwd_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return GSR_ERR_CUDA;
        }
        g_loss_scratch_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_loss_scratch_ptr[dev];
    return GSR_OK;
}

}  // namespace gsr

extern "C" int32_t gsr_loss_fwd_bwd_static(const float *img, const float *gt, int32_t C, int32_t H, int32_t W,
                                           float lambda, float *d_loss, float *dL_dimg, gsr_stream_t stream) {
    if (!img || !gt || !d_loss || !dL_dimg || C <= 0 || H <= 0 || W <= 0 || !(lambda >= 0.f && lambda <= 1.f)) {
        set_error("gsr_loss_fwd_bwd_static: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    const int64_t elems = (int64_t)C * H * W;
    const int64_t nblocks = (int64_t)((W + kLTW - 1) / kLTW) * ((H + kLTH - 1) / kLTH) * C;
    if (elems > kStaticLossMaxElems || nblocks > kStaticLossMaxBlocks) {
        set_error("gsr_loss_fwd_bwd_static: image %d x %d x %d exceeds the fixed scratch (at most %lld values "
                  "and %lld 32x8 pixel blocks); use gsr_loss_fwd_bwd with a workspace",
                  (int)C, (int)H, (int)W, (long long)kStaticLossMaxElems, (long long)kStaticLossMaxBlocks);
        return GSR_ERR_CAPACITY;
    }
    float *base = nullptr;
    int32_t rc = static_loss_scratch(&base);
    if (rc) return rc;
    // every map entry the second pass reads and every partial sum is written
    // by the first pass of the same call, so nothing needs clearing
    float *mA = base, *mB = base + kStaticLossMaxElems, *mC = base + 2 * kStaticLossMaxElems;
    float *part = base + 3 * kStaticLossMaxElems;
    const Win win = ssim_window();
    const dim3 grid((W + kLTW - 1) / kLTW, (H + kLTH - 1) / kLTH, C);
    cudaStream_t st = as_cuda(stream);
    ssim_pass1_kernel<<<grid, 256, 0, st>>>(img, gt, H, W, win, mA, mB, mC, part);
    ssim_pass2_kernel<<<grid, 256, 0, st>>>(img, gt, H, W, win, mA, mB, mC, part, nblocks, lambda, d_loss, dL_dimg);
    return check_launch("ssim kernels (static scratch)");
}
