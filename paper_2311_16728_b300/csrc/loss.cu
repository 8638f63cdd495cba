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

constexpr int kLTW = 32, kLTH = 32, kLR = 5;       // output tile and window radius
constexpr int kRW = kLTW + 2 * kLR, kRH = kLTH + 2 * kLR;
constexpr int kRS = 45;                            // row stride of the staged region (conflict-free)
constexpr int kRun = 4;                            // outputs per thread along a row / column
constexpr int kLThreads = 256;

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

// Stages a (kRH x kRW) region of plane `src` around the tile (zero outside).
__device__ __forceinline__ void stage_region(const float *__restrict__ src, int H, int W, int ox, int oy, float *dst) {
    for (int idx = threadIdx.x; idx < kRH * kRW; idx += kLThreads) {
        const int r = idx / kRW, q = idx % kRW;
        const int gy = oy - kLR + r, gx = ox - kLR + q;
        dst[r * kRS + q] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? src[(int64_t)gy * W + gx] : 0.f;
    }
}

// Pass 1: windowed moments (separable: rows then columns, kRun outputs per
// thread from kRun + 10 staged values), SSIM map, its partials (a, b, c) and
// per-CTA sums of |x - y| and SSIM.
__global__ void __launch_bounds__(kLThreads) ssim_pass1_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                                               int H, int W, Win win, float *__restrict__ mapA,
                                                               float *__restrict__ mapB, float *__restrict__ mapC,
                                                               float *__restrict__ partials) {
    extern __shared__ float sm[];
    float *sX = sm, *sY = sm + kRH * kRS;
    float *sH = sm + 2 * kRH * kRS;  // [5][kRH][kLTW]
    __shared__ float s_red[8];
    const int c = blockIdx.z, ox = blockIdx.x * kLTW, oy = blockIdx.y * kLTH;
    const int64_t plane = (int64_t)H * W, cb = (int64_t)c * plane;
    stage_region(x + cb, H, W, ox, oy, sX);
    stage_region(y + cb, H, W, ox, oy, sY);
    __syncthreads();
    // rows: kRH rows x (kLTW / kRun) runs
    for (int item = threadIdx.x; item < kRH * (kLTW / kRun); item += kLThreads) {
        const int r = item / (kLTW / kRun), j0 = (item % (kLTW / kRun)) * kRun;
        float a[kRun + 10], b[kRun + 10];
#pragma unroll
        for (int k = 0; k < kRun + 10; ++k) {
            a[k] = sX[r * kRS + j0 + k];
            b[k] = sY[r * kRS + j0 + k];
        }
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
            float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) {
                const float w = win.w[k], av = a[o + k], bv = b[o + k];
                mx += w * av;
                my += w * bv;
                xx += w * av * av;
                yy += w * bv * bv;
                xy += w * av * bv;
            }
            float *h = sH + r * kLTW + j0 + o;
            h[0] = mx;
            h[kRH * kLTW] = my;
            h[2 * kRH * kLTW] = xx;
            h[3 * kRH * kLTW] = yy;
            h[4 * kRH * kLTW] = xy;
        }
    }
    __syncthreads();
    // columns: thread = (column, run of kRun rows)
    const int tx = threadIdx.x % kLTW, i0 = (threadIdx.x / kLTW) * kRun;
    float m[5][kRun];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        float col[kRun + 10];
#pragma unroll
        for (int k = 0; k < kRun + 10; ++k) col[k] = sH[q * kRH * kLTW + (i0 + k) * kLTW + tx];
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) s += win.w[k] * col[o + k];
            m[q][o] = s;
        }
    }
    float l1 = 0.f, ssim = 0.f;
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
#pragma unroll
    for (int o = 0; o < kRun; ++o) {
        const int gx = ox + tx, gy = oy + i0 + o;
        if (gx < W && gy < H) {
            const float mx = m[0][o], my = m[1][o];
            const float sxx = m[2][o] - mx * mx, syy = m[3][o] - my * my, sxy = m[4][o] - mx * my;
            const float A1 = 2.f * mx * my + C1, A2 = 2.f * sxy + C2;
            const float B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
            const float iB = 1.0f / (B1 * B2);
            const float S = A1 * A2 * iB;
            const float dS_dmx = 2.f * my * A2 * iB - S * 2.f * mx / B1;
            const float dS_dsxx = -S / B2;
            const float dS_dsxy = 2.f * A1 * iB;
            const int64_t idx = cb + (int64_t)gy * W + gx;
            mapA[idx] = dS_dmx - 2.f * mx * dS_dsxx - my * dS_dsxy;
            mapB[idx] = dS_dsxx;
            mapC[idx] = dS_dsxy;
            const int rr = i0 + o + kLR, qq = tx + kLR;
            l1 += fabsf(sX[rr * kRS + qq] - sY[rr * kRS + qq]);
            ssim += S;
        }
    }
    const float s1 = block_sum_256(l1, s_red);
    const float s2 = block_sum_256(ssim, s_red);
    if (threadIdx.x == 0) {
        const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[2 * b] = s1;
        partials[2 * b + 1] = s2;
    }
}

// Pass 2: blur (a, b, c) (the adjoint of the symmetric window), then
// dL/dx = ((1 - lambda) sign(x - y) - lambda (G*a + 2 x G*b + y G*c)) / (C H W).
// The first CTA also folds the per-CTA sums into the loss, in a fixed order.
__global__ void __launch_bounds__(kLThreads) ssim_pass2_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                                               int H, int W, Win win, const float *__restrict__ mapA,
                                                               const float *__restrict__ mapB,
                                                               const float *__restrict__ mapC,
                                                               const float *__restrict__ partials, int64_t npartials,
                                                               float lambda, float *__restrict__ d_loss,
                                                               float *__restrict__ dx_out) {
    extern __shared__ float sm[];
    float *sM = sm;                  // [3][kRH][kRS]
    float *sH = sm + 3 * kRH * kRS;  // [3][kRH][kLTW]
    const int c = blockIdx.z, ox = blockIdx.x * kLTW, oy = blockIdx.y * kLTH;
    const int64_t plane = (int64_t)H * W, cb = (int64_t)c * plane;
    const float inv_n = (float)(1.0 / ((double)gridDim.z * (double)plane));  // 1 / (C H W)
    stage_region(mapA + cb, H, W, ox, oy, sM);
    stage_region(mapB + cb, H, W, ox, oy, sM + kRH * kRS);
    stage_region(mapC + cb, H, W, ox, oy, sM + 2 * kRH * kRS);
    __syncthreads();
    for (int item = threadIdx.x; item < 3 * kRH * (kLTW / kRun); item += kLThreads) {
        const int q = item / (kRH * (kLTW / kRun)), rem = item % (kRH * (kLTW / kRun));
        const int r = rem / (kLTW / kRun), j0 = (rem % (kLTW / kRun)) * kRun;
        float a[kRun + 10];
#pragma unroll
        for (int k = 0; k < kRun + 10; ++k) a[k] = sM[q * kRH * kRS + r * kRS + j0 + k];
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) s += win.w[k] * a[o + k];
            sH[q * kRH * kLTW + r * kLTW + j0 + o] = s;
        }
    }
    __syncthreads();
    const int tx = threadIdx.x % kLTW, i0 = (threadIdx.x / kLTW) * kRun;
    float g[3][kRun];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float col[kRun + 10];
#pragma unroll
        for (int k = 0; k < kRun + 10; ++k) col[k] = sH[q * kRH * kLTW + (i0 + k) * kLTW + tx];
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) s += win.w[k] * col[o + k];
            g[q][o] = s;
        }
    }
#pragma unroll
    for (int o = 0; o < kRun; ++o) {
        const int gx = ox + tx, gy = oy + i0 + o;
        if (gx < W && gy < H) {
            const int64_t idx = cb + (int64_t)gy * W + gx;
            const float xv = x[idx], yv = y[idx];
            const float d = xv - yv;
            const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
            dx_out[idx] = ((1.f - lambda) * sg - lambda * (g[0][o] + 2.f * xv * g[1][o] + yv * g[2][o])) * inv_n;
        }
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
        __shared__ double s_l1[kLThreads], s_ss[kLThreads];
        const int t = threadIdx.x;
        double a = 0.0, b = 0.0;
        for (int64_t k = t; k < npartials; k += kLThreads) {
            a += (double)partials[2 * k];
            b += (double)partials[2 * k + 1];
        }
        s_l1[t] = a;
        s_ss[t] = b;
        __syncthreads();
        for (int o = kLThreads / 2; o > 0; o >>= 1) {
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

constexpr size_t kPass1Smem = sizeof(float) * (2 * kRH * kRS + 5 * kRH * kLTW);
constexpr size_t kPass2Smem = sizeof(float) * (3 * kRH * kRS + 3 * kRH * kLTW);

static void launch_ssim(const float *img, const float *gt, int C, int H, int W, float lambda, float *d_loss,
                        float *dL_dimg, float *mA, float *mB, float *mC, float *part, int64_t nblocks,
                        cudaStream_t st) {
    // (per device, cheap, and not a stream operation: fine during capture)
    cudaFuncSetAttribute(ssim_pass1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPass1Smem);
    cudaFuncSetAttribute(ssim_pass2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPass2Smem);
    const Win win = ssim_window();
    const dim3 grid((W + kLTW - 1) / kLTW, (H + kLTH - 1) / kLTH, C);
    ssim_pass1_kernel<<<grid, kLThreads, kPass1Smem, st>>>(img, gt, H, W, win, mA, mB, mC, part);
    ssim_pass2_kernel<<<grid, kLThreads, kPass2Smem, st>>>(img, gt, H, W, win, mA, mB, mC, part, nblocks, lambda,
                                                            d_loss, dL_dimg);
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
    launch_ssim(img, gt, C, H, W, lambda, d_loss, dL_dimg, mA, mB, mC, part, L.nblocks, as_cuda(stream));
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
constexpr int64_t kStaticLossMaxBlocks = 16384;   // CTAs of 32 x 32 pixels per channel, summed over channels

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
                  "and %lld 32x32 pixel blocks); use gsr_loss_fwd_bwd with a workspace",
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
    launch_ssim(img, gt, C, H, W, lambda, d_loss, dL_dimg, mA, mB, mC, part, nblocks, as_cuda(stream));
    return check_launch("ssim kernels (static scratch)");
}
