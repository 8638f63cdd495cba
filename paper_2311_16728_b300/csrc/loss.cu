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

#include <string.h>

#include <mutex>

#include "ssim_impl.cuh"

namespace gsr {

// kTma: the staged regions come by TMA (tensor maps tx, ty / ta, tb, tc of
// the C x H x W planes; W a multiple of 4); else the threads stage them.
template <bool kTma>
__global__ void __launch_bounds__(kLThreads, kTma ? 5 : 1) ssim_pass1_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                                               int H, int W, Win win, float *__restrict__ mapA,
                                                               float *__restrict__ mapB, float *__restrict__ mapC,
                                                               float *__restrict__ partials,
                                                               const __grid_constant__ CUtensorMap tx,
                                                               const __grid_constant__ CUtensorMap ty) {
    chain_enter();
    extern __shared__ __align__(128) float sm[];
    __shared__ float s_red[32];
    __shared__ uint64_t s_bar;
    if (kTma) stage_tma_init(&s_bar);
    const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    ssim_pass1_block<kLThreads, kTma>(x, y, H, W, win, mapA, mapB, mapC, partials + 2 * b, blockIdx.x, blockIdx.y,
                                      blockIdx.z, sm, s_red, &tx, &ty, &s_bar, 0u);
}

template <bool kTma>
__global__ void __launch_bounds__(kLThreads, 5) ssim_pass2_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                                               int H, int W, Win win, const float *__restrict__ mapA,
                                                               const float *__restrict__ mapB,
                                                               const float *__restrict__ mapC,
                                                               const float *__restrict__ partials, int64_t npartials,
                                                               float lambda, float *__restrict__ d_loss,
                                                               float *__restrict__ dx_out,
                                                               const __grid_constant__ CUtensorMap ta,
                                                               const __grid_constant__ CUtensorMap tb,
                                                               const __grid_constant__ CUtensorMap tc) {
    chain_enter();
    extern __shared__ __align__(128) float sm[];
    __shared__ double s_dbl[2 * kLThreads];
    __shared__ uint64_t s_bar;
    if (kTma) stage_tma_init(&s_bar);
    ssim_pass2_block<kLThreads, kTma>(x, y, H, W, gridDim.z, win, mapA, mapB, mapC, lambda, 1.0f, dx_out,
                                      blockIdx.x, blockIdx.y, blockIdx.z, sm, &ta, &tb, &tc, &s_bar, 0u);
    // the first CTA folds the per-CTA partial sums, always in the same order
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
        const float L = loss_from_partials<kLThreads>(partials, npartials, (double)gridDim.z * H * W, lambda, s_dbl);
        if (threadIdx.x == 0) *d_loss = L;
    }
}

template <bool kTma> constexpr size_t pass1_smem() { return sizeof(float) * pass1_floats<kTma>(); }
template <bool kTma> constexpr size_t pass2_smem() { return sizeof(float) * pass2_floats<kTma>(); }

// Tensor map of a C x H x W FP32 plane stack for the staging box (48 x 42 x
// 1), zero fill outside; false when TMA cannot take it (W not a multiple of
// 4, a base not 16-byte aligned, no encoder) and the threads stage instead.
static bool plane_map(CUtensorMap *m, const float *base, int C, int H, int W) {
    auto enc = tensor_map_encoder();
    if (!enc || W % 4 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)C};
    const cuuint64_t strides[2] = {(cuuint64_t)W * 4, (cuuint64_t)W * H * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kRP, (cuuint32_t)kRH, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static void launch_ssim(const float *img, const float *gt, int C, int H, int W, float lambda, float *d_loss,
                        float *dL_dimg, float *mA, float *mB, float *mC, float *part, int64_t nblocks,
                        cudaStream_t st) {
    const Win win = ssim_window();
    const dim3 grid((W + kLTW - 1) / kLTW, (H + kLTH - 1) / kLTH, C);
    CUtensorMap t[5];
    const bool tma = plane_map(&t[0], img, C, H, W) && plane_map(&t[1], gt, C, H, W) &&
                     plane_map(&t[2], mA, C, H, W) && plane_map(&t[3], mB, C, H, W) && plane_map(&t[4], mC, C, H, W);
    auto k1 = tma ? ssim_pass1_kernel<true> : ssim_pass1_kernel<false>;
    auto k2 = tma ? ssim_pass2_kernel<true> : ssim_pass2_kernel<false>;
    if (!tma) memset(t, 0, sizeof(t));  // unused by the kernels that stage themselves
    // (per device, cheap, and not a stream operation: fine during capture)
    const size_t s1 = tma ? pass1_smem<true>() : pass1_smem<false>();
    const size_t s2 = tma ? pass2_smem<true>() : pass2_smem<false>();
    cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1);
    cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2);
    launch_chained(k1, dim3(grid), dim3(kLThreads), s1, st, img, gt, H, W, win, mA, mB, mC, part, t[0], t[1]);
    launch_chained(k2, dim3(grid), dim3(kLThreads), s2, st, img, gt, H, W, win, mA, mB, mC, part, nblocks, lambda,
                   d_loss, dL_dimg, t[2], t[3], t[4]);
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

// ---------------------------------------------------------------- luminance loss
// Grayscale views (stereo rigs of Sec. 4): Eq. 4 on the luminance
// Y = 0.299 R + 0.587 G + 0.114 B of the render against a grayscale target.
constexpr float kLumaR = 0.299f, kLumaG = 0.587f, kLumaB = 0.114f;

__global__ void __launch_bounds__(256) luma_kernel(const float *__restrict__ img, int64_t plane,
                                                   float *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < plane) y[i] = kLumaR * img[i] + kLumaG * img[plane + i] + kLumaB * img[2 * plane + i];
}

__global__ void __launch_bounds__(256) luma_grad_kernel(const float *__restrict__ dy, int64_t plane,
                                                        float *__restrict__ dimg) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < plane) {
        const float d = dy[i];
        dimg[i] = kLumaR * d;
        dimg[plane + i] = kLumaG * d;
        dimg[2 * plane + i] = kLumaB * d;
    }
}

extern "C" int32_t gsr_loss_luma_workspace_size(int32_t H, int32_t W, size_t *bytes) {
    if (H <= 0 || W <= 0 || !bytes) {
        set_error("gsr_loss_luma_workspace_size: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    *bytes = loss_layout(1, H, W).total + 2 * al256(sizeof(float) * (size_t)H * W);
    return GSR_OK;
}

extern "C" int32_t gsr_loss_luma_fwd_bwd(const float *img, const float *gt, int32_t H, int32_t W, float lambda,
                                         float *d_loss, float *dL_dimg, void *workspace, size_t workspace_bytes,
                                         gsr_stream_t stream) {
    if (!img || !gt || !d_loss || !dL_dimg || H <= 0 || W <= 0 || !(lambda >= 0.f && lambda <= 1.f)) {
        set_error("gsr_loss_luma_fwd_bwd: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    const LossLayout L = loss_layout(1, H, W);
    const size_t plane_bytes = al256(sizeof(float) * (size_t)H * W);
    if (!workspace || workspace_bytes < L.total + 2 * plane_bytes) {
        set_error("gsr_loss_luma_fwd_bwd: workspace of %zu bytes needed", L.total + 2 * plane_bytes);
        return GSR_ERR_CAPACITY;
    }
    char *ws = static_cast<char *>(workspace);
    float *mA = reinterpret_cast<float *>(ws + L.a), *mB = reinterpret_cast<float *>(ws + L.b);
    float *mC = reinterpret_cast<float *>(ws + L.c), *part = reinterpret_cast<float *>(ws + L.partials);
    float *y = reinterpret_cast<float *>(ws + L.total), *dy = reinterpret_cast<float *>(ws + L.total + plane_bytes);
    const int64_t plane = (int64_t)H * W;
    cudaStream_t st = as_cuda(stream);
    const unsigned blocks = (unsigned)((plane + 255) / 256);
    luma_kernel<<<blocks, 256, 0, st>>>(img, plane, y);
    launch_ssim(y, gt, 1, H, W, lambda, d_loss, dy, mA, mB, mC, part, L.nblocks, st);
    luma_grad_kernel<<<blocks, 256, 0, st>>>(dy, plane, dL_dimg);
    return check_launch("luminance loss kernels");
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
