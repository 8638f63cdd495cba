// mlp.cu -- the learned initialiser of new primitives (the build's answer to
// Photo-SLAM's geometry-based densification, arXiv 2311.16728 Sec. 3.3.1,
// which does not say how new primitives are initialised): a 2308 -> 256 ->
// 256 -> 56 ReLU MLP over multi-level image patches, in BF16 with FP32
// accumulation on the tcgen05 tensor cores (umma_gemm.cuh), trained by MSE
// with Adam on FP32 master weights.
#include <mutex>

#include "umma_gemm.cuh"

namespace gsr {

// ---------------------------------------------------------------- tensor maps
// K-major BF16 matrix [rows x K] (K contiguous, row stride ld elements), box
// of 64 (K) x box_rows rows, 128-byte swizzle.
static int32_t make_map(CUtensorMap *m, const void *base, int64_t rows, int64_t K, int64_t ld, int box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return GSR_ERR_CUDA;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)umma::BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return GSR_ERR_CUDA;
    }
    return GSR_OK;
}

template <int BN, int ST = (BN == 256 ? 4 : 6)>
static int32_t launch_gemm_bn(const void *A, int64_t lda, const void *B, int64_t ldb, int M, int N, int K,
                              const umma::Epilogue &ep, int ksplit, int32_t *d_status, cudaStream_t st) {
    using Cfg = umma::Config<BN, ST>;
    CUtensorMap ma, mb;
    int32_t rc;
    if ((rc = make_map(&ma, A, M, K, lda, umma::BM)) || (rc = make_map(&mb, B, N, K, ldb, BN))) return rc;
    cudaFuncSetAttribute(umma::gemm_kernel<BN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
    const dim3 grid(N / BN, M / umma::BM, ksplit);
    umma::gemm_kernel<BN, ST><<<grid, 192, Cfg::kSmem, st>>>(ma, mb, K, ep, d_status);
    return check_launch("umma gemm_kernel");
}

// D = A B^T with A [M x K], B [N x K] BF16 K-major; M % 128 == 0, N % 64 == 0,
// K % 64 == 0; the widest BN in {256, 128, 64} that divides N, except that a
// short reduction (K <= 256 without split, or bn64) takes BN = 64: there the
// epilogue is most of the work and four times as many CTAs share it.
int32_t gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, int M, int N, int K,
                  const umma::Epilogue &ep_in, int ksplit, int32_t *d_status, cudaStream_t st, bool bn64 = false) {
    umma::Epilogue ep = ep_in;
    ep.vec_mask = ep.mask && aligned16(ep.mask) && ep.ldm % 8 == 0;
    ep.vec_out = ep.out_bf16 && aligned16(ep.out_bf16) && ep.ldo % 8 == 0;
    ep.vec_t = ep.out_bf16_t && aligned16(ep.out_bf16_t) && ep.ldt % 8 == 0;
    if (M <= 0 || N <= 0 || K <= 0 || M % umma::BM || N % 64 || K % umma::BK || ksplit < 1 || !aligned16(A) ||
        !aligned16(B) || lda % 8 || ldb % 8) {
        set_error("gemm_bf16: need M %% 128 == 0, N %% 64 == 0, K %% 64 == 0, 16-byte aligned operands "
                  "(M=%d N=%d K=%d)", M, N, K);
        return GSR_ERR_INVALID_ARG;
    }
    if (ksplit > K / umma::BK) ksplit = K / umma::BK;
    // a reduction of at most 4 k-steps per CTA needs only a 2-stage ring (4 CTAs per SM)
    if (ksplit == 1 && K <= 256) return launch_gemm_bn<64, 2>(A, lda, B, ldb, M, N, K, ep, ksplit, d_status, st);
    if (bn64) return launch_gemm_bn<64>(A, lda, B, ldb, M, N, K, ep, ksplit, d_status, st);
    // split-K over an N that 128 does not divide: 128 x 64 tiles on a 3-stage
    // ring, three CTAs per SM, so the split's CTAs run in one wave
    if (ksplit > 1 && N % 128 != 0) return launch_gemm_bn<64, 3>(A, lda, B, ldb, M, N, K, ep, ksplit, d_status, st);
    // fewer 128 x 256 tiles than two per SM leave a ragged second wave (157
    // tiles on 148 SMs take two tile times): 128 x 128 tiles instead, on a
    // 3-stage ring (two CTAs per SM) when they fit in one wave of those, else
    // on a 2-stage ring (three CTAs per SM)
    const int64_t t256 = (int64_t)(N / 256) * (M / umma::BM) * ksplit;
    if (N % 256 == 0 && t256 < 2 * 148) {
        if (2 * t256 <= 2 * 148) return launch_gemm_bn<128, 3>(A, lda, B, ldb, M, N, K, ep, ksplit, d_status, st);
        return launch_gemm_bn<128, 2>(A, lda, B, ldb, M, N, K, ep, ksplit, d_status, st);
    }
    if (N % 256 == 0) return launch_gemm_bn<256>(A, lda, B, ldb, M, N, K, ep, ksplit, d_status, st);
    if (N % 128 == 0) return launch_gemm_bn<128>(A, lda, B, ldb, M, N, K, ep, ksplit, d_status, st);
    return launch_gemm_bn<64>(A, lda, B, ldb, M, N, K, ep, ksplit, d_status, st);
}

}  // namespace gsr

using namespace gsr;

extern "C" int32_t gsr_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, int32_t M, int32_t N,
                                 int32_t K, const float *bias, int32_t relu, const void *mask, int32_t ldm,
                                 void *out_bf16, int32_t ldo, void *out_bf16_t, int32_t ldt, float *out_f32,
                                 int32_t ldf, int32_t atomic_f32, float *colsum, int64_t valid_rows, int32_t ksplit,
                                 int32_t *d_status, gsr_stream_t stream) {
    umma::Epilogue ep{};
    ep.bias = bias;
    ep.relu = relu;
    ep.mask = static_cast<const __nv_bfloat16 *>(mask);
    ep.ldm = ldm;
    ep.out_bf16 = static_cast<__nv_bfloat16 *>(out_bf16);
    ep.ldo = ldo;
    ep.out_bf16_t = static_cast<__nv_bfloat16 *>(out_bf16_t);
    ep.ldt = ldt;
    ep.out_f32 = out_f32;
    ep.ldf = ldf;
    ep.atomic_f32 = atomic_f32;
    ep.colsum = colsum;
    ep.valid_rows = valid_rows;
    if ((out_f32 && !aligned16(out_f32)) || (out_f32 && ldf % 4)) {
        set_error("gsr_gemm_bf16: out_f32 must be 16-byte aligned with ldf a multiple of 4");
        return GSR_ERR_INVALID_ARG;
    }
    if (!ep.out_bf16 && !ep.out_bf16_t && !ep.out_f32 && !ep.colsum) {
        set_error("gsr_gemm_bf16: no output");
        return GSR_ERR_INVALID_ARG;
    }
    if (ksplit > 1 && ((ep.out_f32 && !atomic_f32) || ep.out_bf16 || ep.out_bf16_t || ep.bias || ep.relu || ep.mask)) {
        set_error("gsr_gemm_bf16: split-K needs an atomic FP32 output and no element-wise epilogue");
        return GSR_ERR_INVALID_ARG;
    }
    return gemm_bf16(A, lda, B, ldb, M, N, K, ep, ksplit, d_status, as_cuda(stream));
}

// ================================================================ the MLP
namespace gsr {

constexpr int kK0 = 2368, kH = 256, kOut = 56, kN3 = 64;  // 2308 inputs padded to kK0

// ---------------------------------------------------------------- patch gather (K13)
// Row m: [level l = 0..2][16 x 16 pixels][RGB] around (u / 2^l, v / 2^l)
// (nearest pixel, clamped), then depth, log keypoint scale, cos, sin of the
// keypoint angle, then zeros up to 2368.  Rows m >= M are zero.
__global__ void __launch_bounds__(256) patch_gather_kernel(const float *__restrict__ l0, const float *__restrict__ l1,
                                                           const float *__restrict__ l2, int W0, int H0,
                                                           const float *__restrict__ kp, int64_t M, int64_t Mpad,
                                                           __nv_bfloat16 *__restrict__ x) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Mpad * kK0) return;
    const int64_t m = e / kK0;
    const int f = (int)(e - m * kK0);
    float val = 0.0f;
    if (m < M) {
        const float *k = kp + 5 * m;
        if (f < 2304) {
            const int l = f / 768, r = f % 768, pix = r / 3, ch = r % 3;
            int W = W0, H = H0;
            for (int i = 0; i < l; ++i) {
                W = (W + 1) / 2;
                H = (H + 1) / 2;
            }
            const float s = 1.0f / (float)(1 << l);
            const int cxp = (int)rintf(k[0] * s), cyp = (int)rintf(k[1] * s);
            const int px = min(max(cxp - 8 + pix % 16, 0), W - 1), py = min(max(cyp - 8 + pix / 16, 0), H - 1);
            const float *img = l == 0 ? l0 : (l == 1 ? l1 : l2);
            val = img[((int64_t)ch * H + py) * W + px];
        } else if (f == 2304) {
            val = k[2];
        } else if (f == 2305) {
            val = k[3];
        } else if (f == 2306) {
            val = cosf(k[4]);
        } else if (f == 2307) {
            val = sinf(k[4]);
        }
    }
    x[e] = __float2bfloat16_rn(val);
}

// out[c][r] = in[r][c] for a rows x cols BF16 matrix (32 x 32 shared tiles)
__global__ void __launch_bounds__(256) transpose_bf16_kernel(const __nv_bfloat16 *__restrict__ in,
                                                             __nv_bfloat16 *__restrict__ out, int64_t rows, int64_t cols) {
    __shared__ __nv_bfloat16 t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[i][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = t[threadIdx.x][i];
    }
}

// ---------------------------------------------------------------- loss (MSE)
// dy = 2 w (y - t) / M on the first 56 columns of valid rows (BF16, both
// layouts), gb3 += sum_m dy (FP32), loss += sum w (y - t)^2 / M.
constexpr int kLossRows = 64;    // rows of one tile
constexpr int kLossTStride = 72; // row stride (BF16) of the transposed tile in shared memory

__global__ void __launch_bounds__(256) mlp_loss_kernel(const float *__restrict__ y, const float *__restrict__ t,
                                                       const float *__restrict__ w, int64_t M, int64_t Mpad,
                                                       __nv_bfloat16 *__restrict__ dy, __nv_bfloat16 *__restrict__ dyT,
                                                       float *__restrict__ gb3, float *__restrict__ d_loss) {
    // tiles of 64 rows, grid-striding: thread = column j = tid % 64 of rows
    // 4 k + tid / 64 (row-major loads and dy stores coalesced); the tile's
    // gradient goes transposed through shared memory so that dyT is written
    // as 16-byte words along the rows.  Column sums and the loss stay in
    // registers until one reduction and one atomic per column (and one for
    // the loss) per block.
    __shared__ __align__(16) __nv_bfloat16 s_t[kN3 * kLossTStride];
    __shared__ float s_g[256], s_l[256];
    const int j = (int)(threadIdx.x & 63), r0 = (int)(threadIdx.x >> 6);
    float lsum = 0.0f, gsum = 0.0f;
    const float wj = j < kOut ? w[j] : 0.0f, inv_m = 1.0f / (float)M;
    constexpr int kPer = kLossRows / 4;
    for (int64_t m0 = (int64_t)kLossRows * blockIdx.x; m0 < Mpad; m0 += (int64_t)kLossRows * gridDim.x) {
        float d[kPer];  // every load of the tile in flight before the first use
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int64_t m = m0 + r0 + 4 * i, e = m * kN3 + j;
            d[i] = (m < M && j < kOut) ? y[e] - t[e] : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int rr = r0 + 4 * i;
            const int64_t e = (m0 + rr) * kN3 + j;
            lsum += wj * d[i] * d[i] * inv_m;
            const float g = 2.0f * wj * d[i] * inv_m;
            gsum += g;
            const __nv_bfloat16 gb = __float2bfloat16_rn(g);
            dy[e] = gb;
            s_t[j * kLossTStride + rr] = gb;
        }
        __syncthreads();
        {  // column c = tid / 4, rows 16 (tid % 4) .. + 15 of the tile: two 16-byte words
            const int c = (int)(threadIdx.x >> 2), q = 16 * (int)(threadIdx.x & 3);
            const uint4 *src = reinterpret_cast<const uint4 *>(s_t + c * kLossTStride + q);
            uint4 *dst = reinterpret_cast<uint4 *>(dyT + (int64_t)c * Mpad + m0 + q);
            dst[0] = src[0];
            dst[1] = src[1];
        }
        __syncthreads();
    }
    s_g[threadIdx.x] = gsum;
    s_l[threadIdx.x] = lsum;
    __syncthreads();
    if (threadIdx.x < kN3) {
        const float s = s_g[threadIdx.x] + s_g[threadIdx.x + 64] + s_g[threadIdx.x + 128] + s_g[threadIdx.x + 192];
        if (s != 0.0f) atomicAdd(gb3 + threadIdx.x, s);
    }
    if (threadIdx.x < 32) {
        float s = 0.0f;
        for (int i = threadIdx.x; i < 256; i += 32) s += s_l[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0 && s != 0.0f) atomicAdd(d_loss, s);
    }
}

// ---------------------------------------------------------------- Adam on the MLP
// p, g, m, v FP32 [rows x cols]; g_t (if set) holds the gradient transposed
// ([cols x rows]).  Writes the BF16 copy (and its transpose) of the updated
// weights; the gradient stays readable until the next step clears it.

// One tensor of the MLP's Adam step.
struct MlpAdamT {
    float *p, *g, *m, *v;
    int g_t, rows, cols;
    __nv_bfloat16 *ph, *phT;
};
struct MlpAdamSet {
    MlpAdamT t[6];
    int64_t off[7];  // element offsets of the tensors in one flat index space
};

// The six tensors' updates in one launch: thread f updates element f of the
// flat index space.
__global__ void __launch_bounds__(256) mlp_adam_all_kernel(const __grid_constant__ MlpAdamSet S, float lr, float b1,
                                                           float b2, float eps, const int32_t *__restrict__ d_step) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= S.off[6]) return;
    int k = 0;
#pragma unroll
    for (int q = 1; q < 6; ++q) k += f >= S.off[q] ? 1 : 0;
    const MlpAdamT &T = S.t[k];
    const int64_t e = f - S.off[k];
    const int r = (int)(e / T.cols), c = (int)(e - (int64_t)r * T.cols);
    const int64_t ge = T.g_t ? (int64_t)c * T.rows + r : e;
    const int t = *d_step + 1;
    const float bc1 = -expm1f((float)t * log1pf(b1 - 1.0f)), bc2 = -expm1f((float)t * log1pf(b2 - 1.0f));
    const float gv = T.g[ge];
    const float mv = b1 * T.m[e] + (1.0f - b1) * gv;
    const float vv = b2 * T.v[e] + (1.0f - b2) * gv * gv;
    const float pv = T.p[e] - lr * (mv / bc1) / (sqrtf(vv / bc2) + eps);
    T.m[e] = mv;
    T.v[e] = vv;
    T.p[e] = pv;
    if (T.ph) T.ph[e] = __float2bfloat16_rn(pv);
    if (T.phT) T.phT[(int64_t)c * T.rows + r] = __float2bfloat16_rn(pv);
}

__global__ void step_advance_mlp_kernel(int32_t *d_step) { *d_step += 1; }

__global__ void __launch_bounds__(256) to_bf16_kernel(const float *__restrict__ p, int rows, int cols,
                                                      __nv_bfloat16 *__restrict__ ph, __nv_bfloat16 *__restrict__ phT) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * cols) return;
    const int r = (int)(e / cols), c = (int)(e - (int64_t)r * cols);
    if (ph) ph[e] = __float2bfloat16_rn(p[e]);
    if (phT) phT[(int64_t)c * rows + r] = __float2bfloat16_rn(p[e]);
}

// ---------------------------------------------------------------- parameters <-> outputs
// Quaternion (w, x, y, z) of a rotation matrix (row-major), Shepperd's method.
__device__ __forceinline__ float4 quat_of(const float *R) {
    const float tr = R[0] + R[4] + R[8];
    float4 q;
    if (tr > 0.0f) {
        const float s = sqrtf(tr + 1.0f) * 2.0f;
        q = make_float4(0.25f * s, (R[7] - R[5]) / s, (R[2] - R[6]) / s, (R[3] - R[1]) / s);
    } else if (R[0] > R[4] && R[0] > R[8]) {
        const float s = sqrtf(1.0f + R[0] - R[4] - R[8]) * 2.0f;
        q = make_float4((R[7] - R[5]) / s, 0.25f * s, (R[1] + R[3]) / s, (R[2] + R[6]) / s);
    } else if (R[4] > R[8]) {
        const float s = sqrtf(1.0f + R[4] - R[0] - R[8]) * 2.0f;
        q = make_float4((R[2] - R[6]) / s, (R[1] + R[3]) / s, 0.25f * s, (R[5] + R[7]) / s);
    } else {
        const float s = sqrtf(1.0f + R[8] - R[0] - R[4]) * 2.0f;
        q = make_float4((R[3] - R[1]) / s, (R[2] + R[6]) / s, (R[5] + R[7]) / s, 0.25f * s);
    }
    return q;
}

__device__ __forceinline__ float4 qmul(float4 a, float4 b) {  // Hamilton product a * b
    return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w, a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                       a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y, a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}

__device__ __forceinline__ float4 qnormalize_pos(float4 q) {  // unit norm, w >= 0
    const float n = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float s = q.x < 0.0f ? -n : n;
    return make_float4(q.x * s, q.y * s, q.z * s, q.w * s);
}

struct CamMLP {
    float R[9], t[3], fx, fy, cx, cy;
};

// target row of keypoint m from Gaussian gids[m]: log-scale relative to
// log(depth / fx) (one pixel at that depth), rotation in the camera frame,
// opacity logit, SH (world frame); columns 56..63 zero.
__global__ void __launch_bounds__(64) mlp_encode_kernel(const float4 *__restrict__ mean_op,
                                                        const float4 *__restrict__ quat,
                                                        const float4 *__restrict__ logscale,
                                                        const float4 *__restrict__ sh, int64_t n,
                                                        const uint32_t *__restrict__ gids,
                                                        const float *__restrict__ kp, int64_t M, CamMLP cam,
                                                        const float *__restrict__ base, float *__restrict__ target) {
    const int64_t m = blockIdx.x;
    const int j = threadIdx.x;
    float val = 0.0f;
    if (m < M) {
        const uint32_t g = gids[m];
        const float lrel = logf(kp[5 * m + 2] / cam.fx);
        if (j < 3) {
            const float4 ls = logscale[g];
            val = (j == 0 ? ls.x : (j == 1 ? ls.y : ls.z)) - lrel;
        } else if (j < 7) {
            const float4 qc = qnormalize_pos(qmul(quat_of(cam.R), qnormalize_pos(quat[g])));
            val = j == 3 ? qc.x : (j == 4 ? qc.y : (j == 5 ? qc.z : qc.w));
        } else if (j == 7) {
            val = mean_op[g].w;
        } else if (j < kOut) {
            const int f = j - 8;
            const float4 s = sh[(int64_t)(f / 4) * n + g];
            val = (f & 3) == 0 ? s.x : ((f & 3) == 1 ? s.y : ((f & 3) == 2 ? s.z : s.w));
        }
    }
    if (base && m < M && j < kOut) val -= base[m * kN3 + j];
    target[m * kN3 + j] = val;
}

// New Gaussian out_offset + m from row m: mean = back-projection of the
// keypoint at its depth, parameters from the row (inverse of the encoding).
__global__ void __launch_bounds__(64) mlp_decode_kernel(const float *__restrict__ y, const float *__restrict__ base,
                                                        const float *__restrict__ kp, int64_t M, CamMLP cam,
                                                        float4 *__restrict__ mean_op, float4 *__restrict__ quat,
                                                        float4 *__restrict__ logscale, float4 *__restrict__ sh,
                                                        int64_t n, int64_t off) {
    __shared__ float row[kN3];
    const int64_t m = blockIdx.x;
    if (m >= M) return;
    const int64_t g = off + m;
    const int j = threadIdx.x;
    row[j] = y[m * kN3 + j] + (base ? base[m * kN3 + j] : 0.0f);
    __syncthreads();
    if (j == 0) {
        const float *k = kp + 5 * m;
        const float d = k[2];
        const float pc[3] = {(k[0] - cam.cx) / cam.fx * d - cam.t[0], (k[1] - cam.cy) / cam.fy * d - cam.t[1],
                             d - cam.t[2]};
        const float *R = cam.R;  // mean = R^T (p_cam - t)
        mean_op[g] = make_float4(R[0] * pc[0] + R[3] * pc[1] + R[6] * pc[2], R[1] * pc[0] + R[4] * pc[1] + R[7] * pc[2],
                                 R[2] * pc[0] + R[5] * pc[1] + R[8] * pc[2], row[7]);
        const float lrel = logf(d / cam.fx);
        logscale[g] = make_float4(row[0] + lrel, row[1] + lrel, row[2] + lrel, 0.0f);
        const float Rt[9] = {R[0], R[3], R[6], R[1], R[4], R[7], R[2], R[5], R[8]};
        quat[g] = qnormalize_pos(qmul(quat_of(Rt), qnormalize_pos(make_float4(row[3], row[4], row[5], row[6]))));
    } else if (j <= 12) {
        const int p = j - 1;  // SH plane
        sh[(int64_t)p * n + g] = make_float4(row[8 + 4 * p], row[9 + 4 * p], row[10 + 4 * p], row[11 + 4 * p]);
    }
}

static CamMLP cam_mlp(const gsr_camera *c) {
    CamMLP k;
    for (int i = 0; i < 9; ++i) k.R[i] = c->R[i];
    for (int i = 0; i < 3; ++i) k.t[i] = c->t[i];
    k.fx = c->fx; k.fy = c->fy; k.cx = c->cx; k.cy = c->cy;
    return k;
}

// ---------------------------------------------------------------- workspace
struct MlpLayout {
    size_t h1, h1t, h2, h2t, y, dy, dyt, dpre2, dpre2t, dpre1t, gW1, gb1, gW2, gb2, gW3t, gb3, total;
};

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

static MlpLayout mlp_layout(int64_t Mpad) {
    MlpLayout L;
    size_t o = 0;
    const size_t bf = 2, f4 = 4, mp = (size_t)Mpad;
    L.h1 = o; o += a256(bf * mp * kH);
    L.h1t = o; o += a256(bf * mp * kH);
    L.h2 = o; o += a256(bf * mp * kH);
    L.h2t = o; o += a256(bf * mp * kH);
    L.y = o; o += a256(f4 * mp * kN3);
    L.dy = o; o += a256(bf * mp * kN3);
    L.dyt = o; o += a256(bf * mp * kN3);
    L.dpre2 = o; o += a256(bf * mp * kH);
    L.dpre2t = o; o += a256(bf * mp * kH);
    L.dpre1t = o; o += a256(bf * mp * kH);
    L.gW1 = o; o += a256(f4 * kH * kK0);
    L.gb1 = o; o += a256(f4 * kH);
    L.gW2 = o; o += a256(f4 * kH * kH);
    L.gb2 = o; o += a256(f4 * kH);
    L.gW3t = o; o += a256(f4 * kH * kN3);
    L.gb3 = o; o += a256(f4 * kN3);
    L.total = o;
    return L;
}

static int32_t check_weights(const gsr_mlp_weights *w, bool need_half) {
    if (!w || !w->W1 || !w->b1 || !w->W2 || !w->b2 || !w->W3 || !w->b3 ||
        (need_half && (!w->W1h || !w->W2h || !w->W2hT || !w->W3h || !w->W3hT))) {
        set_error("gsr_mlp: weight pointer missing");
        return GSR_ERR_INVALID_ARG;
    }
    return GSR_OK;
}

static int ksplit_for(int64_t Mpad, int out_tiles) {
    // enough CTAs to cover the GPU when the reduction runs over the batch
    const int64_t kt = Mpad / umma::BK;
    int s = (int)((296 + out_tiles - 1) / out_tiles);
    if (s > kt) s = (int)kt;
    return s < 1 ? 1 : s;
}

}  // namespace gsr

extern "C" int32_t gsr_mlp_workspace_size(int64_t Mpad, size_t *bytes) {
    if (Mpad <= 0 || Mpad % 128 || !bytes) {
        set_error("gsr_mlp_workspace_size: the padded batch must be a positive multiple of 128");
        return GSR_ERR_INVALID_ARG;
    }
    *bytes = mlp_layout(Mpad).total;
    return GSR_OK;
}

extern "C" int32_t gsr_mlp_sync_weights(const gsr_mlp_weights *w, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = check_weights(w, true))) return rc;
    cudaStream_t st = as_cuda(stream);
    auto conv = [&](const float *p, int rows, int cols, void *ph, void *phT) {
        const int64_t tot = (int64_t)rows * cols;
        to_bf16_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(p, rows, cols, (__nv_bfloat16 *)ph,
                                                                      (__nv_bfloat16 *)phT);
    };
    conv(w->W1, kH, kK0, w->W1h, nullptr);
    conv(w->W2, kH, kH, w->W2h, w->W2hT);
    conv(w->W3, kN3, kH, w->W3h, w->W3hT);
    return check_launch("mlp weight copies");
}

extern "C" int32_t gsr_patch_gather(const float *level0, const float *level1, const float *level2, int32_t W0,
                                    int32_t H0, const float *keypoints, int64_t M, int64_t Mpad, void *x, void *xT,
                                    gsr_stream_t stream) {
    if (!level0 || !level1 || !level2 || W0 <= 0 || H0 <= 0 || M < 0 || Mpad < M || Mpad % 128 || !x ||
        (M > 0 && !keypoints)) {
        set_error("gsr_patch_gather: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    cudaStream_t st = as_cuda(stream);
    const int64_t tot = Mpad * kK0;
    patch_gather_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(level0, level1, level2, W0, H0, keypoints, M,
                                                                       Mpad, (__nv_bfloat16 *)x);
    if (xT) {
        const dim3 grid((unsigned)((kK0 + 31) / 32), (unsigned)((Mpad + 31) / 32));
        transpose_bf16_kernel<<<grid, dim3(32, 8), 0, st>>>((const __nv_bfloat16 *)x, (__nv_bfloat16 *)xT, Mpad, kK0);
    }
    return check_launch("patch gather");
}

// forward into the workspace buffers (h1, h2 and, when training, their transposes)
static int32_t mlp_forward_ws(const gsr_mlp_weights *w, const void *x, int64_t Mpad, float *y, char *ws,
                              const MlpLayout &L, bool train, int32_t *d_status, cudaStream_t st) {
    umma::Epilogue e1{};
    e1.bias = w->b1; e1.relu = 1;
    e1.out_bf16 = (__nv_bfloat16 *)(ws + L.h1); e1.ldo = kH;
    if (train) { e1.out_bf16_t = (__nv_bfloat16 *)(ws + L.h1t); e1.ldt = (int)Mpad; }
    e1.valid_rows = Mpad;
    int32_t rc = gemm_bf16(x, kK0, w->W1h, kK0, (int)Mpad, kH, kK0, e1, 1, d_status, st);
    if (rc) return rc;
    umma::Epilogue e2{};
    e2.bias = w->b2; e2.relu = 1;
    e2.out_bf16 = (__nv_bfloat16 *)(ws + L.h2); e2.ldo = kH;
    if (train) { e2.out_bf16_t = (__nv_bfloat16 *)(ws + L.h2t); e2.ldt = (int)Mpad; }
    e2.valid_rows = Mpad;
    if ((rc = gemm_bf16(ws + L.h1, kH, w->W2h, kH, (int)Mpad, kH, kH, e2, 1, d_status, st))) return rc;
    umma::Epilogue e3{};
    e3.bias = w->b3;
    e3.out_f32 = y; e3.ldf = kN3;
    e3.valid_rows = Mpad;
    return gemm_bf16(ws + L.h2, kH, w->W3h, kH, (int)Mpad, kN3, kH, e3, 1, d_status, st);
}

extern "C" int32_t gsr_mlp_forward(const gsr_mlp_weights *w, const void *x, int64_t Mpad, float *y, void *workspace,
                                   size_t workspace_bytes, int32_t *d_status, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = check_weights(w, true))) return rc;
    if (!x || !y || Mpad <= 0 || Mpad % 128) {
        set_error("gsr_mlp_forward: bad arguments (the padded batch must be a multiple of 128)");
        return GSR_ERR_INVALID_ARG;
    }
    const MlpLayout L = mlp_layout(Mpad);
    if (!workspace || workspace_bytes < L.total) {
        set_error("gsr_mlp_forward: workspace of %zu bytes needed", L.total);
        return GSR_ERR_CAPACITY;
    }
    return mlp_forward_ws(w, x, Mpad, y, static_cast<char *>(workspace), L, false, d_status, as_cuda(stream));
}

extern "C" int32_t gsr_mlp_train_step(const gsr_mlp_weights *w, const gsr_mlp_weights *m, const gsr_mlp_weights *v,
                                      const void *x, const void *xT, const float *target, const float *out_weight,
                                      int64_t M, int64_t Mpad, float lr, float beta1, float beta2, float eps,
                                      int32_t *d_step, float *d_loss, float *y, void *workspace,
                                      size_t workspace_bytes, int32_t *d_status, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = check_weights(w, true)) || (rc = check_weights(m, false)) || (rc = check_weights(v, false))) return rc;
    if (!x || !xT || !target || !out_weight || !d_step || !d_loss || !y || M <= 0 || Mpad < M || Mpad % 128 ||
        !(lr > 0.f)) {
        set_error("gsr_mlp_train_step: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    const MlpLayout L = mlp_layout(Mpad);
    if (!workspace || workspace_bytes < L.total) {
        set_error("gsr_mlp_train_step: workspace of %zu bytes needed", L.total);
        return GSR_ERR_CAPACITY;
    }
    cudaStream_t st = as_cuda(stream);
    char *ws = static_cast<char *>(workspace);
    auto bf = [&](size_t off) { return (__nv_bfloat16 *)(ws + off); };
    auto f32 = [&](size_t off) { return (float *)(ws + off); };
    // gradient accumulators start at zero
    if (cudaMemsetAsync(ws + L.gW1, 0, L.total - L.gW1, st) != cudaSuccess ||
        cudaMemsetAsync(d_loss, 0, sizeof(float), st) != cudaSuccess)
        return check_launch("mlp memset");
    if ((rc = mlp_forward_ws(w, x, Mpad, y, ws, L, true, d_status, st))) return rc;
    const int64_t loss_blocks = Mpad / kLossRows < 2 * 148 ? Mpad / kLossRows : 2 * 148;
    mlp_loss_kernel<<<(unsigned)loss_blocks, 256, 0, st>>>(y, target, out_weight, M, Mpad, bf(L.dy), bf(L.dyt),
                                                           f32(L.gb3), d_loss);
    if ((rc = check_launch("mlp loss"))) return rc;
    // dW3^T = h2^T dy  (K = batch, split)
    umma::Epilogue g3{};
    g3.out_f32 = f32(L.gW3t); g3.ldf = kN3; g3.atomic_f32 = 1; g3.valid_rows = kH;
    // split-K over BN = 64 tiles: ~2 CTAs per SM, each split adds its partial tile atomically
    if ((rc = gemm_bf16(bf(L.h2t), Mpad, bf(L.dyt), Mpad, kH, kN3, (int)Mpad, g3, ksplit_for(Mpad, 8), d_status, st,
                        true)))
        return rc;
    // dpre2 = (dy W3) masked by h2 > 0; both layouts; gb2
    umma::Epilogue d2{};
    d2.mask = (const __nv_bfloat16 *)(ws + L.h2); d2.ldm = kH;
    d2.out_bf16 = bf(L.dpre2); d2.ldo = kH;
    d2.out_bf16_t = bf(L.dpre2t); d2.ldt = (int)Mpad;
    d2.colsum = f32(L.gb2); d2.valid_rows = M;
    if ((rc = gemm_bf16(bf(L.dy), kN3, w->W3hT, kN3, (int)Mpad, kH, kN3, d2, 1, d_status, st))) return rc;
    // dW2 = dpre2^T h1
    umma::Epilogue g2{};
    g2.out_f32 = f32(L.gW2); g2.ldf = kH; g2.atomic_f32 = 1; g2.valid_rows = kH;
    if ((rc = gemm_bf16(bf(L.dpre2t), Mpad, bf(L.h1t), Mpad, kH, kH, (int)Mpad, g2, ksplit_for(Mpad, 8), d_status,
                        st, true)))
        return rc;
    // dpre1^T = ((dpre2 W2) masked by h1 > 0)^T; gb1
    umma::Epilogue d1{};
    d1.mask = (const __nv_bfloat16 *)(ws + L.h1); d1.ldm = kH;
    d1.out_bf16_t = bf(L.dpre1t); d1.ldt = (int)Mpad;
    d1.colsum = f32(L.gb1); d1.valid_rows = M;
    if ((rc = gemm_bf16(bf(L.dpre2), kH, w->W2hT, kH, (int)Mpad, kH, kH, d1, 1, d_status, st))) return rc;
    // dW1 = dpre1^T x
    umma::Epilogue g1{};
    g1.out_f32 = f32(L.gW1); g1.ldf = kK0; g1.atomic_f32 = 1; g1.valid_rows = kH;
    if ((rc = gemm_bf16(bf(L.dpre1t), Mpad, xT, Mpad, kH, kK0, (int)Mpad, g1, ksplit_for(Mpad, 2 * 37), d_status,
                        st)))
        return rc;
    // Adam on every tensor (FP32 masters), refreshed BF16 copies, one launch
    MlpAdamSet S{};
    auto bfp = [](void *q) { return (__nv_bfloat16 *)q; };
    S.t[0] = MlpAdamT{w->W1, f32(L.gW1), m->W1, v->W1, 0, kH, kK0, bfp(w->W1h), nullptr};
    S.t[1] = MlpAdamT{w->b1, f32(L.gb1), m->b1, v->b1, 0, 1, kH, nullptr, nullptr};
    S.t[2] = MlpAdamT{w->W2, f32(L.gW2), m->W2, v->W2, 0, kH, kH, bfp(w->W2h), bfp(w->W2hT)};
    S.t[3] = MlpAdamT{w->b2, f32(L.gb2), m->b2, v->b2, 0, 1, kH, nullptr, nullptr};
    S.t[4] = MlpAdamT{w->W3, f32(L.gW3t), m->W3, v->W3, 1, kN3, kH, bfp(w->W3h), bfp(w->W3hT)};
    S.t[5] = MlpAdamT{w->b3, f32(L.gb3), m->b3, v->b3, 0, 1, kN3, nullptr, nullptr};
    S.off[0] = 0;
    for (int k = 0; k < 6; ++k) S.off[k + 1] = S.off[k] + (int64_t)S.t[k].rows * S.t[k].cols;
    mlp_adam_all_kernel<<<(unsigned)((S.off[6] + 255) / 256), 256, 0, st>>>(S, lr, beta1, beta2, eps, d_step);
    step_advance_mlp_kernel<<<1, 1, 0, st>>>(d_step);
    return check_launch("mlp adam");
}

extern "C" int32_t gsr_mlp_encode_targets(const gsr_gaussians *g, const uint32_t *gids, const float *keypoints,
                                          int64_t M, int64_t Mpad, const gsr_camera *cam, const float *base,
                                          float *target, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_gaussians(g)) || (rc = validate_camera(cam))) return rc;
    if (M < 0 || Mpad < M || !target || (M > 0 && (!gids || !keypoints))) {
        set_error("gsr_mlp_encode_targets: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    if (Mpad == 0) return GSR_OK;
    mlp_encode_kernel<<<(unsigned)Mpad, kN3, 0, as_cuda(stream)>>>(
        reinterpret_cast<const float4 *>(g->mean_op), reinterpret_cast<const float4 *>(g->quat),
        reinterpret_cast<const float4 *>(g->logscale), reinterpret_cast<const float4 *>(g->sh), g->n, gids, keypoints,
        M, cam_mlp(cam), base, target);
    return check_launch("mlp_encode_kernel");
}

extern "C" int32_t gsr_mlp_decode(const float *y, const float *base, const float *keypoints, int64_t M,
                                  const gsr_camera *cam, const gsr_param_buffers *out, int64_t n, int64_t offset,
                                  gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_camera(cam))) return rc;
    if (M < 0 || !out || !out->mean_op || !out->quat || !out->logscale || !out->sh || offset < 0 || offset + M > n ||
        (M > 0 && (!y || !keypoints))) {
        set_error("gsr_mlp_decode: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    if (M == 0) return GSR_OK;
    mlp_decode_kernel<<<(unsigned)M, 64, 0, as_cuda(stream)>>>(
        y, base, keypoints, M, cam_mlp(cam), reinterpret_cast<float4 *>(out->mean_op), reinterpret_cast<float4 *>(out->quat),
        reinterpret_cast<float4 *>(out->logscale), reinterpret_cast<float4 *>(out->sh), n, offset);
    return check_launch("mlp_decode_kernel");
}

extern "C" int32_t gsr_mlp_gradients(void *workspace, int64_t Mpad, gsr_mlp_weights *grads) {
    if (!workspace || !grads || Mpad <= 0 || Mpad % 128) {
        set_error("gsr_mlp_gradients: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    const MlpLayout L = mlp_layout(Mpad);
    char *ws = static_cast<char *>(workspace);
    *grads = gsr_mlp_weights{};
    grads->W1 = (float *)(ws + L.gW1);
    grads->b1 = (float *)(ws + L.gb1);
    grads->W2 = (float *)(ws + L.gW2);
    grads->b2 = (float *)(ws + L.gb2);
    grads->W3 = (float *)(ws + L.gW3t);
    grads->b3 = (float *)(ws + L.gb3);
    return GSR_OK;
}
