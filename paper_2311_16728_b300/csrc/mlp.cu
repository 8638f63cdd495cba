// mlp.cu -- the learned initialiser of new primitives (the build's answer to
// Photo-SLAM's geometry-based densification, arXiv 2311.16728 Sec. 3.3.1,
// which does not say how new primitives are initialised): a 2308 -> 256 ->
// 256 -> 56 ReLU MLP over multi-level image patches, in BF16 with FP32
// accumulation on the tcgen05 tensor cores (umma_gemm.cuh), trained by MSE
// with Adam on FP32 master weights.
#include <cudaTypedefs.h>

#include <mutex>

#include "umma_gemm.cuh"

namespace gsr {

// ---------------------------------------------------------------- tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
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

template <int BN>
static int32_t launch_gemm_bn(const void *A, int64_t lda, const void *B, int64_t ldb, int M, int N, int K,
                              const umma::Epilogue &ep, int ksplit, int32_t *d_status, cudaStream_t st) {
    using Cfg = umma::Config<BN>;
    CUtensorMap ma, mb;
    int32_t rc;
    if ((rc = make_map(&ma, A, M, K, lda, umma::BM)) || (rc = make_map(&mb, B, N, K, ldb, BN))) return rc;
    cudaFuncSetAttribute(umma::gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
    const dim3 grid(N / BN, M / umma::BM, ksplit);
    umma::gemm_kernel<BN><<<grid, 192, Cfg::kSmem, st>>>(ma, mb, K, ep, d_status);
    return check_launch("umma gemm_kernel");
}

// D = A B^T with A [M x K], B [N x K] BF16 K-major; M % 128 == 0, N % 64 == 0,
// K % 64 == 0; the widest BN in {256, 128, 64} that divides N.
int32_t gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, int M, int N, int K,
                  const umma::Epilogue &ep, int ksplit, int32_t *d_status, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0 || M % umma::BM || N % 64 || K % umma::BK || ksplit < 1 || !aligned16(A) ||
        !aligned16(B) || lda % 8 || ldb % 8) {
        set_error("gemm_bf16: need M %% 128 == 0, N %% 64 == 0, K %% 64 == 0, 16-byte aligned operands "
                  "(M=%d N=%d K=%d)", M, N, K);
        return GSR_ERR_INVALID_ARG;
    }
    if (ksplit > K / umma::BK) ksplit = K / umma::BK;
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
