// umma_gemm.cuh -- BF16 x BF16 -> FP32 GEMM on the sm_100-family tensor cores
// (tcgen05.mma, accumulator in tensor memory), operands staged by TMA.
//
//   D[M x N] = A[M x K] * B[N x K]^T      (both operands K-major, row-major
//                                           storage with K contiguous)
//
// CTA tile 128 x BN (BN = 64, 128 or 256), K step 64 (one 128-byte swizzled
// row per operand row).  Warp 0 issues the TMA loads into an mbarrier ring of
// shared-memory stages, warp 1 issues the MMAs (one elected thread), warps
// 2..5 drain the accumulator from tensor memory and apply the epilogue.
// Every wait is bounded; a wait that gives up raises GSR_ERR_TIMEOUT in the
// status word and the CTA winds down (its copies and MMAs are still waited
// for, with a bound, before tensor memory is released).
#pragma once

#include <cuda_bf16.h>

#include "tma.cuh"

namespace gsr {
namespace umma {

constexpr int BM = 128, BK = 64;
using tma::kSpinLimit;
using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_try_wait;
using tma::mbar_wait;
using tma::fence_barrier_init;
using tma::smem_u32;

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
    tma::load_2d(dst, map, c0, c1, bar);
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 B, 8-row groups 1024 B apart (stride
// dimension byte offset), leading-dimension offset unused (1), version bits
// 46-48 = 0b001, swizzle mode 2 (128 B).  The tile base is 1024-B aligned.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x 16 columns of 32-bit words: this thread's row, 16 columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Epilogue of one GEMM (all pointers optional; M, N are the padded extents).
struct Epilogue {
    const float *bias;            // [N]        v += bias[n]
    int relu;                     //            v = max(v, 0)
    const __nv_bfloat16 *mask;    // [M x ldm]  v = mask[m][n] > 0 ? v : 0 (ReLU derivative)
    int ldm;
    __nv_bfloat16 *out_bf16;      // [M x ldo]  row-major BF16
    int ldo;
    __nv_bfloat16 *out_bf16_t;    // [N x ldt]  transposed BF16 (element (n, m))
    int ldt;
    float *out_f32;               // [M x ldf]  FP32 (added atomically when atomic_f32)
    int ldf;
    int atomic_f32;
    float *colsum;                // [N]        colsum[n] += sum over valid rows of v (after mask / relu)
    int64_t valid_rows;           //            rows >= valid_rows are padding: not summed
    int vec_mask, vec_out;        // set by the launcher: mask / out_bf16 rows are 16-byte aligned, so a
                                  // lane moves its 16 columns as two 16-byte words
    int vec_t;                    // set by the launcher: out_bf16_t columns are 16-byte aligned, so the
                                  // warp transposes its 32 x 16 block through shared memory
};

// row stride (BF16 elements) of a warp's transposed 16 x 32 staging block
constexpr int kTStride = 40;

// ST: stages of the shared-memory ring (default 4 for BN = 256, else 6); a
// short reduction takes 2, so that several CTAs fit on an SM.
template <int BN, int ST = (BN == 256 ? 4 : 6)>
struct Config {
    static constexpr int kStages = ST;
    static constexpr int kABytes = BM * BK * 2;
    static constexpr int kBBytes = BN * BK * 2;
    static constexpr int kStageBytes = kABytes + kBBytes;
    static constexpr int kTmemCols = BN < 32 ? 32 : BN;
    static constexpr size_t kSmem = 1024 + (size_t)kStages * kStageBytes + 256;
};

// grid: (N / BN, M / BM, ksplit); K tiles of this CTA: the z-th slice.
template <int BN, int ST = (BN == 256 ? 4 : 6)>
__global__ void __launch_bounds__(192, 4) gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, int K, Epilogue ep,
                                                      int32_t *d_status) {
    using Cfg = Config<BN, ST>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);  // 1024-B aligned stages
    uint8_t *bar_area = smem + (size_t)Cfg::kStages * Cfg::kStageBytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(bar_area);
    uint64_t *empty = full + Cfg::kStages;
    uint64_t *tmem_full = empty + Cfg::kStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tmem_full + 1);
    __shared__ int s_err;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
    const int ktiles = K / BK;
    const int kz = gridDim.z, z = blockIdx.z;
    const int kt0 = (int)((int64_t)ktiles * z / kz), kt1 = (int)((int64_t)ktiles * (z + 1) / kz);
    const int nk = kt1 - kt0;

    if (threadIdx.x == 0) {
        s_err = 0;
        for (int s = 0; s < Cfg::kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tmem_full, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, Cfg::kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            for (int i = 0; i < nk; ++i) {
                const int s = i % Cfg::kStages;
                if (i >= Cfg::kStages && !mbar_wait(&empty[s], ((i / Cfg::kStages) - 1) & 1)) {
                    atomicExch(&s_err, 1);
                    break;
                }
                uint8_t *sa = smem + (size_t)s * Cfg::kStageBytes;
                mbar_expect_tx(&full[s], Cfg::kStageBytes);
                tma_load_2d(sa, &tmA, (kt0 + i) * BK, m0, &full[s]);
                tma_load_2d(sa + Cfg::kABytes, &tmB, (kt0 + i) * BK, n0, &full[s]);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BM, BN);
            for (int i = 0; i < nk; ++i) {
                const int s = i % Cfg::kStages;
                if (!mbar_wait(&full[s], (i / Cfg::kStages) & 1)) {
                    atomicExch(&s_err, 1);
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + (size_t)s * Cfg::kStageBytes);
                const uint64_t da = desc_sw128(sa), db = desc_sw128(sa + Cfg::kABytes);
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)  // 16 BF16 = 32 B per MMA step along K
                    mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc, (i > 0 || k > 0) ? 1u : 0u);
                mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
            }
            mma_commit(tmem_full);  // all MMAs issued so far, done or not, are tracked
        }
    } else {
        // ---------------- epilogue: warps 2..5, lane quarter = warp % 4
        const int q = warp & 3;
        const int m = m0 + 32 * q + lane;
        const bool ok = mbar_wait(tmem_full, 0);
        if (!ok) atomicExch(&s_err, 1);
        tc_fence_after();
        if (ok && nk > 0) {
            const bool row_valid = m < ep.valid_rows;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
                const int nb = n0 + c0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (ep.bias) v[j] += ep.bias[nb + j];
                    if (ep.relu) v[j] = fmaxf(v[j], 0.0f);
                }
                if (ep.mask) {
                    const __nv_bfloat16 *mr = ep.mask + (int64_t)m * ep.ldm + nb;
                    if (ep.vec_mask) {
                        uint4 w[2];
                        w[0] = *reinterpret_cast<const uint4 *>(mr);
                        w[1] = *reinterpret_cast<const uint4 *>(mr + 8);
                        const __nv_bfloat16 *mb = reinterpret_cast<const __nv_bfloat16 *>(w);
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (!(__bfloat162float(mb[j]) > 0.0f)) v[j] = 0.0f;
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (!(__bfloat162float(mr[j]) > 0.0f)) v[j] = 0.0f;
                    }
                }
                if (ep.out_bf16) {
                    __nv_bfloat16 *o = ep.out_bf16 + (int64_t)m * ep.ldo + nb;
                    if (ep.vec_out) {
                        uint4 w[2];
                        __nv_bfloat162 *wb = reinterpret_cast<__nv_bfloat162 *>(w);
#pragma unroll
                        for (int j = 0; j < 16; j += 2) wb[j / 2] = __floats2bfloat162_rn(v[j], v[j + 1]);
                        *reinterpret_cast<uint4 *>(o) = w[0];
                        *reinterpret_cast<uint4 *>(o + 8) = w[1];
                    } else {  // any row stride: one element at a time
#pragma unroll
                        for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16_rn(v[j]);
                    }
                }
                if (ep.out_bf16_t) {
                    if (ep.vec_t) {
                        // the ring's shared memory is free once every MMA has completed:
                        // column j of the warp's block goes to staging row j, then each
                        // lane stores 8 consecutive rows of one column as one 16-byte word
                        __nv_bfloat16 *stg = reinterpret_cast<__nv_bfloat16 *>(smem) + q * 16 * kTStride;
#pragma unroll
                        for (int j = 0; j < 16; ++j) stg[j * kTStride + lane] = __float2bfloat16_rn(v[j]);
                        __syncwarp();
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const int c = 8 * i + (lane >> 2), r8 = 8 * (lane & 3);
                            const uint4 w = *reinterpret_cast<const uint4 *>(stg + c * kTStride + r8);
                            *reinterpret_cast<uint4 *>(ep.out_bf16_t + (int64_t)(nb + c) * ep.ldt + (m0 + 32 * q + r8)) = w;
                        }
                        __syncwarp();
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            ep.out_bf16_t[(int64_t)(nb + j) * ep.ldt + m] = __float2bfloat16_rn(v[j]);
                    }
                }
                if (ep.out_f32) {
                    float *o = ep.out_f32 + (int64_t)m * ep.ldf + nb;
                    if (ep.atomic_f32) {
                        // vector reductions (16-byte aligned: ldf % 4 == 0, nb % 16 == 0)
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            atomicAdd(reinterpret_cast<float4 *>(o + j), make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4 *>(o + j) =
                            make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    }
                }
                if (ep.colsum) {
                    // column sums over the warp's 32 rows by a transposing
                    // butterfly: each stage halves the values a lane keeps (16
                    // shuffles in all); lane l ends with column
                    // 8 b4 + 4 b3 + 2 b2 + b1 of its bits, lanes l and l ^ 1 alike
                    float s16[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) s16[j] = row_valid ? v[j] : 0.0f;
                    float s8[8], s4[4], s2[2];
                    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float keep = b4 ? s16[j + 8] : s16[j], send = b4 ? s16[j] : s16[j + 8];
                        s8[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float keep = b3 ? s8[j + 4] : s8[j], send = b3 ? s8[j] : s8[j + 4];
                        s4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                    }
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const float keep = b2 ? s4[j + 2] : s4[j], send = b2 ? s4[j] : s4[j + 2];
                        s2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                    }
                    float s1 = (b1 ? s2[1] : s2[0]) + __shfl_xor_sync(0xffffffffu, b1 ? s2[0] : s2[1], 2);
                    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
                    const int col = (b4 ? 8 : 0) + (b3 ? 4 : 0) + (b2 ? 2 : 0) + (b1 ? 1 : 0);
                    if ((lane & 1) == 0) atomicAdd(ep.colsum + nb + col, s1);
                }
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (s_err) {
        // wind down: the last copies of the ring and the MMAs must have landed
        // before the shared memory and the tensor memory are given back
        if (threadIdx.x == 0) {
            raise_status(d_status, GSR_ERR_TIMEOUT);
            for (int s = 0; s < Cfg::kStages && s < nk; ++s) {
                const int i = nk - 1 - s;
                mbar_wait(&full[i % Cfg::kStages], (i / Cfg::kStages) & 1);
            }
            mbar_wait(tmem_full, 0);
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, Cfg::kTmemCols);
    }
}

}  // namespace umma
}  // namespace gsr
