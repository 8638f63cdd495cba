// order.cu -- spatial order of the map store (map maintenance, not part of a
// mapping iteration).
//
// The iteration's per-Gaussian kernels (projection and decisions, the chain
// rule, the pose chain) run one thread per Gaussian; when the Gaussians a
// warp holds are spatial neighbours they tend to pass or fail the view's
// visibility decisions together (a warp whose 32 Gaussians are all outside
// the view skips the covariance and its projection), and the visible ones'
// parameter planes are read as runs instead of scattered 16-byte pieces.
// gsr_spatial_order sorts the Gaussians by the Morton code of their means
// (Z-order curve: the bits of the three quantised coordinates interleaved)
// and gsr_permute applies the permutation to any parameter-shaped buffers
// (parameters, Adam moments).
#include <algorithm>

#include "gsr_internal.cuh"

namespace gsr {

constexpr int kOrderThreads = 1024;

// 10 bits of v spread to every third bit (bit b -> bit 3 b)
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void __launch_bounds__(256) morton_kernel(const float4 *__restrict__ mean_op, int64_t n, float lox,
                                                     float loy, float loz, float sx, float sy, float sz,
                                                     uint64_t *__restrict__ keys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = __ldg(mean_op + i);
    auto q = [](float v, float lo, float s) {
        float t = (v - lo) * s;  // in [0, 1024) inside the box
        t = fminf(fmaxf(t, 0.0f), 1023.0f);
        return (uint32_t)t;  // NaN -> 0 after the clamps' NaN handling
    };
    const uint32_t code = spread3(q(p.x, lox, sx)) | (spread3(q(p.y, loy, sy)) << 1) | (spread3(q(p.z, loz, sz)) << 2);
    keys[i] = ((uint64_t)code << 32) | (uint64_t)i;
}

// Stable LSD radix sort of a[0, n) by bits 32 .. 63 (8 bits a pass, the
// passes that can hold set bits of a 30-bit code), by one CTA, through b;
// equal codes keep their (index) order.  The result ends in a (even number
// of passes).
__global__ void __launch_bounds__(kOrderThreads) order_sort_kernel(uint64_t *__restrict__ a, uint64_t *__restrict__ b,
                                                                   int64_t n) {
    constexpr int kWarps = kOrderThreads / 32;
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_wcnt[kWarps * 256];
    __shared__ uint32_t s_tmp[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 32 + 8 * pass;
        for (int d = t; d < 256; d += kOrderThreads) s_base[d] = 0u;
        __syncthreads();
        for (int64_t i = t; i < n; i += kOrderThreads) atomicAdd(&s_base[(uint32_t)(a[i] >> shift) & 0xffu], 1u);
        __syncthreads();
        {  // exclusive scan of the 256 digit counts by the first 8 warps
            uint32_t v = t < 256 ? s_base[t] : 0u, incl = v;
            if (t < 256) {
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                if (lane == 31) s_tmp[wid] = incl;
            }
            __syncthreads();
            if (t < 256) {
                uint32_t add = 0;
                for (int w = 0; w < wid; ++w) add += s_tmp[w];
                s_base[t] = add + incl - v;
            }
            __syncthreads();
        }
        // chunks of the CTA's width in index order: per-warp ranks by digit,
        // warps in order within the chunk, chunks in order -> stable
        for (int64_t c0 = 0; c0 < n; c0 += kOrderThreads) {
            for (int k = t; k < kWarps * 256; k += kOrderThreads) s_wcnt[k] = 0u;
            __syncthreads();
            const int64_t i = c0 + t;
            const bool valid = i < n;
            const uint64_t key = valid ? a[i] : 0ull;
            const uint32_t d = valid ? (uint32_t)(key >> shift) & 0xffu : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t rank = __popc(peers & lt);
            if (valid && rank == 0) s_wcnt[wid * 256 + d] = __popc(peers);
            __syncthreads();
            for (int dd = t; dd < 256; dd += kOrderThreads) {
                uint32_t run = s_base[dd];
                for (int w = 0; w < kWarps; ++w) {
                    const uint32_t c = s_wcnt[w * 256 + dd];
                    s_wcnt[w * 256 + dd] = run;
                    run += c;
                }
                s_base[dd] = run;
            }
            __syncthreads();
            if (valid) b[s_wcnt[wid * 256 + d] + rank] = key;
            __syncthreads();
        }
        uint64_t *tmp = a;
        a = b;
        b = tmp;
    }
}

__global__ void __launch_bounds__(256) order_emit_kernel(const uint64_t *__restrict__ keys, int64_t n,
                                                         uint32_t *__restrict__ perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = (uint32_t)keys[i];
}

// dst plane p, entry i = src plane p, entry perm[i]; blockIdx.y = plane (15)
__global__ void __launch_bounds__(256) permute_kernel(gsr_param_buffers src, gsr_param_buffers dst,
                                                      const uint32_t *__restrict__ perm, int64_t n) {
    const int plane = (int)blockIdx.y;
    const float4 *s;
    float4 *d;
    if (plane == 0) {
        s = reinterpret_cast<const float4 *>(src.mean_op);
        d = reinterpret_cast<float4 *>(dst.mean_op);
    } else if (plane == 1) {
        s = reinterpret_cast<const float4 *>(src.quat);
        d = reinterpret_cast<float4 *>(dst.quat);
    } else if (plane == 2) {
        s = reinterpret_cast<const float4 *>(src.logscale);
        d = reinterpret_cast<float4 *>(dst.logscale);
    } else {
        s = reinterpret_cast<const float4 *>(src.sh) + (int64_t)(plane - 3) * n;
        d = reinterpret_cast<float4 *>(dst.sh) + (int64_t)(plane - 3) * n;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = __ldg(s + perm[i]);
}

}  // namespace gsr

using namespace gsr;

extern "C" int32_t gsr_spatial_order_workspace_size(int64_t n, size_t *bytes) {
    if (n < 0 || !bytes) {
        set_error("gsr_spatial_order_workspace_size: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    *bytes = 2 * sizeof(uint64_t) * (size_t)(n > 0 ? n : 1);
    return GSR_OK;
}

extern "C" int32_t gsr_spatial_order(const gsr_gaussians *g, const float *lo, const float *hi, uint32_t *perm,
                                     void *workspace, size_t workspace_bytes, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_gaussians(g))) return rc;
    if (!lo || !hi || (g->n > 0 && !perm) || g->n > (int64_t)0xffffffffLL) {
        set_error("gsr_spatial_order: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    for (int k = 0; k < 3; ++k)
        if (!(hi[k] > lo[k])) {
            set_error("gsr_spatial_order: the box must have hi > lo on every axis");
            return GSR_ERR_INVALID_ARG;
        }
    size_t need;
    gsr_spatial_order_workspace_size(g->n, &need);
    if (!workspace || workspace_bytes < need) {
        set_error("gsr_spatial_order: workspace of %zu bytes needed", need);
        return GSR_ERR_CAPACITY;
    }
    if (g->n == 0) return GSR_OK;
    cudaStream_t st = as_cuda(stream);
    uint64_t *a = static_cast<uint64_t *>(workspace), *b = a + g->n;
    const unsigned blocks = (unsigned)((g->n + 255) / 256);
    morton_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const float4 *>(g->mean_op), g->n, lo[0], lo[1], lo[2],
                                          1024.0f / (hi[0] - lo[0]), 1024.0f / (hi[1] - lo[1]),
                                          1024.0f / (hi[2] - lo[2]), a);
    order_sort_kernel<<<1, kOrderThreads, 0, st>>>(a, b, g->n);
    order_emit_kernel<<<blocks, 256, 0, st>>>(a, g->n, perm);
    return check_launch("gsr_spatial_order");
}

extern "C" int32_t gsr_permute(const gsr_param_buffers *src, const gsr_param_buffers *dst, const uint32_t *perm,
                               int64_t n, gsr_stream_t stream) {
    if (n < 0 || !src || !dst || (n > 0 && (!perm || !src->mean_op || !src->quat || !src->logscale || !src->sh ||
                                            !dst->mean_op || !dst->quat || !dst->logscale || !dst->sh))) {
        set_error("gsr_permute: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    if (!aligned16(src->mean_op) || !aligned16(src->quat) || !aligned16(src->logscale) || !aligned16(src->sh) ||
        !aligned16(dst->mean_op) || !aligned16(dst->quat) || !aligned16(dst->logscale) || !aligned16(dst->sh)) {
        set_error("gsr_permute: buffers must be 16-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    if (n == 0) return GSR_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 148 * 4);
    permute_kernel<<<dim3((unsigned)blocks, 15), 256, 0, as_cuda(stream)>>>(*src, *dst, perm, n);
    return check_launch("permute_kernel");
}
