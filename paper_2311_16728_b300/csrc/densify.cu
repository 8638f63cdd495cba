// densify.cu -- gradient-driven densification and pruning of the map.
//
// Photo-SLAM (arXiv 2311.16728, Sec. 3.3.1) splits or clones hyper
// primitives with large loss gradients, as 3D Gaussian splatting does, and
// drops nearly transparent ones.  Per input Gaussian i (decisions on FP32
// values, so that they are reproducible bit for bit):
//   g_i = stat_i / count_i (0 if never seen): the mean |dL/d(u, v)| in
//         normalised device coordinates accumulated by the chain rule;
//   prune   when the opacity logit < logit_min;
//   else, when g_i >= grad_thr: split if the largest log-scale >
//         logscale_split (two children at mu + R(q) (s * eps_k), log-scale
//         - shrink, the parent dropped), clone otherwise (the Gaussian and a
//         copy); keep otherwise.
// Survivors keep their Adam moments; new Gaussians (clone copies, split
// children) start with zero moments.  The outputs are written in input order
// to a second store of `cap` Gaussians whose tail [n_out, cap) is filled with
// inert padding (zero quaternion: never visible, never densified), so that a
// caller can keep running fixed-size launches over the whole capacity.
#include "gsr_internal.cuh"

namespace gsr {

constexpr int kDThreads = 256;
constexpr int kDItems = 4;
constexpr int kDTile = kDThreads * kDItems;

struct DensifyK {
    const float4 *p[4], *m[4], *v[4];  // inputs: mean_op, quat, logscale, sh planes (n each)
    float4 *po[4], *mo[4], *vo[4];     // outputs (cap each)
    const float *stat, *count, *eps;
    int64_t n, cap;
    float grad_thr, logit_min, logscale_split, shrink;
};

// 0 = prune (or padding: a zero quaternion), 1 = keep, 2 = clone, 3 = split
__device__ __forceinline__ int densify_kind(const DensifyK &a, int64_t i) {
    const float4 mo = a.p[0][i], q = a.p[1][i], ls = a.p[2][i];
    if (q.x == 0.f && q.y == 0.f && q.z == 0.f && q.w == 0.f) return 0;  // padding
    if (mo.w < a.logit_min) return 0;
    const float c = a.count[i];
    const float g = c > 0.0f ? __fdiv_rn(a.stat[i], c) : 0.0f;
    if (!(g >= a.grad_thr)) return 1;
    const float lmax = fmaxf(ls.x, fmaxf(ls.y, ls.z));
    return lmax > a.logscale_split ? 3 : 2;
}

__device__ __forceinline__ uint32_t outputs_of(int kind) { return kind == 0 ? 0u : (kind == 1 ? 1u : 2u); }

__device__ __forceinline__ uint32_t block_scan_incl(uint32_t v, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < kDThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < kDThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t add = wid > 0 ? s_warp[wid - 1] : 0u;
    __syncthreads();
    return v + add;
}

__global__ void __launch_bounds__(kDThreads) densify_count_kernel(DensifyK a, uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t s_warp[kDThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kDTile + (int64_t)threadIdx.x * kDItems;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kDItems; ++k)
        if (base + k < a.n) c += outputs_of(densify_kind(a, base + k));
    c = block_scan_incl(c, s_warp);
    if (threadIdx.x == kDThreads - 1) block_sums[blockIdx.x] = c;
}

__device__ __forceinline__ void put(float4 *const dst[4], int64_t cap, int64_t o, int plane, float4 val) {
    const int which = plane < 3 ? plane : 3;
    dst[which][plane < 3 ? o : (int64_t)(plane - 3) * cap + o] = val;
}

__device__ __forceinline__ float4 get(const float4 *const src[4], int64_t n, int64_t i, int plane) {
    const int which = plane < 3 ? plane : 3;
    return src[which][plane < 3 ? i : (int64_t)(plane - 3) * n + i];
}

__global__ void __launch_bounds__(kDThreads) densify_emit_kernel(DensifyK a, const uint32_t *__restrict__ block_sums,
                                                                 int64_t nblocks, int64_t *__restrict__ d_n_out,
                                                                 int32_t *__restrict__ d_status) {
    __shared__ uint32_t s_warp[kDThreads / 32];
    __shared__ int64_t s_red[2][kDThreads / 32];
    __shared__ int64_t s_pre, s_total;
    {  // this block's exclusive prefix and the total, over the block sums
        int64_t pre = 0, tot = 0;
        for (int64_t b = threadIdx.x; b < nblocks; b += kDThreads) {
            const int64_t v = block_sums[b];
            tot += v;
            if (b < (int64_t)blockIdx.x) pre += v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pre += __shfl_xor_sync(0xffffffffu, pre, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if ((threadIdx.x & 31) == 0) {
            s_red[0][threadIdx.x >> 5] = pre;
            s_red[1][threadIdx.x >> 5] = tot;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t p = 0, t = 0;
            for (int w = 0; w < kDThreads / 32; ++w) {
                p += s_red[0][w];
                t += s_red[1][w];
            }
            s_pre = p;
            s_total = t;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *d_n_out = s_total;
        if (s_total > a.cap) raise_status(d_status, GSR_ERR_CAPACITY);
    }
    const int64_t base = (int64_t)blockIdx.x * kDTile + (int64_t)threadIdx.x * kDItems;
    int kinds[kDItems];
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kDItems; ++k) {
        kinds[k] = base + k < a.n ? densify_kind(a, base + k) : 0;
        c += outputs_of(kinds[k]);
    }
    const uint32_t incl = block_scan_incl(c, s_warp);
    int64_t o = s_pre + (int64_t)(incl - c);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
    for (int k = 0; k < kDItems; ++k) {
        const int kind = kinds[k];
        if (kind == 0) continue;
        const int64_t i = base + k;
        const int outs = kind == 1 ? 1 : 2;
        if (o + outs > a.cap) {  // overflow: count only (the caller retries with more room)
            o += outs;
            continue;
        }
        if (kind != 3) {
            for (int pl = 0; pl < 3 + kShPlanes; ++pl) {
                const float4 pv = get(a.p, a.n, i, pl);
                put(a.po, a.cap, o, pl, pv);
                put(a.mo, a.cap, o, pl, get(a.m, a.n, i, pl));
                put(a.vo, a.cap, o, pl, get(a.v, a.n, i, pl));
                if (kind == 2) {
                    put(a.po, a.cap, o + 1, pl, pv);
                    put(a.mo, a.cap, o + 1, pl, zero);
                    put(a.vo, a.cap, o + 1, pl, zero);
                }
            }
        } else {
            const float4 mo = a.p[0][i], q = a.p[1][i], ls = a.p[2][i];
            const float nq = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
            const float w = q.x / nq, x = q.y / nq, y = q.z / nq, z = q.w / nq;
            const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                                2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                                2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
            const float s0 = expf(ls.x), s1 = expf(ls.y), s2 = expf(ls.z);
            const float4 lsc = make_float4(__fsub_rn(ls.x, a.shrink), __fsub_rn(ls.y, a.shrink),
                                           __fsub_rn(ls.z, a.shrink), ls.w);
            for (int kk = 0; kk < 2; ++kk) {
                const float *e = a.eps + 6 * i + 3 * kk;
                const float e0 = s0 * e[0], e1 = s1 * e[1], e2 = s2 * e[2];
                const float4 mean = make_float4(mo.x + R[0] * e0 + R[1] * e1 + R[2] * e2,
                                                mo.y + R[3] * e0 + R[4] * e1 + R[5] * e2,
                                                mo.z + R[6] * e0 + R[7] * e1 + R[8] * e2, mo.w);
                put(a.po, a.cap, o + kk, 0, mean);
                put(a.po, a.cap, o + kk, 1, q);
                put(a.po, a.cap, o + kk, 2, lsc);
                for (int pl = 3; pl < 3 + kShPlanes; ++pl) put(a.po, a.cap, o + kk, pl, get(a.p, a.n, i, pl));
                for (int pl = 0; pl < 3 + kShPlanes; ++pl) {
                    put(a.mo, a.cap, o + kk, pl, zero);
                    put(a.vo, a.cap, o + kk, pl, zero);
                }
            }
        }
        o += outs;
    }
}

// inert padding over [n_out, cap): zero everywhere (a zero quaternion is culled)
__global__ void __launch_bounds__(256) densify_pad_kernel(DensifyK a, const int64_t *__restrict__ d_n_out) {
    const int64_t n_out = *d_n_out;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < a.cap; o += (int64_t)gridDim.x * blockDim.x) {
        if (o < n_out) continue;
        for (int pl = 0; pl < 3 + kShPlanes; ++pl) {
            put(a.po, a.cap, o, pl, zero);
            put(a.mo, a.cap, o, pl, zero);
            put(a.vo, a.cap, o, pl, zero);
        }
    }
}

static bool planes_ok(const gsr_param_buffers *b) {
    return b && b->mean_op && b->quat && b->logscale && b->sh && aligned16(b->mean_op) && aligned16(b->quat) &&
           aligned16(b->logscale) && aligned16(b->sh);
}

}  // namespace gsr

using namespace gsr;

extern "C" int32_t gsr_densify_workspace_size(int64_t n, size_t *bytes) {
    if (n < 0 || !bytes) {
        set_error("gsr_densify_workspace_size: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    *bytes = sizeof(uint32_t) * (size_t)((n + kDTile - 1) / kDTile + 1) + 256;
    return GSR_OK;
}

extern "C" int32_t gsr_densify(const gsr_param_buffers *params, const gsr_param_buffers *m,
                               const gsr_param_buffers *v, int64_t n, const float *stat, const float *count,
                               const float *eps, const gsr_densify_config *cfg, const gsr_param_buffers *out_params,
                               const gsr_param_buffers *out_m, const gsr_param_buffers *out_v, int64_t cap,
                               int64_t *d_n_out, void *workspace, size_t workspace_bytes, int32_t *d_status,
                               gsr_stream_t stream) {
    if (n < 0 || cap < 0 || !cfg || !d_n_out || !planes_ok(params) || !planes_ok(m) || !planes_ok(v) ||
        !planes_ok(out_params) || !planes_ok(out_m) || !planes_ok(out_v) || (n > 0 && (!stat || !count || !eps))) {
        set_error("gsr_densify: bad arguments (buffers must be non-NULL and 16-byte aligned)");
        return GSR_ERR_INVALID_ARG;
    }
    size_t need;
    gsr_densify_workspace_size(n, &need);
    if (!workspace || workspace_bytes < need) {
        set_error("gsr_densify: workspace of %zu bytes needed", need);
        return GSR_ERR_CAPACITY;
    }
    DensifyK a;
    const gsr_param_buffers *in[3] = {params, m, v}, *outb[3] = {out_params, out_m, out_v};
    const float4 **ins[3] = {a.p, a.m, a.v};
    float4 **outs[3] = {a.po, a.mo, a.vo};
    for (int k = 0; k < 3; ++k) {
        ins[k][0] = reinterpret_cast<const float4 *>(in[k]->mean_op);
        ins[k][1] = reinterpret_cast<const float4 *>(in[k]->quat);
        ins[k][2] = reinterpret_cast<const float4 *>(in[k]->logscale);
        ins[k][3] = reinterpret_cast<const float4 *>(in[k]->sh);
        outs[k][0] = reinterpret_cast<float4 *>(outb[k]->mean_op);
        outs[k][1] = reinterpret_cast<float4 *>(outb[k]->quat);
        outs[k][2] = reinterpret_cast<float4 *>(outb[k]->logscale);
        outs[k][3] = reinterpret_cast<float4 *>(outb[k]->sh);
    }
    a.stat = stat;
    a.count = count;
    a.eps = eps;
    a.n = n;
    a.cap = cap;
    a.grad_thr = cfg->grad_thr;
    a.logit_min = cfg->logit_min;
    a.logscale_split = cfg->logscale_split;
    a.shrink = cfg->shrink;
    cudaStream_t st = as_cuda(stream);
    uint32_t *block_sums = static_cast<uint32_t *>(workspace);
    const int64_t nb = (n + kDTile - 1) / kDTile;
    int32_t rc;
    if (n > 0) {
        densify_count_kernel<<<(unsigned)nb, kDThreads, 0, st>>>(a, block_sums);
        densify_emit_kernel<<<(unsigned)nb, kDThreads, 0, st>>>(a, block_sums, nb, d_n_out, d_status);
    } else if (cudaMemsetAsync(d_n_out, 0, sizeof(int64_t), st) != cudaSuccess) {
        return check_launch("memset output count");
    }
    if ((rc = check_launch("densify"))) return rc;
    if (cap > 0) densify_pad_kernel<<<148 * 8, 256, 0, st>>>(a, d_n_out);
    return check_launch("densify_pad_kernel");
}
