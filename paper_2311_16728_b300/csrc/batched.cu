// batched.cu -- a window of keyframes at every Gaussian-pyramid level in one
// optimisation iteration (Photo-SLAM, arXiv 2311.16728, Sec. 3.4, Eq. 5):
// instead of supervising one level at a time, all (keyframe, level) views of a
// window are rendered, compared with GP^l(I_gt) (Eq. 4) and back-propagated
// together, L = sum_v w_v L_v, so the gradient is the sum of the single-view
// gradients.
//
//  - gsr_batched_preprocess: one thread per Gaussian projects it into every
//    view (parameters read once; SH read once, coloured per view).
//  - gsr_batched_bin_sort (binning.cu): one binning over all views' records
//    with tiles numbered across views.
//  - gsr_batched_iterate: ONE persistent cooperative launch runs, for every
//    (view, tile) and every (view, channel, 32 x 32 block), the forward
//    blend, both SSIM passes and the backward blend, pulling work from atomic
//    queues; phases are separated by grid barriers whose waits are bounded.
//  - gsr_batched_preprocess_bwd: one thread per Gaussian chains every view's
//    screen-space gradient into the parameter gradient and clears it.
#include <algorithm>
#include <cmath>

#include "chain_impl.cuh"
#include "render_impl.cuh"
#include "render_q4.cuh"
#include "render_warp.cuh"
#include "ssim_impl.cuh"

namespace gsr {

struct ViewsK {
    int nviews;
    CamK cam[kMaxViews];
};

// Views that share a pose (the pyramid levels of one keyframe) share the
// camera-space mean, the near-plane test and the colour; the 3D covariance is
// shared by every view.  Each record is bit-identical to gsr_preprocess's.
constexpr int kPoseMax = 8;  // views per pose group
struct PoseGroups {
    int ngroups;
    int count[kMaxViews];
    int member[kMaxViews][kPoseMax];
};

__global__ void __launch_bounds__(128) batched_preprocess_kernel(GaussK g, const __grid_constant__ ViewsK V,
                                                                 const __grid_constant__ PoseGroups PG,
                                                                 float4 *__restrict__ xy_conic,
                                                                 float4 *__restrict__ c_op_box,
                                                                 float4 *__restrict__ rgb_depth,
                                                                 uint32_t *__restrict__ ntiles,
                                                                 float2 *__restrict__ uv_lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const float4 mo = __ldg(g.mean_op + i), q = __ldg(g.quat + i), ls = __ldg(g.logscale + i);
    Chain shape;
    const bool shape_ok = chain_shape(q, ls, shape);
    const float op = FD(1.0f, FA(1.0f, chain_exp(-mo.w)));
    float sh[48];
    bool have_sh = false;
    const int nc = (g.deg + 1) * (g.deg + 1);
    for (int grp = 0; grp < PG.ngroups; ++grp) {
        Chain pose = shape;
        const bool front = shape_ok && chain_camera(mo, V.cam[PG.member[grp][0]], pose);
        float rgb[3] = {0.f, 0.f, 0.f};
        bool have_rgb = false;
        for (int k = 0; k < PG.count[grp]; ++k) {
            const int v = PG.member[grp][k];
            const CamK &cam = V.cam[v];
            const int64_t r = (int64_t)v * g.n + i;
            Chain c = pose;
            if (!front || !chain_screen(cam, c)) {
                ntiles[r] = 0u;
                continue;
            }
            const float A = FD(c.c, c.det), B = -FD(c.b, c.det), C = FD(c.a, c.det);
            if (!have_rgb) {
                if (!have_sh) {
                    load_sh(g.sh, g.n, i, g.deg, sh);
                    have_sh = true;
                }
                const float3 cc = cam_center(cam);
                float dx = mo.x - cc.x, dy = mo.y - cc.y, dz = mo.z - cc.z;
                const float inv_len = rsqrtf(dx * dx + dy * dy + dz * dz);
                dx *= inv_len; dy *= inv_len; dz *= inv_len;
                float Y[16];
                sh_basis(dx, dy, dz, g.deg, Y, nullptr);
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float acc = 0.5f;
#pragma unroll
                    for (int kk = 0; kk < 16; ++kk)
                        if (kk < nc) acc += sh[3 * kk + ch] * Y[kk];
                    rgb[ch] = fmaxf(acc, 0.0f);
                }
                have_rgb = true;
            }
            const uint32_t bx = (uint32_t)c.x0 | ((uint32_t)c.x1 << 16), by = (uint32_t)c.y0 | ((uint32_t)c.y1 << 16);
            xy_conic[r] = make_float4(c.u, c.v, A, B);
            c_op_box[r] = make_float4(C, op, __uint_as_float(bx), __uint_as_float(by));
            rgb_depth[r] = make_float4(rgb[0], rgb[1], rgb[2], c.zc);
            if (uv_lo) uv_lo[r] = uv_residual(mo, cam, c.u, c.v);
            ntiles[r] = (uint32_t)((c.x1 / cam.tw - c.x0 / cam.tw + 1) * (c.y1 / cam.th - c.y0 / cam.th + 1));
        }
    }
}

// views with identical pose (R and t bit for bit), at most kPoseMax a group
static void pose_groups(const gsr_camera *cams, int nviews, PoseGroups &G) {
    G.ngroups = 0;
    for (int v = 0; v < nviews; ++v) {
        int found = -1;
        for (int q = 0; q < G.ngroups && found < 0; ++q) {
            if (G.count[q] >= kPoseMax) continue;
            const gsr_camera &a = cams[G.member[q][0]], &b = cams[v];
            bool same = true;
            for (int k = 0; k < 9; ++k) same = same && a.R[k] == b.R[k];
            for (int k = 0; k < 3; ++k) same = same && a.t[k] == b.t[k];
            if (same) found = q;
        }
        if (found < 0) {
            found = G.ngroups++;
            G.count[found] = 0;
        }
        G.member[found][G.count[found]++] = v;
    }
}

// ---------------------------------------------------------------- persistent iteration
constexpr int kIterThreads = 128;  // 256-pixel tiles (16 x 16, 32 x 8, 8 x 32) at two pixels per thread
constexpr uint32_t kBarrierSpin = 1u << 24;  // x ~64 ns sleep: about a second

struct IterView {
    float *img, *T_final, *dimg, *mapA, *mapB, *mapC;
    const float *gt;
    uint32_t *n_contrib;
    int W, H, gx, tile_off, loss_off, lbx, lby;
    float weight;
};

struct IterArgs {
    const float4 *xy, *cb, *rd;
    const float2 *uv;  // position residuals of the records (NULL: none)
    const uint32_t *vals;
    const uint2 *ranges;
    const uint32_t *order;  // tiles by decreasing pair count (NULL: natural order)
    int tw, th;
    int depth;  // staging batch of the blend phases (0: one record per thread)
    float bg0, bg1, bg2;
    int nviews, tiles_total, loss_items;
    float lambda;
    Win win;
    float *g0, *g1, *g2;
    float *partials, *losses;
    unsigned *sync;  // [0..3] phase queues, [4] arrivals, [5] generation, [6] abort, [16..23] 4 u64 stamps
    int32_t *d_status;
    IterView view[kMaxViews];
};

__device__ __forceinline__ int next_item(unsigned *counter, int *s_item) {
    __syncthreads();
    if (threadIdx.x == 0) *s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    return *s_item;
}

// next_item for one 64-thread half of the CTA (each half takes its own items)
__device__ __forceinline__ int next_item_half(unsigned *counter, int *s_item) {
    Q4Group<true>::sync();
    if ((threadIdx.x & 63) == 0) *s_item = (int)atomicAdd(counter, 1u);
    Q4Group<true>::sync();
    return *s_item;
}

// Grid-wide barrier of a cooperative launch (all CTAs resident).  Returns
// false when the run was aborted: a wait that exceeded its bound sets the
// abort flag and the timeout status, and every later barrier and phase is
// skipped.
__device__ bool grid_barrier(unsigned *sync, unsigned nblocks, int32_t *status, int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = sync + 5, *vabort = sync + 6;
        int ok = *vabort == 0u;
        if (ok) {
            const unsigned g0 = *vgen;
            __threadfence();
            const unsigned arrived = atomicAdd(sync + 4, 1u) + 1u;
            if (arrived == nblocks) {
                atomicExch(sync + 4, 0u);
                __threadfence();
                atomicAdd(sync + 5, 1u);
            } else {
                uint32_t it = 0;
                while (*vgen == g0) {
                    if (*vabort) {
                        ok = 0;
                        break;
                    }
                    if (++it > kBarrierSpin) {
                        atomicExch(sync + 6, 1u);
                        raise_status(status, GSR_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        *s_ok = ok && *vabort == 0u;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Block 0 records the global timer when it enters the kernel and when it
// leaves each barrier (u64 words at byte 64 of the sync area): a cheap view
// of the phase split of one launch, read back by the host on demand.
__device__ __forceinline__ void phase_stamp(unsigned *sync, int k) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        reinterpret_cast<unsigned long long *>(sync + 16)[k] = t;
    }
}

__device__ __forceinline__ RenderArgs view_args(const IterArgs &a, const IterView &v) {
    RenderArgs r;
    r.xy_conic = a.xy;
    r.c_op_box = a.cb;
    r.rgb_depth = a.rd;
    r.uv_lo = a.uv;
    r.vals = a.vals;
    r.ranges = a.ranges;
    r.W = v.W;
    r.H = v.H;
    r.tw = a.tw;
    r.th = a.th;
    r.depth = a.depth;
    r.gx = v.gx;
    r.tile_off = v.tile_off;
    r.bg0 = a.bg0;
    r.bg1 = a.bg1;
    r.bg2 = a.bg2;
    return r;
}

__device__ __forceinline__ int view_of_tile(const IterArgs &a, int t) {
    int v = 0;
    while (v + 1 < a.nviews && a.view[v + 1].tile_off <= t) ++v;
    return v;
}

// The tile of queue item it: the heavy-first order when the binning wrote
// one (the longest lists start first), else it; -1 outside the window.
__device__ __forceinline__ int ordered_tile(const IterArgs &a, int it) {
    if (!a.order) return it;
    const uint32_t t = __ldg(a.order + it);
    return t < (uint32_t)a.tiles_total ? (int)t : -1;
}

__device__ __forceinline__ int view_of_loss(const IterArgs &a, int t) {
    int v = 0;
    while (v + 1 < a.nviews && a.view[v + 1].loss_off <= t) ++v;
    return v;
}

// kQuad: the views' tiles are 16 x 16 (quadrant warps; box tests from staged
// lane masks), one instance per tiling so the blend loops carry no branch
template <bool kQuad, bool kQ4>
__global__ void __launch_bounds__(kIterThreads, 5) batched_iterate_kernel(const __grid_constant__ IterArgs a) {
    extern __shared__ float4 smem4[];
    float *smf = reinterpret_cast<float *>(smem4);
    __shared__ int s_item, s_ok, s_item2[2];
    __shared__ float s_red[32];
    __shared__ double s_dbl[2 * kIterThreads];
    const unsigned nb = gridDim.x;
    phase_stamp(a.sync, 0);
    // ---- phase 1: forward blend of every (view, tile)
    if (kQuad && a.depth == 0) {
        // every warp takes its own items, one 8 x 8 quadrant of a tile each
        // (render_warp.cuh: it stages for itself), so no CTA barrier ties
        // four quadrants of unequal work together
        const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        Staged *buf = reinterpret_cast<Staged *>(smem4) + 32 * wid;
        for (;;) {
            int it = 0;
            if (lane == 0) it = (int)atomicAdd(a.sync + 0, 1u);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= 4 * a.tiles_total) break;
            const int t = ordered_tile(a, it >> 2);
            if (t < 0) continue;
            const int v = view_of_tile(a, t);
            const IterView &w = a.view[v];
            render_fwd_quadrant<false>(view_args(a, w), t - w.tile_off, it & 3, w.img, w.T_final, w.n_contrib,
                                       nullptr, buf, nullptr);
        }
    } else {
        for (int it = next_item(a.sync + 0, &s_item); it < a.tiles_total; it = next_item(a.sync + 0, &s_item)) {
            const int t = ordered_tile(a, it);
            if (t < 0) continue;
            const int v = view_of_tile(a, t);
            const IterView &w = a.view[v];
            render_fwd_tile<kQuad>(view_args(a, w), t - w.tile_off, w.img, w.T_final, w.n_contrib, nullptr, smem4);
        }
    }
    if (!grid_barrier(a.sync, nb, a.d_status, &s_ok)) return;
    phase_stamp(a.sync, 1);
    // ---- phase 2: SSIM moments of every (view, channel, 32 x 32 block)
    for (int it = next_item(a.sync + 1, &s_item); it < a.loss_items; it = next_item(a.sync + 1, &s_item)) {
        const int v = view_of_loss(a, it);
        const IterView &w = a.view[v];
        const int local = it - w.loss_off, per = w.lbx * w.lby;
        const int c = local / per, rem = local - c * per;
        ssim_pass1_block<kIterThreads>(w.img, w.gt, w.H, w.W, a.win, w.mapA, w.mapB, w.mapC, a.partials + 2 * it,
                                       rem % w.lbx, rem / w.lbx, c, smf, s_red);
    }
    if (!grid_barrier(a.sync, nb, a.d_status, &s_ok)) return;
    phase_stamp(a.sync, 2);
    // ---- phase 3: dL/dI of every view, scaled by its weight; per-view losses
    for (int it = next_item(a.sync + 2, &s_item); it < a.loss_items; it = next_item(a.sync + 2, &s_item)) {
        const int v = view_of_loss(a, it);
        const IterView &w = a.view[v];
        const int local = it - w.loss_off, per = w.lbx * w.lby;
        const int c = local / per, rem = local - c * per;
        ssim_pass2_block<kIterThreads>(w.img, w.gt, w.H, w.W, 3, a.win, w.mapA, w.mapB, w.mapC, a.lambda, w.weight,
                                       w.dimg, rem % w.lbx, rem / w.lbx, c, smf);
    }
    for (int v = blockIdx.x; v < a.nviews; v += gridDim.x) {
        const IterView &w = a.view[v];
        const float L = loss_from_partials<kIterThreads>(a.partials + 2 * w.loss_off, 3 * w.lbx * w.lby,
                                                         3.0 * w.W * w.H, a.lambda, s_dbl);
        if (threadIdx.x == 0) a.losses[v] = L;
    }
    if (!grid_barrier(a.sync, nb, a.d_status, &s_ok)) return;
    phase_stamp(a.sync, 3);
    // ---- phase 4: backward blend of every (view, tile); 16 x 16 tiles run at
    // four pixels per thread, as per-warp halves (default staging) or two
    // tiles at a time, one per 64-thread half of the CTA (staging depths)
    if (kQ4 && a.depth == 0) {
        // every warp takes its own items, one 16 x 8 half of a tile each,
        // staging for itself (render_warp.cuh)
        const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        Staged *buf = reinterpret_cast<Staged *>(smem4) + 32 * wid;
        for (;;) {
            int it = 0;
            if (lane == 0) it = (int)atomicAdd(a.sync + 3, 1u);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= 2 * a.tiles_total) break;
            const int t = ordered_tile(a, it >> 1);
            if (t < 0) continue;
            const int v = view_of_tile(a, t);
            const IterView &w = a.view[v];
            render_bwd_tile_warp(view_args(a, w), t - w.tile_off, it & 1, w.T_final, w.n_contrib, w.dimg, a.g0, a.g1,
                                 a.g2, buf);
        }
    } else if constexpr (kQ4) {
        const int half = (int)(threadIdx.x >> 6);
        float4 *sm = smem4 + half * (render_q4_smem(a.depth > 0 ? a.depth : kQ4Threads) / sizeof(float4));
        for (int it = next_item_half(a.sync + 3, &s_item2[half]); it < a.tiles_total;
             it = next_item_half(a.sync + 3, &s_item2[half])) {
            const int t = ordered_tile(a, it);
            if (t < 0) continue;
            const int v = view_of_tile(a, t);
            const IterView &w = a.view[v];
            render_bwd_tile_q4<true>(view_args(a, w), t - w.tile_off, w.T_final, w.n_contrib, w.dimg, a.g0, a.g1,
                                     a.g2, sm);
        }
    } else {
        for (int it = next_item(a.sync + 3, &s_item); it < a.tiles_total; it = next_item(a.sync + 3, &s_item)) {
            const int t = ordered_tile(a, it);
            if (t < 0) continue;
            const int v = view_of_tile(a, t);
            const IterView &w = a.view[v];
            render_bwd_tile<kQuad>(view_args(a, w), t - w.tile_off, w.T_final, w.n_contrib, w.dimg, a.g0, a.g1,
                                   a.g2, smem4);
        }
    }
}

static size_t iterate_smem(int depth, bool q4) {
    size_t s = render_bwd_smem(depth > 0 ? depth : kIterThreads);
    if (q4 && 2 * render_q4_smem(depth > 0 ? depth : kQ4Threads) > s) s = 2 * render_q4_smem(depth > 0 ? depth : kQ4Threads);
    if (render_fwd_smem(depth > 0 ? depth : kIterThreads) > s) s = render_fwd_smem(depth > 0 ? depth : kIterThreads);
    if (depth == 0 && render_warp_smem(kIterThreads) > s) s = render_warp_smem(kIterThreads);
    if (sizeof(float) * kPass1Floats > s) s = sizeof(float) * kPass1Floats;
    if (sizeof(float) * kPass2Floats > s) s = sizeof(float) * kPass2Floats;
    return s;
}

// ---------------------------------------------------------------- batched chain rule
// The pyramid levels of one keyframe are exact power-of-two scalings of one
// camera (same pose; fx, fy, cx, cy, W, H all scaled by s = 2^-k), so with
// M = J W Sigma W^T J^T at the finest level, level k sees u_k = s u,
// v_k = s v and Sigma'_k = s^2 M + 0.3 I, while the opacity, the view
// direction (hence the colour and its clamp) and the near-plane test are the
// same.  The screen-space gradients of such views therefore merge exactly
// into one view before the chain rule: dL/du += s dL/du_k, dL/dv += s dL/dv_k,
// dL/dM += s^2 dL/dSigma'_k (with dL/dSigma' = -Q dL/dQ Q per view), and the
// opacity and colour gradients add.  The expensive chain then runs once per
// (Gaussian, keyframe) instead of once per (Gaussian, view).
constexpr int kGroupMax = 8;     // views per group
static_assert(kGroupMax <= 8, "member masks are 8-bit");
constexpr int kChainChunk = 128; // Gaussians per CTA

struct ChainGroups {
    int ngroups;
    int count[kMaxViews];
    int member[kMaxViews][kGroupMax];   // view index, finest level first
    float scale[kMaxViews][kGroupMax];  // relative to the group's first view (1, 1/2, 1/4, ...)
};

__global__ void __launch_bounds__(kBwdThreads, 4) batched_chain_kernel(GaussK g, const __grid_constant__ ViewsK V,
                                                                    const __grid_constant__ ChainGroups CG,
                                                                    const float4 *__restrict__ xy_conic,
                                                                    const float4 *__restrict__ c_op_box,
                                                                    const uint32_t *__restrict__ ntiles,
                                                                    const uint32_t *__restrict__ rec_to_c,
                                                                    float4 *__restrict__ g0, float4 *__restrict__ g1,
                                                                    float4 *__restrict__ g2, float4 *__restrict__ d_mo,
                                                                    float4 *__restrict__ d_q, float4 *__restrict__ d_ls,
                                                                    float4 *__restrict__ d_sh,
                                                                    uint32_t *__restrict__ touched) {
    extern __shared__ uint32_t s_rec[];  // kChainChunk x ngroups candidates, then as many member masks
    __shared__ uint32_t s_cnt;
    __shared__ uint32_t s_touch[kChainChunk];
    const int total = kChainChunk * CG.ngroups;  // a multiple of 32: whole warps take part in each ballot
    uint8_t *s_bits = reinterpret_cast<uint8_t *>(s_rec + total);  // members of the group that see the Gaussian
    if (threadIdx.x == 0) s_cnt = 0u;
    for (int k = threadIdx.x; k < kChainChunk; k += kBwdThreads) s_touch[k] = 0u;
    const int64_t base = (int64_t)blockIdx.x * kChainChunk;
    const int lane = threadIdx.x & 31;
    // every visibility word first (independent loads, no ballot in between)
#pragma unroll 4
    for (int k = threadIdx.x; k < total; k += kBwdThreads) {
        const int il = k % kChainChunk, grp = k / kChainChunk;
        const int64_t i = base + il;
        uint32_t bits = 0u;
        if (i < g.n) {
#pragma unroll
            for (int m = 0; m < kGroupMax; ++m)
                if (m < CG.count[grp]) bits |= (ntiles[(int64_t)CG.member[grp][m] * g.n + i] > 0u ? 1u : 0u) << m;
        }
        s_bits[k] = (uint8_t)bits;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < total; k += kBwdThreads) {
        const int il = k % kChainChunk, grp = k / kChainChunk;
        const bool vis = s_bits[k] != 0u;
        const uint32_t msk = __ballot_sync(0xffffffffu, vis);
        uint32_t slot = 0;
        if (lane == 0 && msk) slot = atomicAdd(&s_cnt, (uint32_t)__popc(msk));
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (vis) {
            s_rec[slot + __popc(msk & ((1u << lane) - 1u))] = ((uint32_t)grp << 16) | (uint32_t)il;
            s_touch[il] = 1u;
        }
    }
    __syncthreads();
    if (touched)
        for (int k = threadIdx.x; k < kChainChunk; k += kBwdThreads)
            if (base + k < g.n) touched[base + k] = s_touch[k];
    const uint32_t cnt = s_cnt;
    for (uint32_t k = threadIdx.x; k < cnt; k += kBwdThreads) {
        const int grp = (int)(s_rec[k] >> 16);
        const int il = (int)(s_rec[k] & 0xFFFFu);
        const int64_t i = base + il;
        const uint32_t bits = s_bits[grp * kChainChunk + il];
        // the finest visible view of the group is the base of the merge
        const int mb = __ffs(bits) - 1;
        const int vb = CG.member[grp][mb];
        const CamK &cam = V.cam[vb];
        const float4 mo = __ldg(g.mean_op + i), q = __ldg(g.quat + i), ls = __ldg(g.logscale + i);
        float4 shp[kShPlanes];  // in flight while the decision chain runs
        load_sh_planes(g, i, shp);
        Chain c;
        if (!decide_chain(mo, q, ls, cam, c)) continue;  // cannot happen for a visible record
        ScreenGrad sg = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const float sb = CG.scale[grp][mb];
        for (int m = mb; m < CG.count[grp]; ++m) {
            if (!((bits >> m) & 1u)) continue;
            const int64_t rec = (int64_t)CG.member[grp][m] * g.n + i;
            // records and screen-space gradients: at the record, or at its
            // compact position when the binning gathered the records
            const int64_t r = rec_to_c ? (int64_t)rec_to_c[rec] : rec;
            const float4 G0 = g0[r], G1 = g1[r], G2 = g2[r];
            const float4 xc = __ldg(xy_conic + r), cb = __ldg(c_op_box + r);
            const float s = CG.scale[grp][m] / sb;  // exact: both are powers of two
            float h00, h01, h11;
            conic_grad_to_cov(xc.z, xc.w, cb.x, G0.z, G0.w, G1.x, h00, h01, h11);
            const float s2 = s * s;
            sg.du += s * G0.x;
            sg.dv += s * G0.y;
            sg.Gs00 += s2 * h00;
            sg.Gs01 += s2 * h01;
            sg.Gs11 += s2 * h11;
            sg.dop += G1.y;
            sg.dr += G1.z;
            sg.dg += G1.w;
            sg.db += G2.x;
            // leave the screen-space gradient zeroed for the next iteration
            g0[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            g1[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            g2[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        chain_core(g, cam, i, mo, c, sg, d_mo, d_q, d_ls, d_sh, true, shp);
    }
}

// Groups of views that are exact power-of-two scalings of one camera.
static bool is_scaling(const gsr_camera &a, const gsr_camera &b, float &s) {
    for (int k = 0; k < 9; ++k)
        if (a.R[k] != b.R[k]) return false;
    for (int k = 0; k < 3; ++k)
        if (a.t[k] != b.t[k]) return false;
    s = b.fx / a.fx;
    int e;
    if (!(s > 0.f) || std::frexp(s, &e) != 0.5f) return false;
    return b.fy == a.fy * s && b.cx == a.cx * s && b.cy == a.cy * s && (float)b.width == (float)a.width * s &&
           (float)b.height == (float)a.height * s;
}

static void make_groups(const gsr_camera *cams, int nviews, ChainGroups &G) {
    G.ngroups = 0;
    for (int v = 0; v < nviews; ++v) {
        int found = -1;
        float s = 1.f;
        for (int q = 0; q < G.ngroups && found < 0; ++q)
            if (G.count[q] < kGroupMax && is_scaling(cams[G.member[q][0]], cams[v], s)) found = q;
        if (found < 0) {
            found = G.ngroups++;
            G.count[found] = 0;
            s = 1.f;
        }
        G.member[found][G.count[found]] = v;
        G.scale[found][G.count[found]] = s;
        G.count[found]++;
    }
    // finest first within each group (insertion sort by descending scale)
    for (int q = 0; q < G.ngroups; ++q)
        for (int a = 1; a < G.count[q]; ++a)
            for (int b = a; b > 0 && G.scale[q][b] > G.scale[q][b - 1]; --b) {
                std::swap(G.scale[q][b], G.scale[q][b - 1]);
                std::swap(G.member[q][b], G.member[q][b - 1]);
            }
}

static int32_t views_k(const gsr_camera *cams, int32_t nviews, const gsr_tiling *tiling, ViewsK &V) {
    int32_t rc;
    if (!cams || nviews <= 0 || nviews > kMaxViews) {
        set_error("batched: need 1 .. %d views", kMaxViews);
        return GSR_ERR_INVALID_ARG;
    }
    V.nviews = nviews;
    for (int v = 0; v < nviews; ++v) {
        if ((rc = validate_camera(&cams[v]))) return rc;
        V.cam[v] = make_camk(&cams[v], tiling);
    }
    return GSR_OK;
}

}  // namespace gsr

using namespace gsr;

extern "C" int32_t gsr_batched_preprocess(const gsr_gaussians *g, const gsr_camera *cams, int32_t nviews,
                                          const gsr_tiling *tiling, const gsr_proj *out, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_gaussians(g)) || (rc = validate_tiling(tiling))) return rc;
    ViewsK V;
    if ((rc = views_k(cams, nviews, tiling, V))) return rc;
    if (g->n == 0) return GSR_OK;
    if (!out || !out->xy_conic || !out->c_op_box || !out->rgb_depth || !out->ntiles || !aligned16(out->xy_conic) ||
        !aligned16(out->c_op_box) || !aligned16(out->rgb_depth)) {
        set_error("gsr_batched_preprocess: output records must be non-NULL and 16-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    if (out->uv_lo && (reinterpret_cast<uintptr_t>(out->uv_lo) & 7u)) {
        set_error("gsr_batched_preprocess: uv_lo must be 8-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    PoseGroups PG;
    pose_groups(cams, nviews, PG);
    batched_preprocess_kernel<<<(unsigned)((g->n + 127) / 128), 128, 0, as_cuda(stream)>>>(
        make_gk(g), V, PG, reinterpret_cast<float4 *>(out->xy_conic), reinterpret_cast<float4 *>(out->c_op_box),
        reinterpret_cast<float4 *>(out->rgb_depth), out->ntiles, reinterpret_cast<float2 *>(out->uv_lo));
    return check_launch("batched_preprocess_kernel");
}

extern "C" int32_t gsr_batched_iterate_workspace_size(const gsr_camera *cams, int32_t nviews, size_t *bytes) {
    if (!cams || nviews <= 0 || nviews > kMaxViews || !bytes) {
        set_error("gsr_batched_iterate_workspace_size: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    size_t items = 0, px = 0;
    for (int v = 0; v < nviews; ++v) {
        items += 3 * (size_t)((cams[v].width + kLTW - 1) / kLTW) * ((cams[v].height + kLTH - 1) / kLTH);
        px += 3 * (size_t)cams[v].width * cams[v].height;
    }
    // three SSIM maps per pixel-channel, two partial sums per block, sync words
    *bytes = ((3 * px * sizeof(float) + 255) & ~size_t(255)) + ((2 * items * sizeof(float) + 255) & ~size_t(255)) + 256;
    return GSR_OK;
}

extern "C" int32_t gsr_batched_iterate(const gsr_proj *proj, const uint32_t *vals, const uint32_t *tile_ranges,
                                       const gsr_camera *cams, int32_t nviews, const gsr_tiling *tiling,
                                       const float *bg, float *const *img, float *const *T_final,
                                       uint32_t *const *n_contrib, const float *const *gt, float *const *dL_dimg,
                                       const float *weights, float lambda, float *d_losses, const gsr_grad2d *grad2d,
                                       void *workspace, size_t workspace_bytes, int32_t *d_status,
                                       gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_tiling(tiling))) return rc;
    if (tiling->tile_w * tiling->tile_h != 2 * kIterThreads) {
        set_error("gsr_batched_iterate: the persistent kernel runs 256-pixel tiles (tile_w * tile_h = 256)");
        return GSR_ERR_UNSUPPORTED;
    }
    if (!proj || !tile_ranges || !cams || nviews <= 0 || nviews > kMaxViews || !img || !T_final || !n_contrib ||
        !gt || !dL_dimg || !d_losses || !grad2d || !grad2d->g0 || !grad2d->g1 || !grad2d->g2 ||
        !(lambda >= 0.f && lambda <= 1.f)) {
        set_error("gsr_batched_iterate: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    size_t need;
    if ((rc = gsr_batched_iterate_workspace_size(cams, nviews, &need))) return rc;
    if (!workspace || workspace_bytes < need) {
        set_error("gsr_batched_iterate: workspace of %zu bytes needed", need);
        return GSR_ERR_CAPACITY;
    }
    IterArgs a{};  // passed by value as the kernel parameter
    a.xy = reinterpret_cast<const float4 *>(proj->xy_conic);
    a.cb = reinterpret_cast<const float4 *>(proj->c_op_box);
    a.rd = reinterpret_cast<const float4 *>(proj->rgb_depth);
    a.uv = reinterpret_cast<const float2 *>(proj->uv_lo);
    a.vals = vals;
    a.ranges = reinterpret_cast<const uint2 *>(tile_ranges);
    a.order = proj->tile_order;
    a.tw = tiling->tile_w;
    a.th = tiling->tile_h;
    a.depth = tiling->batch_depth;
    a.bg0 = bg ? bg[0] : 0.f;
    a.bg1 = bg ? bg[1] : 0.f;
    a.bg2 = bg ? bg[2] : 0.f;
    a.nviews = nviews;
    a.lambda = lambda;
    a.win = ssim_window();
    a.g0 = grad2d->g0;
    a.g1 = grad2d->g1;
    a.g2 = grad2d->g2;
    a.losses = d_losses;
    a.d_status = d_status;
    size_t px = 0;
    int tiles = 0, items = 0;
    for (int v = 0; v < nviews; ++v) {
        if ((rc = validate_camera(&cams[v]))) return rc;
        if (!img[v] || !T_final[v] || !n_contrib[v] || !gt[v] || !dL_dimg[v]) {
            set_error("gsr_batched_iterate: NULL image pointer of view %d", v);
            return GSR_ERR_INVALID_ARG;
        }
        IterView &w = a.view[v];
        w.img = img[v];
        w.T_final = T_final[v];
        w.n_contrib = n_contrib[v];
        w.gt = gt[v];
        w.dimg = dL_dimg[v];
        w.W = cams[v].width;
        w.H = cams[v].height;
        w.gx = grid_x(&cams[v], tiling);
        w.tile_off = tiles;
        tiles += grid_x(&cams[v], tiling) * grid_y(&cams[v], tiling);
        w.lbx = (w.W + kLTW - 1) / kLTW;
        w.lby = (w.H + kLTH - 1) / kLTH;
        w.loss_off = items;
        items += 3 * w.lbx * w.lby;
        w.weight = weights ? weights[v] : 1.0f;
        px += 3 * (size_t)w.W * w.H;
    }
    char *ws = static_cast<char *>(workspace);
    float *maps = reinterpret_cast<float *>(ws);
    size_t off = 0;
    for (int v = 0; v < nviews; ++v) {
        const size_t p = 3 * (size_t)a.view[v].W * a.view[v].H;
        a.view[v].mapA = maps + off;
        a.view[v].mapB = maps + px + off;
        a.view[v].mapC = maps + 2 * px + off;
        off += p;
    }
    const size_t maps_bytes = (3 * px * sizeof(float) + 255) & ~size_t(255);
    a.partials = reinterpret_cast<float *>(ws + maps_bytes);
    const size_t part_bytes = (2 * (size_t)items * sizeof(float) + 255) & ~size_t(255);
    a.sync = reinterpret_cast<unsigned *>(ws + maps_bytes + part_bytes);
    a.tiles_total = tiles;
    a.loss_items = items;
    cudaStream_t st = as_cuda(stream);
    if (cudaMemsetAsync(a.sync, 0, 8 * sizeof(unsigned), st) != cudaSuccess) return check_launch("memset sync");
    // 16 x 16 tiles: the backward phase runs two tiles per CTA, one per
    // 64-thread half (four pixels a thread), unless bwd_threads asks for 128
    const bool quad = tiling->tile_w == 16 && tiling->tile_h == 16;
    const bool q4 = quad && tiling->bwd_threads != kIterThreads;
    const size_t smem = iterate_smem(tiling->batch_depth, q4);
    auto kernel = q4 ? batched_iterate_kernel<true, true>
                     : (quad ? batched_iterate_kernel<true, false> : batched_iterate_kernel<false, false>);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kIterThreads, smem);
    if (per_sm < 1) {
        set_error("gsr_batched_iterate: the persistent kernel does not fit on an SM");
        return GSR_ERR_UNSUPPORTED;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(sms * per_sm));
    cfg.blockDim = dim3(kIterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kernel, a) != cudaSuccess) return check_launch("batched_iterate_kernel");
    return check_launch("batched_iterate_kernel");
}

extern "C" int32_t gsr_batched_preprocess_bwd(const gsr_gaussians *g, const gsr_proj *proj, const gsr_proj *compact,
                                              const gsr_camera *cams, int32_t nviews, const gsr_tiling *tiling,
                                              const gsr_grad2d *grad2d, const gsr_param_buffers *grads,
                                              uint32_t *touched, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_gaussians(g)) || (rc = validate_tiling(tiling))) return rc;
    ViewsK V;
    if ((rc = views_k(cams, nviews, tiling, V))) return rc;
    if (g->n == 0) return GSR_OK;
    if (!proj || !proj->ntiles || !grad2d || !grad2d->g0 || !grad2d->g1 || !grad2d->g2 || !grads ||
        !grads->mean_op || !grads->quat || !grads->logscale || !grads->sh) {
        set_error("gsr_batched_preprocess_bwd: NULL pointer");
        return GSR_ERR_INVALID_ARG;
    }
    const gsr_proj *rp = compact ? compact : proj;
    if (!rp->xy_conic || !rp->c_op_box || (compact && !compact->ntiles)) {
        set_error("gsr_batched_preprocess_bwd: NULL record pointer");
        return GSR_ERR_INVALID_ARG;
    }
    ChainGroups CG;
    make_groups(cams, nviews, CG);
    const size_t smem = (sizeof(uint32_t) + sizeof(uint8_t)) * kChainChunk * CG.ngroups;
    batched_chain_kernel<<<(unsigned)((g->n + kChainChunk - 1) / kChainChunk), kBwdThreads, smem, as_cuda(stream)>>>(
        make_gk(g), V, CG, reinterpret_cast<const float4 *>(rp->xy_conic),
        reinterpret_cast<const float4 *>(rp->c_op_box), proj->ntiles, compact ? compact->ntiles : nullptr,
        reinterpret_cast<float4 *>(grad2d->g0),
        reinterpret_cast<float4 *>(grad2d->g1), reinterpret_cast<float4 *>(grad2d->g2),
        reinterpret_cast<float4 *>(grads->mean_op), reinterpret_cast<float4 *>(grads->quat),
        reinterpret_cast<float4 *>(grads->logscale), reinterpret_cast<float4 *>(grads->sh), touched);
    return check_launch("batched_chain_kernel");
}
