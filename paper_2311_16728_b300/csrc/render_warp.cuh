// render_warp.cuh -- forward blend (K5) and backward blend (K7) of the
// tile-based renderer of Photo-SLAM (arXiv 2311.16728) Sec. 3.3, Eq. 3, for
// 16 x 16 tiles with warp-private staging.
//
// Every warp walks its tile's depth-sorted list on its own: 32 records per
// round, one per lane, each tested against the warp's own pixel rectangle
// only; the ballot of the records the warp can see compacts them, in list
// order, into the warp's own 32-record shared-memory buffer, and the blend
// loop visits exactly those.  No block-wide barrier orders the warps of a
// tile, so a warp whose pixels have all terminated stops at once instead of
// staging and waiting for the others, and warps with short visible lists do
// not wait at every round for warps with long ones.  The price is that each
// record's cull test runs once per warp that reads it instead of once per
// tile.  The per-pixel arithmetic and decisions are the block-staged
// routines' (render_impl.cuh, render_q4.cuh), so the image, T_final and
// n_contrib are bit-identical to theirs.
//
// Forward: warp w an 8 x 8 quadrant, two pixels a lane; backward: warp w
// rows 8 w .. 8 w + 7, four pixels a lane.  The one-view kernels run every
// warp as a CTA of its own, so a warp that finishes early frees its slot for
// another tile's warp at once.
#pragma once

#include "render_q4.cuh"

namespace gsr {

constexpr int kWarpFwdThreads = 128, kWarpBwdThreads = 64;  // threads of a tile

// Whether the warp whose pixels span [rx0, rx1] x [ry0, ry1] can see the
// splat at all: the pixel box against the rectangle, then the minimum of the
// quadratic form over their overlap against the alpha threshold (the test
// stage_splat applies per warp, without its prefilter on the alpha
// ellipse's bounding box, which the minimum implies: the two square roots
// and divisions cost more per staged record than the records it drops
// earlier); x0, x1, y0, y1 receive its pixel box.  Every test runs on every
// lane (no divergent early exit).
__device__ __forceinline__ bool warp_may_see(const float4 g, const float4 c, int rx0, int rx1, int ry0, int ry1,
                                             int &x0, int &x1, int &y0, int &y1) {
    const float A = g.z, B = g.w, C = c.x, op = c.y;
    const float tau = 2.0f * __logf(255.0f * op);  // alpha >= 1/255  <=>  d^T Q d <= tau
    const uint32_t bx = __float_as_uint(c.z), by = __float_as_uint(c.w);
    x0 = (int)(bx & 0xffffu);
    x1 = (int)(bx >> 16);
    y0 = (int)(by & 0xffffu);
    y1 = (int)(by >> 16);
    // every test on every lane, combined without short-circuit branches
    const bool boxes = x0 <= rx1 && x1 >= rx0 && y0 <= ry1 && y1 >= ry0;
    const bool near = rect_may_see(g.x, g.y, A, B, C, tau, (float)max(rx0, x0), (float)min(rx1, x1),
                                   (float)max(ry0, y0), (float)min(ry1, y1));
    return (tau > 0.0f) & boxes & near;
}

// The record of a visible splat in the warp's buffer: pre-scaled exponent
// terms as stage_splat writes them, `pad` = the splat's 0-based position in
// the tile's list, lanes[0] = the warp's box lane masks, lanes[1].x = 1 when
// the blend may take its fast path for this splat: the pixel box holds every
// pixel of the warp (`full`) and the opacity cannot reach the alpha clamp.
// The flag is the same for every lane of the warp, so the branch on it
// never diverges; the fast path drops the per-pixel box and clamp tests that
// cannot fail, with the same decisions and arithmetic as the general one.
__device__ __forceinline__ void warp_stage(const RenderArgs &a, uint32_t gid, uint32_t pos, const float4 g,
                                           const float4 c, const uint4 lanes, bool full, Staged &st) {
    st.xy = make_float4(g.x, g.y, g.z * kHalfLog2e, g.w * (2.0f * kHalfLog2e));
    st.cb = make_float4(c.x * kHalfLog2e, c.y, c.z, c.w);
    st.rgb = __ldg(a.rgb_depth + gid);
    st.lo = mean_residual(a, gid);
    st.gid = gid;
    st.pad = pos;
    st.lanes[0] = lanes;
    st.lanes[1] = make_uint4((full && c.y <= kOpNoClamp) ? 1u : 0u, 0u, 0u, 0u);
}

// ---------------------------------------------------------------- K5
// Quadrant `wid` of the tile, by one warp with its 32-record buffer `buf`;
// tile_work (may be NULL): raised (atomic max) to the quadrant's largest
// n_contrib.
template <bool kCount>
__device__ __forceinline__ void render_fwd_quadrant(const RenderArgs &a, int tile, int wid, float *__restrict__ img,
                                                    float *__restrict__ T_final, uint32_t *__restrict__ n_contrib,
                                                    uint32_t *__restrict__ n_blended, Staged *buf,
                                                    uint32_t *__restrict__ tile_work) {
    const int lane = threadIdx.x & 31;
    const int ox = (tile % a.gx) * a.tw, oy = (tile / a.gx) * a.th;
    const int px = ox + 8 * (wid & 1) + (lane & 7), py0 = oy + 8 * (wid >> 1) + 2 * (lane >> 3);
    int rx0, rx1, ry0, ry1;
    warp_rect(a, wid, ox, oy, rx0, rx1, ry0, ry1);
    const bool in0 = px < a.W && py0 < a.H, in1 = px < a.W && py0 + 1 < a.H;
    const uint2 rg = a.ranges[a.tile_off + tile];
    const int begin = (int)rg.x, end = (int)rg.y;
    const float fpx = (float)px;
    const float2 fpy = make_float2((float)py0, (float)(py0 + 1));
    const uint32_t lbit = 1u << lane;  // this lane's bit in the box lane masks
    PairFwd p;
    p.T = make_float2(1.0f, 1.0f);
    p.C0 = p.C1 = p.C2 = make_float2(0.0f, 0.0f);
    p.last0 = p.last1 = p.nb0 = p.nb1 = 0u;
    p.done0 = !in0;
    p.done1 = !in1;
    for (int base = begin; base < end; base += 32) {
        // the warp stops once every one of its pixels has terminated
        if (__all_sync(0xffffffffu, p.done0 && p.done1)) break;
        const int idx = base + lane;
        bool vis = false;
        uint32_t gid = 0u;
        float4 g, c;
        int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
        if (idx < end) {
            gid = a.vals[idx];
            g = __ldg(a.xy_conic + gid);
            c = __ldg(a.c_op_box + gid);
            vis = warp_may_see(g, c, rx0, rx1, ry0, ry1, x0, x1, y0, y1);
        }
        const uint32_t bits = __ballot_sync(0xffffffffu, vis);
        if (vis) {
            const uint2 m = quad_box_lanes(x0, x1, y0, y1, rx0, ry0);
            warp_stage(a, gid, (uint32_t)(idx - begin + 1), g, c, make_uint4(m.x, m.y, 0u, 0u),
                       (m.x & m.y) == 0xffffffffu, buf[__popc(bits & ((1u << lane) - 1u))]);
        }
        __syncwarp();
        const int n = __popc(bits);
        // two splats per round: their alphas are independent, so both are
        // evaluated before they are blended in list order
        for (int j = 0; j < n; j += 2) {
            // and within a round, every eight splats, so that a warp whose
            // pixels all stopped early in the round skips its remaining splats
            if ((j & 7) == 0 && j > 0 && __all_sync(0xffffffffu, p.done0 && p.done1)) break;
            const bool has_b = j + 1 < n;
            const Staged &sa = buf[j], &sb = buf[has_b ? j + 1 : j];
            PixAlpha pa, pb;
            if ((sa.lanes[1].x & sb.lanes[1].x) != 0u) {  // both on the fast path (uniform over the warp)
                pair_alpha<true>(sa.xy, sa.cb, sa.lo, fpx, fpy, true, true, pa);
                pair_alpha<true>(sb.xy, sb.cb, sb.lo, fpx, fpy, true, true, pb);
            } else {
                const uint2 ma = *reinterpret_cast<const uint2 *>(sa.lanes);
                const uint2 mb = *reinterpret_cast<const uint2 *>(sb.lanes);
                pair_alpha(sa.xy, sa.cb, sa.lo, fpx, fpy, (ma.x & lbit) != 0u, (ma.y & lbit) != 0u, pa);
                pair_alpha(sb.xy, sb.cb, sb.lo, fpx, fpy, (mb.x & lbit) != 0u, (mb.y & lbit) != 0u, pb);
            }
            if (!has_b) pb.ok0 = pb.ok1 = false;
            blend_fwd_pair(p, pa.ok0, pa.ok1, pa.a0, pa.a1, sa.rgb, sa.pad);
            blend_fwd_pair(p, pb.ok0, pb.ok1, pb.a0, pb.a1, sb.rgb, sb.pad);
        }
        __syncwarp();
    }
    const int64_t plane = (int64_t)a.W * a.H;
    if (in0) {
        const int64_t pix = (int64_t)py0 * a.W + px;
        img[pix] = p.C0.x + p.T.x * a.bg0;
        img[plane + pix] = p.C1.x + p.T.x * a.bg1;
        img[2 * plane + pix] = p.C2.x + p.T.x * a.bg2;
        T_final[pix] = p.T.x;
        n_contrib[pix] = p.last0;
        if (kCount) n_blended[pix] = p.nb0;
    }
    if (in1) {
        const int64_t pix = (int64_t)(py0 + 1) * a.W + px;
        img[pix] = p.C0.y + p.T.y * a.bg0;
        img[plane + pix] = p.C1.y + p.T.y * a.bg1;
        img[2 * plane + pix] = p.C2.y + p.T.y * a.bg2;
        T_final[pix] = p.T.y;
        n_contrib[pix] = p.last1;
        if (kCount) n_blended[pix] = p.nb1;
    }
    if (tile_work) {
        const uint32_t mx = __reduce_max_sync(0xffffffffu, max(p.last0, p.last1));
        if (lane == 0 && mx) atomicMax(&tile_work[tile], mx);
    }
}

// The whole tile by a CTA of four warps (warp w: quadrant w).
template <bool kCount>
__device__ __forceinline__ void render_fwd_tile_warp(const RenderArgs &a, int tile, float *__restrict__ img,
                                                     float *__restrict__ T_final, uint32_t *__restrict__ n_contrib,
                                                     uint32_t *__restrict__ n_blended, Staged *s_buf,
                                                     uint32_t *__restrict__ tile_work) {
    const int wid = threadIdx.x >> 5;
    render_fwd_quadrant<kCount>(a, tile, wid, img, T_final, n_contrib, n_blended, s_buf + 32 * wid, tile_work);
}

// ---------------------------------------------------------------- K7
// Back to front from the warp's own largest n_contrib; per visible splat the
// arithmetic of render_bwd_tile_q4 (q4_splat_bwd).
// Half `wid` (rows 8 wid .. 8 wid + 7) of the tile, by one warp with its
// 32-record buffer `buf`.
__device__ __forceinline__ void render_bwd_tile_warp(const RenderArgs &a, int tile, int wid,
                                                     const float *__restrict__ T_final,
                                                     const uint32_t *__restrict__ n_contrib,
                                                     const float *__restrict__ dL_dimg, float *__restrict__ g0,
                                                     float *__restrict__ g1, float *__restrict__ g2, Staged *buf) {
    const int lane = (int)(threadIdx.x & 31u), ti = 32 * wid + lane;
    int px, py0, ox, oy;
    q4_pixels(a, tile, ti, px, py0, ox, oy);
    const int rx0 = ox, rx1 = ox + 15, ry0 = oy + 8 * wid, ry1 = ry0 + 7;
    const uint2 rg = a.ranges[a.tile_off + tile];
    const int begin = (int)rg.x;
    const int64_t plane = (int64_t)a.W * a.H;
    PairBwd p[2];
    uint32_t last[4];
    uint32_t mlast = 0u;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float v[2][5];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k = 2 * h + q;
            v[q][0] = v[q][1] = v[q][2] = v[q][3] = v[q][4] = 0.f;
            last[k] = 0u;
            if (px < a.W && py0 + k < a.H) {
                const int64_t pix = (int64_t)(py0 + k) * a.W + px;
                v[q][0] = T_final[pix];
                last[k] = n_contrib[pix];
                v[q][2] = dL_dimg[pix];
                v[q][3] = dL_dimg[plane + pix];
                v[q][4] = dL_dimg[2 * plane + pix];
                // behind the last contributor: the background
                v[q][1] = v[q][2] * a.bg0 + v[q][3] * a.bg1 + v[q][4] * a.bg2;
            }
            mlast = max(mlast, last[k]);
        }
        p[h].T = make_float2(v[0][0], v[1][0]);
        p[h].accd = make_float2(v[0][1], v[1][1]);
        p[h].dC0 = make_float2(v[0][2], v[1][2]);
        p[h].dC1 = make_float2(v[0][3], v[1][3]);
        p[h].dC2 = make_float2(v[0][4], v[1][4]);
    }
    // positions at or beyond the warp's largest n_contrib reach none of its
    // pixels; never past the tile's own list, whatever n_contrib holds
    const uint32_t m = __reduce_max_sync(0xffffffffu, mlast);
    const int stop = min(begin + (int)m, (int)rg.y);
    const float fpx = (float)px;
    const float2 fpy[2] = {make_float2((float)py0, (float)(py0 + 1)), make_float2((float)(py0 + 2), (float)(py0 + 3))};
    // value k of the transposed reduction lands in lane 4k: its gradient slot
    const int kval = (lane >> 2) & 7;
    float *const gk = (kval < 4 ? g0 : g1) + (kval & 3);
    for (int bend = stop; bend > begin; bend -= 32) {
        const int bstart = max(begin, bend - 32);
        const int idx = bstart + lane;
        bool vis = false;
        uint32_t gid = 0u;
        float4 g, c;
        int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
        if (idx < bend) {
            gid = a.vals[idx];
            g = __ldg(a.xy_conic + gid);
            c = __ldg(a.c_op_box + gid);
            vis = warp_may_see(g, c, rx0, rx1, ry0, ry1, x0, x1, y0, y1);
        }
        const uint32_t bits = __ballot_sync(0xffffffffu, vis);
        if (vis) {
            const uint4 m = q4_box_lanes(x0, x1, y0, y1, ox, ry0);
            warp_stage(a, gid, (uint32_t)(idx - begin), g, c, m, (m.x & m.y & m.z & m.w) == 0xffffffffu,
                       buf[__popc(bits & ((1u << lane) - 1u))]);
        }
        __syncwarp();
        // every position of the round below every pixel's n_contrib: no
        // per-splat position test
        if (__all_sync(0xffffffffu, min(min(last[0], last[1]), min(last[2], last[3])) >= (uint32_t)(bend - begin))) {
            for (int j = __popc(bits) - 1; j >= 0; --j) {  // back to front
                const Staged &sj = buf[j];
                if (sj.lanes[1].x) q4_splat_bwd<false, true>(sj, sj.pad, sj.lanes[0], lane, fpx, fpy, last, p, gk, g2);
                else q4_splat_bwd<false>(sj, sj.pad, sj.lanes[0], lane, fpx, fpy, last, p, gk, g2);
            }
        } else {
            for (int j = __popc(bits) - 1; j >= 0; --j) {
                const Staged &sj = buf[j];
                if (sj.lanes[1].x) q4_splat_bwd<true, true>(sj, sj.pad, sj.lanes[0], lane, fpx, fpy, last, p, gk, g2);
                else q4_splat_bwd(sj, sj.pad, sj.lanes[0], lane, fpx, fpy, last, p, gk, g2);
            }
        }
        __syncwarp();
    }
}

// shared memory of warp-staged tiles: 32 records per warp
__host__ __device__ inline size_t render_warp_smem(int threads) { return sizeof(Staged) * 32 * (threads / 32); }

}  // namespace gsr
