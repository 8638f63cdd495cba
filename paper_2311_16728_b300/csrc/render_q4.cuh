// render_q4.cuh -- the backward blend (K7) of the tile-based renderer of
// Photo-SLAM (arXiv 2311.16728) Sec. 3.3, Eq. 3, for 16 x 16 tiles with four
// pixels per thread.
//
// 64 threads, two warps; warp w covers rows 8 w .. 8 w + 7 of the tile, lane l
// column l & 15 and rows 8 w + 4 (l >> 4) + k, k < 4.  The x terms of a
// splat's exponent are shared by a thread's four pixels, and every per-warp
// cost (staging a splat, the warp's visibility test, the loop over visible
// splats, the gradient reduction and its atomics) is paid once per 128
// pixels instead of once per 64.  One splat per round: the four pixels are
// four independent chains.  The per-pixel arithmetic is the two-pixel
// routines' (render_impl.cuh).  (The forward blend keeps two pixels per
// thread: its per-pixel work is small, and the coarser 16 x 8 warp regions
// and later warp-level termination cost it more than the shared overhead
// saves.)
#pragma once

#include "render_impl.cuh"

namespace gsr {

constexpr int kQ4Threads = 64;

__device__ __forceinline__ void q4_pixels(const RenderArgs &a, int tile, int ti, int &px, int &py0, int &ox,
                                          int &oy) {
    ox = (tile % a.gx) * 16;
    oy = (tile / a.gx) * 16;
    const int w = ti >> 5, l = ti & 31;
    px = ox + (l & 15);
    py0 = oy + 8 * w + 4 * (l >> 4);
}

// Lanes of warp w (rows ry0 .. ry0 + 7 of the columns ox .. ox + 15) whose
// k-th pixel lies in the pixel box [x0, x1] x [y0, y1], for k = 0 .. 3.
__device__ __forceinline__ uint4 q4_box_lanes(int x0, int x1, int y0, int y1, int ox, int ry0) {
    const int c0 = max(x0 - ox, 0), c1 = min(x1 - ox, 15);
    if (c0 > c1) return make_uint4(0u, 0u, 0u, 0u);
    const uint32_t cm = (0xffffu >> (15 - c1)) & (0xffffu << c0);  // columns c0 .. c1
    uint32_t m[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int lo = ry0 + k, hi = ry0 + 4 + k;
        m[k] = ((lo >= y0 && lo <= y1) ? cm : 0u) | ((hi >= y0 && hi <= y1) ? (cm << 16) : 0u);
    }
    return make_uint4(m[0], m[1], m[2], m[3]);
}

// Stages Gaussian gid as stage_splat does, for the two 16 x 8 warps: the
// mask of warps that can see it and, for those, the lanes of each pixel slot
// inside its pixel box.  kExact adds the rectangle test of rect_may_see to
// the ellipse's bounding box (the persistent window kernel, whose register
// budget other phases set; in the one-view kernel the extra registers cost
// more than the dropped warps save).
template <bool kExact>
__device__ __forceinline__ void q4_stage(const RenderArgs &a, uint32_t gid, int ox, int oy, Staged &st,
                                         uint32_t &s_mask) {
    const float4 g = __ldg(a.xy_conic + gid), c = __ldg(a.c_op_box + gid);
    st.rgb = __ldg(a.rgb_depth + gid);
    st.lo = mean_residual(a, gid);
    st.gid = gid;
    const float A = g.z, B = g.w, C = c.x, op = c.y;
    st.xy = make_float4(g.x, g.y, A * kHalfLog2e, B * (2.0f * kHalfLog2e));
    st.cb = make_float4(C * kHalfLog2e, op, c.z, c.w);
    uint32_t mask = 0u;
    const float tau = 2.0f * __logf(255.0f * op);  // alpha >= 1/255  <=>  d^T Q d <= tau
    if (tau > 0.0f) {
        const float bb = B * B;
        const float det = __fmaf_rn(A, C, -bb) + __fmaf_rn(-B, B, bb);
        const float ex = sqrtf(tau * C / det) * 1.001f + 0.01f;
        const float ey = sqrtf(tau * A / det) * 1.001f + 0.01f;
        const uint32_t bx = __float_as_uint(c.z), by = __float_as_uint(c.w);
        const int x0 = (int)(bx & 0xffffu), x1 = (int)(bx >> 16), y0 = (int)(by & 0xffffu), y1 = (int)(by >> 16);
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            const int rx0 = ox, rx1 = ox + 15, ry0 = oy + 8 * w, ry1 = ry0 + 7;
            const bool boxes = x0 <= rx1 && x1 >= rx0 && y0 <= ry1 && y1 >= ry0;
            const float cx = fminf(fmaxf(g.x, (float)rx0), (float)rx1);
            const float cy = fminf(fmaxf(g.y, (float)ry0), (float)ry1);
            if (boxes && fabsf(cx - g.x) <= ex && fabsf(cy - g.y) <= ey &&
                (!kExact || rect_may_see(g.x, g.y, A, B, C, tau, (float)max(rx0, x0), (float)min(rx1, x1),
                                         (float)max(ry0, y0), (float)min(ry1, y1)))) {
                mask |= 1u << w;
                st.lanes[w] = q4_box_lanes(x0, x1, y0, y1, ox, ry0);
            }
        }
    }
    s_mask = mask;
}

__device__ __forceinline__ uint32_t q4_lane_bits(const uint4 m, int k) {
    return k == 0 ? m.x : (k == 1 ? m.y : (k == 2 ? m.z : m.w));
}

// The 64 threads of one tile: the whole CTA (kHalf false), or one half of a
// 128-thread CTA that runs two tiles at once (kHalf: thread index modulo 64,
// named barrier 1 + half over its 64 threads).
template <bool kHalf>
struct Q4Group {
    __device__ __forceinline__ static int tid() { return kHalf ? (int)(threadIdx.x & 63) : (int)threadIdx.x; }
    __device__ __forceinline__ static void sync() {
        if constexpr (kHalf) {
            // immediate barrier ids (1, 2): the CTA reserves only the ids it names
            if (threadIdx.x < 64) asm volatile("bar.sync 1, 64;" ::: "memory");
            else asm volatile("bar.sync 2, 64;" ::: "memory");
        } else {
            __syncthreads();
        }
    }
};

// ---------------------------------------------------------------- K7
// The thread's four pixels are two vertical pairs (pixels 2h, 2h + 1 of
// rows py0 + 2h, py0 + 2h + 1), and each pair runs the per-pixel arithmetic
// of pixel_bwd_update in Blackwell's packed FP32 instructions (FFMA2 /
// FADD2 / FMUL2: two independent lanes, each rounded to nearest like the
// scalar operation), so one issue slot does two pixels' work.  A pixel that
// has no contribution from the splat takes the same instructions with
// alpha = 0, G = 0 and a reciprocal of 1, which leave its state and the
// gradient sums exactly unchanged.  Each of the nine gradient sums is kept
// as a pair over the splat's four pixels and folded once.
struct PairBwd {
    float2 T, accd, dC0, dC1, dC2;
};

// The contribution of one staged splat (list position pos, the warp's box
// lane masks lm) to this thread's four pixels and, reduced over the warp, to
// the splat's screen-space gradient: the pixels' alphas a pair at a time,
// their back-to-front updates, and the warp's transposed reduction with its
// atomics into g0 / g1 (lane 4k: value k at gk) and g2.  kPosTest false:
// the caller knows pos lies below every one of the thread's n_contrib.
// kFast: the splat's pixel box holds all of the warp's pixels and its
// opacity cannot reach the clamp (the staged fast-path flag), so the box and
// clamp tests are dropped; decisions and arithmetic are the general path's.
template <bool kPosTest = true, bool kFast = false>
__device__ __forceinline__ void q4_splat_bwd(const Staged &sj, uint32_t pos, const uint4 lm, int lane, float fpx,
                                             const float2 (&fpy)[2], const uint32_t (&last)[4], PairBwd (&p)[2],
                                             float *gk, float *__restrict__ g2) {
    const float4 g = sj.xy, cb = sj.cb;
    const float2 lo = sj.lo;
    const uint32_t lbit = 1u << lane;  // this lane's bit in the box lane masks
    const float dx = FS(FS(fpx, g.x), lo.x);
    const float t = FM(FM(g.z, dx), dx), bdx = FM(g.w, dx);
    // alpha at the four pixels, a pair at a time
    float2 dy[2], al[2], gs[2];
    bool ok[4], cl[4];
    bool any = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        dy[h] = __fadd2_rn(__fadd2_rn(fpy[h], f2(-g.y)), f2(-lo.y));
        const float2 e = __ffma2_rn(__fmul2_rn(f2(cb.x), dy[h]), dy[h], __ffma2_rn(f2(bdx), dy[h], f2(t)));
        gs[h] = make_float2(ex2_approx(e.x), ex2_approx(e.y));
        const float2 raw = __fmul2_rn(f2(cb.y), gs[h]);
        al[h] = kFast ? raw : make_float2(fminf(kAlphaMax, raw.x), fminf(kAlphaMax, raw.y));
        cl[2 * h] = !kFast && raw.x > kAlphaMax;
        cl[2 * h + 1] = !kFast && raw.y > kAlphaMax;
        ok[2 * h] = (!kPosTest || pos < last[2 * h]) && (kFast || (q4_lane_bits(lm, 2 * h) & lbit) != 0u) &&
                    e.x <= 0.0f && al[h].x >= kAlphaMin;
        ok[2 * h + 1] = (!kPosTest || pos < last[2 * h + 1]) &&
                        (kFast || (q4_lane_bits(lm, 2 * h + 1) & lbit) != 0u) && e.y <= 0.0f && al[h].y >= kAlphaMin;
        any = any || ok[2 * h] || ok[2 * h + 1];
    }
    // v2[0 .. 2]: the lane's dpow-weighted moments in dy (sum dpow,
    // sum dpow dy, sum dpow dy^2), from which the five conic and
    // mean sums follow once per lane (dx is the lane's own);
    // v2[5 .. 8]: the opacity and colour sums
    float2 v2[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) v2[q] = make_float2(0.f, 0.f);
    const float A = g.z * (1.0f / kHalfLog2e), B = g.w * (0.5f / kHalfLog2e);
    const float C = cb.x * (1.0f / kHalfLog2e);
    const float4 col = sj.rgb;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const bool o0 = ok[2 * h], o1 = ok[2 * h + 1];
        const bool q0 = o0 && !cl[2 * h], q1 = o1 && !cl[2 * h + 1];
        // alpha of a pixel without a contribution is 0: every update below leaves it unchanged
        const float2 al_e = make_float2(o0 ? al[h].x : 0.f, o1 ? al[h].y : 0.f);
        const float2 al_g = make_float2(q0 ? al[h].x : 0.f, q1 ? al[h].y : 0.f);
        const float2 g_g = make_float2(q0 ? gs[h].x : 0.f, q1 ? gs[h].y : 0.f);
        const float2 one_m = __fadd2_rn(f2(1.0f), neg2(al_e));
        const float2 rc = make_float2(o0 ? __fdividef(1.0f, one_m.x) : 1.0f,
                                      o1 ? __fdividef(1.0f, one_m.y) : 1.0f);
        PairBwd &P = p[h];
        P.T = __fmul2_rn(P.T, rc);  // transmittance in front of this Gaussian
        const float2 aT = __fmul2_rn(al_e, P.T);
        v2[6] = __ffma2_rn(P.dC0, aT, v2[6]);
        v2[7] = __ffma2_rn(P.dC1, aT, v2[7]);
        v2[8] = __ffma2_rn(P.dC2, aT, v2[8]);
        float2 dc = __fmul2_rn(P.dC0, f2(col.x));
        dc = __ffma2_rn(P.dC1, f2(col.y), dc);
        dc = __ffma2_rn(P.dC2, f2(col.z), dc);
        const float2 dalpha = __fmul2_rn(P.T, __fadd2_rn(dc, neg2(P.accd)));
        P.accd = __ffma2_rn(dc, al_e, __fmul2_rn(P.accd, one_m));
        const float2 dpow = __fmul2_rn(dalpha, al_g);
        v2[5] = __ffma2_rn(dalpha, g_g, v2[5]);
        const float2 tdy = __fmul2_rn(dpow, dy[h]);
        v2[0] = __fadd2_rn(v2[0], dpow);
        v2[1] = __fadd2_rn(v2[1], tdy);
        v2[2] = __ffma2_rn(tdy, dy[h], v2[2]);
    }
    if (__any_sync(0xffffffffu, any)) {
        float v[9];
        const float S0 = v2[0].x + v2[0].y, S1 = v2[1].x + v2[1].y, S2 = v2[2].x + v2[2].y;
        v[0] = __fmaf_rn(B, S1, (A * dx) * S0);  // dL/du: sum dpow (A dx + B dy)
        v[1] = __fmaf_rn(C, S1, (B * dx) * S0);  // dL/dv: sum dpow (B dx + C dy)
        v[2] = (-0.5f * dx * dx) * S0;           // dL/dA: sum dpow (-dx^2 / 2)
        v[3] = -dx * S1;                         // dL/dB: sum dpow (-dx dy)
        v[4] = -0.5f * S2;                       // dL/dC: sum dpow (-dy^2 / 2)
#pragma unroll
        for (int q = 5; q < 9; ++q) v[q] = v2[q].x + v2[q].y;
        float v8;
        const float y = warp_transpose_sum(v, v8);
        // one atomic instruction, predicated on the lanes that hold a total
        const uint32_t gid = sj.gid;
        const bool g0g1 = (lane & 3) == 0;
        if (g0g1 || lane == 1) atomicAdd((g0g1 ? gk : g2) + 4 * (int64_t)gid, g0g1 ? y : v8);
    }
}

template <bool kHalf = false, bool kExact = kHalf>
__device__ __forceinline__ void render_bwd_tile_q4(const RenderArgs &a, int tile, const float *__restrict__ T_final,
                                                   const uint32_t *__restrict__ n_contrib,
                                                   const float *__restrict__ dL_dimg, float *__restrict__ g0,
                                                   float *__restrict__ g1, float *__restrict__ g2, float4 *smem) {
    using G = Q4Group<kHalf>;
    constexpr int nthr = kQ4Threads;
    const int D = a.depth > 0 ? a.depth : nthr;
    Staged *s_st = reinterpret_cast<Staged *>(smem);
    uint32_t *s_mask = reinterpret_cast<uint32_t *>(s_st + D);
    uint32_t *s_max = s_mask + D;  // 2 entries
    const int ti = G::tid();
    int px, py0, ox, oy;
    q4_pixels(a, tile, ti, px, py0, ox, oy);
    const int lane = ti & 31, wid = ti >> 5;
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
    // block-wide max of n_contrib: positions at or beyond it are never used
    const uint32_t m = __reduce_max_sync(0xffffffffu, mlast);
    if (lane == 0) s_max[wid] = m;
    G::sync();
    // never past the tile's own list, whatever n_contrib holds
    const int stop = min(begin + (int)max(s_max[0], s_max[1]), (int)rg.y);
    const float fpx = (float)px;
    const float2 fpy[2] = {make_float2((float)py0, (float)(py0 + 1)), make_float2((float)(py0 + 2), (float)(py0 + 3))};
    // value k of the transposed reduction lands in lane 4k: its gradient slot
    const int kval = (lane >> 2) & 7;
    float *const gk = (kval < 4 ? g0 : g1) + (kval & 3);
    for (int bend = stop; bend > begin; bend -= D) {
        const int bstart = max(begin, bend - D);
        G::sync();
        for (int sl = ti; sl < D; sl += nthr) {
            const int idx = bstart + sl;
            if (idx < bend) {
                q4_stage<kExact>(a, a.vals[idx], ox, oy, s_st[sl], s_mask[sl]);
            } else {
                s_mask[sl] = 0u;
            }
        }
        G::sync();
        const int cnt = bend - bstart;
        for (int c0 = ((cnt - 1) >> 5) << 5; c0 >= 0; c0 -= 32) {
            // splats at or beyond the warp's last contributor reach none of its pixels
            const int j0 = c0 + lane;
            uint32_t bits = __ballot_sync(0xffffffffu, j0 < cnt && ((s_mask[j0] >> wid) & 1u) &&
                                                           (uint32_t)(bstart + j0 - begin) < m);
            while (bits) {  // back to front
                const int j = c0 + 31 - __clz(bits);
                bits &= ~(1u << (j - c0));
                const Staged &sj = s_st[j];
                q4_splat_bwd(sj, (uint32_t)(bstart + j - begin), sj.lanes[wid], lane, fpx, fpy, last, p, gk, g2);
            }
        }
    }
}

// shared memory of one tile's 64 threads for a staging batch of `depth`
// records (a multiple of 16 bytes)
__host__ __device__ inline size_t render_q4_smem(int depth = kQ4Threads) {
    return ((sizeof(Staged) + sizeof(uint32_t)) * depth + 2 * sizeof(uint32_t) + 15) / 16 * 16;
}

}  // namespace gsr
