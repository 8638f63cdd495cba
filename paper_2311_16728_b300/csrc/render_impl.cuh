// render_impl.cuh -- per-tile routines of the forward blend (K5) and its
// backward (K7) for the tile-based renderer of Photo-SLAM (arXiv 2311.16728)
// Sec. 3.3, Eq. 3, shared by the one-view kernels (render.cu) and the
// persistent multi-view kernel (batched.cu).  See render.cu for the design.
#pragma once

#include "gsr_internal.cuh"

namespace gsr {

struct RenderArgs {
    const float4 *xy_conic, *c_op_box, *rgb_depth;
    const float2 *uv_lo;  // residuals of the FP64 projected mean (NULL: the FP32 u, v)
    const uint32_t *vals;
    const uint2 *ranges;  // indexed by tile_off + local tile
    int W, H, tw, th, gx, tile_off;
    int depth;  // records staged per round (0: one per thread)
    float bg0, bg1, bg2;
};

constexpr float kHalfLog2e = -0.5f * 1.4426950408889634f;  // exponent of 2 = kHalfLog2e * (d^T Q d)

// Pixel (px, py0) and (px, py0 + 1) of this thread; origin of the tile.  In
// a 16 x 16 tile each warp covers one 8 x 8 quadrant (its lanes: 8 columns x
// 4 pixel pairs), a squarer footprint than 16 x 4 rows, so fewer splats touch
// it; other tile shapes take rows of the tile in thread order.
__device__ __forceinline__ bool quadrant_warps(const RenderArgs &a) { return a.tw == 16 && a.th == 16; }

__device__ __forceinline__ void thread_pixels(const RenderArgs &a, int tile, int &px, int &py0, int &ox, int &oy) {
    ox = (tile % a.gx) * a.tw;
    oy = (tile / a.gx) * a.th;
    const int t = (int)threadIdx.x;
    if (quadrant_warps(a)) {
        const int w = t >> 5, l = t & 31;
        px = ox + 8 * (w & 1) + (l & 7);
        py0 = oy + 8 * (w >> 1) + 2 * (l >> 3);
    } else {
        px = ox + t % a.tw;
        py0 = oy + 2 * (t / a.tw);
    }
}

// pixel rectangle [rx0, rx1] x [ry0, ry1] of warp w (as thread_pixels maps it)
__device__ __forceinline__ void warp_rect(const RenderArgs &a, int w, int ox, int oy, int &rx0, int &rx1, int &ry0,
                                          int &ry1) {
    if (quadrant_warps(a)) {
        rx0 = ox + 8 * (w & 1);
        rx1 = rx0 + 7;
        ry0 = oy + 8 * (w >> 1);
        ry1 = ry0 + 7;
        return;
    }
    const int t0 = 32 * w, t1 = 32 * w + 31;
    rx0 = a.tw >= 32 ? ox + t0 % a.tw : ox;
    rx1 = a.tw >= 32 ? rx0 + 31 : ox + a.tw - 1;
    ry0 = oy + 2 * (t0 / a.tw);
    ry1 = oy + 2 * (t1 / a.tw) + 1;
}

// Lanes of a quadrant warp (its 8 x 8 pixels at (rx0, ry0); lane l holds
// column l & 7 of rows 2 (l >> 3) and 2 (l >> 3) + 1) whose first (.x) and
// second (.y) pixel lie in the pixel box [x0, x1] x [y0, y1].
__device__ __forceinline__ uint2 quad_box_lanes(int x0, int x1, int y0, int y1, int rx0, int ry0) {
    const int c0 = max(x0 - rx0, 0), c1 = min(x1 - rx0, 7);
    if (c0 > c1) return make_uint2(0u, 0u);
    const uint32_t cm = (0xffu >> (7 - c1)) & (0xffu << c0);  // columns c0 .. c1
    uint32_t m0 = 0u, m1 = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = ry0 + 2 * k;
        if (r >= y0 && r <= y1) m0 |= cm << (8 * k);
        if (r + 1 >= y0 && r + 1 <= y1) m1 |= cm << (8 * k);
    }
    return make_uint2(m0, m1);
}

// Residual of the FP64 projected mean (zero without residuals).  The blends
// take a pixel's offset as (px - u) - u_lo: px - u is exact or within an ulp
// of the offset itself near the mean, and subtracting the residual keeps the
// mean to ~1e-6 pixel where the FP32 u alone carries an ulp of u (~1e-4 pixel
// at u ~ 1000).  The offset depends on the pixel and the Gaussian only, not
// on the tiling, so the image stays independent of the tile shape.
__device__ __forceinline__ float2 mean_residual(const RenderArgs &a, uint32_t gid) {
    return a.uv_lo ? __ldg(a.uv_lo + gid) : make_float2(0.0f, 0.0f);
}

// Stages Gaussian gid: exponent coefficients pre-scaled so that
// exponent_2 = a2 dx^2 + b2 dx dy + c2 dy^2 (= -log2(e) d^T Q d / 2), and the
// mask of warps (of a block of nwarps) that can see it.  kQuad (16 x 16
// tiles, quadrant warps): s_lanes[w] also receives, for every warp w that
// can see it, the lanes whose pixels lie in its pixel box, so the blend
// loops test one bit instead of the box.
// Whether some pixel of the rectangle [rx0, rx1] x [ry0, ry1] (pixel
// indices) can reach alpha >= 1/255, i.e. d^T Q d <= tau: a lower bound on
// the continuous minimum of the quadratic form over the rectangle (0 when it
// holds the mean, else the least over the one or two edges that face the
// mean -- the same minimum as over all four, since a ray from the mean
// reaches every other boundary point through them and the form grows along
// it -- each at its clamped 1D vertex, less a bound on the rounding of the
// terms) against tau with a margin far above the FP32 error of this test and
// of the per-pixel alpha.
// Only warps that cannot see the splat are dropped; the per-pixel test
// decides every blend, so the image does not depend on this test.
__device__ __forceinline__ bool rect_may_see(float u, float v, float A, float B, float C, float tau, float rx0,
                                             float rx1, float ry0, float ry1) {
    const bool out_x = u < rx0 || u > rx1, out_y = v < ry0 || v > ry1;
    // both edges are evaluated on every lane (no divergent branch); an edge
    // that does not face the mean does not enter the minimum
    // the vertical edge on the mean's side: dy at its vertex, clamped to the rectangle
    const float dxv = (u < rx0 ? rx0 : rx1) - u;
    const float dyv = fminf(fmaxf(-__fdividef(B * dxv, C), ry0 - v), ry1 - v);
    // the horizontal edge on the mean's side
    const float dyh = (v < ry0 ? ry0 : ry1) - v;
    const float dxh = fminf(fmaxf(-__fdividef(B * dyh, A), rx0 - u), rx1 - u);
    const float t1v = A * dxv * dxv, t2v = 2.0f * B * dxv * dyv, t3v = C * dyv * dyv;
    const float t1h = A * dxh * dxh, t2h = 2.0f * B * dxh * dyh, t3h = C * dyh * dyh;
    const float lv = (t1v + t2v + t3v) - 1e-5f * (fabsf(t1v) + fabsf(t2v) + fabsf(t3v));
    const float lh = (t1h + t2h + t3h) - 1e-5f * (fabsf(t1h) + fabsf(t2h) + fabsf(t3h));
    const float inf = __int_as_float(0x7f800000);
    const float lb = fminf(out_x ? lv : inf, out_y ? lh : inf);
    return !(out_x || out_y) || lb <= tau * 1.001f + 1e-3f;
}

// One staged splat: everything a warp reads per splat in the blend loops, in
// one 96-byte record (one address per splat, the fields at immediate
// offsets).  The warp masks stay in their own array (the ballot reads 32
// consecutive ones).
struct __align__(16) Staged {
    float4 xy;       // mean (u, v), pre-scaled conic terms a2, b2
    float4 cb;       // pre-scaled c2, opacity, packed pixel box
    float4 rgb;      // colour, depth
    float2 lo;       // position residual
    uint32_t gid, pad;
    uint4 lanes[2];  // box lane masks: 4 x uint2 (quadrant warps) or 2 x uint4 (16 x 8 half warps);
                     // warp-private staging: lanes[0] the warp's masks, lanes[1].x its fast-path flag
};
static_assert(sizeof(Staged) == 96, "staged splat record");

template <bool kQuad>
__device__ __forceinline__ void stage_splat(const RenderArgs &a, uint32_t gid, int ox, int oy, int nwarps,
                                            Staged &st, uint32_t &s_mask) {
    const float4 g = __ldg(a.xy_conic + gid), c = __ldg(a.c_op_box + gid);
    st.rgb = __ldg(a.rgb_depth + gid);
    st.lo = mean_residual(a, gid);
    st.gid = gid;
    const float A = g.z, B = g.w, C = c.x, op = c.y;
    st.xy = make_float4(g.x, g.y, A * kHalfLog2e, B * (2.0f * kHalfLog2e));
    st.cb = make_float4(C * kHalfLog2e, op, c.z, c.w);
    uint2 *s_lanes = reinterpret_cast<uint2 *>(st.lanes);
    uint32_t mask = 0u;
    const float tau = 2.0f * __logf(255.0f * op);  // alpha >= 1/255  <=>  d^T Q d <= tau
    if (tau > 0.0f) {
        // A C - B^2 with Kahan's two-FMA scheme: accurate even when the
        // splat is very elongated and the difference cancels
        const float bb = B * B;
        const float det = __fmaf_rn(A, C, -bb) + __fmaf_rn(-B, B, bb);
        const float ex = sqrtf(tau * C / det) * 1.001f + 0.01f;
        const float ey = sqrtf(tau * A / det) * 1.001f + 0.01f;
        const uint32_t bx = __float_as_uint(c.z), by = __float_as_uint(c.w);
        const int x0 = (int)(bx & 0xffffu), x1 = (int)(bx >> 16), y0 = (int)(by & 0xffffu), y1 = (int)(by >> 16);
        for (int w = 0; w < nwarps; ++w) {
            int rx0, rx1, ry0, ry1;
            warp_rect(a, w, ox, oy, rx0, rx1, ry0, ry1);
            const bool boxes = x0 <= rx1 && x1 >= rx0 && y0 <= ry1 && y1 >= ry0;
            const float cx = fminf(fmaxf(g.x, (float)rx0), (float)rx1);
            const float cy = fminf(fmaxf(g.y, (float)ry0), (float)ry1);
            if (boxes && fabsf(cx - g.x) <= ex && fabsf(cy - g.y) <= ey &&
                rect_may_see(g.x, g.y, A, B, C, tau, (float)max(rx0, x0), (float)min(rx1, x1), (float)max(ry0, y0),
                             (float)min(ry1, y1))) {
                mask |= 1u << w;
                if constexpr (kQuad) s_lanes[w] = quad_box_lanes(x0, x1, y0, y1, rx0, ry0);
            }
        }
    }
    s_mask = mask;
}

// alpha of a staged splat at offset (dx, dy); false when the pixel skips it
// (outside the box, positive exponent, or alpha < 1/255).
struct Eval {
    float G, alpha;
    bool clamped;
};

__device__ __forceinline__ bool splat_alpha(float e2, float op, Eval &r) {
    if (e2 > 0.0f) return false;
    r.G = ex2_approx(e2);
    const float raw = FM(op, r.G);
    r.clamped = raw > kAlphaMax;
    r.alpha = fminf(kAlphaMax, raw);
    return r.alpha >= kAlphaMin;
}

// alpha of one staged splat at this thread's two pixels (px, py0), (px, py0 + 1);
// ok = inside the pixel box and alpha >= 1/255
struct PixAlpha {
    float a0, a1;
    bool ok0, ok1;
};

// box test: the staged lane masks (kQuad) or the box itself
template <bool kQuad>
__device__ __forceinline__ void in_box(const float4 cb, const uint2 *lanes, int px, int py0, bool &in0, bool &in1) {
    if constexpr (kQuad) {
        const int lane = threadIdx.x & 31;
        const uint2 m = lanes[threadIdx.x >> 5];
        in0 = (m.x >> lane) & 1u;
        in1 = (m.y >> lane) & 1u;
    } else {
        const uint32_t bx = __float_as_uint(cb.z), by = __float_as_uint(cb.w);
        const bool xin = px >= (int)(bx & 0xffffu) && px <= (int)(bx >> 16);
        const int y0 = (int)(by & 0xffffu), y1 = (int)(by >> 16);
        in0 = xin && py0 >= y0 && py0 <= y1;
        in1 = xin && py0 + 1 >= y0 && py0 + 1 <= y1;
    }
}

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// The exponent and alpha at the thread's two pixels run as one pair in
// Blackwell's packed FP32 instructions (FFMA2 / FMUL2 / FADD2: each lane
// rounded to nearest exactly like the scalar operation), one issue slot for
// both pixels.
// b0, b1: whether the two pixels lie in the splat's pixel box.
// kUnclamped: the caller knows opacity <= kOpNoClamp, so opacity G < 0.99
// and the clamp is the identity (G = 2^e <= 1 up to the 2^-22 error of
// ex2.approx for e <= 0, and a pixel with e > 0 is skipped anyway).
constexpr float kOpNoClamp = 0.98f;

template <bool kUnclamped = false>
__device__ __forceinline__ void pair_alpha(const float4 g, const float4 cb, const float2 lo, float fpx, float2 fpy,
                                           bool b0, bool b1, PixAlpha &r) {
    const float dx = FS(FS(fpx, g.x), lo.x);
    const float t = FM(FM(g.z, dx), dx), bdx = FM(g.w, dx);
    const float2 dy = __fadd2_rn(__fadd2_rn(fpy, f2(-g.y)), f2(-lo.y));
    const float2 e = __ffma2_rn(__fmul2_rn(f2(cb.x), dy), dy, __ffma2_rn(f2(bdx), dy, f2(t)));
    const float2 raw = __fmul2_rn(f2(cb.y), make_float2(ex2_approx(e.x), ex2_approx(e.y)));
    r.a0 = kUnclamped ? raw.x : fminf(kAlphaMax, raw.x);
    r.a1 = kUnclamped ? raw.y : fminf(kAlphaMax, raw.y);
    r.ok0 = b0 && e.x <= 0.0f && r.a0 >= kAlphaMin;
    r.ok1 = b1 && e.y <= 0.0f && r.a1 >= kAlphaMin;
}

template <bool kQuad>
__device__ __forceinline__ void pixel_pair_alpha(const float4 g, const float4 cb, const float2 lo, const uint2 *lanes,
                                                 int px, float fpx, float2 fpy, int py0, PixAlpha &r) {
    bool b0, b1;
    in_box<kQuad>(cb, lanes, px, py0, b0, b1);
    pair_alpha(g, cb, lo, fpx, fpy, b0, b1, r);
}

// Front-to-back blend of one evaluated splat into the thread's two pixels
// (a pair: T, C0, C1, C2 hold pixel 0 in .x and pixel 1 in .y), packed like
// pixel_pair_alpha; a pixel that takes no part (not ok, or already done)
// keeps its state exactly.  Every lane runs every step, without a branch
// around the lanes that have nothing to blend: the divergent branch cost the
// forward blend more than the work it skipped (render_fwd 112.7 -> 104.6 us
// without it and without the select on T, 300k Gaussians, 1200 x 680).
struct PairFwd {
    float2 T, C0, C1, C2;
    uint32_t last0, last1, nb0, nb1;
    bool done0, done1;
};

__device__ __forceinline__ void blend_fwd_pair(PairFwd &p, bool ok0, bool ok1, float a0, float a1,
                                               const float4 &col, uint32_t pos) {
    bool l0 = ok0 && !p.done0, l1 = ok1 && !p.done1;
    const float2 tn = __fmul2_rn(p.T, __fadd2_rn(f2(1.0f), make_float2(-a0, -a1)));
    if (l0 && tn.x < kTMin) { p.done0 = true; l0 = false; }
    if (l1 && tn.y < kTMin) { p.done1 = true; l1 = false; }
    // alpha of a pixel that takes no part is 0: its weight is 0 and
    // T (1 - 0) = T exactly, so T needs no select (T (1 - alpha) = tn otherwise)
    const float2 ae = make_float2(l0 ? a0 : 0.0f, l1 ? a1 : 0.0f);
    const float2 w = __fmul2_rn(ae, p.T);
    p.C0 = __ffma2_rn(f2(col.x), w, p.C0);
    p.C1 = __ffma2_rn(f2(col.y), w, p.C1);
    p.C2 = __ffma2_rn(f2(col.z), w, p.C2);
    p.T = __fmul2_rn(p.T, __fadd2_rn(f2(1.0f), neg2(ae)));
    if (l0) { p.last0 = pos; ++p.nb0; }
    if (l1) { p.last1 = pos; ++p.nb1; }
}

// ---------------------------------------------------------------- K5
// One tile (local index `tile` of the view in `a`), by the whole block.
// tile_work (may be NULL): receives the tile's largest n_contrib, the depth
// of list its backward walks (the cost proxy of the backward's tile order).
template <bool kQuad>
__device__ __forceinline__ void render_fwd_tile(const RenderArgs &a, int tile, float *__restrict__ img,
                                                float *__restrict__ T_final, uint32_t *__restrict__ n_contrib,
                                                uint32_t *__restrict__ n_blended, float4 *smem,
                                                uint32_t *__restrict__ tile_work = nullptr) {
    const int nthr = blockDim.x, nwarps = nthr >> 5, D = a.depth > 0 ? a.depth : nthr;
    Staged *s_st = reinterpret_cast<Staged *>(smem);
    uint32_t *s_mask = reinterpret_cast<uint32_t *>(s_st + D);
    int px, py0, ox, oy;
    thread_pixels(a, tile, px, py0, ox, oy);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool in0 = px < a.W && py0 < a.H, in1 = px < a.W && py0 + 1 < a.H;
    const uint2 rg = a.ranges[a.tile_off + tile];
    const int begin = (int)rg.x, end = (int)rg.y;
    const float fpx = (float)px;
    const float2 fpy = make_float2((float)py0, (float)(py0 + 1));
    PairFwd p;
    p.T = make_float2(1.0f, 1.0f);
    p.C0 = p.C1 = p.C2 = make_float2(0.0f, 0.0f);
    p.last0 = p.last1 = p.nb0 = p.nb1 = 0u;
    p.done0 = !in0;
    p.done1 = !in1;
    for (int base = begin; base < end; base += D) {
        // stop the whole tile once every pixel has terminated
        if (__syncthreads_count(p.done0 && p.done1) == nthr) break;
        for (int sl = (int)threadIdx.x; sl < D; sl += nthr) {
            const int idx = base + sl;
            if (idx < end) stage_splat<kQuad>(a, a.vals[idx], ox, oy, nwarps, s_st[sl], s_mask[sl]);
            else s_mask[sl] = 0u;
        }
        __syncthreads();
        const int cnt = min(D, end - base);
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            // warp-ballot early termination: leave once no pixel of the warp accumulates
            if (__all_sync(0xffffffffu, p.done0 && p.done1)) break;
            uint32_t bits = __ballot_sync(0xffffffffu, c0 + lane < cnt && ((s_mask[c0 + lane] >> wid) & 1u));
            // two splats per round: their alphas are independent, so both are
            // evaluated before they are blended in list order
            while (bits) {
                const int ja = c0 + __ffs(bits) - 1;
                bits &= bits - 1;
                const bool has_b = bits != 0u;
                const int jb = has_b ? c0 + __ffs(bits) - 1 : ja;
                if (has_b) bits &= bits - 1;
                PixAlpha pa, pb;
                const Staged &sa = s_st[ja], &sb = s_st[jb];
                pixel_pair_alpha<kQuad>(sa.xy, sa.cb, sa.lo, reinterpret_cast<const uint2 *>(sa.lanes), px, fpx, fpy,
                                        py0, pa);
                pixel_pair_alpha<kQuad>(sb.xy, sb.cb, sb.lo, reinterpret_cast<const uint2 *>(sb.lanes), px, fpx, fpy,
                                        py0, pb);
                if (!has_b) pb.ok0 = pb.ok1 = false;
                const uint32_t posa = (uint32_t)(base - begin + ja + 1), posb = (uint32_t)(base - begin + jb + 1);
                blend_fwd_pair(p, pa.ok0, pa.ok1, pa.a0, pa.a1, sa.rgb, posa);
                blend_fwd_pair(p, pb.ok0, pb.ok1, pb.a0, pb.a1, sb.rgb, posb);
            }
        }
    }
    const int64_t plane = (int64_t)a.W * a.H;
    if (in0) {
        const int64_t pix = (int64_t)py0 * a.W + px;
        img[pix] = p.C0.x + p.T.x * a.bg0;
        img[plane + pix] = p.C1.x + p.T.x * a.bg1;
        img[2 * plane + pix] = p.C2.x + p.T.x * a.bg2;
        T_final[pix] = p.T.x;
        n_contrib[pix] = p.last0;
        if (n_blended) n_blended[pix] = p.nb0;
    }
    if (in1) {
        const int64_t pix = (int64_t)(py0 + 1) * a.W + px;
        img[pix] = p.C0.y + p.T.y * a.bg0;
        img[plane + pix] = p.C1.y + p.T.y * a.bg1;
        img[2 * plane + pix] = p.C2.y + p.T.y * a.bg2;
        T_final[pix] = p.T.y;
        n_contrib[pix] = p.last1;
        if (n_blended) n_blended[pix] = p.nb1;
    }
    if (tile_work) {  // every thread is past the blend loop (its exit is block-uniform)
        __shared__ uint32_t s_work;
        if (threadIdx.x == 0) s_work = 0u;
        __syncthreads();
        const uint32_t m = __reduce_max_sync(0xffffffffu, max(p.last0, p.last1));
        if ((threadIdx.x & 31) == 0) atomicMax(&s_work, m);
        __syncthreads();
        if (threadIdx.x == 0) tile_work[tile] = s_work;
    }
}


// ---------------------------------------------------------------- K7
// Back to front from each pixel's last contributor.  T_i = T_{i+1} / (1 -
// alpha_i) recovers the transmittance in front of each Gaussian; the colour
// behind it, normalised by T_{i+1}, follows acc <- acc (1 - alpha) + c alpha.
//   dL/dc_i     = dL/dC alpha_i T_i
//   dL/dalpha_i = T_i dL/dC . (c_i - acc)
// then through alpha = opacity exp(power) (zero where the 0.99 clamp holds).
// Only dL/dC . acc enters, and it obeys the same recursion with dL/dC . c_i
// in place of c_i, so the pixel keeps that one scalar (accd) instead of acc.
struct PixelBwd {
    float T, accd, dC0, dC1, dC2;
    uint32_t last;
};

// A staged splat seen from this thread's two pixels: offsets, the original
// conic for the gradient formulas, the pixel-independent factors of the
// exponent's gradient, and each pixel's alpha (ok = the pixel has a
// contribution: inside the box, before its last contributor, alpha above
// the skip threshold).
struct SplatBwd {
    float dx, dy0, dy1, A, B, C;
    float Adx, Bdx, hdx2;  // A dx, B dx, -dx^2 / 2
    Eval e0, e1;
    bool ok0, ok1;
};

// Adds the contribution of a splat with (already evaluated) alpha to this
// pixel's state and to v[9] (dy: this pixel's vertical offset).
__device__ __forceinline__ void pixel_bwd_update(PixelBwd &p, const Eval &ev, const SplatBwd &s, float dy,
                                                 const float4 &col, float v[9]) {
    const float one_m = 1.0f - ev.alpha;
    p.T = __fdividef(p.T, one_m);  // transmittance in front of this Gaussian
    const float aT = ev.alpha * p.T;
    v[6] += p.dC0 * aT;
    v[7] += p.dC1 * aT;
    v[8] += p.dC2 * aT;
    const float dc = p.dC0 * col.x + p.dC1 * col.y + p.dC2 * col.z;
    const float dalpha = p.T * (dc - p.accd);
    p.accd = p.accd * one_m + dc * ev.alpha;
    if (!ev.clamped) {
        const float dpow = dalpha * ev.alpha;
        v[5] += dalpha * ev.G;
        v[0] += dpow * (s.Adx + s.B * dy);
        v[1] += dpow * (s.C * dy + s.Bdx);
        v[2] += dpow * s.hdx2;
        v[3] -= (dpow * s.dx) * dy;
        v[4] += dpow * (-0.5f * dy * dy);
    }
}

template <bool kQuad>
__device__ __forceinline__ void splat_bwd_eval(const float4 g, const float4 cb, const float2 lo, const uint2 *lanes,
                                               int px, float fpx, float fpy0, float fpy1, int py0, bool live0,
                                               bool live1, SplatBwd &r) {
    bool b0, b1;
    in_box<kQuad>(cb, lanes, px, py0, b0, b1);
    r.dx = FS(FS(fpx, g.x), lo.x);
    const float t = FM(FM(g.z, r.dx), r.dx), bdx = FM(g.w, r.dx);
    r.dy0 = FS(FS(fpy0, g.y), lo.y);
    r.dy1 = FS(FS(fpy1, g.y), lo.y);
    const float e0 = __fmaf_rn(FM(cb.x, r.dy0), r.dy0, __fmaf_rn(bdx, r.dy0, t));
    const float e1 = __fmaf_rn(FM(cb.x, r.dy1), r.dy1, __fmaf_rn(bdx, r.dy1, t));
    r.A = g.z * (1.0f / kHalfLog2e);
    r.B = g.w * (0.5f / kHalfLog2e);
    r.C = cb.x * (1.0f / kHalfLog2e);
    r.Adx = r.A * r.dx;
    r.Bdx = r.B * r.dx;
    r.hdx2 = -0.5f * r.dx * r.dx;
    r.ok0 = live0 && b0 && splat_alpha(e0, cb.y, r.e0);
    r.ok1 = live1 && b1 && splat_alpha(e1, cb.y, r.e1);
}

// Sums v[0..8] over the warp without broadcasting every value: each halving
// step keeps half of the values in each lane of a pair and swaps the other
// half (9 shuffles for v[0..7], 5 for v[8]).  Afterwards lane l holds the
// warp total of value (l >> 2) & 7 and every lane holds the total of v[8].
__device__ __forceinline__ float warp_transpose_sum(float v[9], float &v8) {
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = b4 ? v[k] : v[k + 4];
        const float keep = b4 ? v[k + 4] : v[k];
        w[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float x[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = b3 ? w[k] : w[k + 2];
        const float keep = b3 ? w[k + 2] : w[k];
        x[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float y = (b2 ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, b2 ? x[0] : x[1], 4);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    v8 = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v8 += __shfl_xor_sync(0xffffffffu, v8, o);
    return y;
}

template <bool kQuad>
__device__ __forceinline__ void render_bwd_tile(const RenderArgs &a, int tile, const float *__restrict__ T_final,
                                                const uint32_t *__restrict__ n_contrib,
                                                const float *__restrict__ dL_dimg, float *__restrict__ g0,
                                                float *__restrict__ g1, float *__restrict__ g2, float4 *smem) {
    const int nthr = blockDim.x, nwarps = nthr >> 5, D = a.depth > 0 ? a.depth : nthr;
    Staged *s_st = reinterpret_cast<Staged *>(smem);
    uint32_t *s_mask = reinterpret_cast<uint32_t *>(s_st + D);
    uint32_t *s_max = s_mask + D;  // 32 entries
    int px, py0, ox, oy;
    thread_pixels(a, tile, px, py0, ox, oy);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool in0 = px < a.W && py0 < a.H, in1 = px < a.W && py0 + 1 < a.H;
    const uint2 rg = a.ranges[a.tile_off + tile];
    const int begin = (int)rg.x;
    const int64_t plane = (int64_t)a.W * a.H;
    PixelBwd p0{0.f, 0.f, 0.f, 0.f, 0.f, 0u}, p1 = p0;
    if (in0) {
        const int64_t pix = (int64_t)py0 * a.W + px;
        p0.T = T_final[pix];
        p0.last = n_contrib[pix];
        p0.dC0 = dL_dimg[pix];
        p0.dC1 = dL_dimg[plane + pix];
        p0.dC2 = dL_dimg[2 * plane + pix];
        p0.accd = p0.dC0 * a.bg0 + p0.dC1 * a.bg1 + p0.dC2 * a.bg2;  // behind the last contributor: the background
    }
    if (in1) {
        const int64_t pix = (int64_t)(py0 + 1) * a.W + px;
        p1.T = T_final[pix];
        p1.last = n_contrib[pix];
        p1.dC0 = dL_dimg[pix];
        p1.dC1 = dL_dimg[plane + pix];
        p1.dC2 = dL_dimg[2 * plane + pix];
        p1.accd = p1.dC0 * a.bg0 + p1.dC1 * a.bg1 + p1.dC2 * a.bg2;
    }
    // block-wide max of n_contrib: positions at or beyond it are never used
    const uint32_t m = __reduce_max_sync(0xffffffffu, max(p0.last, p1.last));
    if (lane == 0) s_max[wid] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < (unsigned)nwarps ? s_max[threadIdx.x] : 0u;
        v = __reduce_max_sync(0xffffffffu, v);
        if (threadIdx.x == 0) s_max[0] = v;
    }
    __syncthreads();
    // never past the tile's own list, whatever n_contrib holds
    const int stop = min(begin + (int)s_max[0], (int)rg.y);
    const float fpx = (float)px, fpy0 = (float)py0, fpy1 = (float)(py0 + 1);
    // value k of the transposed reduction lands in lane 4k: its gradient slot
    const int kval = (lane >> 2) & 7;
    float *const gk = (kval < 4 ? g0 : g1) + (kval & 3);
    for (int bend = stop; bend > begin; bend -= D) {
        const int bstart = max(begin, bend - D);
        __syncthreads();
        for (int sl = (int)threadIdx.x; sl < D; sl += nthr) {
            const int idx = bstart + sl;
            if (idx < bend) {
                stage_splat<kQuad>(a, a.vals[idx], ox, oy, nwarps, s_st[sl], s_mask[sl]);
            } else {
                s_mask[sl] = 0u;
            }
        }
        __syncthreads();
        const int cnt = bend - bstart;
        for (int c0 = ((cnt - 1) >> 5) << 5; c0 >= 0; c0 -= 32) {
            // splats at or beyond the warp's last contributor reach none of its pixels
            const int j0 = c0 + lane;
            uint32_t bits = __ballot_sync(0xffffffffu, j0 < cnt && ((s_mask[j0] >> wid) & 1u) &&
                                                           (uint32_t)(bstart + j0 - begin) < m);
            // two splats per round, back to front: both are evaluated first
            // (independent), then applied in order, then reduced together
            while (bits) {
                const int ja = c0 + 31 - __clz(bits);
                bits &= ~(1u << (ja - c0));
                const bool has_b = bits != 0u;
                const int jb = has_b ? c0 + 31 - __clz(bits) : ja;
                if (has_b) bits &= ~(1u << (jb - c0));
                const uint32_t posa = (uint32_t)(bstart + ja - begin), posb = (uint32_t)(bstart + jb - begin);
                SplatBwd sa, sb;
                const Staged &ra = s_st[ja], &rb = s_st[jb];
                splat_bwd_eval<kQuad>(ra.xy, ra.cb, ra.lo, reinterpret_cast<const uint2 *>(ra.lanes), px, fpx, fpy0,
                                      fpy1, py0, posa < p0.last, posa < p1.last, sa);
                splat_bwd_eval<kQuad>(rb.xy, rb.cb, rb.lo, reinterpret_cast<const uint2 *>(rb.lanes), px, fpx, fpy0,
                                      fpy1, py0, has_b && posb < p0.last, has_b && posb < p1.last, sb);
                float va[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float vb[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (sa.ok0 || sa.ok1 || sb.ok0 || sb.ok1) {
                    const float4 cola = ra.rgb, colb = rb.rgb;
                    if (sa.ok0) pixel_bwd_update(p0, sa.e0, sa, sa.dy0, cola, va);
                    if (sb.ok0) pixel_bwd_update(p0, sb.e0, sb, sb.dy0, colb, vb);
                    if (sa.ok1) pixel_bwd_update(p1, sa.e1, sa, sa.dy1, cola, va);
                    if (sb.ok1) pixel_bwd_update(p1, sb.e1, sb, sb.dy1, colb, vb);
                }
                const bool anya = __any_sync(0xffffffffu, sa.ok0 || sa.ok1);
                const bool anyb = __any_sync(0xffffffffu, sb.ok0 || sb.ok1);
                if (anya) {
                    float v8;
                    const float y = warp_transpose_sum(va, v8);
                    const uint32_t gid = ra.gid;
                    if ((lane & 3) == 0) atomicAdd(gk + 4 * (int64_t)gid, y);
                    else if (lane == 1) atomicAdd(g2 + 4 * (int64_t)gid, v8);
                }
                if (anyb) {
                    float v8;
                    const float y = warp_transpose_sum(vb, v8);
                    const uint32_t gid = rb.gid;
                    if ((lane & 3) == 0) atomicAdd(gk + 4 * (int64_t)gid, y);
                    else if (lane == 1) atomicAdd(g2 + 4 * (int64_t)gid, v8);
                }
            }
        }
    }
}


// dynamic shared memory of the two tile routines for a staging batch of
// `depth` records
__host__ __device__ inline size_t render_fwd_smem(int depth) {
    return (sizeof(Staged) + sizeof(uint32_t)) * depth;
}
__host__ __device__ inline size_t render_bwd_smem(int depth) {
    return (sizeof(Staged) + sizeof(uint32_t)) * depth + 32 * sizeof(uint32_t);
}

}  // namespace gsr
