// ssim_impl.cuh -- block routines of the Eq. 4 loss (L1 + D-SSIM) of
// Photo-SLAM (arXiv 2311.16728, Sec. 3.3), shared by the one-image kernels
// (loss.cu) and the persistent multi-view kernel (batched.cu).  See loss.cu
// for the maths.
#pragma once

#include <math.h>

#include "tma.cuh"

namespace gsr {

constexpr int kLTW = 32, kLTH = 32, kLR = 5;       // output tile and window radius
constexpr int kRW = kLTW + 2 * kLR, kRH = kLTH + 2 * kLR;
// Staged planes, two layouts of rows oy - 5 .. oy + 36:
//  - staged by the threads: columns ox - 5 .. ox + 36, row stride kRS = 45
//    (the row pass's scalar loads hit distinct banks);
//  - staged by TMA: columns ox - 8 .. ox + 39, row stride kRP = 48 floats (a
//    TMA box starts on a 16-byte column boundary; the window's halo starts at
//    column kRC = 3), read by the row pass in 16-byte loads.
constexpr int kRS = 45;
constexpr int kRP = 48, kRX = 8, kRC = kRX - kLR;
template <bool kTma> struct Region {
    static constexpr int pitch = kTma ? kRP : kRS;    // row stride
    static constexpr int col0 = kTma ? kRX : kLR;     // column of the tile's first output column
    static constexpr int plane = kRH * pitch;         // floats of one staged plane
};
constexpr int kPlane = Region<true>::plane;        // TMA plane: 8064 bytes, a 128-byte multiple
constexpr int kRun = 4;                            // outputs per thread along a row / column
constexpr int kMS = kLTW + 1;                      // row stride of the row-blurred maps (odd: fewer
                                                   // bank conflicts on the row pass's stores)
constexpr int kLThreads = 256;

struct Win {
    float w[11];
};

inline Win ssim_window() {
    Win k;
    double s = 0, v[11];
    for (int i = 0; i < 11; ++i) {
        v[i] = exp(-((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
        s += v[i];
    }
    for (int i = 0; i < 11; ++i) k.w[i] = (float)(v[i] / s);
    return k;
}

// The block sums of a and b (warp shuffles, then the warps' totals by the
// first warp), both in one shared-memory round of two barriers.
template <int NT>
__device__ __forceinline__ float2 block_sum2(float a, float b, float *s_red) {
    constexpr int kW = NT / 32;
    static_assert(2 * kW <= 32, "two partial sums per warp in s_red[32]");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_red[threadIdx.x >> 5] = a;
        s_red[kW + (threadIdx.x >> 5)] = b;
    }
    __syncthreads();
    float ra = 0.f, rb = 0.f;
    if (threadIdx.x < 32) {
        ra = threadIdx.x < kW ? s_red[threadIdx.x] : 0.f;
        rb = threadIdx.x < kW ? s_red[kW + threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ra += __shfl_xor_sync(0xffffffffu, ra, o);
            rb += __shfl_xor_sync(0xffffffffu, rb, o);
        }
    }
    __syncthreads();
    return make_float2(ra, rb);  // valid in thread 0
}

// Stages a (kRH x kRW) region of each of the NP planes src[p] around the
// tile (zero outside) into dst + p kRH kRS: a thread's loads for all planes
// are issued in batches of up to 7 positions before the batch's shared-memory
// stores (one memory round trip per batch: one for 256 threads, two for
// 128); a region inside the image skips the bounds tests.
template <int NT, int NP>
__device__ __forceinline__ void stage_planes(const float *const (&src)[NP], int H, int W, int ox, int oy,
                                             float *dst) {
    constexpr int kN = kRH * kRW, kPer = (kN + NT - 1) / NT, kBatch = 7;
    const int gx0 = ox - kLR, gy0 = oy - kLR;
    const bool interior = gx0 >= 0 && gy0 >= 0 && gx0 + kRW <= W && gy0 + kRH <= H;
#pragma unroll
    for (int j0 = 0; j0 < kPer; j0 += kBatch) {
        float v[NP][kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int idx = (int)threadIdx.x + (j0 + j) * NT;
            const int r = idx / kRW, q = idx - r * kRW;
            const int gy = gy0 + r, gx = gx0 + q;
            const bool ok = j0 + j < kPer && idx < kN && (interior || (gy >= 0 && gy < H && gx >= 0 && gx < W));
#pragma unroll
            for (int pl = 0; pl < NP; ++pl) v[pl][j] = ok ? src[pl][(int64_t)gy * W + gx] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int idx = (int)threadIdx.x + (j0 + j) * NT;
            const int r = idx / kRW, q = idx - r * kRW;
            if (j0 + j < kPer && idx < kN) {
#pragma unroll
                for (int pl = 0; pl < NP; ++pl) dst[pl * kRH * kRS + r * kRS + q] = v[pl][j];
            }
        }
    }
}

// The same regions, copied by the Tensor Memory Accelerator: plane p of the
// C x H x W tensor maps[p] (FP32, zero outside the image), box 48 x 42 x 1
// at column ox - 8 (a multiple of 4: the 16-byte rule of the box's first
// column), row oy - 5, channel c, into dst + p kPlane (128-byte aligned).
// Thread 0 issues the copies on the mbarrier `bar` (one phase per call:
// `parity` alternates between calls); every thread waits, with a bound.
// Returns false, in every thread, when the wait gave up.
template <int NP>
__device__ __forceinline__ bool stage_planes_tma(const CUtensorMap *const (&maps)[NP], int ox, int oy, int c,
                                                 float *dst, uint64_t *bar, uint32_t parity) {
    if (threadIdx.x == 0) {
        tma::mbar_expect_tx(bar, (uint32_t)(NP * kPlane * sizeof(float)));
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) tma::load_3d(dst + pl * kPlane, maps[pl], ox - kRX, oy - kLR, c, bar);
    }
    const bool ok = tma::mbar_wait(bar, parity);
    return __syncthreads_or(!ok) == 0;
}

// One-time set-up of the staging mbarrier of a CTA (before its first
// stage_planes_tma; every thread calls it).
__device__ __forceinline__ void stage_tma_init(uint64_t *bar) {
    if (threadIdx.x == 0) {
        tma::mbar_init(bar, 1);
        tma::fence_barrier_init();
    }
    __syncthreads();
}

template <bool kTma> constexpr size_t pass1_floats() { return 2 * Region<kTma>::plane + 5 * kRH * kMS; }
template <bool kTma> constexpr size_t pass2_floats() { return 3 * Region<kTma>::plane + 3 * kRH * kMS; }
constexpr size_t kPass1Floats = pass1_floats<false>();  // the thread-staged layout
constexpr size_t kPass2Floats = pass2_floats<false>();

__device__ __forceinline__ float2 f2w(float x) { return make_float2(x, x); }

// The separable blurs run two of their maps as one pair in Blackwell's
// packed FP32 instructions (FFMA2 / FMUL2: each lane rounded to nearest like
// the scalar operation), so one issue slot advances two maps: the moments
// (mean x, mean y) and (E x^2, E y^2) as pairs and E xy alone in pass 1, the
// partials (a, b) as a pair and c alone in pass 2.

// Pass 1 on the 32 x 32 output block (bx, by) of channel c: windowed moments
// (separable: rows then columns, kRun outputs per thread from kRun + 10
// staged values), SSIM map, its partials (a, b, c) and the block's sums of
// |x - y| and SSIM into part[0], part[1].
// kTma: x and y come by TMA (tensor maps tmx, tmy, the CTA's mbarrier `bar`
// and its phase parity), else the threads stage them.
template <int NT, bool kTma = false>
__device__ __forceinline__ void ssim_pass1_block(const float *__restrict__ x, const float *__restrict__ y, int H,
                                                 int W, const Win &win, float *__restrict__ mapA,
                                                 float *__restrict__ mapB, float *__restrict__ mapC,
                                                 float *__restrict__ part, int bx, int by, int c, float *sm,
                                                 float *s_red, const CUtensorMap *tmx = nullptr,
                                                 const CUtensorMap *tmy = nullptr, uint64_t *bar = nullptr,
                                                 uint32_t parity = 0u) {
    using Rg = Region<kTma>;
    float *sX = sm, *sY = sm + Rg::plane;
    // row-blurred moments: (mean x, mean y) and (E x^2, E y^2) pairs, then E xy
    float2 *sM2 = reinterpret_cast<float2 *>(sm + 2 * Rg::plane);  // [kRH][kMS]
    float2 *sS2 = sM2 + kRH * kMS;                              // [kRH][kMS]
    float *sXY = reinterpret_cast<float *>(sS2 + kRH * kMS);    // [kRH][kMS]
    const int ox = bx * kLTW, oy = by * kLTH;
    const int64_t plane = (int64_t)H * W, cb = (int64_t)c * plane;
    __syncthreads();  // the previous block's readers of sm are done
    if constexpr (kTma) {
        const CUtensorMap *const maps[2] = {tmx, tmy};
        if (!stage_planes_tma<2>(maps, ox, oy, c, sX, bar, parity)) {
            if (threadIdx.x == 0) part[0] = part[1] = __int_as_float(0x7fc00000);  // the loss reads NaN
            return;
        }
    } else {
        const float *const planes[2] = {x + cb, y + cb};
        stage_planes<NT, 2>(planes, H, W, ox, oy, sX);  // sY = sX + kRH kRS
        __syncthreads();
    }
    // a warp covers four rows of eight runs: its staged loads hit distinct
    // banks (16-byte loads: in each quarter warp), the row-blurred stores
    // (odd row stride kMS) at most two lanes a bank
    if constexpr (!kTma)
    for (int item = threadIdx.x; item < kRH * (kLTW / kRun); item += NT) {
        const int r = item / (kLTW / kRun), j0 = (item % (kLTW / kRun)) * kRun;
        {
            // values and their products once per staged column
            float2 v[kRun + 10], q[kRun + 10];
            float xy[kRun + 10];
#pragma unroll
            for (int k = 0; k < kRun + 10; ++k) {
                v[k] = make_float2(sX[r * kRS + j0 + k], sY[r * kRS + j0 + k]);
                q[k] = __fmul2_rn(v[k], v[k]);
                xy[k] = v[k].x * v[k].y;
            }
#pragma unroll
            for (int o = 0; o < kRun; ++o) {
                float2 m = make_float2(0.f, 0.f), sq = make_float2(0.f, 0.f);
                float sxy = 0.f;
#pragma unroll
                for (int k = 0; k < 11; ++k) {
                    const float w = win.w[k];
                    m = __ffma2_rn(f2w(w), v[o + k], m);
                    sq = __ffma2_rn(f2w(w), q[o + k], sq);
                    sxy = __fmaf_rn(w, xy[o + k], sxy);
                }
                sM2[r * kMS + j0 + o] = m;
                sS2[r * kMS + j0 + o] = sq;
                sXY[r * kMS + j0 + o] = sxy;
            }
        }
    }
    else
    for (int item = threadIdx.x; item < kRH * (kLTW / kRun); item += NT) {
        const int r = item / (kLTW / kRun), j0 = (item % (kLTW / kRun)) * kRun;
        // streamed over the staged columns: five 16-byte loads a plane
        // (columns j0 .. j0 + 19 of the staged row, of which kRC .. kRC + 13
        // are used); each value and its products update the outputs whose
        // window holds it, every sum in ascending tap order
        float2 m[kRun], sq[kRun];
        float sxy[kRun];
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
            m[o] = sq[o] = make_float2(0.f, 0.f);
            sxy[o] = 0.f;
        }
        const float4 *px4 = reinterpret_cast<const float4 *>(sX + r * kRP + j0);
        const float4 *py4 = reinterpret_cast<const float4 *>(sY + r * kRP + j0);
#pragma unroll
        for (int m4 = 0; m4 < 5; ++m4) {
            const float4 a = px4[m4], b = py4[m4];
            const float ax[4] = {a.x, a.y, a.z, a.w}, by[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * m4 + i - kRC;  // staged column k of the window run
                if (k < 0 || k >= kRun + 10) continue;
                const float2 v = make_float2(ax[i], by[i]);
                const float2 q = __fmul2_rn(v, v);
                const float xy = v.x * v.y;
#pragma unroll
                for (int o = 0; o < kRun; ++o) {
                    if (k - o < 0 || k - o > 10) continue;
                    const float w = win.w[k - o];
                    m[o] = __ffma2_rn(f2w(w), v, m[o]);
                    sq[o] = __ffma2_rn(f2w(w), q, sq[o]);
                    sxy[o] = __fmaf_rn(w, xy, sxy[o]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
            sM2[r * kMS + j0 + o] = m[o];
            sS2[r * kMS + j0 + o] = sq[o];
            sXY[r * kMS + j0 + o] = sxy[o];
        }
    }
    __syncthreads();
    float l1 = 0.f, ssim = 0.f;
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    // columns: virtual thread = (column, run of kRun rows); 256 of them
    for (int vt = threadIdx.x; vt < kLTW * (kLTH / kRun); vt += NT) {
        const int tx = vt % kLTW, i0 = (vt / kLTW) * kRun;
        float2 mm[kRun], ss[kRun];
        float sxyv[kRun];
        {
            float2 cm[kRun + 10], cs[kRun + 10];
            float cx[kRun + 10];
#pragma unroll
            for (int k = 0; k < kRun + 10; ++k) {
                cm[k] = sM2[(i0 + k) * kMS + tx];
                cs[k] = sS2[(i0 + k) * kMS + tx];
                cx[k] = sXY[(i0 + k) * kMS + tx];
            }
#pragma unroll
            for (int o = 0; o < kRun; ++o) {
                float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
                float e = 0.f;
#pragma unroll
                for (int k = 0; k < 11; ++k) {
                    const float w = win.w[k];
                    a = __ffma2_rn(f2w(w), cm[o + k], a);
                    b = __ffma2_rn(f2w(w), cs[o + k], b);
                    e = __fmaf_rn(w, cx[o + k], e);
                }
                mm[o] = a;
                ss[o] = b;
                sxyv[o] = e;
            }
        }
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
            const int gx = ox + tx, gy = oy + i0 + o;
            if (gx < W && gy < H) {
                const float mx = mm[o].x, my = mm[o].y;
                const float sxx = ss[o].x - mx * mx, syy = ss[o].y - my * my, sxy = sxyv[o] - mx * my;
                const float A1 = 2.f * mx * my + C1, A2 = 2.f * sxy + C2;
                const float B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
                const float iB = __fdividef(1.0f, B1 * B2);  // B1 B2 >= C1 C2 > 0: the fast reciprocal (2 ulp)
                const float S = A1 * A2 * iB;
                // 1 / B1 = B2 iB and 1 / B2 = B1 iB: one division per pixel
                const float dS_dmx = 2.f * my * A2 * iB - S * 2.f * mx * (B2 * iB);
                const float dS_dsxx = -S * (B1 * iB);
                const float dS_dsxy = 2.f * A1 * iB;
                const int64_t idx = cb + (int64_t)gy * W + gx;
                mapA[idx] = dS_dmx - 2.f * mx * dS_dsxx - my * dS_dsxy;
                mapB[idx] = dS_dsxx;
                mapC[idx] = dS_dsxy;
                const int rr = i0 + o + kLR, qq = tx + Rg::col0;
                l1 += fabsf(sX[rr * Rg::pitch + qq] - sY[rr * Rg::pitch + qq]);
                ssim += S;
            }
        }
    }
    const float2 s12 = block_sum2<NT>(l1, ssim, s_red);
    if (threadIdx.x == 0) {
        part[0] = s12.x;
        part[1] = s12.y;
    }
}

// Pass 2 on block (bx, by) of channel c: blur (a, b, c) (the adjoint of the
// symmetric window), then
// dL/dx = scale ((1 - lambda) sign(x - y) - lambda (G*a + 2 x G*b + y G*c)) / (C H W).
// kTma: (a, b, c) come by TMA (tensor maps tma_a, tma_b, tma_c, the CTA's
// mbarrier `bar` and its phase parity), else the threads stage them.
template <int NT, bool kTma = false>
__device__ __forceinline__ void ssim_pass2_block(const float *__restrict__ x, const float *__restrict__ y, int H,
                                                 int W, int C, const Win &win, const float *__restrict__ mapA,
                                                 const float *__restrict__ mapB, const float *__restrict__ mapC,
                                                 float lambda, float scale, float *__restrict__ dx_out, int bx, int by,
                                                 int c, float *sm, const CUtensorMap *tma_a = nullptr,
                                                 const CUtensorMap *tma_b = nullptr,
                                                 const CUtensorMap *tma_c = nullptr, uint64_t *bar = nullptr,
                                                 uint32_t parity = 0u) {
    using Rg = Region<kTma>;
    float *sM = sm;                                                  // [3][kRH][pitch]
    float2 *sAB = reinterpret_cast<float2 *>(sm + 3 * Rg::plane);    // [kRH][kMS] row-blurred (a, b)
    float *sCh = reinterpret_cast<float *>(sAB + kRH * kMS);      // [kRH][kMS] row-blurred c
    const int ox = bx * kLTW, oy = by * kLTH;
    const int64_t plane = (int64_t)H * W, cb = (int64_t)c * plane;
    const float inv_n = (float)((double)scale / ((double)C * (double)plane));
    // one column run per thread: its rendered and target values are loaded
    // before the staging, in flight during the copy and both blurs
    constexpr bool kEarly = kTma && NT == kLTW * (kLTH / kRun);
    float xs[kRun], ys[kRun];
    if constexpr (kEarly) {
        const int tx = (int)threadIdx.x % kLTW, i0 = ((int)threadIdx.x / kLTW) * kRun;
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
            const int gx = ox + tx, gy = oy + i0 + o;
            const bool in = gx < W && gy < H;
            const int64_t idx = cb + (int64_t)(in ? gy : 0) * W + (in ? gx : 0);
            xs[o] = x[idx];
            ys[o] = y[idx];
        }
    }
    __syncthreads();
    if constexpr (kTma) {
        const CUtensorMap *const maps[3] = {tma_a, tma_b, tma_c};
        if (!stage_planes_tma<3>(maps, ox, oy, c, sM, bar, parity)) {
            for (int k = threadIdx.x; k < kLTW * kLTH; k += NT) {  // the gradient reads NaN
                const int gx = ox + k % kLTW, gy = oy + k / kLTW;
                if (gx < W && gy < H) dx_out[cb + (int64_t)gy * W + gx] = __int_as_float(0x7fc00000);
            }
            return;
        }
    } else {
        const float *const planes[3] = {mapA + cb, mapB + cb, mapC + cb};
        stage_planes<NT, 3>(planes, H, W, ox, oy, sM);
        __syncthreads();
    }
    // a warp covers four rows of eight runs (as in pass 1)
    if constexpr (!kTma)
    for (int item = threadIdx.x; item < kRH * (kLTW / kRun); item += NT) {
        const int r = item / (kLTW / kRun), j0 = (item % (kLTW / kRun)) * kRun;
        {
            float2 ab[kRun + 10];
            float cc[kRun + 10];
#pragma unroll
            for (int k = 0; k < kRun + 10; ++k) {
                ab[k] = make_float2(sM[r * kRS + j0 + k], sM[kRH * kRS + r * kRS + j0 + k]);
                cc[k] = sM[2 * kRH * kRS + r * kRS + j0 + k];
            }
#pragma unroll
            for (int o = 0; o < kRun; ++o) {
                float2 s2 = make_float2(0.f, 0.f);
                float s1 = 0.f;
#pragma unroll
                for (int k = 0; k < 11; ++k) {
                    s2 = __ffma2_rn(f2w(win.w[k]), ab[o + k], s2);
                    s1 = __fmaf_rn(win.w[k], cc[o + k], s1);
                }
                sAB[r * kMS + j0 + o] = s2;
                sCh[r * kMS + j0 + o] = s1;
            }
        }
    }
    else
    for (int item = threadIdx.x; item < kRH * (kLTW / kRun); item += NT) {
        const int r = item / (kLTW / kRun), j0 = (item % (kLTW / kRun)) * kRun;
        // streamed over the staged columns as in pass 1
        float2 s2[kRun];
        float s1[kRun];
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
            s2[o] = make_float2(0.f, 0.f);
            s1[o] = 0.f;
        }
        const float4 *pa4 = reinterpret_cast<const float4 *>(sM + r * kRP + j0);
        const float4 *pb4 = reinterpret_cast<const float4 *>(sM + kPlane + r * kRP + j0);
        const float4 *pc4 = reinterpret_cast<const float4 *>(sM + 2 * kPlane + r * kRP + j0);
#pragma unroll
        for (int m4 = 0; m4 < 5; ++m4) {
            const float4 a = pa4[m4], b = pb4[m4], c4 = pc4[m4];
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w}, cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * m4 + i - kRC;
                if (k < 0 || k >= kRun + 10) continue;
                const float2 ab = make_float2(av[i], bv[i]);
#pragma unroll
                for (int o = 0; o < kRun; ++o) {
                    if (k - o < 0 || k - o > 10) continue;
                    s2[o] = __ffma2_rn(f2w(win.w[k - o]), ab, s2[o]);
                    s1[o] = __fmaf_rn(win.w[k - o], cv[i], s1[o]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
            sAB[r * kMS + j0 + o] = s2[o];
            sCh[r * kMS + j0 + o] = s1[o];
        }
    }
    __syncthreads();
    for (int vt = threadIdx.x; vt < kLTW * (kLTH / kRun); vt += NT) {
        const int tx = vt % kLTW, i0 = (vt / kLTW) * kRun;
        // this thread's rendered and target values, in flight during the blur
        if constexpr (!kEarly) {
#pragma unroll
            for (int o = 0; o < kRun; ++o) {
                const int gx = ox + tx, gy = oy + i0 + o;
                const bool in = gx < W && gy < H;
                const int64_t idx = cb + (int64_t)(in ? gy : 0) * W + (in ? gx : 0);
                xs[o] = x[idx];
                ys[o] = y[idx];
            }
        }
        float2 gab[kRun];
        float gc[kRun];
        {
            float2 cab[kRun + 10];
            float ccc[kRun + 10];
#pragma unroll
            for (int k = 0; k < kRun + 10; ++k) {
                cab[k] = sAB[(i0 + k) * kMS + tx];
                ccc[k] = sCh[(i0 + k) * kMS + tx];
            }
#pragma unroll
            for (int o = 0; o < kRun; ++o) {
                float2 s2 = make_float2(0.f, 0.f);
                float s1 = 0.f;
#pragma unroll
                for (int k = 0; k < 11; ++k) {
                    s2 = __ffma2_rn(f2w(win.w[k]), cab[o + k], s2);
                    s1 = __fmaf_rn(win.w[k], ccc[o + k], s1);
                }
                gab[o] = s2;
                gc[o] = s1;
            }
        }
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
            const int gx = ox + tx, gy = oy + i0 + o;
            if (gx < W && gy < H) {
                const int64_t idx = cb + (int64_t)gy * W + gx;
                const float xv = xs[o], yv = ys[o];
                const float d = xv - yv;
                const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                dx_out[idx] = ((1.f - lambda) * sg - lambda * (gab[o].x + 2.f * xv * gab[o].y + yv * gc[o])) * inv_n;
            }
        }
    }
}

// Loss of one image from its per-block partial sums, folded in a fixed order
// by one block of NT threads (s_dbl: 2 NT doubles).
template <int NT>
__device__ __forceinline__ float loss_from_partials(const float *__restrict__ partials, int64_t npartials,
                                                    double count, float lambda, double *s_dbl) {
    double *s_l1 = s_dbl, *s_ss = s_dbl + NT;
    const int t = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (int64_t k = t; k < npartials; k += NT) {
        a += (double)partials[2 * k];
        b += (double)partials[2 * k + 1];
    }
    __syncthreads();
    s_l1[t] = a;
    s_ss[t] = b;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (t < o) {
            s_l1[t] += s_l1[t + o];
            s_ss[t] += s_ss[t + o];
        }
        __syncthreads();
    }
    const float L = (float)((1.0 - lambda) * s_l1[0] / count + lambda * (1.0 - s_ss[0] / count));
    __syncthreads();
    return L;
}

}  // namespace gsr
