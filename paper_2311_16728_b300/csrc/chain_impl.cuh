// chain_impl.cuh -- parameter access and the per-Gaussian chain rule (K8)
// from screen-space gradients to the 59 parameters, for the EWA splatting
// cited by Eq. 3 of Photo-SLAM (arXiv 2311.16728, Sec. 3.3); shared by the
// one-view kernels (preprocess.cu) and the multi-view ones (batched.cu).
#pragma once

#include "gsr_internal.cuh"

namespace gsr {

struct GaussK {
    const float4 *mean_op, *quat, *logscale, *sh;
    int64_t n;
    int deg;
};

inline GaussK make_gk(const gsr_gaussians *g) {
    return GaussK{reinterpret_cast<const float4 *>(g->mean_op), reinterpret_cast<const float4 *>(g->quat),
                  reinterpret_cast<const float4 *>(g->logscale), reinterpret_cast<const float4 *>(g->sh), g->n,
                  g->sh_degree};
}

// camera centre C = -R^T t
__device__ __forceinline__ float3 cam_center(const CamK &cam) {
    const float *R = cam.R, *t = cam.t;
    return make_float3(-(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]), -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]),
                       -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2]));
}

__device__ __forceinline__ void load_sh(const float4 *__restrict__ sh, int64_t n, int64_t i, int deg, float out[48]) {
    const int planes = sh_planes(deg);
#pragma unroll
    for (int j = 0; j < kShPlanes; ++j) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < planes) v = __ldg(sh + (int64_t)j * n + i);
        out[4 * j + 0] = v.x;
        out[4 * j + 1] = v.y;
        out[4 * j + 2] = v.z;
        out[4 * j + 3] = v.w;
    }
}

// K8: screen-space gradients (du, dv, dA, dB, dC, dopacity, dr, dg, db) of one
// Gaussian -> dL/d(mean, opacity logit, quaternion, log-scale, SH), added to
// the gradient planes.  Only visible Gaussians have work, and they are a
// small fraction of the map, so each CTA first compacts the visible indices
// of its chunk in shared memory and then runs the chain on full warps.
constexpr int kBwdThreads = 128;
constexpr int kBwdChunk = 1024;  // Gaussians per CTA

// The CTA's chunk is kBwdChunk / kBwdThreads runs of kBwdThreads consecutive
// Gaussians, run j starting at Gaussian (j * gridDim.x + blockIdx.x) *
// kBwdThreads: every CTA samples the whole index range, so the visible
// Gaussians spread over the CTAs even when the store is in a spatial order
// (they are then contiguous, and whole chunks would be visible or not, with
// the grid a single wave).  Slot k of the chunk is Gaussian chunk_index(k).
__device__ __forceinline__ int64_t chunk_index(uint32_t k) {
    return ((int64_t)(k / kBwdThreads) * gridDim.x + blockIdx.x) * kBwdThreads + (k % kBwdThreads);
}

// Slots k (0 .. kBwdChunk-1) of the visible Gaussians of this CTA's chunk
// into s_idx[0 .. *s_cnt - 1] (s_cnt zero on entry; a barrier must follow).
// Every visibility word is loaded before the first ballot, so the chunk costs
// one memory round trip, not one per iteration.
__device__ __forceinline__ void compact_visible(const uint32_t *__restrict__ ntiles, int64_t n, uint32_t *s_idx,
                                                uint32_t *s_cnt) {
    constexpr int kIt = kBwdChunk / kBwdThreads;
    const int lane = threadIdx.x & 31;
    uint32_t nt[kIt];
#pragma unroll
    for (int j = 0; j < kIt; ++j) {
        const int64_t i = chunk_index((uint32_t)(j * kBwdThreads) + threadIdx.x);
        nt[j] = i < n ? __ldg(ntiles + i) : 0u;
    }
#pragma unroll
    for (int j = 0; j < kIt; ++j) {
        const bool vis = nt[j] > 0u;
        const uint32_t m = __ballot_sync(0xffffffffu, vis);
        uint32_t slot = 0;
        if (lane == 0 && m) slot = atomicAdd(s_cnt, (uint32_t)__popc(m));
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (vis) s_idx[slot + __popc(m & ((1u << lane) - 1u))] = (uint32_t)(j * kBwdThreads + (int)threadIdx.x);
    }
}

// Screen-space gradient of one Gaussian in one view, with the conic part
// already taken to the dilated 2D covariance: Gs = dL/dSigma' (symmetric).
struct ScreenGrad {
    float du, dv, Gs00, Gs01, Gs11, dop, dr, dg, db;
};

// conic Q = Sigma'^-1 = [[A, B], [B, C]] and G_Q = [[dA, dB/2], [dB/2, dC]]
// -> G_Sigma' = -Q G_Q Q
__device__ __forceinline__ void conic_grad_to_cov(float A, float B, float C, float dA, float dB, float dC, float &Gs00,
                                                  float &Gs01, float &Gs11) {
    const float hB = 0.5f * dB;
    const float t00 = A * dA + B * hB, t01 = A * hB + B * dC;
    const float t10 = B * dA + C * hB, t11 = B * hB + C * dC;
    Gs00 = -(t00 * A + t01 * B);
    Gs11 = -(t10 * B + t11 * C);
    Gs01 = -0.5f * ((t00 * B + t01 * C) + (t10 * A + t11 * B));
}

__device__ __forceinline__ void add4(float4 *p, float4 v, bool atomic) {
    if (atomic) {
        atomicAdd(p, v);  // 128-bit global float atomic (sm_90 and later)
    } else {
        const float4 a = *p;
        *p = make_float4(a.x + v.x, a.y + v.y, a.z + v.z, a.w + v.w);
    }
}

// Number of camera pose gradient values: dL/dR (9, row-major, R taken as a
// general 3 x 3 matrix), dL/dt (3), dL/dphi (3) for the left perturbation
// R <- exp([phi]x) R, t <- exp([phi]x) t (a rotation about the camera centre).
constexpr int kPoseGrad = 15;

// Chain rule of one Gaussian from its screen-space gradient in camera `cam`
// (c = the forward chain of that camera) to the 59 parameters.  Each plane's
// gradient goes to sink(plane, value): planes 3 .. 3 + sh_planes - 1 (SH) as
// soon as that SH plane has been read, then 0 (mean, opacity logit), 1
// (quaternion), 2 (log-scale).  kPose: this Gaussian's part of the camera pose
// gradient is added to pose[kPoseGrad].  shp (may be NULL): the Gaussian's SH
// planes already in registers (load_sh_planes), else they are read here.
template <class Sink, bool kPose = false>
__device__ __forceinline__ void chain_core_to(const GaussK &g, const CamK &cam, int64_t i, const float4 mo,
                                              const Chain &c, const ScreenGrad &sg, Sink &sink,
                                              float *pose = nullptr, const float4 *shp = nullptr) {
    const float du = sg.du, dv = sg.dv, dop = sg.dop;
    const float *W = cam.R;
    // ---- colour and SH, streamed one float4 plane at a time
    const float3 cc = cam_center(cam);
    const float dirx = mo.x - cc.x, diry = mo.y - cc.y, dirz = mo.z - cc.z;
    const float inv_len = 1.0f / sqrtf(dirx * dirx + diry * diry + dirz * dirz);
    const float vx = dirx * inv_len, vy = diry * inv_len, vz = dirz * inv_len;
    float Y[16];
    float3 dY[16];
    sh_basis(vx, vy, vz, g.deg, Y, dY);
    const int nc = (g.deg + 1) * (g.deg + 1);
    const int planes = sh_planes(g.deg);
    // raw colour decides the clamp: first pass over the planes
    float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int j = 0; j < kShPlanes; ++j) {
        if (j >= planes) break;
        const float4 v = shp ? shp[j] : __ldg(g.sh + (int64_t)j * g.n + i);
        const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int f = 4 * j + t, k = f / 3, ch = f % 3;
            if (k < nc) raw[ch] += e[t] * Y[k];
        }
    }
    const float dcol[3] = {raw[0] > 0.0f ? sg.dr : 0.0f, raw[1] > 0.0f ? sg.dg : 0.0f, raw[2] > 0.0f ? sg.db : 0.0f};
    float3 dvh = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < kShPlanes; ++j) {
        if (j >= planes) break;
        const float4 v = shp ? shp[j] : __ldg(g.sh + (int64_t)j * g.n + i);
        const float e[4] = {v.x, v.y, v.z, v.w};
        float d[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int f = 4 * j + t, k = f / 3, ch = f % 3;
            d[t] = 0.0f;
            if (k < nc) {
                d[t] = dcol[ch] * Y[k];
                const float w = dcol[ch] * e[t];
                dvh.x += w * dY[k].x;
                dvh.y += w * dY[k].y;
                dvh.z += w * dY[k].z;
            }
        }
        sink(3 + j, make_float4(d[0], d[1], d[2], d[3]));
    }
    const float vd = dvh.x * vx + dvh.y * vy + dvh.z * vz;
    // dL/d(mean - camera centre) through the view direction
    const float ddx = (dvh.x - vx * vd) * inv_len, ddy = (dvh.y - vy * vd) * inv_len,
                ddz = (dvh.z - vz * vd) * inv_len;
    float dmx = ddx, dmy = ddy, dmz = ddz;
    // ---- opacity (the same FP32 opacity the forward used)
    const float sig = FD(1.0f, FA(1.0f, chain_exp(-mo.w)));
    const float dlogit = dop * sig * (1.0f - sig);
    const float Gs00 = sg.Gs00, Gs01 = sg.Gs01, Gs11 = sg.Gs11;
    // ---- T = J W, J with the clamped x/z, y/z
    const float limx = 1.3f * (0.5f * (float)cam.W / cam.fx), limy = 1.3f * (0.5f * (float)cam.H / cam.fy);
    const bool clx = c.txz < -limx || c.txz > limx, cly = c.tyz < -limy || c.tyz > limy;
    const float qx = fminf(limx, fmaxf(-limx, c.txz)), qy = fminf(limy, fmaxf(-limy, c.tyz));
    const float iz = 1.0f / c.zc, iz2 = iz * iz;
    const float J00 = cam.fx * iz, J02 = -cam.fx * qx * iz, J11 = cam.fy * iz, J12 = -cam.fy * qy * iz;
    float T[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T[j] = J00 * W[j] + J02 * W[6 + j];
        T[3 + j] = J11 * W[3 + j] + J12 * W[6 + j];
    }
    const float S[9] = {c.Sig[0], c.Sig[1], c.Sig[2], c.Sig[1], c.Sig[3], c.Sig[4], c.Sig[2], c.Sig[4], c.Sig[5]};
    const float Gs[4] = {Gs00, Gs01, Gs01, Gs11};
    // G_Sig = T^T G_S' T
    float GS[9];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
            GS[3 * k + l] = T[k] * (Gs[0] * T[l] + Gs[1] * T[3 + l]) + T[3 + k] * (Gs[2] * T[l] + Gs[3] * T[3 + l]);
    // G_T = 2 G_S' T Sig
    float TS[6];
#pragma unroll
    for (int i2 = 0; i2 < 2; ++i2)
#pragma unroll
        for (int l = 0; l < 3; ++l)
            TS[3 * i2 + l] = T[3 * i2] * S[l] + T[3 * i2 + 1] * S[3 + l] + T[3 * i2 + 2] * S[6 + l];
    float GT[6];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        GT[l] = 2.0f * (Gs[0] * TS[l] + Gs[1] * TS[3 + l]);
        GT[3 + l] = 2.0f * (Gs[2] * TS[l] + Gs[3] * TS[3 + l]);
    }
    // G_J = G_T W^T (entries 00, 02, 11, 12 are the only live ones of J)
    const float GJ00 = GT[0] * W[0] + GT[1] * W[1] + GT[2] * W[2];
    const float GJ02 = GT[0] * W[6] + GT[1] * W[7] + GT[2] * W[8];
    const float GJ11 = GT[3] * W[3] + GT[4] * W[4] + GT[5] * W[5];
    const float GJ12 = GT[3] * W[6] + GT[4] * W[7] + GT[5] * W[8];
    const float X = c.xc, Yc = c.yc;
    float dpx = 0.f, dpy = 0.f, dpz = 0.f;
    dpz += -(GJ00 * cam.fx + GJ11 * cam.fy) * iz2;
    // J02 = -fx qx / z with qx = clamp(x / z)
    if (!clx) {
        dpx += -GJ02 * cam.fx * iz2;
        dpz += GJ02 * cam.fx * (qx * iz2 + X * iz2 * iz);
    } else {
        dpz += GJ02 * cam.fx * qx * iz2;
    }
    if (!cly) {
        dpy += -GJ12 * cam.fy * iz2;
        dpz += GJ12 * cam.fy * (qy * iz2 + Yc * iz2 * iz);
    } else {
        dpz += GJ12 * cam.fy * qy * iz2;
    }
    // u = fx x / z + cx, v = fy y / z + cy
    dpx += du * cam.fx * iz;
    dpy += dv * cam.fy * iz;
    dpz += -(du * cam.fx * X + dv * cam.fy * Yc) * iz2;
    dmx += W[0] * dpx + W[3] * dpy + W[6] * dpz;
    dmy += W[1] * dpx + W[4] * dpy + W[7] * dpz;
    dmz += W[2] * dpx + W[5] * dpy + W[8] * dpz;
    if constexpr (kPose) {
        // the pose enters through p = W mean + t, through T = J W
        // (G_W = J^T G_T) and through the camera centre -W^T t of the view
        // direction; under the left rotation dp = phi x p, dW = [phi]x W and
        // the centre stays: <G_W, [phi]x W> = phi . (N21 - N12, N02 - N20,
        // N10 - N01) with N = G_W W^T
        float GW[9];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            GW[b] = J00 * GT[b];
            GW[3 + b] = J11 * GT[3 + b];
            GW[6 + b] = J02 * GT[b] + J12 * GT[3 + b];
        }
        const float mu[3] = {mo.x, mo.y, mo.z}, dp[3] = {dpx, dpy, dpz}, dd[3] = {ddx, ddy, ddz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) pose[3 * a + b] += dp[a] * mu[b] + GW[3 * a + b] + dd[b] * cam.t[a];
            pose[9 + a] += dp[a] + W[3 * a] * dd[0] + W[3 * a + 1] * dd[1] + W[3 * a + 2] * dd[2];
        }
        float N[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                N[3 * a + b] = GW[3 * a] * W[3 * b] + GW[3 * a + 1] * W[3 * b + 1] + GW[3 * a + 2] * W[3 * b + 2];
        pose[12] += Yc * dpz - c.zc * dpy + N[7] - N[5];
        pose[13] += c.zc * dpx - X * dpz + N[2] - N[6];
        pose[14] += X * dpy - Yc * dpx + N[3] - N[1];
    }
    // ---- Sig = M M^T, M = Rq diag(s):  G_M = 2 G_Sig M
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * r + j] = c.Rq[3 * r + j] * c.s[j];
    float GR[9], dls[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float ds = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float gm = 2.0f * (GS[3 * r] * M[j] + GS[3 * r + 1] * M[3 + j] + GS[3 * r + 2] * M[6 + j]);
            ds += gm * c.Rq[3 * r + j];
            GR[3 * r + j] = gm * c.s[j];
        }
        dls[j] = ds * c.s[j];
    }
    // rotation entries -> normalised quaternion (w, x, y, z)
    const float w = c.qn[0], x = c.qn[1], y = c.qn[2], z = c.qn[3];
    float dw = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
    float dx2 = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] -
                       2.f * x * GR[8]);
    float dy2 = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] -
                       2.f * y * GR[8]);
    float dz2 = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] +
                       x * GR[6] + y * GR[7]);
    const float qd = dw * w + dx2 * x + dy2 * y + dz2 * z;
    const float iq = 1.0f / c.qnorm;
    dw = (dw - w * qd) * iq;
    dx2 = (dx2 - x * qd) * iq;
    dy2 = (dy2 - y * qd) * iq;
    dz2 = (dz2 - z * qd) * iq;
    sink(0, make_float4(dmx, dmy, dmz, dlogit));
    sink(1, make_float4(dw, dx2, dy2, dz2));
    sink(2, make_float4(dls[0], dls[1], dls[2], 0.0f));
}

// sink that adds into the gradient planes (atomically when several threads
// may add to the same Gaussian), or stores into them (store: the caller's
// gradients of this Gaussian are replaced)
struct AddSink {
    float4 *d_mo, *d_q, *d_ls, *d_sh;
    int64_t n, i;
    bool atomic, store;
    __device__ __forceinline__ void operator()(int plane, float4 v) const {
        float4 *p = plane == 0 ? d_mo + i : (plane == 1 ? d_q + i : (plane == 2 ? d_ls + i : d_sh + (int64_t)(plane - 3) * n + i));
        if (store) *p = v;
        else add4(p, v, atomic);
    }
};

// sink that discards the parameter gradients (pose-only passes)
struct NullSink {
    __device__ __forceinline__ void operator()(int, float4) const {}
};

__device__ __forceinline__ void chain_core(const GaussK &g, const CamK &cam, int64_t i, const float4 mo, const Chain &c,
                                           const ScreenGrad &sg, float4 *__restrict__ d_mo, float4 *__restrict__ d_q,
                                           float4 *__restrict__ d_ls, float4 *__restrict__ d_sh, bool atomic,
                                           const float4 *shp = nullptr) {
    AddSink sink{d_mo, d_q, d_ls, d_sh, g.n, i, atomic, false};
    chain_core_to(g, cam, i, mo, c, sg, sink, nullptr, shp);
}

// The SH planes of Gaussian i in registers (planes beyond the degree zero).
__device__ __forceinline__ void load_sh_planes(const GaussK &g, int64_t i, float4 shp[kShPlanes]) {
    const int planes = sh_planes(g.deg);
#pragma unroll
    for (int j = 0; j < kShPlanes; ++j)
        shp[j] = j < planes ? __ldg(g.sh + (int64_t)j * g.n + i) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// One view: the screen-space gradient of record i (g0, g1, g2) chained into
// the parameter gradients of Gaussian i (one thread per Gaussian).  Every
// input of the Gaussian is loaded first, so its loads share one memory round
// trip that overlaps the decision chain (these kernels run few warps per SM,
// each bound by the latency of its own chain).
__device__ __forceinline__ void chain_one_gaussian(const GaussK &g, const CamK &cam, int64_t i,
                                                   const float4 *__restrict__ g0, const float4 *__restrict__ g1,
                                                   const float4 *__restrict__ g2, float4 *__restrict__ d_mo,
                                                   float4 *__restrict__ d_q, float4 *__restrict__ d_ls,
                                                   float4 *__restrict__ d_sh, float *__restrict__ dstat,
                                                   float *__restrict__ dcount, bool store = false) {
    const float4 mo = __ldg(g.mean_op + i), q = __ldg(g.quat + i), ls = __ldg(g.logscale + i);
    const float4 G0 = g0[i], G1 = g1[i], G2 = g2[i];
    float4 shp[kShPlanes];
    load_sh_planes(g, i, shp);
    Chain c;
    if (!decide_chain(mo, q, ls, cam, c)) return;  // cannot happen for a visible Gaussian
    if (dstat) {  // |dL/d(u, v)| in normalised device coordinates
        const float gu = G0.x * (0.5f * (float)cam.W), gv = G0.y * (0.5f * (float)cam.H);
        dstat[i] += sqrtf(gu * gu + gv * gv);
        dcount[i] += 1.0f;
    }
    float A, B, C, sig;
    chain_conic_opacity(c, mo.w, A, B, C, sig);
    ScreenGrad sg;
    sg.du = G0.x;
    sg.dv = G0.y;
    conic_grad_to_cov(A, B, C, G0.z, G0.w, G1.x, sg.Gs00, sg.Gs01, sg.Gs11);
    sg.dop = G1.y;
    sg.dr = G1.z;
    sg.dg = G1.w;
    sg.db = G2.x;
    AddSink sink{d_mo, d_q, d_ls, d_sh, g.n, i, false, store};
    chain_core_to(g, cam, i, mo, c, sg, sink, nullptr, shp);
}

}  // namespace gsr
