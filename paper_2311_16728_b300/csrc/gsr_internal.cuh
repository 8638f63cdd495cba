// gsr_internal.cuh -- device helpers shared by the libgsr kernels (sm_103a).
//
// Holds the FP32 decision chain (cull, depth, 3-sigma radius, pixel box) of
// the EWA projection cited by Eq. 3 of Photo-SLAM (arXiv 2311.16728,
// Sec. 3.3), the real SH basis used for the colour c_i of Eq. 3 (SH in R^16
// per channel, Sec. 3.1) and the per-pixel alpha of Eq. 3.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsr.h"

namespace gsr {

// ---------------------------------------------------------------- host side
void set_error(const char *fmt, ...);
int32_t check_launch(const char *what);  // GSR_OK or GSR_ERR_CUDA (+ message)
inline cudaStream_t as_cuda(gsr_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }
inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
int32_t validate_gaussians(const gsr_gaussians *g);
int32_t validate_camera(const gsr_camera *c);
int32_t validate_tiling(const gsr_tiling *t);
inline int grid_x(const gsr_camera *c, const gsr_tiling *t) { return (c->width + t->tile_w - 1) / t->tile_w; }
inline int grid_y(const gsr_camera *c, const gsr_tiling *t) { return (c->height + t->tile_h - 1) / t->tile_h; }

// ---------------------------------------------------------------- chained launches
// The kernels of one mapping iteration run back to back on one stream.  A
// kernel launched by launch_chained may be scheduled while the kernel before
// it in the stream is still finishing (programmatic dependent launch): its
// CTAs take SM slots that the predecessor's last wave leaves free and get
// through their launch before the predecessor has ended.  Every such kernel
// calls chain_enter() first, before it touches global memory:
// griddepcontrol.wait returns once every grid it depends on has completed
// and its memory operations are visible (at once when the kernel was
// launched without the attribute, or after a non-kernel node), so what the
// kernel computes is what a plainly serialised launch computes.  chain_enter
// then lets the next chained kernel be scheduled (griddepcontrol.
// launch_dependents); that kernel in turn waits for this one to complete.
__device__ __forceinline__ void chain_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... P, typename... A>
inline cudaError_t launch_chained(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                  A &&...args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// status bit set by kernels in the caller's device status word
__device__ __forceinline__ void raise_status(int32_t *d_status, int code) {
    if (d_status) atomicOr(d_status, 1 << code);
}

// Counting-sort bases of NB classes ordered from the last class down: c[b]
// <- sum of c[b'] over b' > b, by the first warp of the block (the other
// threads return at once; the caller synchronises afterwards).
template <int NB>
__device__ __forceinline__ void desc_class_bases(uint32_t *c) {
    if (threadIdx.x >= 32) return;
    constexpr int K = (NB + 31) / 32;
    const int lane = (int)threadIdx.x;
    uint32_t v[K], sum = 0u;
#pragma unroll
    for (int k = 0; k < K; ++k) {  // lane l takes the classes NB - 1 - (l K + k)
        const int r = lane * K + k;
        v[k] = r < NB ? c[NB - 1 - r] : 0u;
        sum += v[k];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    uint32_t run = inc - sum;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int r = lane * K + k;
        if (r < NB) c[NB - 1 - r] = run;
        run += v[k];
    }
}

// ---------------------------------------------------------------- constants
constexpr float kNear = 0.2f;        // near plane (reading; the paper names none)
constexpr float kAlphaMax = 0.99f;   // alpha clamp
constexpr float kAlphaMin = 1.0f / 255.0f;  // alpha skip threshold
constexpr float kTMin = 1e-4f;       // stop before T drops below this
constexpr int kShPlanes = 12;        // 48 SH floats as 12 float4 planes

// Views of a batched call: records of view v are [v n_per_view, (v + 1)
// n_per_view); its tiles are numbered from toff[v] (row-major, gx[v] wide).
constexpr int kMaxViews = 64;
struct ViewTiles {
    int nviews;
    int64_t n_per_view;
    int gx[kMaxViews];
    uint32_t toff[kMaxViews];
};

// Camera as a kernel argument (by value).
struct CamK {
    float R[9], t[3];
    float fx, fy, cx, cy;
    int W, H;
    int tw, th, gx, gy;
};

inline CamK make_camk(const gsr_camera *c, const gsr_tiling *t) {
    CamK k;
    for (int i = 0; i < 9; ++i) k.R[i] = c->R[i];
    for (int i = 0; i < 3; ++i) k.t[i] = c->t[i];
    k.fx = c->fx; k.fy = c->fy; k.cx = c->cx; k.cy = c->cy;
    k.W = c->width; k.H = c->height;
    k.tw = t ? t->tile_w : 16; k.th = t ? t->tile_h : 16;
    k.gx = (k.W + k.tw - 1) / k.tw; k.gy = (k.H + k.th - 1) / k.th;
    return k;
}

// ---------------------------------------------------------------- FP32 chain
// Every step is one correctly rounded binary32 operation (explicit _rn
// intrinsics keep nvcc from contracting into FMAs); the order is part of the
// definition so that tile keys are reproducible bit for bit.
#define FM(a, b) __fmul_rn((a), (b))
#define FA(a, b) __fadd_rn((a), (b))
#define FS(a, b) __fsub_rn((a), (b))
#define FD(a, b) __fdiv_rn((a), (b))

// exp for the chain: Cody-Waite reduction x = k ln2 + r (ln2 split in a
// 9-trailing-zero high part and a low part), then the degree-7 Taylor
// polynomial of e^r in Horner form, scaled by the exact power of two 2^k.
__device__ __forceinline__ float chain_exp(float x) {
    const float xc = fminf(fmaxf(x, -80.0f), 80.0f);
    const float k = rintf(FM(xc, 1.44269502f));
    float r = FS(xc, FM(k, 0.693145752f));
    r = FS(r, FM(k, 1.42860677e-06f));
    float p = 1.98412698e-04f;               // 1/7!
    p = FA(FM(p, r), 1.38888889e-03f);       // 1/6!
    p = FA(FM(p, r), 8.33333377e-03f);       // 1/5!
    p = FA(FM(p, r), 4.16666679e-02f);       // 1/4!
    p = FA(FM(p, r), 1.66666672e-01f);       // 1/3!
    p = FA(FM(p, r), 0.5f);
    p = FA(FM(p, r), 1.0f);
    p = FA(FM(p, r), 1.0f);
    return FM(p, __int_as_float(((int)k + 127) << 23));
}

// Outputs of the chain for one Gaussian.
struct Chain {
    float xc, yc, zc;        // camera-space mean
    float s[3];              // chain_exp(logscale)
    float qn[4], qnorm;      // normalised quaternion, |q|
    float Rq[9];             // rotation of qn
    float Sig[6];            // 3D covariance xx xy xz yy yz zz
    float txz, tyz;          // x/z, y/z (unclamped)
    float a, b, c, det;      // Sigma' (dilated) and its determinant
    float u, v;              // projected mean
    int radius;
    int x0, x1, y0, y1;      // inclusive clipped pixel box
};

// The view-independent part of the decision chain: scales, normalised
// quaternion, its rotation and the 3D covariance (false for a zero
// quaternion).
__device__ __forceinline__ bool chain_shape(const float4 q, const float4 ls, Chain &o) {
    o.s[0] = chain_exp(ls.x);
    o.s[1] = chain_exp(ls.y);
    o.s[2] = chain_exp(ls.z);
    const float nn = FA(FA(FA(FM(q.x, q.x), FM(q.y, q.y)), FM(q.z, q.z)), FM(q.w, q.w));
    if (!(nn > 0.0f)) return false;
    o.qnorm = __fsqrt_rn(nn);
    const float w = FD(q.x, o.qnorm), x = FD(q.y, o.qnorm), y = FD(q.z, o.qnorm), z = FD(q.w, o.qnorm);
    o.qn[0] = w; o.qn[1] = x; o.qn[2] = y; o.qn[3] = z;
    const float xx = FM(x, x), yy = FM(y, y), zz = FM(z, z);
    const float xy = FM(x, y), xz = FM(x, z), yz = FM(y, z);
    const float wx = FM(w, x), wy = FM(w, y), wz = FM(w, z);
    float *Rq = o.Rq;
    Rq[0] = FS(1.0f, FM(2.0f, FA(yy, zz)));
    Rq[1] = FM(2.0f, FS(xy, wz));
    Rq[2] = FM(2.0f, FA(xz, wy));
    Rq[3] = FM(2.0f, FA(xy, wz));
    Rq[4] = FS(1.0f, FM(2.0f, FA(xx, zz)));
    Rq[5] = FM(2.0f, FS(yz, wx));
    Rq[6] = FM(2.0f, FS(xz, wy));
    Rq[7] = FM(2.0f, FA(yz, wx));
    Rq[8] = FS(1.0f, FM(2.0f, FA(xx, yy)));
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        M[3 * i + 0] = FM(Rq[3 * i + 0], o.s[0]);
        M[3 * i + 1] = FM(Rq[3 * i + 1], o.s[1]);
        M[3 * i + 2] = FM(Rq[3 * i + 2], o.s[2]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            const float v = FA(FA(FM(M[3 * i], M[3 * j]), FM(M[3 * i + 1], M[3 * j + 1])), FM(M[3 * i + 2], M[3 * j + 2]));
            const int k = i == 0 ? j : (i == 1 ? 2 + j : 5);  // xx xy xz yy yz zz
            o.Sig[k] = v;
        }
    return true;
}

// Camera-space mean and near-plane test of the decision chain.
__device__ __forceinline__ bool chain_camera(const float4 mo, const CamK &cam, Chain &o) {
    const float *R = cam.R;
    o.xc = FA(FA(FA(FM(R[0], mo.x), FM(R[1], mo.y)), FM(R[2], mo.z)), cam.t[0]);
    o.yc = FA(FA(FA(FM(R[3], mo.x), FM(R[4], mo.y)), FM(R[5], mo.z)), cam.t[1]);
    o.zc = FA(FA(FA(FM(R[6], mo.x), FM(R[7], mo.y)), FM(R[8], mo.z)), cam.t[2]);
    return o.zc > kNear;
}

// The rest of the chain for one camera (intrinsics and image of `cam`), from
// the shape part and the camera-space mean already in o.
__device__ __forceinline__ bool chain_screen(const CamK &cam, Chain &o) {
    const float *R = cam.R;
    float S[9];
    S[0] = o.Sig[0]; S[1] = o.Sig[1]; S[2] = o.Sig[2];
    S[3] = o.Sig[1]; S[4] = o.Sig[3]; S[5] = o.Sig[4];
    S[6] = o.Sig[2]; S[7] = o.Sig[4]; S[8] = o.Sig[5];
    const float limx = FM(1.3f, FD(FM(0.5f, (float)cam.W), cam.fx));
    const float limy = FM(1.3f, FD(FM(0.5f, (float)cam.H), cam.fy));
    o.txz = FD(o.xc, o.zc);
    o.tyz = FD(o.yc, o.zc);
    const float qx = fminf(limx, fmaxf(-limx, o.txz));
    const float qy = fminf(limy, fmaxf(-limy, o.tyz));
    const float J00 = FD(cam.fx, o.zc), J02 = -FD(FM(cam.fx, qx), o.zc);
    const float J11 = FD(cam.fy, o.zc), J12 = -FD(FM(cam.fy, qy), o.zc);
    float T[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T[j] = FA(FM(J00, R[j]), FM(J02, R[6 + j]));
        T[3 + j] = FA(FM(J11, R[3 + j]), FM(J12, R[6 + j]));
    }
    float U[6];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            U[3 * i + j] = FA(FA(FM(T[3 * i], S[j]), FM(T[3 * i + 1], S[3 + j])), FM(T[3 * i + 2], S[6 + j]));
    o.a = FA(FA(FA(FM(U[0], T[0]), FM(U[1], T[1])), FM(U[2], T[2])), 0.3f);
    o.b = FA(FA(FM(U[0], T[3]), FM(U[1], T[4])), FM(U[2], T[5]));
    o.c = FA(FA(FA(FM(U[3], T[3]), FM(U[4], T[4])), FM(U[5], T[5])), 0.3f);
    o.det = FS(FM(o.a, o.c), FM(o.b, o.b));
    if (!(o.det > 0.0f)) return false;
    const float mid = FM(0.5f, FA(o.a, o.c));
    const float disc = fmaxf(0.1f, FS(FM(mid, mid), o.det));
    const float lam = FA(mid, __fsqrt_rn(disc));
    const float r = ceilf(FM(3.0f, __fsqrt_rn(lam)));
    o.u = FA(FM(cam.fx, o.txz), cam.cx);
    o.v = FA(FM(cam.fy, o.tyz), cam.cy);
    o.radius = (int)r;
    const float fx0 = ceilf(FS(o.u, r)), fx1 = floorf(FA(o.u, r));
    const float fy0 = ceilf(FS(o.v, r)), fy1 = floorf(FA(o.v, r));
    if (fx1 < 0.0f || fy1 < 0.0f || fx0 > (float)(cam.W - 1) || fy0 > (float)(cam.H - 1)) return false;
    o.x0 = fx0 < 0.0f ? 0 : (int)fx0;
    o.x1 = fx1 > (float)(cam.W - 1) ? cam.W - 1 : (int)fx1;
    o.y0 = fy0 < 0.0f ? 0 : (int)fy0;
    o.y1 = fy1 > (float)(cam.H - 1) ? cam.H - 1 : (int)fy1;
    return o.x0 <= o.x1 && o.y0 <= o.y1;
}

// The whole decision chain of one Gaussian in one view: camera-space mean,
// near plane, 3D covariance, EWA projection, 3-sigma radius, pixel box.
// Returns false when the Gaussian is culled (behind the near plane, zero
// quaternion, degenerate covariance or a box that misses the image).
__device__ __forceinline__ bool decide_chain(const float4 mo, const float4 q, const float4 ls, const CamK &cam,
                                             Chain &o) {
    if (!chain_camera(mo, cam, o)) return false;
    if (!chain_shape(q, ls, o)) return false;
    return chain_screen(cam, o);
}

// Conic (inverse of the dilated 2D covariance) and opacity in the chain's
// FP32: these feed the tile cull below and are the values the render uses.
__device__ __forceinline__ void chain_conic_opacity(const Chain &c, float logit, float &A, float &B, float &C,
                                                    float &op) {
    A = FD(c.c, c.det);
    B = -FD(c.b, c.det);
    C = FD(c.a, c.det);
    op = FD(1.0f, FA(1.0f, chain_exp(-logit)));
}

// The projected mean beyond FP32: the chain's u, v carry an error of about
// an ulp of u (~1e-4 pixel at u ~ 1000), which moves alpha by ~1e-4 relative
// for a splat a pixel wide.  The same projection, u = fx X / Z + cx with
// X = R mean + t from the FP32 inputs, is evaluated in double-float
// arithmetic (each value an unevaluated sum hi + lo of two floats, ~2^-44
// relative): products split exactly by FMA (TwoProduct), sums by Knuth's
// TwoSum, the division by one correction step, as in Dekker (1971).  The
// residuals against the chain's u, v let the blends evaluate alpha at the
// mean to ~1e-6 pixel; the chain keeps deciding boxes, keys and culling.
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e) {
    s = FA(a, b);
    const float bb = FS(s, a);
    e = FA(FS(a, FS(s, bb)), FS(b, bb));
}

// (hi, lo) += a b
__device__ __forceinline__ void df_add_prod(float &hi, float &lo, float a, float b) {
    const float p = FM(a, b), pe = __fmaf_rn(a, b, -p);
    float s, se;
    df_two_sum(hi, p, s, se);
    hi = s;
    lo = FA(lo, FA(se, pe));
}

// R[3 r .. 3 r + 2] . mean + t[r] as hi + lo
__device__ __forceinline__ void df_row(const float *R, float t, const float4 mo, float &hi, float &lo) {
    hi = t;
    lo = 0.0f;
    df_add_prod(hi, lo, R[0], mo.x);
    df_add_prod(hi, lo, R[1], mo.y);
    df_add_prod(hi, lo, R[2], mo.z);
    const float s = FA(hi, lo);  // renormalise
    lo = FS(lo, FS(s, hi));
    hi = s;
}

// residual of f (X / Z) + c against the FP32 value w (near it)
__device__ __forceinline__ float df_screen_residual(float f, float c, float xh, float xl, float zh, float zl,
                                                    float w) {
    const float q1 = FD(xh, zh);
    const float p = FM(q1, zh), pe = __fmaf_rn(q1, zh, -p);
    const float r = FA(FS(FS(xh, p), pe), FS(xl, FM(q1, zl)));  // X - q1 Z
    const float q2 = FD(r, zh);                                 // X / Z = q1 + q2
    const float m = FM(f, q1), me = __fmaf_rn(f, q1, -m);
    float s, se;
    df_two_sum(m, c, s, se);
    return FA(FS(s, w), FA(FA(se, me), FM(f, q2)));
}

__device__ __forceinline__ float2 uv_residual(const float4 mo, const CamK &cam, float u, float v) {
    float xh, xl, yh, yl, zh, zl;
    df_row(cam.R, cam.t[0], mo, xh, xl);
    df_row(cam.R + 3, cam.t[1], mo, yh, yl);
    df_row(cam.R + 6, cam.t[2], mo, zh, zl);
    return make_float2(df_screen_residual(cam.fx, cam.cx, xh, xl, zh, zl, u),
                       df_screen_residual(cam.fy, cam.cy, yh, yl, zh, zl, v));
}

// Tile cull.  A (Gaussian, tile) pair is kept when opacity exp(-q_min / 2)
// >= 0.5 / 255, q_min being the continuous minimum of d^T Sigma'^-1 d over
// R = tile x pixel box: 0 when the mean lies in R, else the least over the
// edges of R that face the mean (the vertical one on the mean's side when u
// is outside [x0, x1], the horizontal one when v is outside [y0, y1]; a ray
// from the mean to any other boundary point enters R through one of them
// first, and the form grows along the ray), each minimised at its clamped 1D
// vertex.  A dropped pair has alpha < 1/255 at every pixel by a factor-two
// margin, so the per-pixel skip would drop it anyway: the image does not
// depend on this cull or on the tiling.
constexpr float kTileAlphaMin = 0x1.010102p-9f;  // 0.5 / 255 in binary32

__device__ __forceinline__ float qform32(float A, float B, float C, float dx, float dy) {
    return FA(FA(FM(FM(A, dx), dx), FM(FM(FM(2.0f, B), dx), dy)), FM(FM(C, dy), dy));
}

__device__ __forceinline__ bool tile_keep(float u, float v, float A, float B, float C, float op, float x0, float x1,
                                          float y0, float y1) {
    // both edges on every lane, no divergent branch: the lanes of a warp
    // test different tiles and Gaussians; edges that do not face the mean
    // (and the mean inside) are selected away
    const bool out_x = u < x0 || u > x1, out_y = v < y0 || v > y1;
    const float dx = FS(u < x0 ? x0 : x1, u);
    const float ys = fminf(fmaxf(FS(v, FD(FM(B, dx), C)), y0), y1);
    const float qx = qform32(A, B, C, dx, FS(ys, v));
    const float dy = FS(v < y0 ? y0 : y1, v);
    const float xs = fminf(fmaxf(FS(u, FD(FM(B, dy), A)), x0), x1);
    const float qy = qform32(A, B, C, FS(xs, u), dy);
    float q = out_x ? qx : __int_as_float(0x7f800000);
    q = out_y ? fminf(q, qy) : q;
    q = (u >= x0 && u <= x1 && v >= y0 && v <= y1) ? 0.0f : q;
    return FM(op, chain_exp(FM(-0.5f, q))) >= kTileAlphaMin;
}

// Tile (tx, ty) of a Gaussian with pixel box [x0, x1] x [y0, y1]: keep?
__device__ __forceinline__ bool tile_keep_at(int tx, int ty, int tw, int th, float u, float v, float A, float B,
                                             float C, float op, int x0, int x1, int y0, int y1) {
    const int rx0 = max(tx * tw, x0), rx1 = min(tx * tw + tw - 1, x1);
    const int ry0 = max(ty * th, y0), ry1 = min(ty * th + th - 1, y1);
    return tile_keep(u, v, A, B, C, op, (float)rx0, (float)rx1, (float)ry0, (float)ry1);
}

// Record of one projected Gaussian as the binning kernels read it back.
struct Splat {
    float u, v, A, B, C, op;
    int x0, x1, y0, y1;
};

__device__ __forceinline__ Splat load_splat(const float4 *xy_conic, const float4 *c_op_box, int64_t i) {
    const float4 a = xy_conic[i], b = c_op_box[i];
    const uint32_t bx = __float_as_uint(b.z), by = __float_as_uint(b.w);
    return Splat{a.x, a.y, a.z, a.w, b.x, b.y, (int)(bx & 0xffffu), (int)(bx >> 16), (int)(by & 0xffffu),
                 (int)(by >> 16)};
}

// Number of kept tiles of one Gaussian, computed by the whole warp (every
// lane passes the same splat; the result is returned to every lane).
__device__ __forceinline__ uint32_t warp_count_tiles(const Splat &s, int tw, int th) {
    const int tx0 = s.x0 / tw, ty0 = s.y0 / th;
    const int ntx = s.x1 / tw - tx0 + 1, total = ntx * (s.y1 / th - ty0 + 1);
    uint32_t c = 0;
    for (int k = (int)(threadIdx.x & 31); k < total; k += 32)
        c += tile_keep_at(tx0 + k % ntx, ty0 + k / ntx, tw, th, s.u, s.v, s.A, s.B, s.C, s.op, s.x0, s.x1, s.y0, s.y1)
                 ? 1u
                 : 0u;
    return __reduce_add_sync(0xffffffffu, c);
}

__device__ __forceinline__ Splat shfl_splat(const Splat &s, int src) {
    Splat o;
    o.u = __shfl_sync(0xffffffffu, s.u, src);
    o.v = __shfl_sync(0xffffffffu, s.v, src);
    o.A = __shfl_sync(0xffffffffu, s.A, src);
    o.B = __shfl_sync(0xffffffffu, s.B, src);
    o.C = __shfl_sync(0xffffffffu, s.C, src);
    o.op = __shfl_sync(0xffffffffu, s.op, src);
    o.x0 = __shfl_sync(0xffffffffu, s.x0, src);
    o.x1 = __shfl_sync(0xffffffffu, s.x1, src);
    o.y0 = __shfl_sync(0xffffffffu, s.y0, src);
    o.y1 = __shfl_sync(0xffffffffu, s.y1, src);
    return o;
}

constexpr int kSmallBoxTiles = 8;  // boxes with more tiles are counted / emitted by a whole warp

// ---------------------------------------------------------------- SH basis
// Real orthonormal SH with the Condon-Shortley phase, index l*l + l + m,
// written as the textbook polynomials in the unit direction (x, y, z).
namespace shc {
constexpr float Y00 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float C1 = 0.4886025119029199f;     // sqrt(3/(4 pi))
constexpr float C2a = 1.0925484305920792f;    // sqrt(15/pi)/2
constexpr float C2b = 0.31539156525252005f;   // sqrt(5/pi)/4
constexpr float C2c = 0.5462742152960396f;    // sqrt(15/pi)/4
constexpr float C3a = 0.5900435899266435f;    // sqrt(35/(2 pi))/4
constexpr float C3b = 2.890611442640554f;     // sqrt(105/pi)/2
constexpr float C3c = 0.4570457994644658f;    // sqrt(21/(2 pi))/4
constexpr float C3d = 0.3731763325901154f;    // sqrt(7/pi)/4
constexpr float C3e = 1.445305721320277f;     // sqrt(105/pi)/4
}  // namespace shc

// Y[16] at unit direction d; dY (optional) = gradient of the polynomial form.
__device__ __forceinline__ void sh_basis(float x, float y, float z, int deg, float Y[16], float3 *dY) {
    using namespace shc;
    Y[0] = Y00;
    if (dY) dY[0] = make_float3(0.f, 0.f, 0.f);
    if (deg < 1) return;
    Y[1] = -C1 * y; Y[2] = C1 * z; Y[3] = -C1 * x;
    if (dY) {
        dY[1] = make_float3(0.f, -C1, 0.f);
        dY[2] = make_float3(0.f, 0.f, C1);
        dY[3] = make_float3(-C1, 0.f, 0.f);
    }
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = C2a * x * y;
    Y[5] = -C2a * y * z;
    Y[6] = C2b * (3.f * zz - 1.f);
    Y[7] = -C2a * x * z;
    Y[8] = C2c * (xx - yy);
    if (dY) {
        dY[4] = make_float3(C2a * y, C2a * x, 0.f);
        dY[5] = make_float3(0.f, -C2a * z, -C2a * y);
        dY[6] = make_float3(0.f, 0.f, 6.f * C2b * z);
        dY[7] = make_float3(-C2a * z, 0.f, -C2a * x);
        dY[8] = make_float3(2.f * C2c * x, -2.f * C2c * y, 0.f);
    }
    if (deg < 3) return;
    Y[9] = -C3a * y * (3.f * xx - yy);
    Y[10] = C3b * x * y * z;
    Y[11] = -C3c * y * (5.f * zz - 1.f);
    Y[12] = C3d * z * (5.f * zz - 3.f);
    Y[13] = -C3c * x * (5.f * zz - 1.f);
    Y[14] = C3e * z * (xx - yy);
    Y[15] = -C3a * x * (xx - 3.f * yy);
    if (dY) {
        dY[9] = make_float3(-6.f * C3a * x * y, -C3a * (3.f * xx - 3.f * yy), 0.f);
        dY[10] = make_float3(C3b * y * z, C3b * x * z, C3b * x * y);
        dY[11] = make_float3(0.f, -C3c * (5.f * zz - 1.f), -10.f * C3c * y * z);
        dY[12] = make_float3(0.f, 0.f, C3d * (15.f * zz - 3.f));
        dY[13] = make_float3(-C3c * (5.f * zz - 1.f), 0.f, -10.f * C3c * x * z);
        dY[14] = make_float3(2.f * C3e * x * z, -2.f * C3e * y * z, C3e * (xx - yy));
        dY[15] = make_float3(-C3a * (3.f * xx - 3.f * yy), 6.f * C3a * x * y, 0.f);
    }
}

// Number of float4 SH planes that hold the first (deg+1)^2 coefficients x 3.
__host__ __device__ __forceinline__ int sh_planes(int deg) { return (3 * (deg + 1) * (deg + 1) + 3) / 4; }

// ---------------------------------------------------------------- alpha
// alpha of Eq. 3 at pixel offset d = (px - u, py - v) with conic (A, B, C):
// power = -(A dx^2 + C dy^2)/2 - B dx dy, G = exp(power), alpha = min(0.99,
// opacity G).  Written with explicit rounding so the forward and backward
// kernels take bit-identical skip / clamp / stop decisions.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float splat_power(float A, float B, float C, float dx, float dy) {
    const float q = FA(FM(FM(A, dx), dx), FM(FM(C, dy), dy));
    return FS(FM(-0.5f, q), FM(FM(B, dx), dy));
}

__device__ __forceinline__ float splat_gauss(float power) { return ex2_approx(FM(power, 1.4426950408889634f)); }

// pixel box packed as x0 | x1 << 16 (and y0 | y1 << 16)
__device__ __forceinline__ bool in_box(uint32_t bx, uint32_t by, int px, int py) {
    const int x0 = (int)(bx & 0xffffu), x1 = (int)(bx >> 16);
    const int y0 = (int)(by & 0xffffu), y1 = (int)(by >> 16);
    return px >= x0 && px <= x1 && py >= y0 && py <= y1;
}

}  // namespace gsr
