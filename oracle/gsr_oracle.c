/*
 * gsr_oracle.c -- plain, slow FP64 CPU oracle for differentiable 3D-Gaussian
 * rasterisation as used by Photo-SLAM's photorealistic mapping.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: it exists so that tests, the smoke check and the CPU
 * baseline timer have an independent statement of what the CUDA path must
 * compute.  It shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * What it follows (Photo-SLAM, arXiv 2311.16728):
 *   - Sec. 3.1  hyper primitive = position P, rotation r, scaling s,
 *               density sigma, SH colour (16 coefficients per channel).
 *   - Sec. 3.3, Eq. 3  C(R,t) = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j)
 *               (the printed product index (1 - alpha_i) is a typo and is
 *               read as (1 - alpha_j)); alpha_i = sigma_i * G(R,t,P_i,r_i,s_i)
 *               with G the 3D-Gaussian splatting footprint it cites.
 *   - Sec. 3.3, Eq. 4  L = (1-lambda)|I_r - I_gt|_1 + lambda (1 - SSIM).
 *   - Sec. 3.4, Eq. 5  Gaussian pyramid levels GP^l(I_gt).
 *   - Sec. 4.1  lambda = 0.2, three pyramid levels.
 *   - Sec. 3.3.1  densification: split or clone primitives with large
 *               loss gradients, prune transparent ones (3DGS rules as the
 *               reading; thresholds are parameters).
 *   - Sec. 3.3.1  new primitives at keypoints (their default initial shape
 *               is a reading: 3-nearest-neighbour scale, identity rotation,
 *               opacity 0.1, DC colour of the keypoint pixel).
 * Where the paper is silent the readings are the ones listed in the design
 * notes: EWA splat with 0.3 px dilation, 3-sigma pixel-square footprint,
 * alpha clamp 0.99, skip below 1/255, stop before T(1-alpha) < 1e-4, near
 * plane z > 0.2, integer pixel centres, black background, colour clamp at 0.
 *
 * Precision: everything is FP64 except the "decision chain" (cull, depth,
 * 3-sigma radius, pixel box), which is a fixed sequence of IEEE FP32
 * operations so that tile keys are bit-identical with any implementation
 * that performs the same sequence.  This file must be compiled with
 * -ffp-contract=off and without -ffast-math.
 *
 * Parity unpinned: nothing here is unpinned; every function is checked by the
 * non-GPU tests against closed forms, library routines, brute force or
 * finite differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NO_CLAMP 1 /* drop the alpha <= 0.99 clamp            */
#define ORC_NO_SKIP 2  /* drop the alpha < 1/255 skip             */
#define ORC_NO_TERM 4  /* drop the T(1-alpha) < 1e-4 termination  */

#define ORC_ALPHA_MAX 0.99
#define ORC_ALPHA_MIN (1.0 / 255.0)
#define ORC_T_MIN 1e-4
#define ORC_DILATION 0.3
#define ORC_NEAR 0.2f

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Real spherical harmonics, degree <= 3, from the associated-Legendre        */
/* definition.  With z = cos(theta) and (x + i y) = sin(theta) e^{i phi} on   */
/* the unit sphere,                                                           */
/*   P_l^m(z) = (-1)^m (1 - z^2)^{m/2} d^m P_l / dz^m   (Condon-Shortley)     */
/*   Y_l^0    = K_l^0 P_l(z)                                                  */
/*   Y_l^{+m} = sqrt2 K_l^m (-1)^m (d^m P_l/dz^m)(z) Re[(x + i y)^m]          */
/*   Y_l^{-m} = sqrt2 K_l^m (-1)^m (d^m P_l/dz^m)(z) Im[(x + i y)^m]          */
/*   K_l^m    = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)                             */
/* i.e. Y_real = sqrt2 Re/Im of the complex Y_l^m.  Index = l*l + l + m.      */
/* The same polynomial form extends Y off the sphere; its gradient, projected */
/* onto the tangent plane, is the direction derivative used by the backward.  */
/* ------------------------------------------------------------------------- */

static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

/* coefficients c[0..3] of P_l(z) = sum_k c[k] z^k, Bonnet recurrence
 * (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1}. */
static void legendre_coeffs(int l, double c[4]) {
    double p0[4] = {1, 0, 0, 0}, p1[4] = {0, 1, 0, 0}, p2[4];
    if (l == 0) { memcpy(c, p0, sizeof p0); return; }
    for (int n = 1; n < l; ++n) {
        for (int k = 0; k < 4; ++k) {
            double zp = (k > 0) ? p1[k - 1] : 0.0;
            p2[k] = ((2 * n + 1) * zp - n * p0[k]) / (n + 1);
        }
        memcpy(p0, p1, sizeof p0);
        memcpy(p1, p2, sizeof p1);
    }
    memcpy(c, p1, sizeof p1);
}

/* value of the m-th derivative of a cubic polynomial with coefficients c */
static double poly_deriv(const double c[4], int m, double z) {
    double s = 0.0;
    for (int k = m; k < 4; ++k) {
        double f = factorial(k) / factorial(k - m);
        s += c[k] * f * pow(z, k - m);
    }
    return s;
}

/* (x + i y)^m, and its partial derivatives in x and y */
static void xiy_pow(double x, double y, int m, double *re, double *im) {
    double r = 1.0, i = 0.0;
    for (int k = 0; k < m; ++k) {
        double nr = r * x - i * y, ni = r * y + i * x;
        r = nr;
        i = ni;
    }
    *re = r;
    *im = i;
}

void orc_sh_basis(const double v[3], int degree, double *Y, double *dY) {
    const double x = v[0], y = v[1], z = v[2];
    for (int k = 0; k < 16; ++k) {
        Y[k] = 0.0;
        if (dY) dY[3 * k] = dY[3 * k + 1] = dY[3 * k + 2] = 0.0;
    }
    for (int l = 0; l <= degree; ++l) {
        double c[4];
        legendre_coeffs(l, c);
        for (int m = 0; m <= l; ++m) {
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
            double Q = poly_deriv(c, m, z);    /* d^m P_l / dz^m     */
            double Qz = poly_deriv(c, m + 1, z); /* its z-derivative  */
            double re, im, re1 = 0.0, im1 = 0.0;
            xiy_pow(x, y, m, &re, &im);
            if (m > 0) xiy_pow(x, y, m - 1, &re1, &im1);
            /* d/dx (x+iy)^m = m (x+iy)^{m-1};  d/dy (x+iy)^m = i m (x+iy)^{m-1} */
            double dre_dx = m * re1, dim_dx = m * im1;
            double dre_dy = -m * im1, dim_dy = m * re1;
            if (m == 0) {
                int idx = l * l + l;
                Y[idx] = K * Q;
                if (dY) { dY[3 * idx + 2] = K * Qz; }
            } else {
                double a = sqrt(2.0) * K * ((m & 1) ? -1.0 : 1.0);
                int ip = l * l + l + m, in = l * l + l - m;
                Y[ip] = a * Q * re;
                Y[in] = a * Q * im;
                if (dY) {
                    dY[3 * ip + 0] = a * Q * dre_dx;
                    dY[3 * ip + 1] = a * Q * dre_dy;
                    dY[3 * ip + 2] = a * Qz * re;
                    dY[3 * in + 0] = a * Q * dim_dx;
                    dY[3 * in + 1] = a * Q * dim_dy;
                    dY[3 * in + 2] = a * Qz * im;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* FP32 decision chain.  Every line below is one IEEE-754 binary32 operation, */
/* rounded to nearest even; the order of operations is part of the definition */
/* (tile keys and pixel boxes must be bit-identical across implementations).  */
/* exp() is a fixed Cody-Waite range reduction followed by a degree-7 Taylor  */
/* polynomial (Horner), so that no platform exp enters a key.                 */
/* ------------------------------------------------------------------------- */

float orc_chain_exp(float x) {
    float xc = fminf(fmaxf(x, -80.0f), 80.0f);
    float t = xc * 1.44269502f;            /* log2(e) rounded to binary32   */
    float k = rintf(t);
    float r = xc - k * 0.693145752f;       /* ln2 high part, 9 trailing 0s  */
    r = r - k * 1.42860677e-06f;           /* ln2 low part                  */
    float p = 1.98412698e-04f;             /* 1/7!                          */
    p = p * r + 1.38888889e-03f;           /* 1/6!                          */
    p = p * r + 8.33333377e-03f;           /* 1/5!                          */
    p = p * r + 4.16666679e-02f;           /* 1/4!                          */
    p = p * r + 1.66666672e-01f;           /* 1/3!                          */
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    return ldexpf(p, (int)k);
}

typedef struct {
    int visible;
    float depth;
    float u, v;
    int radius;
    int box[4];     /* x0, x1, y0, y1 inclusive, clipped to the image */
    float conic[3]; /* A, B, C of Sigma'^-1 in the chain's FP32        */
    float opacity;  /* sigmoid(logit) in the chain's FP32               */
} orc_decision;

/* cam layout (floats): R[9] row-major world->camera, t[3], fx, fy, cx, cy */
static orc_decision decide_one(const float *mo, const float *q, const float *ls, const float *cam,
                               int W, int H) {
    orc_decision d;
    memset(&d, 0, sizeof d);
    const float *R = cam, *t = cam + 9;
    const float fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    const float mx = mo[0], my = mo[1], mz = mo[2];
    float xc = ((R[0] * mx + R[1] * my) + R[2] * mz) + t[0];
    float yc = ((R[3] * mx + R[4] * my) + R[5] * mz) + t[1];
    float zc = ((R[6] * mx + R[7] * my) + R[8] * mz) + t[2];
    d.depth = zc;
    if (!(zc > ORC_NEAR)) return d;
    float s0 = orc_chain_exp(ls[0]), s1 = orc_chain_exp(ls[1]), s2 = orc_chain_exp(ls[2]);
    float nn = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    if (!(nn > 0.0f)) return d;
    float nrm = sqrtf(nn);
    float w = q[0] / nrm, x = q[1] / nrm, y = q[2] / nrm, z = q[3] / nrm;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float Rq[9];
    Rq[0] = 1.0f - 2.0f * (yy + zz);
    Rq[1] = 2.0f * (xy - wz);
    Rq[2] = 2.0f * (xz + wy);
    Rq[3] = 2.0f * (xy + wz);
    Rq[4] = 1.0f - 2.0f * (xx + zz);
    Rq[5] = 2.0f * (yz - wx);
    Rq[6] = 2.0f * (xz - wy);
    Rq[7] = 2.0f * (yz + wx);
    Rq[8] = 1.0f - 2.0f * (xx + yy);
    float M[9];
    for (int i = 0; i < 3; ++i) {
        M[3 * i + 0] = Rq[3 * i + 0] * s0;
        M[3 * i + 1] = Rq[3 * i + 1] * s1;
        M[3 * i + 2] = Rq[3 * i + 2] * s2;
    }
    float S[9];
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            float v = (M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1]) + M[3 * i + 2] * M[3 * j + 2];
            S[3 * i + j] = v;
            S[3 * j + i] = v;
        }
    float limx = 1.3f * ((0.5f * (float)W) / fx);
    float limy = 1.3f * ((0.5f * (float)H) / fy);
    float txz = xc / zc, tyz = yc / zc;
    float qx = fminf(limx, fmaxf(-limx, txz));
    float qy = fminf(limy, fmaxf(-limy, tyz));
    float J00 = fx / zc, J02 = -((fx * qx) / zc);
    float J11 = fy / zc, J12 = -((fy * qy) / zc);
    float T[6];
    for (int j = 0; j < 3; ++j) {
        T[j] = J00 * R[j] + J02 * R[6 + j];
        T[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
    }
    float U[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            U[3 * i + j] = (T[3 * i] * S[j] + T[3 * i + 1] * S[3 + j]) + T[3 * i + 2] * S[6 + j];
    float a = ((U[0] * T[0] + U[1] * T[1]) + U[2] * T[2]) + 0.3f;
    float b = (U[0] * T[3] + U[1] * T[4]) + U[2] * T[5];
    float c = ((U[3] * T[3] + U[4] * T[4]) + U[5] * T[5]) + 0.3f;
    float det = a * c - b * b;
    if (!(det > 0.0f)) return d;
    float mid = 0.5f * (a + c);
    float disc = fmaxf(0.1f, mid * mid - det);
    float lam = mid + sqrtf(disc);
    float r = ceilf(3.0f * sqrtf(lam));
    float u = fx * txz + cx;
    float v = fy * tyz + cy;
    float fx0 = ceilf(u - r), fx1 = floorf(u + r);
    float fy0 = ceilf(v - r), fy1 = floorf(v + r);
    d.u = u;
    d.v = v;
    d.radius = (int)r;
    if (fx1 < 0.0f || fy1 < 0.0f || fx0 > (float)(W - 1) || fy0 > (float)(H - 1)) return d;
    int x0 = fx0 < 0.0f ? 0 : (int)fx0;
    int x1 = fx1 > (float)(W - 1) ? W - 1 : (int)fx1;
    int y0 = fy0 < 0.0f ? 0 : (int)fy0;
    int y1 = fy1 > (float)(H - 1) ? H - 1 : (int)fy1;
    if (x0 > x1 || y0 > y1) return d;
    d.box[0] = x0;
    d.box[1] = x1;
    d.box[2] = y0;
    d.box[3] = y1;
    d.visible = 1;
    d.conic[0] = c / det;
    d.conic[1] = -(b / det);
    d.conic[2] = a / det;
    d.opacity = 1.0f / (1.0f + orc_chain_exp(-mo[3]));
    return d;
}

int orc_decide(int64_t n, const float *mean_op, const float *quat, const float *logscale,
               const float *cam, int W, int H, uint8_t *visible, float *depth, int32_t *box,
               float *uv, int32_t *radius, float *conic, float *opacity) {
    if (n < 0 || W <= 0 || H <= 0) return 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        orc_decision d = decide_one(mean_op + 4 * i, quat + 4 * i, logscale + 4 * i, cam, W, H);
        visible[i] = (uint8_t)d.visible;
        depth[i] = d.depth;
        for (int k = 0; k < 4; ++k) box[4 * i + k] = d.box[k];
        if (uv) { uv[2 * i] = d.u; uv[2 * i + 1] = d.v; }
        if (radius) radius[i] = d.radius;
        if (conic) for (int k = 0; k < 3; ++k) conic[3 * i + k] = d.conic[k];
        if (opacity) opacity[i] = d.opacity;
    }
    return 0;
}

/* Tile cull of the decision chain.  A (Gaussian, tile) pair is kept when the
 * Gaussian's largest alpha over the rectangle R = tile x pixel box, computed
 * from the continuous minimum q_min of d^T Sigma'^-1 d over R, reaches
 * half of the 1/255 skip threshold:  opacity exp(-q_min / 2) >= 0.5 / 255.
 * Pixels of a dropped pair would all have alpha < 1/255 by a factor-two
 * margin, so they are skipped by the per-pixel rule anyway: the image does
 * not change and stays independent of the tile shape.  q_min is 0 when the
 * projected mean lies in R, else the smallest value over the edges of R that
 * face the mean (one or two), each minimised in closed form (the 1D
 * quadratic's vertex, clamped). */
#define ORC_TILE_ALPHA_MIN 0x1.010102p-9f /* 0.5 / 255 in binary32 */

static float qform32(float A, float B, float C, float dx, float dy) {
    return ((A * dx) * dx + ((2.0f * B) * dx) * dy) + (C * dy) * dy;
}

static int tile_keep(float u, float v, const float *conic, float op, float x0, float x1, float y0,
                     float y1) {
    const float A = conic[0], B = conic[1], C = conic[2];
    float q;
    if (u >= x0 && u <= x1 && v >= y0 && v <= y1) {
        q = 0.0f;
    } else {
        /* The minimum lies on the edges that face the mean: a ray from the
           mean to any other boundary point enters the rectangle through one
           of them first, and the form grows along a ray from the mean.  So
           only the vertical edge on the mean's side (when u is outside
           [x0, x1]) and the horizontal edge on its side (when v is outside
           [y0, y1]) are evaluated. */
        q = INFINITY;
        if (u < x0 || u > x1) {
            const float dx = (u < x0 ? x0 : x1) - u;
            float ys = v - (B * dx) / C;
            ys = fminf(fmaxf(ys, y0), y1);
            const float dy = ys - v;
            q = qform32(A, B, C, dx, dy);
        }
        if (v < y0 || v > y1) {
            const float dy = (v < y0 ? y0 : y1) - v;
            float xs = u - (B * dy) / A;
            xs = fminf(fmaxf(xs, x0), x1);
            const float dx = xs - u;
            q = fminf(q, qform32(A, B, C, dx, dy));
        }
    }
    return op * orc_chain_exp(-0.5f * q) >= ORC_TILE_ALPHA_MIN;
}

int orc_tile_keep(float u, float v, const float *conic, float op, float x0, float x1, float y0, float y1) {
    return tile_keep(u, v, conic, op, x0, x1, y0, y1);
}

/* ------------------------------------------------------------------------- */
/* Tile keys: one (key, gid) pair per (visible Gaussian, tile of its pixel    */
/* box that survives the tile cull above); key = tile << 32 | bits(depth).    */
/* Sorted by (key, gid) and per-tile [begin, end) ranges; empty tiles [0, 0). */
/* ------------------------------------------------------------------------- */

typedef struct { uint64_t key; uint32_t val; } kv_t;

static int kv_cmp(const void *a, const void *b) {
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->val != y->val) return x->val < y->val ? -1 : 1;
    return 0;
}

static uint32_t float_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* keep[tile-in-box] decisions of Gaussian i, row-major over its box's tiles */
static int64_t gaussian_tiles(const int32_t *b, const float *uv, const float *conic, float op, int tw,
                              int th, int gx, uint32_t *tiles_out) {
    int64_t k = 0;
    for (int ty = b[2] / th; ty <= b[3] / th; ++ty)
        for (int tx = b[0] / tw; tx <= b[1] / tw; ++tx) {
            const int rx0 = tx * tw > b[0] ? tx * tw : b[0];
            const int rx1 = tx * tw + tw - 1 < b[1] ? tx * tw + tw - 1 : b[1];
            const int ry0 = ty * th > b[2] ? ty * th : b[2];
            const int ry1 = ty * th + th - 1 < b[3] ? ty * th + th - 1 : b[3];
            if (!tile_keep(uv[0], uv[1], conic, op, (float)rx0, (float)rx1, (float)ry0, (float)ry1)) continue;
            if (tiles_out) tiles_out[k] = (uint32_t)(ty * gx + tx);
            ++k;
        }
    return k;
}

int orc_keys(int64_t n, const uint8_t *visible, const float *depth, const int32_t *box, const float *uv,
             const float *conic, const float *opacity, int W, int H, int tw, int th, uint64_t *keys,
             uint32_t *vals, int64_t cap, int64_t *npairs, uint32_t *ranges) {
    if (tw <= 0 || th <= 0) return 1;
    const int gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!visible[i]) continue;
        total += gaussian_tiles(box + 4 * i, uv + 2 * i, conic + 3 * i, opacity[i], tw, th, gx, NULL);
    }
    *npairs = total;
    if (total > cap) return 2;
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (size_t)(total > 0 ? total : 1));
    uint32_t *tl = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(gx * gy));
    if (!kv || !tl) return 3;
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!visible[i]) continue;
        const int64_t m = gaussian_tiles(box + 4 * i, uv + 2 * i, conic + 3 * i, opacity[i], tw, th, gx, tl);
        for (int64_t j = 0; j < m; ++j) {
            kv[k].key = ((uint64_t)tl[j] << 32) | float_bits(depth[i]);
            kv[k].val = (uint32_t)i;
            ++k;
        }
    }
    free(tl);
    qsort(kv, (size_t)total, sizeof(kv_t), kv_cmp);
    for (int t = 0; t < gx * gy; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
    for (int64_t j = 0; j < total; ++j) {
        keys[j] = kv[j].key;
        vals[j] = kv[j].val;
        uint32_t tile = (uint32_t)(kv[j].key >> 32);
        if (j == 0 || (uint32_t)(kv[j - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)j;
        ranges[2 * tile + 1] = (uint32_t)(j + 1);
    }
    free(kv);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* FP64 projection of one Gaussian (EWA splatting, cited by Eq. 3).          */
/* ------------------------------------------------------------------------- */

typedef struct {
    double mu[3];          /* world-space mean                           */
    double pc[3];          /* camera-space mean                          */
    double s[3];           /* exp(logscale)                              */
    double qn[4], qnorm;   /* normalised quaternion (w,x,y,z), |q|       */
    double Rq[9];          /* rotation of the normalised quaternion      */
    double M[9];           /* Rq diag(s)                                 */
    double Sig[9];         /* 3D covariance M M^T                        */
    double qx, qy;         /* clamped x/z, y/z                           */
    int clx, cly;          /* 1 when the clamp is active                 */
    double J[6];           /* 2x3 Jacobian of the projection             */
    double T[6];           /* J W                                        */
    double cov2[3];        /* a', b', c' of Sigma' (dilated)             */
    double conic[3];       /* A, B, C of Sigma'^-1                       */
    double u, v;           /* projected mean                             */
    double opacity;        /* sigmoid(logit)                             */
    double rgb_raw[3];     /* SH colour + 0.5 before the clamp           */
    double rgb[3];         /* max(0, rgb_raw)                            */
    double dir[3], dirn;   /* mean - camera centre, its norm             */
    double vh[3];          /* unit view direction                        */
    double Y[16], dY[48];  /* SH basis and its gradient                  */
} orc_pre;

typedef struct {
    double R[9], t[3], fx, fy, cx, cy, campos[3];
    int W, H;
} orc_cam;

/* The FP64 path takes the camera in FP64 (an FP32 camera widens exactly);
 * the decision chain keeps its FP32 copy. */
static orc_cam make_cam(const double *cam, int W, int H) {
    orc_cam c;
    for (int i = 0; i < 9; ++i) c.R[i] = cam[i];
    for (int i = 0; i < 3; ++i) c.t[i] = cam[9 + i];
    c.fx = cam[12]; c.fy = cam[13]; c.cx = cam[14]; c.cy = cam[15];
    c.W = W; c.H = H;
    /* camera centre C = -R^T t */
    for (int j = 0; j < 3; ++j)
        c.campos[j] = -(c.R[j] * c.t[0] + c.R[3 + j] * c.t[1] + c.R[6 + j] * c.t[2]);
    return c;
}

static void project_one(const double *mo, const double *q, const double *ls, const double *sh,
                        int deg, const orc_cam *cam, orc_pre *p) {
    const double *W = cam->R;
    for (int i = 0; i < 3; ++i) p->mu[i] = mo[i];
    for (int i = 0; i < 3; ++i)
        p->pc[i] = W[3 * i] * mo[0] + W[3 * i + 1] * mo[1] + W[3 * i + 2] * mo[2] + cam->t[i];
    for (int i = 0; i < 3; ++i) p->s[i] = exp(ls[i]);
    p->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) p->qn[i] = q[i] / p->qnorm;
    const double w = p->qn[0], x = p->qn[1], y = p->qn[2], z = p->qn[3];
    double *Rq = p->Rq;
    Rq[0] = 1 - 2 * (y * y + z * z); Rq[1] = 2 * (x * y - w * z);     Rq[2] = 2 * (x * z + w * y);
    Rq[3] = 2 * (x * y + w * z);     Rq[4] = 1 - 2 * (x * x + z * z); Rq[5] = 2 * (y * z - w * x);
    Rq[6] = 2 * (x * z - w * y);     Rq[7] = 2 * (y * z + w * x);     Rq[8] = 1 - 2 * (x * x + y * y);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) p->M[3 * i + j] = Rq[3 * i + j] * p->s[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += p->M[3 * i + k] * p->M[3 * j + k];
            p->Sig[3 * i + j] = acc;
        }
    const double X = p->pc[0], Yc = p->pc[1], Z = p->pc[2];
    const double limx = 1.3 * (0.5 * cam->W / cam->fx), limy = 1.3 * (0.5 * cam->H / cam->fy);
    double tx = X / Z, ty = Yc / Z;
    p->clx = (tx < -limx || tx > limx);
    p->cly = (ty < -limy || ty > limy);
    p->qx = tx < -limx ? -limx : (tx > limx ? limx : tx);
    p->qy = ty < -limy ? -limy : (ty > limy ? limy : ty);
    double *J = p->J;
    J[0] = cam->fx / Z; J[1] = 0; J[2] = -cam->fx * p->qx / Z;
    J[3] = 0; J[4] = cam->fy / Z; J[5] = -cam->fy * p->qy / Z;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += J[3 * i + k] * W[3 * k + j];
            p->T[3 * i + j] = acc;
        }
    double C2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += p->T[3 * i + k] * p->Sig[3 * k + l] * p->T[3 * j + l];
            C2[2 * i + j] = acc;
        }
    p->cov2[0] = C2[0] + ORC_DILATION;
    p->cov2[1] = C2[1];
    p->cov2[2] = C2[3] + ORC_DILATION;
    double det = p->cov2[0] * p->cov2[2] - p->cov2[1] * p->cov2[1];
    p->conic[0] = p->cov2[2] / det;
    p->conic[1] = -p->cov2[1] / det;
    p->conic[2] = p->cov2[0] / det;
    p->u = cam->fx * X / Z + cam->cx;
    p->v = cam->fy * Yc / Z + cam->cy;
    p->opacity = 1.0 / (1.0 + exp(-mo[3]));
    for (int i = 0; i < 3; ++i) p->dir[i] = mo[i] - cam->campos[i];
    p->dirn = sqrt(p->dir[0] * p->dir[0] + p->dir[1] * p->dir[1] + p->dir[2] * p->dir[2]);
    for (int i = 0; i < 3; ++i) p->vh[i] = p->dir[i] / p->dirn;
    orc_sh_basis(p->vh, deg, p->Y, p->dY);
    const int nc = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0;
        for (int k = 0; k < nc; ++k) acc += sh[3 * k + ch] * p->Y[k];
        p->rgb_raw[ch] = acc + 0.5;
        p->rgb[ch] = p->rgb_raw[ch] > 0 ? p->rgb_raw[ch] : 0.0;
    }
}

/* Parameters arrive planar, as the product stores them:
 *   mean_op[4n] (x, y, z, opacity logit), quat[4n] (w, x, y, z),
 *   logscale[4n] (3 + pad), sh[12][n][4] = 48 floats per Gaussian,
 *   coefficient-major: float f of the 48 is coefficient f/3, channel f%3.  */
static void gather_sh(const double *sh, int64_t n, int64_t i, double out[48]) {
    for (int j = 0; j < 12; ++j)
        for (int e = 0; e < 4; ++e) out[4 * j + e] = sh[((int64_t)j * n + i) * 4 + e];
}

typedef struct { float depth; int64_t gid; } ord_t;

static int ord_cmp(const void *a, const void *b) {
    const ord_t *x = (const ord_t *)a, *y = (const ord_t *)b;
    if (x->depth != y->depth) return x->depth < y->depth ? -1 : 1;
    return x->gid < y->gid ? -1 : (x->gid > y->gid ? 1 : 0);
}

/* visible Gaussians sorted by (FP32 depth, index) */
static int64_t depth_order(int64_t n, const uint8_t *visible, const float *depth, int64_t **out) {
    int64_t nv = 0;
    for (int64_t i = 0; i < n; ++i) nv += visible[i] ? 1 : 0;
    ord_t *o = (ord_t *)malloc(sizeof(ord_t) * (size_t)(nv > 0 ? nv : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i)
        if (visible[i]) { o[k].depth = depth[i]; o[k].gid = i; ++k; }
    qsort(o, (size_t)nv, sizeof(ord_t), ord_cmp);
    int64_t *ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
    for (int64_t j = 0; j < nv; ++j) ids[j] = o[j].gid;
    free(o);
    *out = ids;
    return nv;
}

static orc_pre *project_all(int64_t n, const double *mean_op, const double *quat,
                            const double *logscale, const double *sh, int deg, const orc_cam *cam,
                            const uint8_t *visible) {
    orc_pre *pre = (orc_pre *)calloc((size_t)(n > 0 ? n : 1), sizeof(orc_pre));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (!visible[i]) continue;
        double shi[48];
        gather_sh(sh, n, i, shi);
        project_one(mean_op + 4 * i, quat + 4 * i, logscale + 4 * i, shi, deg, cam, &pre[i]);
    }
    return pre;
}

static double rel_margin(double a, double thr) { return fabs(a - thr) / thr; }

/* One contribution of a Gaussian at a pixel, kept for the backward. */
typedef struct {
    int64_t gid;
    double alpha, T, dx, dy, G; /* T = transmittance in front of it      */
    int clamped;                /* alpha hit the 0.99 clamp              */
} contrib_t;

/* Walk one pixel front to back over the depth-ordered visible Gaussians whose
 * pixel box contains it; returns the number of contributions written to cs
 * and the final transmittance. */
static int64_t pixel_walk(int px, int py, const int64_t *order, int64_t nv, const orc_pre *pre,
                          const int32_t *box, int flags, contrib_t *cs, double *T_out,
                          double *margin_out, int64_t *nconsidered) {
    double T = 1.0, margin = INFINITY;
    int64_t nc = 0, considered = 0;
    for (int64_t j = 0; j < nv; ++j) {
        const int64_t g = order[j];
        const int32_t *b = box + 4 * g;
        if (px < b[0] || px > b[1] || py < b[2] || py > b[3]) continue;
        ++considered;
        const orc_pre *p = &pre[g];
        double dx = px - p->u, dy = py - p->v;
        double power = -0.5 * (p->conic[0] * dx * dx + p->conic[2] * dy * dy) - p->conic[1] * dx * dy;
        if (power > 0.0) continue;
        double G = exp(power);
        double araw = p->opacity * G;
        double alpha = araw;
        int clamped = 0;
        if (!(flags & ORC_NO_CLAMP)) {
            double m = rel_margin(araw, ORC_ALPHA_MAX);
            if (m < margin) margin = m;
            if (araw > ORC_ALPHA_MAX) { alpha = ORC_ALPHA_MAX; clamped = 1; }
        }
        if (!(flags & ORC_NO_SKIP)) {
            double m = rel_margin(alpha, ORC_ALPHA_MIN);
            if (m < margin) margin = m;
            if (alpha < ORC_ALPHA_MIN) continue;
        }
        double Tn = T * (1.0 - alpha);
        if (!(flags & ORC_NO_TERM)) {
            double m = rel_margin(Tn, ORC_T_MIN);
            if (m < margin) margin = m;
            if (Tn < ORC_T_MIN) break;
        }
        if (cs) {
            cs[nc].gid = g; cs[nc].alpha = alpha; cs[nc].T = T;
            cs[nc].dx = dx; cs[nc].dy = dy; cs[nc].G = G; cs[nc].clamped = clamped;
        }
        ++nc;
        T = Tn;
    }
    *T_out = T;
    if (margin_out) *margin_out = margin;
    if (nconsidered) *nconsidered = considered;
    return nc;
}

/* Forward render of rows [y_begin, y_end).  img is planar 3 x H x W.
 * n_contrib[p] = number of Gaussians blended at pixel p; margin[p] = smallest
 * relative distance of any alpha / transmittance decision at p to its
 * threshold (pixels with a tiny margin may legitimately differ between an
 * FP32 and an FP64 evaluation). */
int orc_render(int64_t n, const double *mean_op, const double *quat, const double *logscale,
               const double *sh, int deg, const double *camf, int W, int H, const double *bg,
               const uint8_t *visible, const float *depth, const int32_t *box, int flags,
               int y_begin, int y_end, double *img, double *T_final, int32_t *n_contrib,
               double *margin) {
    if (deg < 0 || deg > 3 || y_begin < 0 || y_end > H || y_begin > y_end) return 1;
    orc_cam cam = make_cam(camf, W, H);
    orc_pre *pre = project_all(n, mean_op, quat, logscale, sh, deg, &cam, visible);
    int64_t *order;
    int64_t nv = depth_order(n, visible, depth, &order);
#pragma omp parallel
    {
        contrib_t *cs = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(nv > 0 ? nv : 1));
#pragma omp for schedule(dynamic, 1)
        for (int py = y_begin; py < y_end; ++py) {
            for (int px = 0; px < W; ++px) {
                double T, mg;
                int64_t nc = pixel_walk(px, py, order, nv, pre, box, flags, cs, &T, &mg, NULL);
                double C[3] = {0, 0, 0};
                for (int64_t k = 0; k < nc; ++k) {
                    const orc_pre *p = &pre[cs[k].gid];
                    for (int ch = 0; ch < 3; ++ch) C[ch] += p->rgb[ch] * cs[k].alpha * cs[k].T;
                }
                const int64_t pix = (int64_t)py * W + px;
                for (int ch = 0; ch < 3; ++ch) img[(int64_t)ch * W * H + pix] = C[ch] + T * bg[ch];
                if (T_final) T_final[pix] = T;
                if (n_contrib) n_contrib[pix] = (int32_t)nc;
                if (margin) margin[pix] = mg;
            }
        }
        free(cs);
    }
    free(order);
    free(pre);
    return 0;
}

/* Chain the per-Gaussian screen-space gradients g2 = (du, dv, dA, dB, dC,
 * dopacity, dr, dg, db) to the 60-float parameter gradient layout
 * (mean x y z, opacity logit, quat w x y z, logscale 0 1 2, pad, sh[48]).
 * pose (may be NULL) receives (+=) this Gaussian's part of the camera pose
 * gradient, 15 values: dL/dR (row-major, R taken as a general 3 x 3 matrix),
 * dL/dt, and dL/dphi for the left perturbation R <- exp([phi]x) R,
 * t <- exp([phi]x) t (a rotation about the camera centre); pose_mag (may be
 * NULL) the absolute values of the same parts. */
static void chain_one(const orc_pre *p, const orc_cam *cam, const double *sh, int deg,
                      const double *g2, double *out, double *pose, double *pose_mag) {
    const double *W = cam->R;
    double dmean[3] = {0, 0, 0}, dpc[3] = {0, 0, 0};
    /* colour: c = max(0, sum_k sh_k Y_k(vhat) + 0.5) */
    const int nc = (deg + 1) * (deg + 1);
    double dcol[3], dvh[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) dcol[ch] = (p->rgb_raw[ch] > 0) ? g2[6 + ch] : 0.0;
    for (int k = 0; k < 16; ++k)
        for (int ch = 0; ch < 3; ++ch) out[12 + 3 * k + ch] = (k < nc) ? dcol[ch] * p->Y[k] : 0.0;
    for (int k = 0; k < nc; ++k)
        for (int ch = 0; ch < 3; ++ch)
            for (int a = 0; a < 3; ++a) dvh[a] += dcol[ch] * sh[3 * k + ch] * p->dY[3 * k + a];
    double vd = dvh[0] * p->vh[0] + dvh[1] * p->vh[1] + dvh[2] * p->vh[2];
    double ddir[3]; /* dL/d(mean - camera centre) through the view direction */
    for (int a = 0; a < 3; ++a) ddir[a] = (dvh[a] - p->vh[a] * vd) / p->dirn;
    for (int a = 0; a < 3; ++a) dmean[a] += ddir[a];
    /* opacity */
    out[3] = g2[5] * p->opacity * (1.0 - p->opacity);
    /* conic -> Sigma' : G_S' = -Q G_Q Q with G_Q = [[dA, dB/2], [dB/2, dC]] */
    double Q[4] = {p->conic[0], p->conic[1], p->conic[1], p->conic[2]};
    double GQ[4] = {g2[2], 0.5 * g2[3], 0.5 * g2[3], g2[4]};
    double tmp[4], GS2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) tmp[2 * i + j] = Q[2 * i] * GQ[j] + Q[2 * i + 1] * GQ[2 + j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) GS2[2 * i + j] = -(tmp[2 * i] * Q[j] + tmp[2 * i + 1] * Q[2 + j]);
    /* Sigma' = T Sig T^T + 0.3 I :  G_Sig = T^T G_S' T,  G_T = 2 G_S' T Sig */
    double GSig[9], GT[6];
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            double acc = 0;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) acc += p->T[3 * i + k] * GS2[2 * i + j] * p->T[3 * j + l];
            GSig[3 * k + l] = acc;
        }
    for (int i = 0; i < 2; ++i)
        for (int l = 0; l < 3; ++l) {
            double acc = 0;
            for (int j = 0; j < 2; ++j)
                for (int k = 0; k < 3; ++k) acc += GS2[2 * i + j] * p->T[3 * j + k] * p->Sig[3 * k + l];
            GT[3 * i + l] = 2.0 * acc;
        }
    /* T = J W : G_J = G_T W^T */
    double GJ[6];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += GT[3 * i + j] * W[3 * k + j];
            GJ[3 * i + k] = acc;
        }
    const double X = p->pc[0], Yc = p->pc[1], Z = p->pc[2];
    const double fx = cam->fx, fy = cam->fy;
    /* J00 = fx/Z, J02 = -fx qx/Z, J11 = fy/Z, J12 = -fy qy/Z, qx = clamp(X/Z) */
    double dqx_dX = p->clx ? 0.0 : 1.0 / Z, dqx_dZ = p->clx ? 0.0 : -X / (Z * Z);
    double dqy_dY = p->cly ? 0.0 : 1.0 / Z, dqy_dZ = p->cly ? 0.0 : -Yc / (Z * Z);
    dpc[2] += GJ[0] * (-fx / (Z * Z)) + GJ[4] * (-fy / (Z * Z));
    dpc[0] += GJ[2] * (-fx / Z) * dqx_dX;
    dpc[2] += GJ[2] * (fx * p->qx / (Z * Z) - fx / Z * dqx_dZ);
    dpc[1] += GJ[5] * (-fy / Z) * dqy_dY;
    dpc[2] += GJ[5] * (fy * p->qy / (Z * Z) - fy / Z * dqy_dZ);
    /* u = fx X/Z + cx, v = fy Y/Z + cy */
    dpc[0] += g2[0] * fx / Z;
    dpc[1] += g2[1] * fy / Z;
    dpc[2] += -g2[0] * fx * X / (Z * Z) - g2[1] * fy * Yc / (Z * Z);
    /* pc = W mean + t */
    for (int a = 0; a < 3; ++a) dmean[a] += W[a] * dpc[0] + W[3 + a] * dpc[1] + W[6 + a] * dpc[2];
    out[0] = dmean[0]; out[1] = dmean[1]; out[2] = dmean[2];
    if (pose) {
        /* the pose enters through pc = W mean + t, through T = J W (G_W = J^T G_T)
         * and through the camera centre C = -W^T t of the view direction
         * mean - C (G_C = -ddir) */
        double c[15], GWc[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) GWc[3 * a + b] = p->J[a] * GT[b] + p->J[3 + a] * GT[3 + b];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                c[3 * a + b] = dpc[a] * p->mu[b] + GWc[3 * a + b] + ddir[b] * cam->t[a];
        for (int a = 0; a < 3; ++a)
            c[9 + a] = dpc[a] + W[3 * a] * ddir[0] + W[3 * a + 1] * ddir[1] + W[3 * a + 2] * ddir[2];
        /* left rotation: d pc = phi x pc, d W = [phi]x W, the centre is fixed;
         * <G, [phi]x W> = phi . (N21 - N12, N02 - N20, N10 - N01), N = G W^T */
        double N[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                N[3 * a + b] = GWc[3 * a] * W[3 * b] + GWc[3 * a + 1] * W[3 * b + 1] + GWc[3 * a + 2] * W[3 * b + 2];
        const double *pc = p->pc;
        c[12] = pc[1] * dpc[2] - pc[2] * dpc[1] + N[7] - N[5];
        c[13] = pc[2] * dpc[0] - pc[0] * dpc[2] + N[2] - N[6];
        c[14] = pc[0] * dpc[1] - pc[1] * dpc[0] + N[3] - N[1];
        for (int k = 0; k < 15; ++k) {
            pose[k] += c[k];
            if (pose_mag) pose_mag[k] += fabs(c[k]);
        }
    }
    /* Sig = M M^T, M = Rq diag(s) : G_M = 2 G_Sig M */
    double GM[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += GSig[3 * i + k] * p->M[3 * k + j];
            GM[3 * i + j] = 2.0 * acc;
        }
    double GR[9];
    for (int j = 0; j < 3; ++j) {
        double ds = 0;
        for (int i = 0; i < 3; ++i) {
            ds += GM[3 * i + j] * p->Rq[3 * i + j];
            GR[3 * i + j] = GM[3 * i + j] * p->s[j];
        }
        out[8 + j] = ds * p->s[j];
    }
    out[11] = 0.0;
    /* rotation entries as functions of the normalised quaternion (w,x,y,z) */
    const double w = p->qn[0], x = p->qn[1], y = p->qn[2], z = p->qn[3];
    /* dR_ij / d(w, x, y, z) */
    const double dR[9][4] = {
        {0, 0, -4 * y, -4 * z},        {-2 * z, 2 * y, 2 * x, -2 * w}, {2 * y, 2 * z, 2 * w, 2 * x},
        {2 * z, 2 * y, 2 * x, 2 * w},  {0, -4 * x, 0, -4 * z},         {-2 * x, -2 * w, 2 * z, 2 * y},
        {-2 * y, 2 * z, -2 * w, 2 * x}, {2 * x, 2 * w, 2 * z, 2 * y},  {0, -4 * x, -4 * y, 0}};
    double dqn[4] = {0, 0, 0, 0};
    for (int e = 0; e < 9; ++e)
        for (int a = 0; a < 4; ++a) dqn[a] += GR[e] * dR[e][a];
    double qd = dqn[0] * p->qn[0] + dqn[1] * p->qn[1] + dqn[2] * p->qn[2] + dqn[3] * p->qn[3];
    for (int a = 0; a < 4; ++a) out[4 + a] = (dqn[a] - p->qn[a] * qd) / p->qnorm;
}

/* Backward of the render: given dL/dimg (planar 3 x H x W) over rows
 * [y_begin, y_end), writes grad[60 n] (= dL/dparams, overwritten) and
 * grad2d[9 n] (screen-space gradients du dv dA dB dC dopacity dr dg db).
 * The per-pixel blend state is kept exactly (no division recompute).
 * grad2d_mag (may be NULL) receives, per screen-space gradient element, the
 * sum over pixels of the magnitude of that pixel's term with every inner sum
 * taken in absolute value: the scale against which a finite-precision
 * evaluation of the same sum can err (its condition magnitude). */
int orc_render_bwd(int64_t n, const double *mean_op, const double *quat, const double *logscale,
                   const double *sh, int deg, const double *camf, int W, int H, const double *bg,
                   const uint8_t *visible, const float *depth, const int32_t *box, int flags,
                   int y_begin, int y_end, const double *dimg, double *grad, double *grad2d,
                   double *grad2d_mag) {
    if (deg < 0 || deg > 3 || y_begin < 0 || y_end > H || y_begin > y_end) return 1;
    orc_cam cam = make_cam(camf, W, H);
    orc_pre *pre = project_all(n, mean_op, quat, logscale, sh, deg, &cam, visible);
    int64_t *order;
    int64_t nv = depth_order(n, visible, depth, &order);
    const int nthr = orc_num_threads();
    const int nacc = 18; /* 9 gradients + 9 condition magnitudes */
    double *acc = (double *)calloc((size_t)nthr * (size_t)(n > 0 ? n : 1) * nacc, sizeof(double));
#pragma omp parallel
    {
#ifdef _OPENMP
        const int tid = omp_get_thread_num();
#else
        const int tid = 0;
#endif
        double *g2 = acc + (size_t)tid * (size_t)n * nacc;
        contrib_t *cs = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(nv > 0 ? nv : 1));
#pragma omp for schedule(dynamic, 1)
        for (int py = y_begin; py < y_end; ++py) {
            for (int px = 0; px < W; ++px) {
                double Tf;
                int64_t nc = pixel_walk(px, py, order, nv, pre, box, flags, cs, &Tf, NULL, NULL);
                const int64_t pix = (int64_t)py * W + px;
                double dC[3];
                for (int ch = 0; ch < 3; ++ch) dC[ch] = dimg[(int64_t)ch * W * H + pix];
                /* S = colour accumulated behind the current Gaussian, incl. background */
                double S[3];
                for (int ch = 0; ch < 3; ++ch) S[ch] = bg[ch] * Tf;
                for (int64_t k = nc - 1; k >= 0; --k) {
                    const contrib_t *c = &cs[k];
                    const orc_pre *p = &pre[c->gid];
                    double *o = g2 + nacc * c->gid, *om = o + 9;
                    double dalpha = 0.0, dalpha_mag = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        o[6 + ch] += dC[ch] * c->alpha * c->T;
                        om[6 + ch] += fabs(dC[ch] * c->alpha * c->T);
                        dalpha += dC[ch] * (p->rgb[ch] * c->T - S[ch] / (1.0 - c->alpha));
                        dalpha_mag += fabs(dC[ch]) * (fabs(p->rgb[ch]) * c->T + fabs(S[ch]) / (1.0 - c->alpha));
                    }
                    for (int ch = 0; ch < 3; ++ch) S[ch] += p->rgb[ch] * c->alpha * c->T;
                    if (c->clamped) continue; /* alpha = 0.99 does not depend on anything */
                    /* alpha = opacity * exp(power) */
                    o[5] += dalpha * c->G;
                    om[5] += dalpha_mag * c->G;
                    double dpow = dalpha * c->alpha, dpow_mag = dalpha_mag * c->alpha;
                    const double A = p->conic[0], B = p->conic[1], Cc = p->conic[2];
                    o[0] += dpow * (A * c->dx + B * c->dy);
                    o[1] += dpow * (Cc * c->dy + B * c->dx);
                    o[2] += dpow * (-0.5 * c->dx * c->dx);
                    o[3] += dpow * (-c->dx * c->dy);
                    o[4] += dpow * (-0.5 * c->dy * c->dy);
                    om[0] += dpow_mag * (fabs(A * c->dx) + fabs(B * c->dy));
                    om[1] += dpow_mag * (fabs(Cc * c->dy) + fabs(B * c->dx));
                    om[2] += dpow_mag * 0.5 * c->dx * c->dx;
                    om[3] += dpow_mag * fabs(c->dx * c->dy);
                    om[4] += dpow_mag * 0.5 * c->dy * c->dy;
                }
            }
        }
        free(cs);
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < nacc; ++k) {
            double s = 0.0;
            for (int t = 0; t < nthr; ++t) s += acc[((size_t)t * (size_t)n + (size_t)i) * nacc + k];
            if (k < 9 && grad2d) grad2d[9 * i + k] = s;
            if (k >= 9 && grad2d_mag) grad2d_mag[9 * i + k - 9] = s;
            acc[(size_t)i * nacc + k] = s; /* thread 0 slot now holds the total */
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double *o = grad + 60 * i;
        for (int k = 0; k < 60; ++k) o[k] = 0.0;
        if (!visible[i]) continue;
        double shi[48];
        gather_sh(sh, n, i, shi);
        chain_one(&pre[i], &cam, shi, deg, acc + (size_t)i * nacc, o, NULL, NULL);
    }
    free(acc);
    free(order);
    free(pre);
    return 0;
}

/* Screen-space chain only (for checking the per-Gaussian chain rule by itself):
 * given g2[9n] computes grad[60n]. */
int orc_chain(int64_t n, const double *mean_op, const double *quat, const double *logscale,
              const double *sh, int deg, const double *camf, int W, int H, const uint8_t *visible,
              const double *g2, double *grad) {
    orc_cam cam = make_cam(camf, W, H);
    orc_pre *pre = project_all(n, mean_op, quat, logscale, sh, deg, &cam, visible);
    for (int64_t i = 0; i < n; ++i) {
        double *o = grad + 60 * i;
        for (int k = 0; k < 60; ++k) o[k] = 0.0;
        if (!visible[i]) continue;
        double shi[48];
        gather_sh(sh, n, i, shi);
        chain_one(&pre[i], &cam, shi, deg, g2 + 9 * i, o, NULL, NULL);
    }
    free(pre);
    return 0;
}

/* Camera pose gradient (pose refinement against the map): given the
 * screen-space gradients g2[9n] of the visible Gaussians, pose[15] receives
 * the sum over them of their parts (chain_one): dL/dR (9, row-major), dL/dt
 * (3), dL/dphi (3; the gradient along the translation of the same left
 * perturbation is dL/dt).  pose_mag[15] (may be NULL) receives the sums of
 * the parts' absolute values. */
int orc_pose_grad(int64_t n, const double *mean_op, const double *quat, const double *logscale,
                  const double *sh, int deg, const double *camf, int W, int H, const uint8_t *visible,
                  const double *g2, double *pose, double *pose_mag) {
    orc_cam cam = make_cam(camf, W, H);
    orc_pre *pre = project_all(n, mean_op, quat, logscale, sh, deg, &cam, visible);
    double o[60];
    for (int k = 0; k < 15; ++k) {
        pose[k] = 0.0;
        if (pose_mag) pose_mag[k] = 0.0;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (!visible[i]) continue;
        double shi[48];
        gather_sh(sh, n, i, shi);
        chain_one(&pre[i], &cam, shi, deg, g2 + 9 * i, o, pose, pose_mag);
    }
    free(pre);
    return 0;
}

/* Per-Gaussian FP64 screen-space quantities (for closed-form checks):
 * out[16 n] = u, v, A, B, C, opacity, r, g, b, depth, a', b', c', rgb_raw r g b */
int orc_project(int64_t n, const double *mean_op, const double *quat, const double *logscale,
                const double *sh, int deg, const double *camf, int W, int H, const uint8_t *visible,
                double *out) {
    orc_cam cam = make_cam(camf, W, H);
    orc_pre *pre = project_all(n, mean_op, quat, logscale, sh, deg, &cam, visible);
    for (int64_t i = 0; i < n; ++i) {
        const orc_pre *p = &pre[i];
        double *o = out + 16 * i;
        o[0] = p->u; o[1] = p->v;
        o[2] = p->conic[0]; o[3] = p->conic[1]; o[4] = p->conic[2];
        o[5] = p->opacity;
        o[6] = p->rgb[0]; o[7] = p->rgb[1]; o[8] = p->rgb[2];
        o[9] = p->pc[2];
        o[10] = p->cov2[0]; o[11] = p->cov2[1]; o[12] = p->cov2[2];
        o[13] = p->rgb_raw[0]; o[14] = p->rgb_raw[1]; o[15] = p->rgb_raw[2];
    }
    free(pre);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Eq. 4 photometric loss: (1-lambda) mean|x - y| + lambda (1 - mean SSIM).   */
/* SSIM (Wang et al. 2004) per channel with an 11x11 Gaussian window of       */
/* sigma 1.5 normalised to 1, zero padding ("same" output), C1 = 0.01^2,      */
/* C2 = 0.03^2, dynamic range 1, averaged over every pixel and channel.       */
/* Images are planar C x H x W.  dimg (may be NULL) receives dL/dx.           */
/* ------------------------------------------------------------------------- */

static void ssim_window(double w[11]) {
    double s = 0;
    for (int i = 0; i < 11; ++i) { w[i] = exp(-((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5)); s += w[i]; }
    for (int i = 0; i < 11; ++i) w[i] /= s;
}

int orc_ssim_map(const double *x, const double *y, int C, int H, int W, double *smap) {
    double w[11];
    ssim_window(w);
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
#pragma omp parallel for collapse(2) schedule(static)
    for (int c = 0; c < C; ++c)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                const double *X = x + (int64_t)c * H * W, *Yv = y + (int64_t)c * H * W;
                double mx = 0, my = 0, ex2 = 0, ey2 = 0, exy = 0;
                for (int a = -5; a <= 5; ++a)
                    for (int b = -5; b <= 5; ++b) {
                        int ii = i + a, jj = j + b;
                        if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                        double wt = w[a + 5] * w[b + 5];
                        double xv = X[(int64_t)ii * W + jj], yv = Yv[(int64_t)ii * W + jj];
                        mx += wt * xv; my += wt * yv;
                        ex2 += wt * xv * xv; ey2 += wt * yv * yv; exy += wt * xv * yv;
                    }
                double sxx = ex2 - mx * mx, syy = ey2 - my * my, sxy = exy - mx * my;
                smap[(int64_t)c * H * W + (int64_t)i * W + j] =
                    ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2));
            }
    return 0;
}

int orc_loss(const double *x, const double *y, int C, int H, int W, double lambda, double *loss,
             double *dimg) {
    const int64_t npx = (int64_t)C * H * W;
    if (npx <= 0) return 1;
    double w[11];
    ssim_window(w);
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double *smap = (double *)malloc(sizeof(double) * (size_t)npx);
    /* per-pixel partials of S w.r.t. the raw moments (mx, E[x^2], E[xy]) */
    double *pa = (double *)malloc(sizeof(double) * (size_t)npx);
    double *pb = (double *)malloc(sizeof(double) * (size_t)npx);
    double *pc = (double *)malloc(sizeof(double) * (size_t)npx);
#pragma omp parallel for collapse(2) schedule(static)
    for (int c = 0; c < C; ++c)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                const double *X = x + (int64_t)c * H * W, *Yv = y + (int64_t)c * H * W;
                double mx = 0, my = 0, ex2 = 0, ey2 = 0, exy = 0;
                for (int a = -5; a <= 5; ++a)
                    for (int b = -5; b <= 5; ++b) {
                        int ii = i + a, jj = j + b;
                        if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                        double wt = w[a + 5] * w[b + 5];
                        double xv = X[(int64_t)ii * W + jj], yv = Yv[(int64_t)ii * W + jj];
                        mx += wt * xv; my += wt * yv;
                        ex2 += wt * xv * xv; ey2 += wt * yv * yv; exy += wt * xv * yv;
                    }
                double sxx = ex2 - mx * mx, syy = ey2 - my * my, sxy = exy - mx * my;
                double A1 = 2 * mx * my + C1, A2 = 2 * sxy + C2;
                double B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
                double S = (A1 * A2) / (B1 * B2);
                double dS_dmx = (2 * my * A2) / (B1 * B2) - S * (2 * mx) / B1;
                double dS_dsxx = -S / B2;
                double dS_dsxy = 2 * A1 / (B1 * B2);
                const int64_t o = (int64_t)c * H * W + (int64_t)i * W + j;
                smap[o] = S;
                pa[o] = dS_dmx - 2 * mx * dS_dsxx - my * dS_dsxy;
                pb[o] = dS_dsxx;
                pc[o] = dS_dsxy;
            }
    double l1 = 0, ss = 0;
    for (int64_t k = 0; k < npx; ++k) { l1 += fabs(x[k] - y[k]); ss += smap[k]; }
    *loss = (1 - lambda) * l1 / npx + lambda * (1 - ss / npx);
    if (dimg) {
#pragma omp parallel for collapse(2) schedule(static)
        for (int c = 0; c < C; ++c)
            for (int i = 0; i < H; ++i)
                for (int j = 0; j < W; ++j) {
                    const int64_t base = (int64_t)c * H * W;
                    const int64_t o = base + (int64_t)i * W + j;
                    double ga = 0, gb = 0, gc = 0;
                    for (int a = -5; a <= 5; ++a)
                        for (int b = -5; b <= 5; ++b) {
                            int ii = i + a, jj = j + b;
                            if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                            double wt = w[a + 5] * w[b + 5];
                            const int64_t q = base + (int64_t)ii * W + jj;
                            ga += wt * pa[q]; gb += wt * pb[q]; gc += wt * pc[q];
                        }
                    double dsum = ga + 2 * x[o] * gb + y[o] * gc;
                    double diff = x[o] - y[o];
                    double sg = diff > 0 ? 1.0 : (diff < 0 ? -1.0 : 0.0);
                    dimg[o] = (1 - lambda) * sg / npx - lambda * dsum / npx;
                }
    }
    free(smap); free(pa); free(pb); free(pc);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Eq. 5 Gaussian pyramid, one level down: separable binomial [1 4 6 4 1]/16, */
/* reflect-101 border, keep even pixels; output ceil(H/2) x ceil(W/2).        */
/* ------------------------------------------------------------------------- */

static int reflect101(int i, int n) {
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * (n - 1) - i;
    }
    return i;
}

int orc_pyramid_down(const double *in, int C, int H, int W, double *out) {
    const double k[5] = {1 / 16.0, 4 / 16.0, 6 / 16.0, 4 / 16.0, 1 / 16.0};
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    for (int c = 0; c < C; ++c)
        for (int i = 0; i < Ho; ++i)
            for (int j = 0; j < Wo; ++j) {
                double s = 0;
                for (int a = 0; a < 5; ++a)
                    for (int b = 0; b < 5; ++b) {
                        int ii = reflect101(2 * i + a - 2, H), jj = reflect101(2 * j + b - 2, W);
                        s += k[a] * k[b] * in[(int64_t)c * H * W + (int64_t)ii * W + jj];
                    }
                out[(int64_t)c * Ho * Wo + (int64_t)i * Wo + j] = s;
            }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adam (Kingma & Ba 2015) with bias correction; step is the 1-based index    */
/* of this update.  lr[k] is the learning rate of element k.                  */
/* ------------------------------------------------------------------------- */

int orc_adam(int64_t count, double *p, const double *g, double *m, double *v, const double *lr,
             int step, double b1, double b2, double eps) {
    if (step < 1) return 1;
    const double bc1 = 1 - pow(b1, step), bc2 = 1 - pow(b2, step);
    for (int64_t k = 0; k < count; ++k) {
        m[k] = b1 * m[k] + (1 - b1) * g[k];
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k];
        double mh = m[k] / bc1, vh = v[k] / bc2;
        p[k] -= lr[k] * mh / (sqrt(vh) + eps);
    }
    return 0;
}

/* PSNR in dB of img (clamped to [0,1]) against gt, peak 1. */
double orc_psnr(const double *img, const double *gt, int64_t count) {
    double se = 0;
    for (int64_t k = 0; k < count; ++k) {
        double a = img[k] < 0 ? 0 : (img[k] > 1 ? 1 : img[k]);
        double d = a - gt[k];
        se += d * d;
    }
    double mse = se / (double)count;
    return 10.0 * log10(1.0 / mse);
}

/* Default initialisation of new primitives created at keypoints.  Photo-SLAM
 * adds primitives at inactive ORB keypoints (Sec. 3.3.1, geometry-based
 * densification) without stating their initial shape; the reading is the
 * 3D-Gaussian-splatting convention:
 *   mean      = R^T (d K^-1 [u v 1]^T - t)      (keypoint u, v at depth d)
 *   log-scale = log sqrt(mean squared distance to the 3 nearest other map
 *               points), the same on all three axes (mean squared distance
 *               floored at 1e-7 m^2; 1e-4 m^2 when the map has no other point)
 *   rotation  = identity, opacity logit = logit(0.1)
 *   SH        = DC (I(p) - 0.5) / Y_00 at the keypoint's nearest pixel p of
 *               the level-0 image, higher bands 0.
 * kp: M x 5 floats (u, v, depth, log keypoint scale, angle); cam: R (9),
 * t (3), fx, fy, cx, cy as floats; ref: the map's means (n_ref x 3 doubles),
 * of which entries offset .. offset + M - 1 are the new primitives and are
 * replaced by their back-projected means; each primitive's own entry is not
 * its neighbour.  Outputs are M x 3, M x 3, M x 4, M, M x 48 (coefficient-
 * major: 16 coefficients x RGB). */
int orc_default_init(const double *img, int W, int H, const float *kp, int64_t M, const float *cam,
                     const double *ref, int64_t n_ref, int64_t offset, double *mean, double *logscale, double *quat,
                     double *logit, double *sh) {
    if (M < 0 || n_ref < offset + M) return 1;
    double R[9], t[3];
    for (int k = 0; k < 9; ++k) R[k] = cam[k];
    for (int k = 0; k < 3; ++k) t[k] = cam[9 + k];
    const double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    for (int64_t m = 0; m < M; ++m) {
        const double u = kp[5 * m], v = kp[5 * m + 1], d = kp[5 * m + 2];
        const double pc[3] = {(u - cx) / fx * d - t[0], (v - cy) / fy * d - t[1], d - t[2]};
        for (int r = 0; r < 3; ++r) mean[3 * m + r] = R[r] * pc[0] + R[3 + r] * pc[1] + R[6 + r] * pc[2];
    }
    const double y00 = 0.5 / sqrt(M_PI);
    const double lg = log(0.1 / 0.9);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t m = 0; m < M; ++m) {
        double best[3] = {INFINITY, INFINITY, INFINITY};
        int found = 0;
        for (int64_t j = 0; j < n_ref; ++j) {
            if (j == offset + m) continue;
            const double *q = (j >= offset && j < offset + M) ? mean + 3 * (j - offset) : ref + 3 * j;
            const double dx = q[0] - mean[3 * m], dy = q[1] - mean[3 * m + 1], dz = q[2] - mean[3 * m + 2];
            const double d2 = dx * dx + dy * dy + dz * dz;
            ++found;
            if (d2 < best[2]) {
                best[2] = d2;
                if (best[2] < best[1]) { double s = best[1]; best[1] = best[2]; best[2] = s; }
                if (best[1] < best[0]) { double s = best[0]; best[0] = best[1]; best[1] = s; }
            }
        }
        const int k = found < 3 ? found : 3;
        double msd = 1e-4;
        if (k > 0) {
            msd = 0;
            for (int a = 0; a < k; ++a) msd += best[a];
            msd /= k;
            if (msd < 1e-7) msd = 1e-7;
        }
        const double ls = 0.5 * log(msd);
        for (int a = 0; a < 3; ++a) logscale[3 * m + a] = ls;
        quat[4 * m] = 1.0;
        quat[4 * m + 1] = quat[4 * m + 2] = quat[4 * m + 3] = 0.0;
        logit[m] = lg;
        /* nearest pixel: round half up, clamped to the image */
        const float uf = kp[5 * m], vf = kp[5 * m + 1];
        int px = (int)floor((double)uf) + ((double)uf - floor((double)uf) >= 0.5);
        int py = (int)floor((double)vf) + ((double)vf - floor((double)vf) >= 0.5);
        px = px < 0 ? 0 : (px > W - 1 ? W - 1 : px);
        py = py < 0 ? 0 : (py > H - 1 ? H - 1 : py);
        for (int c = 0; c < 48; ++c) sh[48 * m + c] = 0.0;
        for (int ch = 0; ch < 3; ++ch) sh[48 * m + ch] = (img[((int64_t)ch * H + py) * W + px] - 0.5) / y00;
    }
    return 0;
}

/* Gradient-driven densification and pruning of the map (Photo-SLAM Sec.
 * 3.3.1: split or clone primitives with large loss gradients, after 3D
 * Gaussian splatting; prune nearly transparent ones).  Decisions, per input
 * Gaussian i, on FP32 values:
 *   g_i = stat_i / count_i (0 if count_i = 0): the mean |dL/d(u, v)| in
 *         normalised device coordinates over the iterations that saw it;
 *   prune  when the opacity logit < logit_min (opacity below its sigmoid),
 *          and drop padding (a zero quaternion: an empty slot of the store);
 *   else densify when g_i >= grad_thr:
 *     split when its largest log-scale > logscale_split: two children,
 *           mean mu + R(q) (s * eps_k) (eps_k = eps[6 i + 3 k ..], s the
 *           scales), log-scale - shrink, the rest copied; the parent goes;
 *     clone otherwise: the Gaussian and a copy;
 *   else keep.
 * Outputs in input order (a clone: original first).  src[o] = input index,
 * kind[o] = 0 kept, 1 clone copy, 2 / 3 split child 0 / 1; mean_out and
 * logscale_out (o x 3) in FP64 (split means from FP64 arithmetic on the FP32
 * inputs).  Returns 1 if the outputs exceed cap. */
int orc_densify(int64_t n, const float *mean_op, const float *quat, const float *logscale, const float *stat,
                const float *count, const float *eps, float grad_thr, float logit_min, float logscale_split,
                float shrink, int64_t cap, int64_t *n_out, int64_t *src, int32_t *kind, double *mean_out,
                double *logscale_out) {
    int64_t o = 0;
    for (int64_t i = 0; i < n; ++i) {
        const float g = count[i] > 0.0f ? stat[i] / count[i] : 0.0f;
        const float *mo = mean_op + 4 * i, *q = quat + 4 * i, *ls = logscale + 4 * i;
        if (q[0] == 0.0f && q[1] == 0.0f && q[2] == 0.0f && q[3] == 0.0f) continue; /* padding */
        if (mo[3] < logit_min) continue;
        const int densify = g >= grad_thr;
        const float lmax = ls[0] > ls[1] ? (ls[0] > ls[2] ? ls[0] : ls[2]) : (ls[1] > ls[2] ? ls[1] : ls[2]);
        const int split = densify && lmax > logscale_split;
        const int outs = split || densify ? 2 : 1;
        if (o + outs > cap) return 1;
        if (!split) {
            for (int k = 0; k < outs; ++k, ++o) {
                src[o] = i;
                kind[o] = k;
                for (int c = 0; c < 3; ++c) {
                    mean_out[3 * o + c] = mo[c];
                    logscale_out[3 * o + c] = ls[c];
                }
            }
            continue;
        }
        /* rotation of the normalised quaternion (w, x, y, z) */
        const double nq = sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3]);
        const double w = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
        const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                             2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                             2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
        const double s[3] = {exp((double)ls[0]), exp((double)ls[1]), exp((double)ls[2])};
        for (int k = 0; k < 2; ++k, ++o) {
            const float *e = eps + 6 * i + 3 * k;
            src[o] = i;
            kind[o] = 2 + k;
            for (int r = 0; r < 3; ++r)
                mean_out[3 * o + r] = mo[r] + R[3 * r] * s[0] * e[0] + R[3 * r + 1] * s[1] * e[1] + R[3 * r + 2] * s[2] * e[2];
            for (int c = 0; c < 3; ++c) logscale_out[3 * o + c] = (double)(float)(ls[c] - shrink);
        }
    }
    *n_out = o;
    return 0;
}
