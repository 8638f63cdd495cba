// init.cu -- default initialisation of new primitives at keypoints.
//
// Photo-SLAM adds hyper primitives at inactive ORB keypoints (arXiv
// 2311.16728, Sec. 3.3.1, geometry-based densification) without saying how
// their shape is initialised.  This is the 3D-Gaussian-splatting convention,
// the fallback of the learned initialiser (mlp.cu):
//   mean      = R^T (d K^-1 [u v 1]^T - t)
//   log-scale = log sqrt(mean squared distance to the 3 nearest other map
//               points) on all three axes
//   rotation  = identity, opacity logit = logit(0.1)
//   SH DC     = (I(p) - 0.5) / Y_00 at the keypoint's nearest pixel, other
//               bands 0.
// The nearest-neighbour search is brute force over the whole map: the map is
// split into slices, each CTA keeps the 3 least squared distances of 128
// query points over one slice (slice staged through shared memory), and a
// second kernel merges the slices' candidates.
#include <algorithm>

#include "gsr_internal.cuh"

namespace gsr {

constexpr int kKnnThreads = 128;
constexpr int kKnnTile = 1024;        // map points per shared-memory tile
constexpr float kY00 = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
constexpr float kLogitTenth = -2.1972245773362196f;  // log(0.1 / 0.9)

struct CamI {
    float R[9], t[3], fx, fy, cx, cy;
};

__global__ void __launch_bounds__(128) init_fields_kernel(const float *__restrict__ img, int W, int H,
                                                          const float *__restrict__ kp, int64_t M, CamI cam,
                                                          float4 *__restrict__ mean_op, float4 *__restrict__ quat,
                                                          float4 *__restrict__ sh, int64_t n, int64_t off) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int64_t g = off + m;
    const float u = kp[5 * m], v = kp[5 * m + 1], d = kp[5 * m + 2];
    const float pc[3] = {(u - cam.cx) / cam.fx * d - cam.t[0], (v - cam.cy) / cam.fy * d - cam.t[1], d - cam.t[2]};
    const float *R = cam.R;  // mean = R^T (p_cam - t)
    mean_op[g] = make_float4(R[0] * pc[0] + R[3] * pc[1] + R[6] * pc[2], R[1] * pc[0] + R[4] * pc[1] + R[7] * pc[2],
                             R[2] * pc[0] + R[5] * pc[1] + R[8] * pc[2], kLogitTenth);
    quat[g] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    // nearest pixel, half up (u - floor(u) is exact), clamped to the image
    const float fu = floorf(u), fv = floorf(v);
    int px = (int)fu + ((u - fu) >= 0.5f ? 1 : 0), py = (int)fv + ((v - fv) >= 0.5f ? 1 : 0);
    px = min(max(px, 0), W - 1);
    py = min(max(py, 0), H - 1);
    const int64_t plane = (int64_t)W * H, pix = (int64_t)py * W + px;
    const float r = (img[pix] - 0.5f) / kY00, gr = (img[plane + pix] - 0.5f) / kY00,
                b = (img[2 * plane + pix] - 0.5f) / kY00;
    // coefficient-major planes: plane 0 = (c0 r, c0 g, c0 b, c1 r)
    sh[g] = make_float4(r, gr, b, 0.0f);
    for (int p = 1; p < kShPlanes; ++p) sh[(int64_t)p * n + g] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ void keep3(float d2, float &b0, float &b1, float &b2) {
    if (d2 < b2) {
        b2 = d2;
        if (b2 < b1) {
            const float s = b1;
            b1 = b2;
            b2 = s;
        }
        if (b1 < b0) {
            const float s = b0;
            b0 = b1;
            b1 = s;
        }
    }
}

// blockIdx.x: 128 query points; blockIdx.y: map slice [y * slice, (y + 1) * slice)
__global__ void __launch_bounds__(kKnnThreads) knn_partial_kernel(const float4 *__restrict__ mean_op, int64_t n,
                                                                  int64_t off, int64_t M, int64_t slice,
                                                                  float *__restrict__ part) {
    __shared__ float4 s_pts[kKnnTile];
    const int64_t q = (int64_t)blockIdx.x * kKnnThreads + threadIdx.x;
    const int64_t self = off + q;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < M) p = mean_op[self];
    float b0 = INFINITY, b1 = INFINITY, b2 = INFINITY;
    const int64_t j0 = (int64_t)blockIdx.y * slice, j1 = min(n, j0 + slice);
    for (int64_t t0 = j0; t0 < j1; t0 += kKnnTile) {
        const int cnt = (int)min((int64_t)kKnnTile, j1 - t0);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kKnnThreads) s_pts[k] = mean_op[t0 + k];
        __syncthreads();
        const int skip = (self >= t0 && self < t0 + cnt) ? (int)(self - t0) : -1;
        for (int k = 0; k < cnt; ++k) {
            const float4 o = s_pts[k];
            const float dx = o.x - p.x, dy = o.y - p.y, dz = o.z - p.z;
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (k != skip) keep3(d2, b0, b1, b2);
        }
    }
    if (q < M) {
        float *o = part + ((int64_t)q * gridDim.y + blockIdx.y) * 3;
        o[0] = b0;
        o[1] = b1;
        o[2] = b2;
    }
}

__global__ void __launch_bounds__(128) knn_merge_kernel(const float *__restrict__ part, int slices, int64_t M,
                                                        float4 *__restrict__ logscale, int64_t off) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= M) return;
    float b0 = INFINITY, b1 = INFINITY, b2 = INFINITY;
    const float *c = part + q * slices * 3;
    for (int k = 0; k < 3 * slices; ++k) keep3(c[k], b0, b1, b2);
    float sum = 0.f;
    int cnt = 0;
    if (b0 < INFINITY) { sum += b0; ++cnt; }
    if (b1 < INFINITY) { sum += b1; ++cnt; }
    if (b2 < INFINITY) { sum += b2; ++cnt; }
    float msd = 1e-4f;  // no other map point: 1 cm
    if (cnt > 0) msd = fmaxf(sum / (float)cnt, 1e-7f);
    const float ls = 0.5f * logf(msd);
    logscale[off + q] = make_float4(ls, ls, ls, 0.0f);
}

static int knn_slices(int64_t M, int64_t n) {
    if (M <= 0) return 1;
    const int64_t qb = (M + kKnnThreads - 1) / kKnnThreads;
    int64_t s = (4 * 148 + qb - 1) / qb;  // about four CTAs per SM
    s = std::max<int64_t>(1, std::min<int64_t>(s, 64));
    s = std::min<int64_t>(s, std::max<int64_t>(1, n / kKnnTile));
    return (int)s;
}

}  // namespace gsr

using namespace gsr;

extern "C" int32_t gsr_default_init_workspace_size(int64_t M, int64_t n, size_t *bytes) {
    if (M < 0 || n < 0 || !bytes) {
        set_error("gsr_default_init_workspace_size: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    *bytes = (size_t)M * knn_slices(M, n) * 3 * sizeof(float) + 256;
    return GSR_OK;
}

extern "C" int32_t gsr_default_init(const float *img0, int32_t W, int32_t H, const float *keypoints, int64_t M,
                                    const gsr_camera *cam, const gsr_param_buffers *map, int64_t n, int64_t offset,
                                    void *workspace, size_t workspace_bytes, gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_camera(cam))) return rc;
    if (M < 0 || W <= 0 || H <= 0 || !map || !map->mean_op || !map->quat || !map->logscale || !map->sh ||
        offset < 0 || offset + M > n || (M > 0 && (!img0 || !keypoints))) {
        set_error("gsr_default_init: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    if (!aligned16(map->mean_op) || !aligned16(map->quat) || !aligned16(map->logscale) || !aligned16(map->sh)) {
        set_error("gsr_default_init: parameter planes must be 16-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    if (M == 0) return GSR_OK;
    size_t need;
    gsr_default_init_workspace_size(M, n, &need);
    if (!workspace || workspace_bytes < need) {
        set_error("gsr_default_init: workspace of %zu bytes needed", need);
        return GSR_ERR_CAPACITY;
    }
    if (M > (int64_t)0x7fffffff * kKnnThreads) {
        set_error("gsr_default_init: too many keypoints");
        return GSR_ERR_UNSUPPORTED;
    }
    CamI c;
    for (int i = 0; i < 9; ++i) c.R[i] = cam->R[i];
    for (int i = 0; i < 3; ++i) c.t[i] = cam->t[i];
    c.fx = cam->fx;
    c.fy = cam->fy;
    c.cx = cam->cx;
    c.cy = cam->cy;
    cudaStream_t st = as_cuda(stream);
    float4 *mo = reinterpret_cast<float4 *>(map->mean_op);
    init_fields_kernel<<<(unsigned)((M + 127) / 128), 128, 0, st>>>(img0, W, H, keypoints, M, c, mo,
                                                                  reinterpret_cast<float4 *>(map->quat),
                                                                  reinterpret_cast<float4 *>(map->sh), n, offset);
    if ((rc = check_launch("init_fields_kernel"))) return rc;
    const int S = knn_slices(M, n);
    const int64_t slice = (n + S - 1) / S;
    float *part = static_cast<float *>(workspace);
    knn_partial_kernel<<<dim3((unsigned)((M + kKnnThreads - 1) / kKnnThreads), (unsigned)S), kKnnThreads, 0, st>>>(
        mo, n, offset, M, slice, part);
    if ((rc = check_launch("knn_partial_kernel"))) return rc;
    knn_merge_kernel<<<(unsigned)((M + 127) / 128), 128, 0, st>>>(part, S, M,
                                                                  reinterpret_cast<float4 *>(map->logscale), offset);
    return check_launch("knn_merge_kernel");
}
