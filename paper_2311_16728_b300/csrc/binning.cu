// binning.cu -- tile binning for the tile-based renderer of Photo-SLAM
// (arXiv 2311.16728) Sec. 3.3: one (key, Gaussian) pair per tile a
// Gaussian's pixel box touches, key = tile << 32 | bits(depth), sorted by an
// in-house stable LSD radix sort, then per-tile [begin, end) ranges.
//
// The pair count is data dependent; every kernel reads it from device memory
// (clamped to the caller's capacity) so the whole sequence can be captured
// in a CUDA graph with fixed launch shapes.
#include "gsr_internal.cuh"

namespace gsr {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;  // Gaussians per thread in the scan / emit kernels
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;  // pairs per thread per block tile
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

__device__ __forceinline__ int64_t clamp_count(const int64_t *d_count, int64_t cap) {
    const int64_t c = *d_count;
    return c < cap ? c : cap;
}

// inclusive block-wide scan of one u32 per thread (256 threads)
__device__ __forceinline__ uint32_t block_incl_scan_256(uint32_t v, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < 8 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < 8) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t add = wid > 0 ? s_warp[wid - 1] : 0u;
    __syncthreads();
    return v + add;
}

// ---------------------------------------------------------------- K2: scan + emit
__global__ void __launch_bounds__(kScanThreads) tiles_reduce_kernel(const uint32_t *__restrict__ ntiles, int64_t n,
                                                                    uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t s_warp[8];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += ntiles[base + k];
    s = block_incl_scan_256(s, s_warp);
    if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = s;
}

// one block: exclusive scan of the per-block sums (64-bit), total -> *d_num_pairs
__global__ void __launch_bounds__(1024) tiles_scan_blocks_kernel(const uint32_t *__restrict__ block_sums,
                                                                 int64_t nblocks, int64_t *__restrict__ block_offsets,
                                                                 int64_t *__restrict__ d_num_pairs, int64_t cap,
                                                                 int32_t *__restrict__ d_status) {
    __shared__ int64_t s_part[1024];
    const int t = threadIdx.x;
    const int64_t per = (nblocks + 1023) / 1024;
    const int64_t b0 = t * per;
    int64_t s = 0;
    for (int64_t k = 0; k < per; ++k)
        if (b0 + k < nblocks) s += block_sums[b0 + k];
    s_part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int64_t v = t >= o ? s_part[t - o] : 0;
        __syncthreads();
        s_part[t] += v;
        __syncthreads();
    }
    int64_t run = s_part[t] - s;  // exclusive prefix of this thread's chunk
    for (int64_t k = 0; k < per; ++k)
        if (b0 + k < nblocks) {
            block_offsets[b0 + k] = run;
            run += block_sums[b0 + k];
        }
    if (t == 1023) {
        const int64_t total = s_part[1023];
        *d_num_pairs = total;
        if (total > cap) raise_status(d_status, GSR_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(kScanThreads) emit_pairs_kernel(
    const uint32_t *__restrict__ ntiles, const float4 *__restrict__ c_op_box, const float4 *__restrict__ rgb_depth,
    int64_t n, const int64_t *__restrict__ block_offsets, int tw, int th, int gx, int64_t cap,
    uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    __shared__ uint32_t s_warp[8];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t cnt[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        cnt[k] = (base + k < n) ? ntiles[base + k] : 0u;
        s += cnt[k];
    }
    const uint32_t incl = block_incl_scan_256(s, s_warp);
    int64_t off = block_offsets[blockIdx.x] + (int64_t)(incl - s);
#pragma unroll 1
    for (int k = 0; k < kScanItems; ++k) {
        if (cnt[k] == 0u) continue;
        const int64_t i = base + k;
        const float4 cb = __ldg(c_op_box + i);
        const uint32_t bx = __float_as_uint(cb.z), by = __float_as_uint(cb.w);
        const int tx0 = (int)(bx & 0xffffu) / tw, tx1 = (int)(bx >> 16) / tw;
        const int ty0 = (int)(by & 0xffffu) / th, ty1 = (int)(by >> 16) / th;
        const uint32_t dbits = __float_as_uint(__ldg(&rgb_depth[i].w));
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                if (off < cap) {
                    keys[off] = ((uint64_t)(uint32_t)(ty * gx + tx) << 32) | dbits;
                    vals[off] = (uint32_t)i;
                }
                ++off;
            }
    }
}

// ---------------------------------------------------------------- K3: radix sort
// One pass = histogram of the digit per block tile, per-digit scan over
// blocks, then a stable scatter (warp match_any ranks, warps in order).
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t *__restrict__ keys,
                                                                  const int64_t *__restrict__ d_count, int64_t cap,
                                                                  int shift, int nblocks,
                                                                  uint32_t *__restrict__ hist) {
    __shared__ uint32_t s_hist[kRadix];
    s_hist[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t count = clamp_count(d_count, cap);
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int k = 0; k < kSortItems; ++k) {
        const int64_t idx = base + (int64_t)k * kSortThreads + threadIdx.x;
        if (idx < count) atomicAdd(&s_hist[(uint32_t)(keys[idx] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_hist[threadIdx.x];
}

// grid = 256 blocks (one per digit): exclusive scan over blocks, digit total
__global__ void __launch_bounds__(256) radix_digit_scan_kernel(uint32_t *__restrict__ hist, int nblocks,
                                                               uint32_t *__restrict__ digit_total) {
    __shared__ uint32_t s_warp[8];
    uint32_t *row = hist + (int64_t)blockIdx.x * nblocks;
    const int per = (nblocks + 255) / 256;
    const int b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nblocks) s += row[b0 + k];
    const uint32_t incl = block_incl_scan_256(s, s_warp);
    uint32_t run = incl - s;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nblocks) {
            const uint32_t v = row[b0 + k];
            row[b0 + k] = run;
            run += v;
        }
    if (threadIdx.x == 255) digit_total[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(
    const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, uint64_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, const int64_t *__restrict__ d_count, int64_t cap, int shift, int nblocks,
    const uint32_t *__restrict__ hist, const uint32_t *__restrict__ digit_total) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t s_base[kRadix];            // running output position per digit
    __shared__ uint32_t s_wcount[kWarps][kRadix];  // per-warp digit counts of one sub-tile
    __shared__ uint32_t s_warp[8];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int64_t count = clamp_count(d_count, cap);
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    if (base >= count) return;
    {
        const uint32_t tot = digit_total[t];
        const uint32_t incl = block_incl_scan_256(tot, s_warp);
        s_base[t] = (incl - tot) + hist[(int64_t)t * nblocks + blockIdx.x];
    }
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s_wcount[w][t] = 0u;
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll 1
    for (int k = 0; k < kSortItems; ++k) {
        const int64_t idx = base + (int64_t)k * kSortThreads + t;
        const bool valid = idx < count;
        uint64_t key = 0;
        uint32_t val = 0, d = kRadix;  // sentinel digit for the tail
        if (valid) {
            key = keys_in[idx];
            val = vals_in[idx];
            d = (uint32_t)(key >> shift) & (kRadix - 1);
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) s_wcount[wid][d] = __popc(peers);
        __syncthreads();
        // digit t: exclusive prefix over warps, advance the running base
        uint32_t run = s_base[t];
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = s_wcount[w][t];
            s_wcount[w][t] = run;
            run += c;
        }
        s_base[t] = run;
        __syncthreads();
        if (valid) {
            const uint32_t pos = s_wcount[wid][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s_wcount[w][t] = 0u;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- K4: tile ranges
__global__ void __launch_bounds__(256) tile_ranges_kernel(const uint64_t *__restrict__ keys,
                                                          const int64_t *__restrict__ d_count, int64_t cap,
                                                          uint2 *__restrict__ ranges) {
    const int64_t count = clamp_count(d_count, cap);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint32_t tile = (uint32_t)(keys[i] >> 32);
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != tile) ranges[tile].x = (uint32_t)i;
    if (i == count - 1 || (uint32_t)(keys[i + 1] >> 32) != tile) ranges[tile].y = (uint32_t)(i + 1);
}

// ---------------------------------------------------------------- host side
static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct SortLayout {
    size_t keys_alt, vals_alt, block_sums, block_offsets, hist, digit_total, total;
    int64_t scan_blocks, sort_blocks;
};

static SortLayout sort_layout(int64_t n, int64_t cap) {
    SortLayout L;
    L.scan_blocks = (n + kScanTile - 1) / kScanTile;
    L.sort_blocks = (cap + kSortTile - 1) / kSortTile;
    size_t off = 0;
    L.keys_alt = off; off += align256(sizeof(uint64_t) * (size_t)(cap > 0 ? cap : 1));
    L.vals_alt = off; off += align256(sizeof(uint32_t) * (size_t)(cap > 0 ? cap : 1));
    L.block_sums = off; off += align256(sizeof(uint32_t) * (size_t)(L.scan_blocks > 0 ? L.scan_blocks : 1));
    L.block_offsets = off; off += align256(sizeof(int64_t) * (size_t)(L.scan_blocks > 0 ? L.scan_blocks : 1));
    L.hist = off; off += align256(sizeof(uint32_t) * kRadix * (size_t)(L.sort_blocks > 0 ? L.sort_blocks : 1));
    L.digit_total = off; off += align256(sizeof(uint32_t) * kRadix);
    L.total = off;
    return L;
}

static int radix_passes(int64_t tiles) {
    int bits = 0;
    while ((int64_t(1) << bits) < tiles) ++bits;
    return (32 + bits + kRadixBits - 1) / kRadixBits;
}

// Sort (keys, vals) of *d_count pairs in place on 64-bit keys over `passes`
// 8-bit digits.  The data start in the buffer pair selected by `start_in_alt`
// and end in (keys, vals).
static int32_t radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                                const int64_t *d_count, int64_t cap, int passes, uint32_t *hist,
                                uint32_t *digit_total, int nblocks, cudaStream_t st) {
    uint64_t *kin = (passes & 1) ? keys_alt : keys, *kout = (passes & 1) ? keys : keys_alt;
    uint32_t *vin = (passes & 1) ? vals_alt : vals, *vout = (passes & 1) ? vals : vals_alt;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * kRadixBits;
        radix_hist_kernel<<<nblocks, kSortThreads, 0, st>>>(kin, d_count, cap, shift, nblocks, hist);
        radix_digit_scan_kernel<<<kRadix, 256, 0, st>>>(hist, nblocks, digit_total);
        radix_scatter_kernel<<<nblocks, kSortThreads, 0, st>>>(kin, vin, kout, vout, d_count, cap, shift, nblocks,
                                                               hist, digit_total);
        uint64_t *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
    }
    return check_launch("radix sort");
}

}  // namespace gsr

using namespace gsr;

extern "C" int32_t gsr_bin_sort_workspace_size(int64_t n, int64_t pair_capacity, const gsr_camera *cam,
                                               const gsr_tiling *tiling, size_t *bytes) {
    if (n < 0 || pair_capacity < 0 || !bytes) {
        set_error("gsr_bin_sort_workspace_size: bad arguments");
        return GSR_ERR_INVALID_ARG;
    }
    (void)cam;
    (void)tiling;
    *bytes = sort_layout(n, pair_capacity).total;
    return GSR_OK;
}

extern "C" int32_t gsr_bin_sort(const gsr_proj *proj, int64_t n, const gsr_camera *cam, const gsr_tiling *tiling,
                                uint64_t *keys, uint32_t *vals, int64_t pair_capacity, uint32_t *tile_ranges,
                                int64_t *d_num_pairs, void *workspace, size_t workspace_bytes, int32_t *d_status,
                                gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_camera(cam)) || (rc = validate_tiling(tiling))) return rc;
    if (!proj || (n > 0 && (!proj->ntiles || !proj->c_op_box || !proj->rgb_depth)) || n < 0 || pair_capacity < 0 ||
        !tile_ranges || !d_num_pairs || (pair_capacity > 0 && (!keys || !vals))) {
        set_error("gsr_bin_sort: NULL pointer or negative size");
        return GSR_ERR_INVALID_ARG;
    }
    if (n > 0xffffffffLL || pair_capacity > 0xffffffffLL) {
        set_error("gsr_bin_sort: n and pair_capacity must fit in 32 bits");
        return GSR_ERR_UNSUPPORTED;
    }
    const SortLayout L = sort_layout(n, pair_capacity);
    if (!workspace || workspace_bytes < L.total) {
        set_error("gsr_bin_sort: workspace of %zu bytes needed, %zu given", L.total, workspace_bytes);
        return GSR_ERR_CAPACITY;
    }
    cudaStream_t st = as_cuda(stream);
    char *ws = static_cast<char *>(workspace);
    uint64_t *keys_alt = reinterpret_cast<uint64_t *>(ws + L.keys_alt);
    uint32_t *vals_alt = reinterpret_cast<uint32_t *>(ws + L.vals_alt);
    uint32_t *block_sums = reinterpret_cast<uint32_t *>(ws + L.block_sums);
    int64_t *block_offsets = reinterpret_cast<int64_t *>(ws + L.block_offsets);
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + L.hist);
    uint32_t *digit_total = reinterpret_cast<uint32_t *>(ws + L.digit_total);
    const int gx = grid_x(cam, tiling), gy = grid_y(cam, tiling);
    const int64_t tiles = (int64_t)gx * gy;
    if (cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)tiles, st) != cudaSuccess)
        return check_launch("memset tile ranges");
    if (n == 0) {
        if (cudaMemsetAsync(d_num_pairs, 0, sizeof(int64_t), st) != cudaSuccess)
            return check_launch("memset pair count");
        return GSR_OK;
    }
    const int passes = radix_passes(tiles);
    // emit into the buffer that makes the last pass land in (keys, vals)
    uint64_t *emit_k = (passes & 1) ? keys_alt : keys;
    uint32_t *emit_v = (passes & 1) ? vals_alt : vals;
    const int64_t sb = L.scan_blocks;
    tiles_reduce_kernel<<<(unsigned)sb, kScanThreads, 0, st>>>(proj->ntiles, n, block_sums);
    tiles_scan_blocks_kernel<<<1, 1024, 0, st>>>(block_sums, sb, block_offsets, d_num_pairs, pair_capacity,
                                                 d_status);
    emit_pairs_kernel<<<(unsigned)sb, kScanThreads, 0, st>>>(
        proj->ntiles, reinterpret_cast<const float4 *>(proj->c_op_box),
        reinterpret_cast<const float4 *>(proj->rgb_depth), n, block_offsets, tiling->tile_w, tiling->tile_h, gx,
        pair_capacity, emit_k, emit_v);
    if ((rc = check_launch("emit pairs"))) return rc;
    if (pair_capacity == 0) return GSR_OK;
    if ((rc = radix_sort_pairs(keys, vals, keys_alt, vals_alt, d_num_pairs, pair_capacity, passes, hist, digit_total,
                               (int)L.sort_blocks, st)))
        return rc;
    const unsigned rb = (unsigned)((pair_capacity + 255) / 256);
    tile_ranges_kernel<<<rb, 256, 0, st>>>(keys, d_num_pairs, pair_capacity, reinterpret_cast<uint2 *>(tile_ranges));
    return check_launch("tile_ranges_kernel");
}
