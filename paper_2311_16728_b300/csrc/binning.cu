// binning.cu -- tile binning for the tile-based renderer of Photo-SLAM
// (arXiv 2311.16728) Sec. 3.3: one (tile, Gaussian) pair per kept tile of a
// Gaussian's pixel box, ordered by the 64-bit key tile << 32 | bits(depth)
// (ties by Gaussian index), plus per-tile [begin, end) ranges.
//
// The order is produced by an in-house stable LSD radix sort in two stages
// that together sort the full 64-bit key:
//   1. the ~10^5 visible Gaussians are sorted once by their 32 depth bits
//      (4 passes of 8 bits over N_visible, not over the pairs);
//   2. their box tiles are expanded in that depth order, culled (see
//      tile_keep) and compacted, and the pairs are stably sorted by the tile
//      bits only (ceil(log2 tiles) bits, one or two passes over the pairs).
// Stable passes over the low 32 bits followed by stable passes over the high
// bits are exactly an LSD sort of the 64-bit key; doing the low passes
// before duplication sorts 10^5 items instead of 10^6.
//
// Counts are data dependent: every kernel reads them from device memory
// (clamped to capacity) so the whole sequence has fixed launch shapes and can
// be captured in a CUDA graph.
#include "gsr_internal.cuh"

namespace gsr {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;  // Gaussians per thread in the scan / compaction / emit kernels
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kSortThreads = 256;
constexpr int kSortItems = 4;   // elements per thread per block tile (short per-block chains)
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 256;     // bins of one pass (a pass uses at most 8 bits)

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

// Sum of block_sums[0 .. b) (the exclusive prefix of block b) and, when
// `total` is not NULL, of all of them.  Block-cooperative; few hundred blocks.
__device__ __forceinline__ int64_t block_prefix(const uint32_t *block_sums, int64_t nblocks, int64_t b,
                                                int64_t *total, int64_t *s_red) {
    int64_t pre = 0, all = 0;
    for (int64_t k = threadIdx.x; k < nblocks; k += kScanThreads) {
        const uint32_t v = block_sums[k];
        all += v;
        if (k < b) pre += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pre += __shfl_xor_sync(0xffffffffu, pre, o);
        all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_red[wid] = pre;
        s_red[8 + wid] = all;
    }
    __syncthreads();
    int64_t p = 0, a = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        p += s_red[w];
        a += s_red[8 + w];
    }
    __syncthreads();
    if (total) *total = a;
    return p;
}

// ---------------------------------------------------------------- visible compaction
__global__ void __launch_bounds__(kScanThreads) vis_count_kernel(const uint32_t *__restrict__ ntiles, int64_t n,
                                                                 uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t s_warp[8];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += ntiles[base + k] > 0u ? 1u : 0u;
    s = block_incl_scan_256(s, s_warp);
    if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = s;
}

// visible Gaussians in index order -> (depth bits, index), count -> *d_nvis
__global__ void __launch_bounds__(kScanThreads) vis_compact_kernel(
    const uint32_t *__restrict__ ntiles, const float4 *__restrict__ rgb_depth, int64_t n,
    const uint32_t *__restrict__ block_sums, int64_t nblocks, uint32_t *__restrict__ dkey,
    uint32_t *__restrict__ dval, int64_t *__restrict__ d_nvis) {
    __shared__ uint32_t s_warp[8];
    __shared__ int64_t s_red[16];
    int64_t total;
    const int64_t pre = block_prefix(block_sums, nblocks, blockIdx.x, &total, s_red);
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_nvis = total;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    bool vis[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        vis[k] = base + k < n && ntiles[base + k] > 0u;
        s += vis[k] ? 1u : 0u;
    }
    const uint32_t incl = block_incl_scan_256(s, s_warp);
    int64_t pos = pre + (int64_t)(incl - s);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (vis[k]) {
            dkey[pos] = __float_as_uint(__ldg(&rgb_depth[base + k].w));
            dval[pos] = (uint32_t)(base + k);
            ++pos;
        }
}

// ---------------------------------------------------------------- pair expansion
// Candidates are the (Gaussian, box tile) slots of the depth-ordered visible
// list.  One thread per candidate runs the tile cull, so a few near-camera
// Gaussians with thousands of box tiles spread over the whole GPU instead of
// serialising in the warps that hold them; an ordered compaction of the kept
// candidates then yields the pairs in depth order (row-major within a box).
__global__ void __launch_bounds__(kScanThreads) cand_count_kernel(const uint32_t *__restrict__ ntiles,
                                                                  const uint32_t *__restrict__ order,
                                                                  const int64_t *__restrict__ d_nvis, int64_t cap_n,
                                                                  uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t s_warp[8];
    const int64_t nv = clamp_count(d_nvis, cap_n);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < nv) s += ntiles[order[base + k]];
    s = block_incl_scan_256(s, s_warp);
    if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = s;
}

// coff[i] = first candidate slot of item i; coff[nv] = *d_ncand = total.  If
// the candidates exceed their capacity, the GSR_ERR_CAPACITY bit is set and
// *d_num_pairs receives the candidate count (an upper bound on the pairs).
__global__ void __launch_bounds__(kScanThreads) cand_offsets_kernel(
    const uint32_t *__restrict__ ntiles, const uint32_t *__restrict__ order, const int64_t *__restrict__ d_nvis,
    int64_t cap_n, const uint32_t *__restrict__ block_sums, int64_t nblocks, int64_t cand_cap,
    uint32_t *__restrict__ coff, int64_t *__restrict__ d_ncand, int64_t *__restrict__ d_num_pairs,
    int32_t *__restrict__ d_status) {
    __shared__ uint32_t s_warp[8];
    __shared__ int64_t s_red[16];
    int64_t total;
    const int64_t pre = block_prefix(block_sums, nblocks, blockIdx.x, &total, s_red);
    const int64_t nv = clamp_count(d_nvis, cap_n);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *d_ncand = total;
        coff[nv] = (uint32_t)total;
        if (total > cand_cap) {
            *d_num_pairs = total;
            raise_status(d_status, GSR_ERR_CAPACITY);
        }
    }
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t cnt[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        cnt[k] = base + k < nv ? ntiles[order[base + k]] : 0u;
        s += cnt[k];
    }
    const uint32_t incl = block_incl_scan_256(s, s_warp);
    int64_t off = pre + (int64_t)(incl - s);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < nv) {
            coff[base + k] = (uint32_t)off;
            off += cnt[k];
        }
}

constexpr int kExpandThreads = 256;
constexpr int kExpandItems = 4;
constexpr int kExpandTile = kExpandThreads * kExpandItems;

// largest i in [0, n) with a[i] <= x (a ascending, a[0] <= x), by one warp
__device__ __forceinline__ int64_t warp_upper_index(const uint32_t *a, int64_t n, uint32_t x) {
    int64_t lo = 0, hi = n;  // answer in [lo, hi)
    const int lane = threadIdx.x & 31;
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t probe = lo + (int64_t)lane * step;
        const bool le = probe < hi && a[probe] <= x;
        const uint32_t m = __ballot_sync(0xffffffffu, le);
        const int last = 31 - __clz(m);  // highest lane whose probe is <= x (lane 0 always is)
        const int64_t nlo = lo + (int64_t)last * step;
        hi = nlo + step < hi ? nlo + step : hi;
        lo = nlo;
    }
    return lo;
}

__global__ void __launch_bounds__(kExpandThreads) expand_kernel(
    const uint32_t *__restrict__ coff, const uint32_t *__restrict__ order, const float4 *__restrict__ xy_conic,
    const float4 *__restrict__ c_op_box, const int64_t *__restrict__ d_nvis, int64_t cap_n,
    const int64_t *__restrict__ d_ncand, int64_t cand_cap, int tw, int th, const ViewTiles vt,
    uint8_t *__restrict__ flag, uint32_t *__restrict__ ctile, uint32_t *__restrict__ cgid) {
    __shared__ uint32_t s_off[kExpandTile + 1];
    __shared__ int64_t s_i0;
    __shared__ int s_m;
    const int64_t ncand = clamp_count(d_ncand, cand_cap);
    const int64_t nv = clamp_count(d_nvis, cap_n);
    const int64_t s0 = (int64_t)blockIdx.x * kExpandTile;
    if (s0 >= ncand) return;
    const int64_t s_last = (s0 + kExpandTile < ncand ? s0 + kExpandTile : ncand) - 1;
    if (threadIdx.x < 32) {
        const int64_t i0 = warp_upper_index(coff, nv, (uint32_t)s0);
        const int64_t i1 = warp_upper_index(coff, nv, (uint32_t)s_last);
        if (threadIdx.x == 0) {
            s_i0 = i0;
            s_m = (int)(i1 - i0 + 1);  // every item owns >= 1 slot, so m <= kExpandTile
        }
    }
    __syncthreads();
    const int64_t i0 = s_i0;
    const int m = s_m;
    for (int j = threadIdx.x; j <= m; j += kExpandThreads) s_off[j] = coff[i0 + j];
    __syncthreads();
#pragma unroll 1
    for (int r = 0; r < kExpandItems; ++r) {
        const int64_t slot = s0 + (int64_t)r * kExpandThreads + threadIdx.x;
        if (slot >= ncand) break;
        int lo = 0, hi = m;  // s_off[lo] <= slot < s_off[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] <= (uint32_t)slot) lo = mid;
            else hi = mid;
        }
        const uint32_t gid = order[i0 + lo];
        const int k = (int)((uint32_t)slot - s_off[lo]);
        const Splat sp = load_splat(xy_conic, c_op_box, gid);
        const int tx0 = sp.x0 / tw, ntx = sp.x1 / tw - tx0 + 1;
        const int tx = tx0 + k % ntx, ty = sp.y0 / th + k / ntx;
        flag[slot] = tile_keep_at(tx, ty, tw, th, sp.u, sp.v, sp.A, sp.B, sp.C, sp.op, sp.x0, sp.x1, sp.y0, sp.y1)
                         ? 1
                         : 0;
        const int v = (int)((int64_t)gid / vt.n_per_view);  // view of this record
        ctile[slot] = vt.toff[v] + (uint32_t)(ty * vt.gx[v] + tx);
        cgid[slot] = gid;
    }
}

__global__ void __launch_bounds__(kScanThreads) kept_count_kernel(const uint8_t *__restrict__ flag,
                                                                  const int64_t *__restrict__ d_ncand,
                                                                  int64_t cand_cap,
                                                                  uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t s_warp[8];
    const int64_t nc = clamp_count(d_ncand, cand_cap);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < nc) s += flag[base + k];
    s = block_incl_scan_256(s, s_warp);
    if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kScanThreads) kept_compact_kernel(
    const uint8_t *__restrict__ flag, const uint32_t *__restrict__ ctile, const uint32_t *__restrict__ cgid,
    const int64_t *__restrict__ d_ncand, int64_t cand_cap, const uint32_t *__restrict__ block_sums,
    int64_t nblocks, int64_t cap, uint32_t *__restrict__ tkey, uint32_t *__restrict__ tval,
    int64_t *__restrict__ d_num_pairs, int64_t *__restrict__ d_written, int32_t *__restrict__ d_status) {
    __shared__ uint32_t s_warp[8];
    __shared__ int64_t s_red[16];
    int64_t total;
    const int64_t pre = block_prefix(block_sums, nblocks, blockIdx.x, &total, s_red);
    const int64_t nc_raw = *d_ncand;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // pairs actually present for the sort, whatever overflowed upstream
        *d_written = total < cap ? total : cap;
        if (nc_raw <= cand_cap) {
            *d_num_pairs = total;
            if (total > cap) raise_status(d_status, GSR_ERR_CAPACITY);
        }
    }
    const int64_t nc = nc_raw < cand_cap ? nc_raw : cand_cap;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
    uint8_t f[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        f[k] = base + k < nc ? flag[base + k] : 0;
        s += f[k];
    }
    const uint32_t incl = block_incl_scan_256(s, s_warp);
    int64_t pos = pre + (int64_t)(incl - s);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (f[k]) {
            if (pos < cap) {
                tkey[pos] = ctile[base + k];
                tval[pos] = cgid[base + k];
            }
            ++pos;
        }
}

// ---------------------------------------------------------------- radix sort passes
// One stable pass on u32 keys (digit = (key >> shift) & mask, <= 8 bits) with
// u32 values: per-block digit histogram, per-digit scan over blocks, scatter
// (warp match_any ranks, warps in order).
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint32_t *__restrict__ keys,
                                                                  const int64_t *__restrict__ d_count, int64_t cap,
                                                                  int shift, uint32_t mask, int nblocks,
                                                                  uint32_t *__restrict__ hist) {
    __shared__ uint32_t s_hist[kRadix];
    s_hist[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t count = clamp_count(d_count, cap);
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const uint32_t lane_lt = (1u << (threadIdx.x & 31)) - 1u;
#pragma unroll 4
    for (int k = 0; k < kSortItems; ++k) {
        const int64_t idx = base + (int64_t)k * kSortThreads + threadIdx.x;
        const bool valid = idx < count;
        const uint32_t d = valid ? (keys[idx] >> shift) & mask : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & lane_lt) == 0u) atomicAdd(&s_hist[d], (uint32_t)__popc(peers));
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
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, uint32_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, const int64_t *__restrict__ d_count, int64_t cap, int shift, uint32_t mask,
    int nblocks, const uint32_t *__restrict__ hist, const uint32_t *__restrict__ digit_total) {
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
        if (base + (int64_t)k * kSortThreads >= count) break;  // block-uniform
        const int64_t idx = base + (int64_t)k * kSortThreads + t;
        const bool valid = idx < count;
        uint32_t key = 0, val = 0, d = kRadix;  // sentinel digit for the tail
        if (valid) {
            key = keys_in[idx];
            val = vals_in[idx];
            d = (key >> shift) & mask;
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) s_wcount[wid][d] = __popc(peers);
        __syncthreads();
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

// ---------------------------------------------------------------- ranges + 64-bit keys
__global__ void __launch_bounds__(256) finalize_kernel(const uint32_t *__restrict__ tkey,
                                                       const uint32_t *__restrict__ vals,
                                                       const float4 *__restrict__ rgb_depth,
                                                       const int64_t *__restrict__ d_count, int64_t cap,
                                                       uint32_t ntiles_total, uint64_t *__restrict__ keys,
                                                       uint2 *__restrict__ ranges) {
    const int64_t count = clamp_count(d_count, cap);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint32_t tile = tkey[i];
    if (tile >= ntiles_total) return;  // cannot happen for emitted pairs; keeps every write in bounds
    keys[i] = ((uint64_t)tile << 32) | __float_as_uint(__ldg(&rgb_depth[vals[i]].w));
    if (i == 0 || tkey[i - 1] != tile) ranges[tile].x = (uint32_t)i;
    if (i == count - 1 || tkey[i + 1] != tile) ranges[tile].y = (uint32_t)(i + 1);
}

// ---------------------------------------------------------------- host side
static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct SortLayout {
    size_t block_sums, dkey, dval, dkey2, dval2, nvis, tkey, tkey2, tval2, hist, digit_total;
    size_t coff, ncand, written, flag, ctile, cgid, cblock_sums, total;
    int64_t scan_blocks, nsort_blocks, psort_blocks, cand_cap, cand_blocks, expand_blocks;
};

// Candidates (box tiles before the cull) get twice the pair capacity.
static SortLayout sort_layout(int64_t n, int64_t cap) {
    SortLayout L;
    const int64_t n1 = n > 0 ? n : 1, c1 = cap > 0 ? cap : 1;
    L.cand_cap = 2 * c1 > 1024 ? 2 * c1 : 1024;
    L.scan_blocks = (n1 + kScanTile - 1) / kScanTile;
    L.nsort_blocks = (n1 + kSortTile - 1) / kSortTile;
    L.psort_blocks = (c1 + kSortTile - 1) / kSortTile;
    L.cand_blocks = (L.cand_cap + kScanTile - 1) / kScanTile;
    L.expand_blocks = (L.cand_cap + kExpandTile - 1) / kExpandTile;
    const int64_t hist_blocks = L.nsort_blocks > L.psort_blocks ? L.nsort_blocks : L.psort_blocks;
    size_t off = 0;
    L.coff = off; off += align256(sizeof(uint32_t) * (size_t)(n1 + 1));
    L.ncand = off; off += align256(sizeof(int64_t));
    L.written = off; off += align256(sizeof(int64_t));
    L.flag = off; off += align256(sizeof(uint8_t) * (size_t)L.cand_cap);
    L.ctile = off; off += align256(sizeof(uint32_t) * (size_t)L.cand_cap);
    L.cgid = off; off += align256(sizeof(uint32_t) * (size_t)L.cand_cap);
    L.cblock_sums = off; off += align256(sizeof(uint32_t) * (size_t)L.cand_blocks);
    L.block_sums = off; off += align256(sizeof(uint32_t) * (size_t)L.scan_blocks);
    L.dkey = off; off += align256(sizeof(uint32_t) * (size_t)n1);
    L.dval = off; off += align256(sizeof(uint32_t) * (size_t)n1);
    L.dkey2 = off; off += align256(sizeof(uint32_t) * (size_t)n1);
    L.dval2 = off; off += align256(sizeof(uint32_t) * (size_t)n1);
    L.nvis = off; off += align256(sizeof(int64_t));
    L.tkey = off; off += align256(sizeof(uint32_t) * (size_t)c1);
    L.tkey2 = off; off += align256(sizeof(uint32_t) * (size_t)c1);
    L.tval2 = off; off += align256(sizeof(uint32_t) * (size_t)c1);
    L.hist = off; off += align256(sizeof(uint32_t) * kRadix * (size_t)hist_blocks);
    L.digit_total = off; off += align256(sizeof(uint32_t) * kRadix);
    L.total = off;
    return L;
}

static int ceil_log2(int64_t x) {
    int b = 0;
    while ((int64_t(1) << b) < x) ++b;
    return b;
}

// Stable LSD passes over `bits` bits starting at `shift0`: `passes` passes
// of ceil(bits / passes) bits.  Data start in (k, v); after an odd number of
// passes they end in (k2, v2), after an even number back in (k, v).
static void radix_passes(uint32_t *k, uint32_t *v, uint32_t *k2, uint32_t *v2, const int64_t *d_count, int64_t cap,
                         int shift0, int bits, int passes, uint32_t *hist, uint32_t *digit_total, int nblocks,
                         cudaStream_t st) {
    const int per = passes > 0 ? (bits + passes - 1) / passes : 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = shift0 + p * per;
        const int b = (shift0 + bits - shift) < per ? (shift0 + bits - shift) : per;
        const uint32_t mask = (1u << b) - 1u;
        radix_hist_kernel<<<nblocks, kSortThreads, 0, st>>>(k, d_count, cap, shift, mask, nblocks, hist);
        radix_digit_scan_kernel<<<kRadix, 256, 0, st>>>(hist, nblocks, digit_total);
        radix_scatter_kernel<<<nblocks, kSortThreads, 0, st>>>(k, v, k2, v2, d_count, cap, shift, mask, nblocks, hist,
                                                               digit_total);
        uint32_t *t = k; k = k2; k2 = t;
        t = v; v = v2; v2 = t;
    }
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

namespace gsr {
// Binning of n records spread over the views of vt (tiles numbered 0 .. tiles - 1).
int32_t bin_sort_impl(const gsr_proj *proj, int64_t n, const ViewTiles &vt, int64_t tiles, const gsr_tiling *tiling,
                      uint64_t *keys, uint32_t *vals, int64_t pair_capacity, uint32_t *tile_ranges,
                      int64_t *d_num_pairs, void *workspace, size_t workspace_bytes, int32_t *d_status,
                      gsr_stream_t stream) {
    int32_t rc;
    if (!proj || (n > 0 && (!proj->ntiles || !proj->xy_conic || !proj->c_op_box || !proj->rgb_depth)) || n < 0 ||
        pair_capacity < 0 || !tile_ranges || !d_num_pairs || (pair_capacity > 0 && (!keys || !vals))) {
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
    auto u32 = [&](size_t off) { return reinterpret_cast<uint32_t *>(ws + off); };
    uint32_t *block_sums = u32(L.block_sums), *hist = u32(L.hist), *digit_total = u32(L.digit_total);
    uint32_t *dkey = u32(L.dkey), *dval = u32(L.dval), *dkey2 = u32(L.dkey2), *dval2 = u32(L.dval2);
    uint32_t *tkey = u32(L.tkey), *tkey2 = u32(L.tkey2), *tval2 = u32(L.tval2);
    int64_t *d_nvis = reinterpret_cast<int64_t *>(ws + L.nvis);
    if (cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)tiles, st) != cudaSuccess)
        return check_launch("memset tile ranges");
    if (n == 0) {
        if (cudaMemsetAsync(d_num_pairs, 0, sizeof(int64_t), st) != cudaSuccess)
            return check_launch("memset pair count");
        return GSR_OK;
    }
    const float4 *xy = reinterpret_cast<const float4 *>(proj->xy_conic);
    const float4 *cb = reinterpret_cast<const float4 *>(proj->c_op_box);
    const float4 *rd = reinterpret_cast<const float4 *>(proj->rgb_depth);
    const unsigned sb = (unsigned)L.scan_blocks;
    // 1. visible Gaussians -> (depth bits, index), then the four depth passes
    vis_count_kernel<<<sb, kScanThreads, 0, st>>>(proj->ntiles, n, block_sums);
    vis_compact_kernel<<<sb, kScanThreads, 0, st>>>(proj->ntiles, rd, n, block_sums, L.scan_blocks, dkey, dval, d_nvis);
    radix_passes(dkey, dval, dkey2, dval2, d_nvis, n, 0, 32, 4, hist, digit_total, (int)L.nsort_blocks, st);
    if ((rc = check_launch("depth sort"))) return rc;
    // 2. pairs in depth order, then the tile passes (ending in tkey / vals)
    const int tbits = ceil_log2(tiles);
    const int tpasses = (tbits + 7) / 8;
    uint32_t *ek = (tpasses & 1) ? tkey2 : tkey;
    uint32_t *ev = (tpasses & 1) ? tval2 : vals;
    uint32_t *coff = u32(L.coff), *ctile = u32(L.ctile), *cgid = u32(L.cgid), *cblock_sums = u32(L.cblock_sums);
    uint8_t *flag = reinterpret_cast<uint8_t *>(ws + L.flag);
    int64_t *d_ncand = reinterpret_cast<int64_t *>(ws + L.ncand);
    int64_t *d_written = reinterpret_cast<int64_t *>(ws + L.written);
    cand_count_kernel<<<sb, kScanThreads, 0, st>>>(proj->ntiles, dval, d_nvis, n, block_sums);
    cand_offsets_kernel<<<sb, kScanThreads, 0, st>>>(proj->ntiles, dval, d_nvis, n, block_sums, L.scan_blocks,
                                                     L.cand_cap, coff, d_ncand, d_num_pairs, d_status);
    expand_kernel<<<(unsigned)L.expand_blocks, kExpandThreads, 0, st>>>(
        coff, dval, xy, cb, d_nvis, n, d_ncand, L.cand_cap, tiling->tile_w, tiling->tile_h, vt, flag, ctile, cgid);
    kept_count_kernel<<<(unsigned)L.cand_blocks, kScanThreads, 0, st>>>(flag, d_ncand, L.cand_cap, cblock_sums);
    kept_compact_kernel<<<(unsigned)L.cand_blocks, kScanThreads, 0, st>>>(flag, ctile, cgid, d_ncand, L.cand_cap,
                                                                          cblock_sums, L.cand_blocks, pair_capacity,
                                                                          ek, ev, d_num_pairs, d_written, d_status);
    if ((rc = check_launch("pair expansion"))) return rc;
    if (pair_capacity == 0) return GSR_OK;
    radix_passes(ek, ev, (tpasses & 1) ? tkey : tkey2, (tpasses & 1) ? vals : tval2, d_written, pair_capacity, 0,
                 tbits, tpasses, hist, digit_total, (int)L.psort_blocks, st);
    const unsigned rb = (unsigned)((pair_capacity + 255) / 256);
    finalize_kernel<<<rb, 256, 0, st>>>(tkey, vals, rd, d_written, pair_capacity, (uint32_t)tiles, keys,
                                        reinterpret_cast<uint2 *>(tile_ranges));
    return check_launch("finalize_kernel");
}
}  // namespace gsr

extern "C" int32_t gsr_bin_sort(const gsr_proj *proj, int64_t n, const gsr_camera *cam, const gsr_tiling *tiling,
                                uint64_t *keys, uint32_t *vals, int64_t pair_capacity, uint32_t *tile_ranges,
                                int64_t *d_num_pairs, void *workspace, size_t workspace_bytes, int32_t *d_status,
                                gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_camera(cam)) || (rc = validate_tiling(tiling))) return rc;
    ViewTiles vt{};
    vt.nviews = 1;
    vt.n_per_view = n > 0 ? n : 1;
    vt.gx[0] = grid_x(cam, tiling);
    vt.toff[0] = 0;
    const int64_t tiles = (int64_t)grid_x(cam, tiling) * grid_y(cam, tiling);
    return bin_sort_impl(proj, n, vt, tiles, tiling, keys, vals, pair_capacity, tile_ranges, d_num_pairs, workspace,
                         workspace_bytes, d_status, stream);
}

extern "C" int32_t gsr_batched_bin_sort(const gsr_proj *proj, int64_t n_per_view, const gsr_camera *cams,
                                        int32_t nviews, const gsr_tiling *tiling, uint64_t *keys, uint32_t *vals,
                                        int64_t pair_capacity, uint32_t *tile_ranges, int64_t *d_num_pairs,
                                        void *workspace, size_t workspace_bytes, int32_t *d_status,
                                        gsr_stream_t stream) {
    int32_t rc;
    if ((rc = validate_tiling(tiling))) return rc;
    if (!cams || nviews <= 0 || nviews > kMaxViews || n_per_view < 0) {
        set_error("gsr_batched_bin_sort: need 1 .. %d views and n_per_view >= 0", kMaxViews);
        return GSR_ERR_INVALID_ARG;
    }
    ViewTiles vt{};
    vt.nviews = nviews;
    vt.n_per_view = n_per_view > 0 ? n_per_view : 1;
    int64_t tiles = 0;
    for (int v = 0; v < nviews; ++v) {
        if ((rc = validate_camera(&cams[v]))) return rc;
        vt.gx[v] = grid_x(&cams[v], tiling);
        vt.toff[v] = (uint32_t)tiles;
        tiles += (int64_t)grid_x(&cams[v], tiling) * grid_y(&cams[v], tiling);
    }
    if (n_per_view * nviews > 0xffffffffLL) {
        set_error("gsr_batched_bin_sort: n_per_view x views must fit in 32 bits");
        return GSR_ERR_UNSUPPORTED;
    }
    return bin_sort_impl(proj, n_per_view * nviews, vt, tiles, tiling, keys, vals, pair_capacity, tile_ranges,
                         d_num_pairs, workspace, workspace_bytes, d_status, stream);
}
