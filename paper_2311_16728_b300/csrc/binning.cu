// binning.cu -- tile binning for the tile-based renderer of Photo-SLAM
// (arXiv 2311.16728) Sec. 3.3: one (tile, Gaussian) pair per kept tile of a
// Gaussian's pixel box, ordered by the 64-bit key tile << 32 | bits(depth)
// (ties by Gaussian index), plus per-tile [begin, end) ranges.
//
// In-house bucket sort by tile, then a sort inside each tile:
//   1. the visible records are compacted in index order;
//   2. an exclusive scan of their box-tile counts numbers the candidates
//      (record, box tile);
//   3. expansion: one thread per candidate runs the tile cull (tile_keep); a
//      kept pair is appended to an unordered list (one atomic per block and
//      chunk of candidates) and counted in its tile (an atomic on the tile's
//      range word, whose return value is the pair's rank in the tile);
//   4. one CTA scans the tile counts into [begin, end) ranges and lists the
//      non-empty tiles by length class;
//   5. scatter: every kept pair goes to its tile's segment at the rank the
//      counting atomic returned;
//   6. each segment is sorted on (depth bits << 32 | index) -- unique keys --
//      in shared memory by a bitonic network (a stable LSD radix sort in
//      global memory for the rare segment longer than shared memory), and
//      written out as key = tile << 32 | depth bits, value = index.
// The result is exactly the order of a stable sort of all pairs by the
// 64-bit key.  Counts stay on the device (kernels read them back), so the
// whole sequence has fixed launch shapes and can be captured in a CUDA graph.
#include "gsr_internal.cuh"

namespace gsr {

constexpr int kScanThreads = 256;
// records per thread in the count / compaction kernels: 8, or 32 when that
// keeps the block count (whose prefix every compaction block sums) at most
// kScanBlocksMax -- the batched window has views x n records
constexpr int kScanItems = 8, kScanItemsBig = 32;
constexpr int64_t kScanBlocksMax = 512;

constexpr int kRadix = 256;  // digits of one pass of the long-segment radix sort

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

// Exclusive running maximum over a block of 256 threads (0 for thread 0).
__device__ __forceinline__ uint32_t block_excl_max_256(uint32_t v, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl = max(incl, t);
    }
    const uint32_t prev_lane = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < 8 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w = max(w, t);
        }
        if (lane < 8) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = max(wid > 0 ? s_warp[wid - 1] : 0u, lane > 0 ? prev_lane : 0u);
    __syncthreads();
    return excl;
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

// ---------------------------------------------------------------- visible records and candidates
// Pass 1: per block of kScanThreads x I records, the number of visible
// records and of their box tiles (the candidates).  Warp w of block b takes
// the 32 I records from (8 b + w) 32 I on, lane l record 32 j + l of them
// (coalesced loads).  It also zeroes the per-tile counters (the range words)
// and the kept-pair counter for the passes that follow.
template <int I>
__global__ void __launch_bounds__(kScanThreads) count_kernel(const uint32_t *__restrict__ ntiles, int64_t n,
                                                             uint32_t *__restrict__ vis_sums,
                                                             uint32_t *__restrict__ cand_sums,
                                                             uint32_t *__restrict__ ranges, int64_t range_words,
                                                             unsigned long long *__restrict__ d_kept) {
    __shared__ uint32_t s_warp[8];
    for (int64_t w = (int64_t)blockIdx.x * kScanThreads + threadIdx.x; w < range_words;
         w += (int64_t)gridDim.x * kScanThreads)
        ranges[w] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_kept = 0ull;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t wbase = ((int64_t)blockIdx.x * (kScanThreads / 32) + wid) * (32 * I);
    uint32_t v = 0, c = 0;
#pragma unroll
    for (int j = 0; j < I; ++j) {
        const int64_t e = wbase + 32 * j + lane;
        const uint32_t t = e < n ? ntiles[e] : 0u;
        v += t > 0u ? 1u : 0u;
        c += t;
    }
    v = block_incl_scan_256(v, s_warp);
    c = block_incl_scan_256(c, s_warp);
    if (threadIdx.x == kScanThreads - 1) {
        vis_sums[blockIdx.x] = v;
        cand_sums[blockIdx.x] = c;
    }
}

// Records of the visible list gathered into dense arrays (position = rank in
// index order) with rec_to_c[record] = position: the later passes then read
// and accumulate into arrays that stay in L2 instead of the sparse
// views x n ones.  All NULL: no gathering.
struct Gather {
    const float4 *xy, *cb, *rd;
    float4 *cxy, *ccb, *crd;
    uint32_t *rec_to_c;
    const float2 *uv;  // position residuals (both NULL: none)
    float2 *cuv;
};

// Pass 2: the visible records in index order (order[]), the first candidate
// slot of each (coff[], with coff[nv] = the candidate total), *d_nvis and
// *d_ncand, and the gathered records when gt.cxy is set.  Candidate numbers
// are 32-bit: a frame with 2^32 or more candidates sets GSR_ERR_UNSUPPORTED
// and expands nothing.
template <int I>
__global__ void __launch_bounds__(kScanThreads, 4) compact_kernel(const uint32_t *__restrict__ ntiles, int64_t n,
                                                               const uint32_t *__restrict__ vis_sums,
                                                               const uint32_t *__restrict__ cand_sums,
                                                               int64_t nblocks, uint32_t *__restrict__ order,
                                                               uint32_t *__restrict__ coff,
                                                               int64_t *__restrict__ d_nvis,
                                                               int64_t *__restrict__ d_ncand,
                                                               int32_t *__restrict__ d_status, Gather gt) {
    __shared__ uint32_t s_warp[8];
    __shared__ int64_t s_red[16];
    int64_t vis_total, cand_total;
    const int64_t vis_pre = block_prefix(vis_sums, nblocks, blockIdx.x, &vis_total, s_red);
    const int64_t cand_pre = block_prefix(cand_sums, nblocks, blockIdx.x, &cand_total, s_red);
    const bool too_many = cand_total > (int64_t)0xffffffffLL;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *d_nvis = vis_total;
        *d_ncand = too_many ? 0 : cand_total;
        coff[vis_total] = (uint32_t)cand_total;
        if (too_many) raise_status(d_status, GSR_ERR_UNSUPPORTED);
    }
    // the records of count_kernel's warp layout, in index order within the warp
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t wbase = ((int64_t)blockIdx.x * (kScanThreads / 32) + wid) * (32 * I);
    uint32_t t[I];
    uint32_t v = 0, c = 0;
#pragma unroll
    for (int j = 0; j < I; ++j) {
        const int64_t e = wbase + 32 * j + lane;
        t[j] = e < n ? ntiles[e] : 0u;
        v += t[j] > 0u ? 1u : 0u;
        c += t[j];
    }
    // warps' exclusive offsets within the block (lane 0 carries the warp's totals)
    const uint32_t wv = __reduce_add_sync(0xffffffffu, v), wc = __reduce_add_sync(0xffffffffu, c);
    const uint32_t vi = block_incl_scan_256(lane == 0 ? wv : 0u, s_warp);
    const uint32_t ci = block_incl_scan_256(lane == 0 ? wc : 0u, s_warp);
    int64_t pos = vis_pre + (int64_t)(__shfl_sync(0xffffffffu, vi, 0) - wv);
    int64_t off = cand_pre + (int64_t)(__shfl_sync(0xffffffffu, ci, 0) - wc);
#pragma unroll
    for (int j = 0; j < I; ++j) {
        const uint32_t tj = t[j];
        const bool vis = tj > 0u;
        const uint32_t m = __ballot_sync(0xffffffffu, vis);
        uint32_t inc = tj;  // inclusive warp scan of the candidate counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (vis) {
            const int64_t p = pos + __popc(m & lt), e = wbase + 32 * j + lane;
            order[p] = (uint32_t)e;
            coff[p] = (uint32_t)(off + (int64_t)(inc - tj));
            if (gt.cxy) {
                gt.cxy[p] = __ldg(gt.xy + e);
                gt.ccb[p] = __ldg(gt.cb + e);
                gt.crd[p] = __ldg(gt.rd + e);
                if (gt.cuv) gt.cuv[p] = __ldg(gt.uv + e);
                gt.rec_to_c[e] = (uint32_t)p;
            }
        }
        pos += __popc(m);
        off += __shfl_sync(0xffffffffu, inc, 31);
    }
}

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

constexpr int kExpandThreads = 256;
constexpr int kExpandItems = 4;
constexpr int kExpandTile = kExpandThreads * kExpandItems;
constexpr int kExpandGrid = 148 * 4;  // one wave at four CTAs per SM (56 registers), grid-stride over chunks
constexpr int kExpandGroup = 16;      // chunks of a block whose ends are searched together

// Kept pairs: kept_ts[p] = global tile << 32 | rank of the pair within its
// tile (from the atomic that counts the tile's pairs in counts[2 t]),
// kept_sk[p] = depth bits << 32 | record; positions p from one atomic per
// block and chunk on *d_kept (pairs beyond `cap` are counted, not stored).
__global__ void __launch_bounds__(kExpandThreads) expand_kernel(
    const uint32_t *__restrict__ coff, const uint32_t *__restrict__ order, const float4 *__restrict__ xy_conic,
    const float4 *__restrict__ c_op_box, const float4 *__restrict__ rgb_depth, const int64_t *__restrict__ d_nvis,
    int64_t cap_n, const int64_t *__restrict__ d_ncand, int tw, int th, const ViewTiles vt, uint32_t ntiles_total,
    uint32_t *__restrict__ counts, uint64_t *__restrict__ kept_ts, uint64_t *__restrict__ kept_sk, int64_t cap,
    unsigned long long *__restrict__ d_kept, bool compact) {
    chain_enter();  // lets the chained tile scan be scheduled
    __shared__ uint32_t s_off[kExpandTile + 1];
    __shared__ __align__(16) uint4 s_meta[kExpandTile];
    __shared__ __align__(16) uint32_t s_map[kExpandTile];
    __shared__ uint32_t s_depth[kExpandTile];
    __shared__ uint32_t s_warp[8];
    __shared__ int64_t s_ci[2 * kExpandGroup];
    __shared__ unsigned long long s_base;
    const int64_t ncand = *d_ncand;
    const int64_t nv = clamp_count(d_nvis, cap_n);
    const int64_t nchunks = (ncand + kExpandTile - 1) / kExpandTile;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // this block's chunks are blockIdx.x + k gridDim.x; a group of up to
    // kExpandGroup of them first finds the visible items at both ends of each
    // chunk, one warp per search, all searches in flight together
    for (int64_t cg = blockIdx.x; cg < nchunks; cg += (int64_t)gridDim.x * kExpandGroup) {
        const int64_t left = (nchunks - cg + gridDim.x - 1) / gridDim.x;
        const int kn = left < kExpandGroup ? (int)left : kExpandGroup;
        __syncthreads();  // the previous group is done with the shared words
        for (int q = wid; q < 2 * kn; q += kExpandThreads / 32) {
            const int64_t c0 = (cg + (int64_t)(q >> 1) * gridDim.x) * kExpandTile;
            const int64_t slot = (q & 1) ? (c0 + kExpandTile < ncand ? c0 + kExpandTile : ncand) - 1 : c0;
            const int64_t idx = warp_upper_index(coff, nv, (uint32_t)slot);
            if (lane == 0) s_ci[q] = idx;
        }
        __syncthreads();
    for (int kc = 0; kc < kn; ++kc) {
        const int64_t s0 = (cg + (int64_t)kc * gridDim.x) * kExpandTile;
        const int64_t i0 = s_ci[2 * kc];
        const int m = (int)(s_ci[2 * kc + 1] - i0 + 1);  // every visible item owns >= 1 slot, so m <= kExpandTile
        __syncthreads();  // the previous chunk is done with s_off, s_meta, s_map
        reinterpret_cast<uint4 *>(s_map)[threadIdx.x] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        // per visible item of the chunk (once, not per candidate): its first
        // slot, the pair value, its box in tiles and the index of its first
        // tile; the first chunk slot of each item marks the slot map
        for (int j = threadIdx.x; j <= m; j += kExpandThreads) {
            const uint32_t off = coff[i0 + j];
            s_off[j] = off;
            if (j < m) {
                const uint32_t rec = order[i0 + j];
                // the pair's value: the record, or its position in the visible
                // list when the records were gathered into compact arrays
                const uint32_t gid = compact ? (uint32_t)(i0 + j) : rec;
                const float4 b = __ldg(c_op_box + gid);
                const uint32_t bx = __float_as_uint(b.z), by = __float_as_uint(b.w);
                const int tx0 = (int)(bx & 0xffffu) / tw, ty0 = (int)(by & 0xffffu) / th;
                const int ntx = (int)(bx >> 16) / tw - tx0 + 1;
                const int v = vt.nviews > 1 ? (int)(rec / (uint32_t)vt.n_per_view) : 0;  // view of this record
                s_meta[j] = make_uint4(gid, vt.toff[v] + (uint32_t)(ty0 * vt.gx[v] + tx0),
                                       ((uint32_t)vt.gx[v] << 16) | (uint32_t)ntx, ((uint32_t)ty0 << 16) | (uint32_t)tx0);
                s_depth[j] = __float_as_uint(__ldg(&rgb_depth[gid].w));
                const int64_t start = (int64_t)off - s0;
                if (start < kExpandTile) s_map[start > 0 ? start : 0] = (uint32_t)j;
            }
        }
        __syncthreads();
        {  // slot -> item: running maximum of the marks
            uint4 q = reinterpret_cast<uint4 *>(s_map)[threadIdx.x];
            q.y = max(q.y, q.x);
            q.z = max(q.z, q.y);
            q.w = max(q.w, q.z);
            const uint32_t carry = block_excl_max_256(q.w, s_warp);
            q.x = max(q.x, carry);
            q.y = max(q.y, carry);
            q.z = max(q.z, carry);
            q.w = max(q.w, carry);
            reinterpret_cast<uint4 *>(s_map)[threadIdx.x] = q;
        }
        __syncthreads();
        uint32_t tiles[kExpandItems], gids[kExpandItems], depth[kExpandItems];
        uint32_t mine = 0;  // bit r: this thread's candidate of round r is kept
#pragma unroll
        for (int r = 0; r < kExpandItems; ++r) {
            const int kl = r * kExpandThreads + (int)threadIdx.x;
            const int64_t slot = s0 + kl;
            tiles[r] = 0;
            gids[r] = 0;
            depth[r] = 0;
            if (slot < ncand) {
                const int lo = (int)s_map[kl];
                const uint4 meta = s_meta[lo];
                const int k = (int)((uint32_t)slot - s_off[lo]);
                const int ntx = (int)(meta.z & 0xffffu), gxv = (int)(meta.z >> 16);
                // k = q ntx + rr; q < 2^16, so the rounded quotient is off by
                // at most one and one correction step makes it exact
                int q = __float2int_rz(__fmul_rn(__int2float_rn(k), __frcp_rn(__int2float_rn(ntx))));
                int rr = k - q * ntx;
                if (rr < 0) {
                    --q;
                    rr += ntx;
                } else if (rr >= ntx) {
                    ++q;
                    rr -= ntx;
                }
                const uint32_t gid = meta.x;
                const Splat sp = load_splat(xy_conic, c_op_box, gid);
                const int tx = (int)(meta.w & 0xffffu) + rr, ty = (int)(meta.w >> 16) + q;
                const uint32_t tile = meta.y + (uint32_t)(q * gxv + rr);
                if (tile < ntiles_total &&
                    tile_keep_at(tx, ty, tw, th, sp.u, sp.v, sp.A, sp.B, sp.C, sp.op, sp.x0, sp.x1, sp.y0, sp.y1)) {
                    mine |= 1u << r;
                    tiles[r] = tile;
                    gids[r] = gid;
                    depth[r] = s_depth[lo];
                }
            }
        }
        // one atomic per block and chunk reserves the block's slots
        const uint32_t c = (uint32_t)__popc(mine);
        const uint32_t incl = block_incl_scan_256(c, s_warp);
        if (threadIdx.x == kExpandThreads - 1) s_base = incl ? atomicAdd(d_kept, (unsigned long long)incl) : 0ull;
        __syncthreads();
        unsigned long long pos = s_base + (unsigned long long)(incl - c);
#pragma unroll
        for (int r = 0; r < kExpandItems; ++r)
            if (mine & (1u << r)) {
                const uint32_t rank = atomicAdd(&counts[2 * (size_t)tiles[r]], 1u);
                if (pos < (unsigned long long)cap) {
                    kept_ts[pos] = ((uint64_t)tiles[r] << 32) | rank;
                    kept_sk[pos] = ((uint64_t)depth[r] << 32) | gids[r];
                }
                ++pos;
            }
    }
    }
}

// ---------------------------------------------------------------- tile scan
constexpr int kTileScanThreads = 1024;
constexpr uint32_t kWarpTile = 512;      // segments this short are sorted by one warp, in registers
constexpr uint32_t kSmallTile = 1024;    // longest segment of the one-block shared-memory sort
constexpr uint32_t kLargeTile = 16384;   // longest segment sorted in shared memory
// length classes of the heavy-first tile order: 16 pairs each, the last open
constexpr int kOrderBuckets = 64;
__device__ __forceinline__ int order_bucket(uint32_t n) { return (int)min((n + 15u) >> 4, (uint32_t)kOrderBuckets - 1u); }
// the warp-sorted segments (1 .. kWarpTile pairs) are whole length classes of
// that order, the last non-empty ones
static_assert(kWarpTile % 16 == 0 && kWarpTile / 16 < kOrderBuckets - 1, "warp segments end on a class boundary");

__device__ __forceinline__ uint32_t block_incl_scan_1024(uint32_t v, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t add = wid > 0 ? s_warp[wid - 1] : 0u;
    __syncthreads();
    return v + add;
}

// One CTA.  ranges[2 t] holds tile t's pair count on entry; on exit
// ranges[2 t], [2 t + 1] = [begin, end) of its segment, or [0, 0) for an
// empty tile.  Non-empty tiles are listed for the sort by length: up to
// kWarpTile from the front of `list`, up to kSmallTile in `list2`, longer
// ones from the back of `list`.  On pair overflow every range is empty.
// tile_work (may be NULL) is zeroed for the forward blend to raise.
__global__ void __launch_bounds__(kTileScanThreads) tile_scan_kernel(
    uint32_t *__restrict__ ranges, uint32_t T, const unsigned long long *__restrict__ d_kept, int64_t cap,
    uint32_t *__restrict__ list, uint32_t *__restrict__ list2, uint32_t *__restrict__ list_counts,
    int64_t *__restrict__ d_written, int64_t *__restrict__ d_num_pairs, int32_t *__restrict__ d_status,
    uint32_t *__restrict__ order, uint32_t *__restrict__ tile_work) {
    chain_enter();
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_small, s_large, s_mid;
    __shared__ uint32_t s_bucket[kOrderBuckets];
    const unsigned long long K = *d_kept;
    const bool overflow = K > (unsigned long long)cap;
    for (int b = threadIdx.x; b < kOrderBuckets; b += kTileScanThreads) s_bucket[b] = 0u;
    if (threadIdx.x == 0) {
        s_small = 0u;
        s_large = 0u;
        s_mid = 0u;
        *d_num_pairs = (int64_t)K;
        *d_written = overflow ? 0 : (int64_t)K;
        if (overflow) raise_status(d_status, GSR_ERR_CAPACITY);
    }
    __syncthreads();
    // rounds of kTileScanThreads x 4 tiles: each thread loads its four
    // tiles' counts at once (two 16-byte words when aligned), one block scan
    // per round, the running total carried between rounds
    constexpr uint32_t kPer = 4;
    const bool vec = (reinterpret_cast<uintptr_t>(ranges) & 15u) == 0u;
    uint32_t carried = 0;
    uint32_t c[kPer];  // the last round's counts stay for the tile order (one round: every tile's)
    for (uint32_t r0 = 0; r0 < T; r0 += kTileScanThreads * kPer) {
        const uint32_t t0 = r0 + threadIdx.x * kPer;
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k) c[k] = 0u;
        if (!overflow) {
            if (vec && t0 + kPer <= T) {
                const uint4 a = __ldcg(reinterpret_cast<const uint4 *>(ranges + 2 * (size_t)t0));
                const uint4 b = __ldcg(reinterpret_cast<const uint4 *>(ranges + 2 * (size_t)t0 + 4));
                c[0] = a.x;
                c[1] = a.z;
                c[2] = b.x;
                c[3] = b.z;
            } else {
#pragma unroll
                for (uint32_t k = 0; k < kPer; ++k)
                    if (t0 + k < T) c[k] = ranges[2 * (size_t)(t0 + k)];
            }
        }
        const uint32_t sum = c[0] + c[1] + c[2] + c[3];
        const uint32_t incl = block_incl_scan_1024(sum, s_warp);
        const uint32_t round_total = s_warp[31];
        uint32_t off = carried + incl - sum;
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k) {
            const uint32_t t = t0 + k;
            if (t >= T) break;
            const uint32_t n = c[k];
            ranges[2 * (size_t)t] = n ? off : 0u;
            ranges[2 * (size_t)t + 1] = n ? off + n : 0u;
            if (tile_work) tile_work[t] = 0u;  // raised by the forward blend
            if (n) {
                if (n <= kWarpTile) list[atomicAdd(&s_small, 1u)] = t;
                else if (n <= kSmallTile) list2[atomicAdd(&s_mid, 1u)] = t;
                else list[(size_t)cap - 1 - atomicAdd(&s_large, 1u)] = t;
            }
            if (order) atomicAdd(&s_bucket[order_bucket(n)], 1u);
            off += n;
        }
        carried += round_total;
        __syncthreads();  // s_warp is rewritten by the next round's scan
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        list_counts[0] = s_small;
        list_counts[1] = s_large;
        list_counts[2] = s_mid;
    }
    if (!order) return;
    // tiles by decreasing pair count for the blend kernels: a counting sort
    // on kOrderBuckets length classes, the longest class first
    desc_class_bases<kOrderBuckets>(s_bucket);
    __syncthreads();
    if (T <= kTileScanThreads * kPer) {  // one round: the counts are still in registers
        const uint32_t t0 = threadIdx.x * kPer;
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k)
            if (t0 + k < T) order[atomicAdd(&s_bucket[order_bucket(overflow ? 0u : c[k])], 1u)] = t0 + k;
        return;
    }
    for (uint32_t t = threadIdx.x; t < T; t += kTileScanThreads) {
        const uint2 r = __ldcg(reinterpret_cast<const uint2 *>(ranges) + t);
        order[atomicAdd(&s_bucket[order_bucket(r.y - r.x)], 1u)] = t;
    }
}

// the tile order of a view without pairs
__global__ void identity_order_kernel(uint32_t *__restrict__ order, uint32_t T) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) order[t] = t;
}

// every stored kept pair goes to its tile's segment at its rank; a thread
// takes four pairs a round (a grid stride apart), all loads issued first
__global__ void __launch_bounds__(256) scatter_kernel(const uint64_t *__restrict__ kept_ts,
                                                      const uint64_t *__restrict__ kept_sk,
                                                      const int64_t *__restrict__ d_written, int64_t cap,
                                                      const uint32_t *__restrict__ ranges,
                                                      uint64_t *__restrict__ seg) {
    constexpr int kU = 4;
    const int64_t w = *d_written;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < w; i0 += kU * stride) {
        uint64_t ts[kU], sk[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int64_t i = i0 + k * stride;
            ts[k] = i < w ? kept_ts[i] : 0ull;
            sk[k] = i < w ? kept_sk[i] : 0ull;
        }
        uint32_t b[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) b[k] = i0 + k * stride < w ? ranges[2 * (size_t)(ts[k] >> 32)] : 0u;
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const uint64_t pos = (uint64_t)b[k] + (uint32_t)ts[k];
            if (i0 + k * stride < w && pos < (uint64_t)cap) seg[pos] = sk[k];
        }
    }
}

// ---------------------------------------------------------------- per-tile sort
// Ascending bitonic network over s[0, P) (P a power of two) by NT threads.
// Stages whose partner distance j is below 32 stay inside aligned chunks of
// 64 entries, so each warp runs them on its own chunks with warp barriers;
// only the wider stages take a block barrier.
__device__ __forceinline__ void cmp_swap(uint64_t *s, uint32_t a, uint32_t j, uint32_t k) {
    const uint32_t b = a + j;
    const uint64_t x = s[a], y = s[b];
    if ((x > y) == ((a & k) == 0)) {
        s[a] = y;
        s[b] = x;
    }
}

template <int NT>
__device__ __forceinline__ void bitonic_sort(uint64_t *s, uint32_t P) {
    constexpr int kWarps = NT / 32;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t C = P < 64 ? P : 64;  // chunk of the warp-local stages
    // j is a power of two: the lower element of pair i is 2 j (i / j) + i % j,
    // i.e. i with a zero bit inserted at bit log2(j)
    for (uint32_t k = 2; k <= P; k <<= 1) {
        uint32_t j = k >> 1;
        for (; j >= 32; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P / 2; i += NT) cmp_swap(s, ((i & ~(j - 1)) << 1) | (i & (j - 1)), j, k);
            __syncthreads();
        }
        for (uint32_t c = wid; c < P / C; c += kWarps) {
            for (uint32_t jj = j; jj > 0; jj >>= 1) {
                if (lane < C / 2) cmp_swap(s, c * C + (((lane & ~(jj - 1)) << 1) | (lane & (jj - 1))), jj, k);
                __syncwarp();
            }
        }
        __syncthreads();
    }
}

// The same network over P <= 32 E entries held in one warp's registers,
// lane-major: entry i = E lane + e sits in v[e] of that lane, so partners at
// distance J < E are registers of the same lane and partners at J >= E are
// J / E lanes apart (one shuffle each).  With E = P / 32 the first log2(E)
// merge levels and the short stages of every later level stay in registers.
// Only the in-register stages are unrolled at compile time (their register
// indices must be constants); the levels beyond E and their shuffle stages
// are runtime loops, which keeps the code of the five E instances small
// (the warps of one launch run all of them at once).

// In-register stages J, J / 2, .., 1 of a level K >= E: the direction of
// every pair is the lane's (ascending when bit K / E of the lane is clear).
template <int E, uint32_t J>
__device__ __forceinline__ void reg_stages(uint64_t (&v)[E], bool up) {
    if constexpr (J >= 1) {
#pragma unroll
        for (uint32_t e = 0; e < (uint32_t)E; ++e)
            if ((e & J) == 0) {
                const uint64_t a = v[e], b = v[e | J];
                if ((a > b) == up) {
                    v[e] = b;
                    v[e | J] = a;
                }
            }
        if constexpr (J > 1) reg_stages<E, J / 2>(v, up);
    }
}

// Levels K = 2 .. E / 2, all in registers: the direction of a pair is bit K
// of its entries' in-lane index e (from level E on it is a bit of the lane).
template <int E, uint32_t K, uint32_t J>
__device__ __forceinline__ void reg_level(uint64_t (&v)[E]) {
#pragma unroll
    for (uint32_t e = 0; e < (uint32_t)E; ++e)
        if ((e & J) == 0) {
            const bool up = (e & K) == 0;
            const uint64_t a = v[e], b = v[e | J];
            if ((a > b) == up) {
                v[e] = b;
                v[e | J] = a;
            }
        }
    if constexpr (J > 1) reg_level<E, K, J / 2>(v);
}

template <int E, uint32_t K>
__device__ __forceinline__ void reg_levels(uint64_t (&v)[E]) {
    if constexpr (K < (uint32_t)E) {
        reg_level<E, K, K / 2>(v);
        reg_levels<E, 2 * K>(v);
    }
}

template <int E>
__device__ __forceinline__ void warp_sort_regs(uint64_t (&v)[E], uint32_t lane, uint32_t P) {
    reg_levels<E, 2>(v);
    for (uint32_t k = E > 1 ? (uint32_t)E : 2u; k <= P; k <<= 1) {
        const uint32_t kl = k / (uint32_t)E;
        for (uint32_t jl = kl >> 1; jl >= 1; jl >>= 1) {  // stages J = K / 2 .. E, J / E lanes apart
            // the lane keeps the smaller key when it is the lower one of an
            // ascending pair (or the upper one of a descending pair): one
            // decision, one 64-bit select (keys are unique)
            const bool keep_min = ((lane & jl) == 0) == ((lane & kl) == 0);
#pragma unroll
            for (uint32_t e = 0; e < (uint32_t)E; ++e) {
                const uint64_t o = __shfl_xor_sync(0xffffffffu, v[e], jl);
                if ((o < v[e]) == keep_min) v[e] = o;
            }
        }
        reg_stages<E, (uint32_t)E / 2>(v, (lane & kl) == 0);
    }
}

// The warp's transpose buffer: entry i at word i + i / 32, so that both the
// lane-major writes (entry E lane + e, any E <= 16) and the row reads (entry
// 32 e + lane) hit 32 distinct banks.
constexpr uint32_t kTransposeWords = kWarpTile + kWarpTile / 32;
__device__ __forceinline__ uint32_t transpose_word(uint32_t i) { return i + (i >> 5); }

// Tile t's segment seg[b, b + L) (L <= 32 E) sorted by one warp in
// registers and emitted: loaded coalesced (the input order is free); the
// lane-major sorted order goes through the warp's shared buffer `tr`
// (kTransposeWords words), the depth halves and then the index halves, so
// that every store of keys and vals covers 32 consecutive entries.
template <int E>
__device__ __forceinline__ void warp_tile_sort(const uint64_t *__restrict__ seg, uint32_t t, uint32_t b, uint32_t L,
                                               uint32_t P, uint32_t lane, uint64_t *__restrict__ keys,
                                               uint32_t *__restrict__ vals, uint32_t *tr) {
    static_assert(32 * E <= (int)kWarpTile, "a warp segment fits the transpose buffer");
    uint64_t v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t i = 32u * e + lane;
        v[e] = i < L ? seg[b + i] : ~0ull;
    }
    warp_sort_regs<E>(v, lane, P);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
        for (int e = 0; e < E; ++e)
            tr[transpose_word((uint32_t)E * lane + e)] = half ? (uint32_t)v[e] : (uint32_t)(v[e] >> 32);
        __syncwarp();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint32_t i = 32u * e + lane;
            if (i < L) {
                const uint32_t w = tr[transpose_word(i)];
                if (half) vals[b + i] = w;
                else keys[b + i] = ((uint64_t)t << 32) | w;
            }
        }
        __syncwarp();  // the buffer is free again
    }
}

// sorted (depth << 32 | index) of tile t -> keys (tile << 32 | depth), vals
template <int NT>
__device__ __forceinline__ void emit_sorted(const uint64_t *s, uint32_t L, uint32_t tile, uint32_t begin,
                                            uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    for (uint32_t i = threadIdx.x; i < L; i += NT) {
        const uint64_t v = s[i];
        keys[begin + i] = ((uint64_t)tile << 32) | (v >> 32);
        vals[begin + i] = (uint32_t)v;
    }
}

template <int NT>
__device__ __forceinline__ void smem_tile_sort(const uint64_t *__restrict__ seg, uint32_t tile, uint32_t begin,
                                               uint32_t L, uint64_t *s, uint64_t *__restrict__ keys,
                                               uint32_t *__restrict__ vals) {
    uint32_t P = 1;
    while (P < L) P <<= 1;
    for (uint32_t i = threadIdx.x; i < P; i += NT) s[i] = i < L ? seg[begin + i] : ~0ull;
    __syncthreads();
    bitonic_sort<NT>(s, P);
    emit_sorted<NT>(s, L, tile, begin, keys, vals);
    __syncthreads();
}

// Exclusive scan in place of the 256 words h[0 .. 255] by the first 256
// threads of a block (NT >= 256; every thread calls it); s_tmp: 8 words.
template <int NT>
__device__ __forceinline__ void block_excl_scan_hist(uint32_t *h, uint32_t *s_tmp) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    uint32_t v = t < 256 ? h[t] : 0u, incl = v;
    if (t < 256) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) s_tmp[wid] = incl;
    }
    __syncthreads();
    if (t < 256) {
        uint32_t add = 0;
        for (int w = 0; w < wid; ++w) add += s_tmp[w];
        h[t] = add + incl - v;
    }
    __syncthreads();
}

// Stable LSD radix sort of the entries a[0, L) (depth bits << 32 | value) by
// their depth, 8 bits per pass over the depth bits that vary within the
// segment, through b; returns the buffer that holds the result.  Entries of
// equal depth keep their input order (fix_depth_ties orders them).  Shared
// words: s_hist 256, s_wcnt (NT / 32) x 256, s_tmp 9.
template <int NT>
__device__ uint64_t *block_radix_sort_depth(uint64_t *a, uint64_t *b, uint32_t L, uint32_t *s_hist,
                                            uint32_t *s_wcnt, uint32_t *s_tmp) {
    constexpr int kWarps = NT / 32;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    if (t == 0) s_tmp[8] = 0u;
    __syncthreads();
    const uint32_t d0 = (uint32_t)(a[0] >> 32);
    uint32_t x = 0;
    for (uint32_t i = t; i < L; i += NT) x |= (uint32_t)(a[i] >> 32) ^ d0;
    x = __reduce_or_sync(0xffffffffu, x);
    if (lane == 0 && x) atomicOr(&s_tmp[8], x);
    __syncthreads();
    const uint32_t vary = s_tmp[8];
    if (vary == 0u) return a;  // one depth: nothing to order here
    const int lo = __ffs(vary) - 1, hi = 31 - __clz(vary);
    for (int shift = 32 + (lo & ~7); shift <= 32 + hi; shift += 8) {
        for (int d = t; d < 256; d += NT) s_hist[d] = 0u;
        __syncthreads();
        for (uint32_t i = t; i < L; i += NT) atomicAdd(&s_hist[(uint32_t)(a[i] >> shift) & 0xffu], 1u);
        __syncthreads();
        block_excl_scan_hist<NT>(s_hist, s_tmp);
        // chunks of NT entries in index order: per-warp ranks by digit, warps
        // in order within the chunk, chunks in order -> stable
        for (uint32_t c0 = 0; c0 < L; c0 += NT) {
            for (int k = t; k < kWarps * 256; k += NT) s_wcnt[k] = 0u;
            __syncthreads();
            const uint32_t i = c0 + (uint32_t)t;
            const bool valid = i < L;
            const uint64_t key = valid ? a[i] : 0ull;
            const uint32_t d = valid ? (uint32_t)(key >> shift) & 0xffu : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t rank = __popc(peers & lt);
            if (valid && rank == 0) s_wcnt[wid * 256 + d] = __popc(peers);
            __syncthreads();
            for (int dd = t; dd < 256; dd += NT) {
                uint32_t run = s_hist[dd];
                for (int w = 0; w < kWarps; ++w) {
                    const uint32_t c = s_wcnt[w * 256 + dd];
                    s_wcnt[w * 256 + dd] = run;
                    run += c;
                }
                s_hist[dd] = run;
            }
            __syncthreads();
            if (valid) b[s_wcnt[wid * 256 + d] + rank] = key;
            __syncthreads();
        }
        uint64_t *tmp = a;
        a = b;
        b = tmp;
    }
    return a;
}

// r[0, L) sorted by depth: each run of equal depth is sorted by value (the
// whole 64-bit entry) by the thread at its start.  Runs are rare and short;
// the depth bits of a run are equal, so reordering one never changes what
// the other threads compare.
template <int NT>
__device__ __forceinline__ void fix_depth_ties(uint64_t *r, uint32_t L) {
    for (uint32_t i = threadIdx.x; i + 1 < L; i += NT) {
        const uint32_t di = (uint32_t)(r[i] >> 32);
        if ((uint32_t)(r[i + 1] >> 32) != di) continue;
        if (i > 0 && (uint32_t)(r[i - 1] >> 32) == di) continue;
        uint32_t j = i + 1;
        while (j + 1 < L && (uint32_t)(r[j + 1] >> 32) == di) ++j;
        for (uint32_t p = i + 1; p <= j; ++p) {
            const uint64_t v = r[p];
            uint32_t q = p;
            while (q > i && r[q - 1] > v) {
                r[q] = r[q - 1];
                --q;
            }
            r[q] = v;
        }
    }
    __syncthreads();
}

// Tile t's segment seg[begin, begin + L) sorted in shared memory by the radix
// sort (s_a, s_b: L entries each), then emitted.
template <int NT>
__device__ __forceinline__ void smem_tile_radix(const uint64_t *__restrict__ seg, uint32_t tile, uint32_t begin,
                                                uint32_t L, uint64_t *s_a, uint64_t *s_b, uint32_t *s_hist,
                                                uint32_t *s_wcnt, uint32_t *s_tmp, uint64_t *__restrict__ keys,
                                                uint32_t *__restrict__ vals) {
    for (uint32_t i = threadIdx.x; i < L; i += NT) s_a[i] = seg[begin + i];
    __syncthreads();
    uint64_t *r = block_radix_sort_depth<NT>(s_a, s_b, L, s_hist, s_wcnt, s_tmp);
    fix_depth_ties<NT>(r, L);
    emit_sorted<NT>(r, L, tile, begin, keys, vals);
    __syncthreads();
}

constexpr int kSmallSortThreads = 256;
constexpr int kLargeSortThreads = 1024;
constexpr int kSortGrid = 148 * 8;


// Segments up to kWarpTile: one warp each, in registers; segments up to
// kSmallTile: one block each, in shared memory.  Both classes are spread
// over the whole grid.
__global__ void __launch_bounds__(kSmallSortThreads) sort_small_kernel(const uint32_t *__restrict__ list,
                                                                       const uint32_t *__restrict__ list2,
                                                                       const uint32_t *__restrict__ order,
                                                                       const uint32_t *__restrict__ list_counts,
                                                                       const uint32_t *__restrict__ ranges,
                                                                       const uint64_t *__restrict__ seg,
                                                                       uint64_t *__restrict__ keys,
                                                                       uint32_t *__restrict__ vals) {
    chain_enter();  // lets the chained long-segment sort be scheduled
    constexpr int kWarps = kSmallSortThreads / 32;
    // the warps' transpose buffers share the block sort's arrays: the block
    // segments start after a barrier that ends every warp segment
    constexpr size_t kBlockBytes = sizeof(uint64_t) * 2 * kSmallTile + sizeof(uint32_t) * (1 + kWarps) * 256;
    static_assert(sizeof(uint32_t) * kWarps * kTransposeWords <= kBlockBytes, "transpose buffers fit");
    __shared__ __align__(16) unsigned char s_raw[kBlockBytes];
    __shared__ uint32_t s_tmp[9];
    uint64_t *const s_a = reinterpret_cast<uint64_t *>(s_raw), *const s_b = s_a + kSmallTile;
    uint32_t *const s_hist = reinterpret_cast<uint32_t *>(s_b + kSmallTile), *const s_wcnt = s_hist + 256;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t *const s_tr = reinterpret_cast<uint32_t *>(s_raw) + wid * kTransposeWords;
    const uint32_t n_warp = list_counts[0], n_block = list_counts[2];
    // with the heavy-first tile order, the warp segments (1 .. kWarpTile
    // pairs) are its entries after the longer segments: the longest go first
    if (order) list = order + list_counts[1] + list_counts[2];
    for (uint32_t e = blockIdx.x * kWarps + wid; e < n_warp; e += gridDim.x * kWarps) {
        const uint32_t t = list[e];
        const uint32_t b = ranges[2 * (size_t)t], L = ranges[2 * (size_t)t + 1] - b;
        uint32_t P = 1;
        while (P < L) P <<= 1;
        // E = P / 32 entries a lane (at least one)
        if (P <= 32) warp_tile_sort<1>(seg, t, b, L, P, lane, keys, vals, s_tr);
        else if (P <= 64) warp_tile_sort<2>(seg, t, b, L, P, lane, keys, vals, s_tr);
        else if (P <= 128) warp_tile_sort<4>(seg, t, b, L, P, lane, keys, vals, s_tr);
        else if (P <= 256) warp_tile_sort<8>(seg, t, b, L, P, lane, keys, vals, s_tr);
        else warp_tile_sort<16>(seg, t, b, L, P, lane, keys, vals, s_tr);
    }
    if (blockIdx.x < n_block) __syncthreads();  // the transpose buffers are free
    for (uint32_t e = blockIdx.x; e < n_block; e += gridDim.x) {
        const uint32_t t = list2[e];
        const uint32_t b = ranges[2 * (size_t)t], L = ranges[2 * (size_t)t + 1] - b;
        smem_tile_radix<kSmallSortThreads>(seg, t, b, L, s_a, s_b, s_hist, s_wcnt, s_tmp, keys, vals);
    }
}

// Stable LSD radix sort of a[0, L) (64-bit keys, 8 passes of 8 bits) through
// b[0, L), by one CTA of NT threads; the result ends in a.  Shared memory:
// kRadix digit bases + (NT / 32) x kRadix per-warp counts.
template <int NT>
__device__ void cta_radix_sort64(uint64_t *a, uint64_t *b, uint32_t L, uint32_t *s_base, uint32_t *s_wcount,
                                 uint32_t *s_warp) {
    constexpr int kWarps = NT / 32;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 8 * pass;
        for (int d = t; d < kRadix; d += NT) s_base[d] = 0u;
        __syncthreads();
        for (uint32_t i = t; i < L; i += NT) atomicAdd(&s_base[(a[i] >> shift) & 0xffu], 1u);
        __syncthreads();
        if (t == 0) {  // exclusive scan of 256 digit counts (once per pass)
            uint32_t run = 0;
            for (int d = 0; d < kRadix; ++d) {
                const uint32_t c = s_base[d];
                s_base[d] = run;
                run += c;
            }
        }
        __syncthreads();
        for (uint32_t c0 = 0; c0 < L; c0 += NT) {
            for (int k = t; k < kWarps * kRadix; k += NT) s_wcount[k] = 0u;
            __syncthreads();
            const uint32_t i = c0 + t;
            const bool valid = i < L;
            const uint64_t key = valid ? a[i] : 0ull;
            const uint32_t d = valid ? (uint32_t)((key >> shift) & 0xffu) : (uint32_t)kRadix;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t rank = __popc(peers & lt);
            if (valid && rank == 0) s_wcount[wid * kRadix + d] = __popc(peers);
            __syncthreads();
            for (int dd = t; dd < kRadix; dd += NT) {  // per-warp offsets within the chunk, warps in order
                uint32_t run = s_base[dd];
                for (int w = 0; w < kWarps; ++w) {
                    const uint32_t c = s_wcount[w * kRadix + dd];
                    s_wcount[w * kRadix + dd] = run;
                    run += c;
                }
                s_base[dd] = run;
            }
            __syncthreads();
            if (valid) b[s_wcount[wid * kRadix + d] + rank] = key;
            __syncthreads();
        }
        uint64_t *tmp = a;
        a = b;
        b = tmp;
    }
    (void)s_warp;
}

// Segments longer than kSmallTile: in shared memory up to kLargeTile, else
// the radix sort in global memory with `spare` (the kept-pair list, free by
// now, indexed like the segments) as the second buffer.
__global__ void __launch_bounds__(kLargeSortThreads) sort_large_kernel(const uint32_t *__restrict__ list,
                                                                       const uint32_t *__restrict__ list_counts,
                                                                       int64_t cap,
                                                                       const uint32_t *__restrict__ ranges,
                                                                       uint64_t *__restrict__ seg,
                                                                       uint64_t *__restrict__ spare,
                                                                       uint64_t *__restrict__ keys,
                                                                       uint32_t *__restrict__ vals) {
    // the last kernel of the binning: lets the chained forward blend after it be scheduled
    chain_enter();
    extern __shared__ uint64_t s_big[];  // kLargeTile entries
    __shared__ uint32_t s_base[kRadix];
    __shared__ uint32_t s_warp[32];
    const uint32_t cnt = list_counts[1];
    for (uint32_t e = blockIdx.x; e < cnt; e += gridDim.x) {
        const uint32_t t = list[(size_t)cap - 1 - e];
        const uint32_t b = ranges[2 * (size_t)t], L = ranges[2 * (size_t)t + 1] - b;
        if (L <= kLargeTile / 2) {
            // s_big: two halves of kLargeTile / 2 entries, then the per-warp digit counts
            uint32_t *s_w = reinterpret_cast<uint32_t *>(s_big + kLargeTile);
            smem_tile_radix<kLargeSortThreads>(seg, t, b, L, s_big, s_big + kLargeTile / 2, s_base, s_w, s_warp,
                                               keys, vals);
        } else if (L <= kLargeTile) {
            smem_tile_sort<kLargeSortThreads>(seg, t, b, L, s_big, keys, vals);
        } else {
            // s_big serves as the per-warp digit counts (32 x 256 words)
            cta_radix_sort64<kLargeSortThreads>(seg + b, spare + b, L, s_base,
                                                reinterpret_cast<uint32_t *>(s_big), s_warp);
            emit_sorted<kLargeSortThreads>(seg + b, L, t, b, keys, vals);  // 8 passes end in seg
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------- host side
static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct SortLayout {
    size_t order, block_sums, cand_sums, coff, counters, kept_ts, kept_sk, seg, list, list2, total;
    int64_t scan_blocks;
    int scan_items;
};

static SortLayout sort_layout(int64_t n, int64_t cap) {
    SortLayout L;
    const int64_t n1 = n > 0 ? n : 1, c1 = cap > 0 ? cap : 1;
    const int64_t small_tile = (int64_t)kScanThreads * kScanItems, big_tile = (int64_t)kScanThreads * kScanItemsBig;
    L.scan_items = (n1 + small_tile - 1) / small_tile > kScanBlocksMax ? kScanItemsBig : kScanItems;
    const int64_t tile = L.scan_items == kScanItems ? small_tile : big_tile;
    L.scan_blocks = (n1 + tile - 1) / tile;
    size_t off = 0;
    L.order = off; off += align256(sizeof(uint32_t) * (size_t)n1);
    L.block_sums = off; off += align256(sizeof(uint32_t) * (size_t)L.scan_blocks);
    L.cand_sums = off; off += align256(sizeof(uint32_t) * (size_t)L.scan_blocks);
    L.coff = off; off += align256(sizeof(uint32_t) * (size_t)(n1 + 1));
    L.counters = off; off += 256;  // nvis, ncand, kept, written (int64) + 3 list counts (u32)
    L.kept_ts = off; off += align256(sizeof(uint64_t) * (size_t)c1);
    L.kept_sk = off; off += align256(sizeof(uint64_t) * (size_t)c1);
    L.seg = off; off += align256(sizeof(uint64_t) * (size_t)c1);
    L.list = off; off += align256(sizeof(uint32_t) * (size_t)c1);
    L.list2 = off; off += align256(sizeof(uint32_t) * (size_t)c1);
    L.total = off;
    return L;
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
                      gsr_stream_t stream, const gsr_proj *compact = nullptr) {
    int32_t rc;
    if (!proj || (n > 0 && (!proj->ntiles || !proj->xy_conic || !proj->c_op_box || !proj->rgb_depth)) || n < 0 ||
        pair_capacity < 0 || !tile_ranges || !d_num_pairs || (pair_capacity > 0 && (!keys || !vals))) {
        set_error("gsr_bin_sort: NULL pointer or negative size");
        return GSR_ERR_INVALID_ARG;
    }
    if (n > 0xffffffffLL || pair_capacity > 0xffffffffLL || tiles > 0xffffffffLL) {
        set_error("gsr_bin_sort: n, pair_capacity and the tile count must fit in 32 bits");
        return GSR_ERR_UNSUPPORTED;
    }
    const SortLayout L = sort_layout(n, pair_capacity);
    if (!workspace || workspace_bytes < L.total) {
        set_error("gsr_bin_sort: workspace of %zu bytes needed, %zu given", L.total, workspace_bytes);
        return GSR_ERR_CAPACITY;
    }
    cudaStream_t st = as_cuda(stream);
    char *ws = static_cast<char *>(workspace);
    if (n == 0) {
        if (cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)tiles, st) != cudaSuccess ||
            cudaMemsetAsync(d_num_pairs, 0, sizeof(int64_t), st) != cudaSuccess)
            return check_launch("memset ranges and pair count");
        if (proj->tile_order && tiles > 0) {
            identity_order_kernel<<<(unsigned)((tiles + 255) / 256), 256, 0, st>>>(proj->tile_order, (uint32_t)tiles);
            return check_launch("identity_order_kernel");
        }
        return GSR_OK;
    }
    uint32_t *order = reinterpret_cast<uint32_t *>(ws + L.order);
    uint32_t *vis_sums = reinterpret_cast<uint32_t *>(ws + L.block_sums);
    uint32_t *cand_sums = reinterpret_cast<uint32_t *>(ws + L.cand_sums);
    uint32_t *coff = reinterpret_cast<uint32_t *>(ws + L.coff);
    int64_t *d_nvis = reinterpret_cast<int64_t *>(ws + L.counters);
    int64_t *d_ncand = d_nvis + 1;
    unsigned long long *d_kept = reinterpret_cast<unsigned long long *>(d_nvis + 2);
    int64_t *d_written = d_nvis + 3;
    uint32_t *list_counts = reinterpret_cast<uint32_t *>(d_nvis + 4);
    uint64_t *kept_ts = reinterpret_cast<uint64_t *>(ws + L.kept_ts);
    uint64_t *kept_sk = reinterpret_cast<uint64_t *>(ws + L.kept_sk);
    uint64_t *seg = reinterpret_cast<uint64_t *>(ws + L.seg);
    uint32_t *list = reinterpret_cast<uint32_t *>(ws + L.list);
    uint32_t *list2 = reinterpret_cast<uint32_t *>(ws + L.list2);
    if (compact && (!compact->xy_conic || !compact->c_op_box || !compact->rgb_depth || !compact->ntiles ||
                    !aligned16(compact->xy_conic) || !aligned16(compact->c_op_box) || !aligned16(compact->rgb_depth))) {
        set_error("gsr_batched_bin_sort: compact record arrays must be non-NULL and 16-byte aligned");
        return GSR_ERR_INVALID_ARG;
    }
    if (compact && proj->uv_lo && (!compact->uv_lo || (reinterpret_cast<uintptr_t>(compact->uv_lo) & 7u))) {
        set_error("gsr_batched_bin_sort: records with uv_lo need an 8-byte aligned compact uv_lo");
        return GSR_ERR_INVALID_ARG;
    }
    const gsr_proj *rp = compact ? compact : proj;  // the records the pairs index
    const float4 *xy = reinterpret_cast<const float4 *>(rp->xy_conic);
    const float4 *cb = reinterpret_cast<const float4 *>(rp->c_op_box);
    const float4 *rd = reinterpret_cast<const float4 *>(rp->rgb_depth);
    const unsigned sb = (unsigned)L.scan_blocks;
    // The binning's wave-sized grids (record scans, expansion, scatter,
    // per-tile sorts) are launched plainly, not chained: a chained launch
    // would place their CTAs around the predecessor's last ones, unevenly
    // (all seven chained took 77 us instead of 70 us on the 300k / 1200 x 680
    // mapping step).  The one-CTA tile scan and the long-segment sort are
    // chained (their predecessors trigger them at entry): 69.9 -> 68.4 us.
    // 1-2. visible records in index order and their candidate offsets (the
    // first pass also zeroes the tile counters and the kept-pair counter)
    auto count = L.scan_items == kScanItems ? count_kernel<kScanItems> : count_kernel<kScanItemsBig>;
    count<<<sb, kScanThreads, 0, st>>>(proj->ntiles, n, vis_sums, cand_sums, tile_ranges, 2 * tiles, d_kept);
    Gather gt{};
    if (compact)
        gt = Gather{reinterpret_cast<const float4 *>(proj->xy_conic), reinterpret_cast<const float4 *>(proj->c_op_box),
                    reinterpret_cast<const float4 *>(proj->rgb_depth), reinterpret_cast<float4 *>(compact->xy_conic),
                    reinterpret_cast<float4 *>(compact->c_op_box), reinterpret_cast<float4 *>(compact->rgb_depth),
                    compact->ntiles, reinterpret_cast<const float2 *>(proj->uv_lo),
                    proj->uv_lo ? reinterpret_cast<float2 *>(compact->uv_lo) : nullptr};
    auto compact_k = L.scan_items == kScanItems ? compact_kernel<kScanItems> : compact_kernel<kScanItemsBig>;
    compact_k<<<sb, kScanThreads, 0, st>>>(proj->ntiles, n, vis_sums, cand_sums, L.scan_blocks, order, coff, d_nvis,
                                           d_ncand, d_status, gt);
    // 3. cull + unordered kept list + tile counts (in the range words)
    expand_kernel<<<kExpandGrid, kExpandThreads, 0, st>>>(coff, order, xy, cb, rd, d_nvis, n, d_ncand,
                                                          tiling->tile_w, tiling->tile_h, vt, (uint32_t)tiles,
                                                          tile_ranges, kept_ts, kept_sk, pair_capacity, d_kept,
                                                          compact != nullptr);
    if ((rc = check_launch("pair expansion"))) return rc;
    // 4-6. ranges, scatter into tile segments, sort each segment
    launch_chained(tile_scan_kernel, dim3(1), dim3(kTileScanThreads), 0, st, tile_ranges, (uint32_t)tiles, d_kept,
                   pair_capacity, list, list2, list_counts, d_written, d_num_pairs, d_status, proj->tile_order,
                   proj->tile_order ? proj->tile_work : nullptr);
    if (pair_capacity == 0) return check_launch("tile_scan_kernel");
    scatter_kernel<<<kSortGrid, 256, 0, st>>>(kept_ts, kept_sk, d_written, pair_capacity, tile_ranges, seg);
    sort_small_kernel<<<kSortGrid, kSmallSortThreads, 0, st>>>(list, list2, proj->tile_order, list_counts,
                                                                 tile_ranges, seg, keys, vals);
    const size_t big = sizeof(uint64_t) * kLargeTile + sizeof(uint32_t) * (kLargeSortThreads / 32) * 256;
    static_assert(sizeof(uint64_t) * kLargeTile >= sizeof(uint32_t) * (kLargeSortThreads / 32) * kRadix,
                  "the long-segment sort reuses the shared array for its per-warp counts");
    cudaFuncSetAttribute(sort_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big);
    launch_chained(sort_large_kernel, dim3(148), dim3(kLargeSortThreads), big, st, list, list_counts, pair_capacity,
                   tile_ranges, seg, kept_sk, keys, vals);
    return check_launch("tile sort");
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
                                        const gsr_proj *compact, void *workspace, size_t workspace_bytes,
                                        int32_t *d_status, gsr_stream_t stream) {
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
                         d_num_pairs, workspace, workspace_bytes, d_status, stream, compact);
}
