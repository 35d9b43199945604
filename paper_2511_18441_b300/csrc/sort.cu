// Binning and sorting of (tile, depth) keys, written for this library.
//
// The front-to-back order of Eq. 3 (ReCoGS, arXiv 2511.18441, Sec. 3.1) is
// obtained per 16x16 tile by a stable LSD radix sort of (tile, depth) keys.
// All pairs of one Gaussian share its depth, so the low (depth) digits are
// sorted once per visible Gaussian, before the pairs are expanded; the
// expansion keeps that order and a second stable radix sort over the tile
// bits finishes the LSD sort. The result is the same sequence a full 64-bit
// (tile << 32 | depth) LSD sort of all pairs would produce, with far fewer
// bytes moved: 32-bit depth keys over V Gaussians plus ~13 tile bits over
// P pairs instead of ~45 bits over P pairs.
//
// Radix pass = upsweep (per-block digit counts) + per-digit scan over blocks
// + downsweep (stable block-local ranking with warp match, then a
// digit-ordered scatter). No pass waits on another block: there is no
// inter-block spinning anywhere in this file.
#include "recogs_internal.cuh"

namespace recogs {

// ---------------------------------------------------------------------------
// block-wide exclusive scan helpers (blockDim.x == 1024 or 256)

template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* s_warp,
                                                         uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < THREADS / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < THREADS / 32) s_warp[lane] = wi - w;
        if (lane == THREADS / 32 - 1) s_warp[32] = wi;
    }
    __syncthreads();
    const uint32_t r = s_warp[warp] + inc - x;
    if (total) *total = s_warp[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// small exclusive scan in one block (block sums, <= a few hundred thousand)

// The total saturates at 0xffffffff when the sum does not fit in 32 bits.
__global__ void __launch_bounds__(1024) scan_small_kernel(const uint32_t* __restrict__ in,
                                                          uint32_t* __restrict__ out, int n,
                                                          uint32_t* __restrict__ total) {
    __shared__ uint32_t s_warp[33];
    unsigned long long carry = 0;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t x = i < n ? in[i] : 0u;
        uint32_t t;
        const uint32_t e = block_exclusive_scan<1024>(x, s_warp, &t);
        if (out && i < n) out[i] = (uint32_t)carry + e;
        carry += t;
    }
    if (threadIdx.x == 0 && total) *total = carry > 0xffffffffull ? 0xffffffffu : (uint32_t)carry;
}

int launch_scan_small(const uint32_t* in, uint32_t* out, int n, int, uint32_t* total,
                      cudaStream_t st) {
    scan_small_kernel<<<1, 1024, 0, st>>>(in, out, n, total);
    return 1;
}

// ---------------------------------------------------------------------------
// stable compaction of visible Gaussians into (depth key, index) pairs

__global__ void __launch_bounds__(kPrepThreads)
    compact_kernel(const uint32_t* __restrict__ count, const uint32_t* __restrict__ zkey, int n,
                   const uint32_t* __restrict__ block_offsets, const DevCounters* __restrict__ ctr,
                   uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
    __shared__ uint32_t s_warp[33];
    const int i = blockIdx.x * kPrepThreads + threadIdx.x;
    const bool vis = i < n && count[i] > 0;
    const uint32_t pos = block_exclusive_scan<kPrepThreads>(vis ? 1u : 0u, s_warp, nullptr);
    if (vis) {
        const uint32_t zmin = ~ctr->zmin_inv;
        const uint32_t o = block_offsets[blockIdx.x] + pos;
        keys_out[o] = zkey[i] - zmin;
        vals_out[o] = (uint32_t)i;
    }
}

int launch_compact(const uint32_t* count, const uint32_t* zkey, int n, const uint32_t* block_offsets,
                   const DevCounters* counters, uint32_t* keys_out, uint32_t* vals_out,
                   cudaStream_t st) {
    if (n == 0) return 0;
    compact_kernel<<<(n + kPrepThreads - 1) / kPrepThreads, kPrepThreads, 0, st>>>(
        count, zkey, n, block_offsets, counters, keys_out, vals_out);
    return 1;
}

// ---------------------------------------------------------------------------
// radix sort passes

__global__ void __launch_bounds__(kSortThreads)
    radix_upsweep(const uint32_t* __restrict__ keys, int n, int shift, int nbits,
                  uint32_t* __restrict__ table) {
    __shared__ uint32_t hist[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[d] = 0;
    __syncthreads();
    const uint32_t mask = (1u << nbits) - 1u;
    const int base = blockIdx.x * kSortTile;
#pragma unroll 4
    for (int k = 0; k < kSortItemsPerThread; ++k) {
        const int i = base + k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&hist[(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    const int nb = gridDim.x;
    for (int d = threadIdx.x; d < (1 << nbits); d += kSortThreads)
        table[d * nb + blockIdx.x] = hist[d];
}

// One block per digit: exclusive scan of that digit's counts across blocks,
// digit total to digit_totals[d].
__global__ void __launch_bounds__(1024) radix_scan(uint32_t* __restrict__ table, int nb,
                                                   uint32_t* __restrict__ digit_totals) {
    __shared__ uint32_t s_warp[33];
    uint32_t* row = table + (size_t)blockIdx.x * nb;
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t x = i < nb ? row[i] : 0u;
        uint32_t t;
        const uint32_t e = block_exclusive_scan<1024>(x, s_warp, &t);
        if (i < nb) row[i] = carry + e;
        carry += t;
    }
    if (threadIdx.x == 0) digit_totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kSortThreads)
    radix_downsweep(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int n,
                    int shift, int nbits, const uint32_t* __restrict__ table,
                    const uint32_t* __restrict__ digit_totals) {
    constexpr int W = kSortThreads / 32;
    constexpr int PER_WARP = kSortTile / W;       // 512 consecutive items per warp
    __shared__ uint32_t s_keys[kSortTile];
    __shared__ uint32_t s_vals[kSortTile];
    __shared__ uint32_t s_wcnt[W][kRadix];        // per-warp digit counters -> warp offsets
    __shared__ uint32_t s_bstart[kRadix];         // block-local start of each digit
    __shared__ uint32_t s_gbase[kRadix];          // global start of each digit for this block
    __shared__ uint32_t s_warp[33];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t mask = (1u << nbits) - 1u;
    const int nb = gridDim.x;
    const int base = blockIdx.x * kSortTile;
    const int nblk = min(kSortTile, n - base);

    // global digit bases: exclusive scan of digit totals + this block's offset
    {
        const int d = threadIdx.x;  // kSortThreads == kRadix
        const uint32_t tot = d < (1 << nbits) ? digit_totals[d] : 0u;
        const uint32_t ex = block_exclusive_scan<kSortThreads>(tot, s_warp, nullptr);
        s_gbase[d] = d < (1 << nbits) ? ex + table[d * nb + blockIdx.x] : 0u;
        for (int w = 0; w < W; ++w) s_wcnt[w][d] = 0;
    }
    __syncthreads();

    // stable warp-local ranking: item order = (iteration, lane) within the warp
    uint32_t key[kSortItemsPerThread], val[kSortItemsPerThread], rank[kSortItemsPerThread];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kSortItemsPerThread; ++k) {
        const int li = warp * PER_WARP + k * 32 + lane;
        const bool ok = li < nblk;
        key[k] = ok ? keys_in[base + li] : 0u;
        val[k] = ok ? vals_in[base + li] : 0u;
        const uint32_t d = ok ? ((key[k] >> shift) & mask) : (uint32_t)kRadix;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = ok ? s_wcnt[warp][d] : 0u;
        __syncwarp();
        if (ok && (peers & lt) == 0) s_wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[k] = before + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: exclusive offsets across warps, block totals, block-local starts
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t c = s_wcnt[w][d];
            s_wcnt[w][d] = run;
            run += c;
        }
        s_bstart[d] = block_exclusive_scan<kSortThreads>(run, s_warp, nullptr);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItemsPerThread; ++k) {
        const int li = warp * PER_WARP + k * 32 + lane;
        if (li < nblk) {
            const uint32_t d = (key[k] >> shift) & mask;
            const uint32_t p = s_bstart[d] + s_wcnt[warp][d] + rank[k];
            s_keys[p] = key[k];
            s_vals[p] = val[k];
        }
    }
    __syncthreads();
    // digit-ordered scatter: consecutive slots of one digit go to consecutive addresses
    for (int j = threadIdx.x; j < nblk; j += kSortThreads) {
        const uint32_t k = s_keys[j];
        const uint32_t d = (k >> shift) & mask;
        const uint32_t g = s_gbase[d] + (uint32_t)j - s_bstart[d];
        keys_out[g] = k;
        vals_out[g] = s_vals[j];
    }
}

int radix_sort_pairs(SortBuffers& b, int n, int bits, cudaStream_t st, int* launches) {
    int cur = 0;
    if (n <= 1 || bits <= 0) return 0;
    const int nb = (n + kSortTile - 1) / kSortTile;
    for (int shift = 0; shift < bits; shift += kRadixBits) {
        const int nbits = min(kRadixBits, bits - shift);
        radix_upsweep<<<nb, kSortThreads, 0, st>>>(b.keys[cur], n, shift, nbits, b.table);
        radix_scan<<<1 << nbits, 1024, 0, st>>>(b.table, nb, b.digit_totals);
        radix_downsweep<<<nb, kSortThreads, 0, st>>>(b.keys[cur], b.vals[cur], b.keys[cur ^ 1],
                                                      b.vals[cur ^ 1], n, shift, nbits, b.table,
                                                      b.digit_totals);
        *launches += 3;
        cur ^= 1;
    }
    return cur;
}

// ---------------------------------------------------------------------------
// pair expansion in depth order

// Blocked assignment: thread t of block b owns sorted Gaussians
// b*4096 + t*16 .. +15.
__global__ void __launch_bounds__(kSortThreads)
    pair_block_sums(const uint32_t* __restrict__ ids, const uint32_t* __restrict__ count, int v,
                    uint32_t* __restrict__ sums) {
    __shared__ uint32_t s_warp[33];
    const int base = blockIdx.x * kSortTile + threadIdx.x * kSortItemsPerThread;
    uint32_t acc = 0;
#pragma unroll 4
    for (int k = 0; k < kSortItemsPerThread; ++k) {
        const int j = base + k;
        if (j < v) acc += count[ids[j]];
    }
    uint32_t tot;
    block_exclusive_scan<kSortThreads>(acc, s_warp, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

int launch_pair_block_sums(const uint32_t* sorted_ids, const uint32_t* count, int v, uint32_t* sums,
                           cudaStream_t st) {
    pair_block_sums<<<(v + kSortTile - 1) / kSortTile, kSortThreads, 0, st>>>(sorted_ids, count, v,
                                                                                 sums);
    return 1;
}

__global__ void __launch_bounds__(kSortThreads)
    emit_kernel(const uint32_t* __restrict__ ids, const uint32_t* __restrict__ count,
                const uint2* __restrict__ rect, int v, const uint32_t* __restrict__ block_offsets,
                int tiles_x, uint32_t* __restrict__ tile_keys, uint32_t* __restrict__ vals) {
    __shared__ uint32_t s_warp[33];
    const int base = blockIdx.x * kSortTile + threadIdx.x * kSortItemsPerThread;
    uint32_t acc = 0;
#pragma unroll 4
    for (int k = 0; k < kSortItemsPerThread; ++k) {
        const int j = base + k;
        if (j < v) acc += count[ids[j]];
    }
    uint32_t o = block_offsets[blockIdx.x] + block_exclusive_scan<kSortThreads>(acc, s_warp, nullptr);
    for (int k = 0; k < kSortItemsPerThread; ++k) {
        const int j = base + k;
        if (j >= v) break;
        const uint32_t id = ids[j];
        const uint2 r = rect[id];
        const uint32_t x0 = r.x & 0xffffu, x1 = r.x >> 16, y0 = r.y & 0xffffu, y1 = r.y >> 16;
        for (uint32_t y = y0; y <= y1; ++y)
            for (uint32_t x = x0; x <= x1; ++x) {
                tile_keys[o] = y * (uint32_t)tiles_x + x;
                vals[o] = id;
                ++o;
            }
    }
}

int launch_emit(const uint32_t* sorted_ids, const uint32_t* count, const uint2* rect, int v,
                const uint32_t* block_offsets, int tiles_x, uint32_t* tile_keys, uint32_t* vals,
                cudaStream_t st) {
    emit_kernel<<<(v + kSortTile - 1) / kSortTile, kSortThreads, 0, st>>>(
        sorted_ids, count, rect, v, block_offsets, tiles_x, tile_keys, vals);
    return 1;
}

// ---------------------------------------------------------------------------
// tile ranges [begin, end) from the sorted tile keys (ranges pre-zeroed)

__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t* __restrict__ tiles, int p,
                                                     uint2* __restrict__ ranges) {
    const int j = blockIdx.x * 256 + threadIdx.x;
    if (j >= p) return;
    const uint32_t t = tiles[j];
    if (j == 0 || tiles[j - 1] != t) ranges[t].x = (uint32_t)j;
    if (j == p - 1 || tiles[j + 1] != t) ranges[t].y = (uint32_t)(j + 1);
}

int launch_ranges(const uint32_t* sorted_tiles, int p, uint2* ranges, cudaStream_t st) {
    if (p == 0) return 0;
    ranges_kernel<<<(p + 255) / 256, 256, 0, st>>>(sorted_tiles, p, ranges);
    return 1;
}

}  // namespace recogs
