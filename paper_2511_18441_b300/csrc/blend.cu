// Per-tile front-to-back alpha blending (Eq. 3 of ReCoGS, arXiv 2511.18441,
// Sec. 3.1) with HWC output (Sec. 4.2).
//
// One CTA of 256 threads per 16x16 tile, one thread per pixel; tiles are
// launched heaviest first (the tile order of the tile scan). Each warp owns an 8x4-pixel
// sub-tile made of four 4x2-pixel groups of 8 lanes. Each batch of up to 256
// (or 128) depth-sorted Gaussians is gathered by one thread per Gaussian (the next
// batch is prefetched into registers while the current one is blended) and
// staged in shared memory with a 32-bit mask of the groups its alpha >= 1/255
// box meets. The four groups of a warp then walk their own hit lists in
// depth order in lockstep (same instructions, a different Gaussian per
// group), so a warp iterates as often as its busiest group, not as often as
// the union of its groups' lists. Pixels stop at the transmittance cut-off, a
// warp stops when all its pixels have, and the CTA stops fetching when every
// pixel has.
#include "recogs_internal.cuh"

// Resident CTAs per SM the register allocation is held to (a tuning knob).
#ifndef RECOGS_BLEND_MIN_BLOCKS
#define RECOGS_BLEND_MIN_BLOCKS 6
#endif

namespace recogs {

// 2^x with the PTX approximate base-2 exponential (relative error ~2^-22).
__device__ __forceinline__ float exp2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Group mask of a Gaussian with centre (u, v) in this tile's frame whose
// alpha >= 1/255 box has half extents (ex, ey). The tile's 16x16 pixels are
// split into 32 groups of 4x2 pixels (a 4 x 8 grid of groups); warp w owns
// the four groups of its 8x4 sub-tile (column w & 1, row w >> 1) and they
// occupy bits 4w .. 4w+3 (bit 4w + (col & 1) + 2 (row & 1)). A bit is set for
// every group whose pixel centres the box meets; the box is widened slightly
// so that rounding never drops a pixel the per-pixel test would keep.
__device__ __forceinline__ uint32_t group_mask(float u, float v, float ex, float ey) {
    ex = ex * 1.0001f + 0.01f;
    ey = ey * 1.0001f + 0.01f;
    // group columns c (4 px wide) with 4c <= u + ex and 4c + 3 >= u - ex;
    // group rows r (2 px tall) with 2r <= v + ey and 2r + 1 >= v - ey
    const float c0 = fmaxf(ceilf((u - ex - 3.0f) * 0.25f), 0.0f);
    const float c1 = fminf(floorf((u + ex) * 0.25f), 3.0f);
    const float r0 = fmaxf(ceilf((v - ey - 1.0f) * 0.5f), 0.0f);
    const float r1 = fminf(floorf((v + ey) * 0.5f), 7.0f);
    if (!(c0 <= c1) || !(r0 <= r1)) return 0u;
    const int ic0 = (int)c0, ic1 = (int)c1, ir0 = (int)r0, ir1 = (int)r1;
    uint32_t mask = 0u;
    for (int r = ir0; r <= ir1; ++r)
        for (int c = ic0; c <= ic1; ++c)
            mask |= 1u << (4 * ((c >> 1) + 2 * (r >> 1)) + (c & 1) + 2 * (r & 1));
    return mask;
}

// BATCH (128 or 256) Gaussians are staged per batch; threads below BATCH
// gather them.
template <int BATCH>
__global__ void __launch_bounds__(kBlendThreads, RECOGS_BLEND_MIN_BLOCKS)
    blend_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
                 const uint32_t* __restrict__ ids, const float4* __restrict__ rec, int width,
                 int height, int tiles_x, float bg0, float bg1, float bg2, float* __restrict__ image,
                 float* __restrict__ final_T, DevCounters* __restrict__ ctr) {
    static_assert(BATCH == 128 || BATCH == 256, "blend batch");
    __shared__ float4 s_a[BATCH];     // (u, v, q0, q1), centre in this tile's frame
    __shared__ float4 s_b[BATCH];     // (q2, log2 sigma, r, g)
    __shared__ float s_c[BATCH];      // b
    __shared__ uint32_t s_m[BATCH];   // group mask

    const int tile = (int)order[blockIdx.x];
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> 3;                // 4x2-pixel group inside the warp's 8x4 sub-tile
    // pixel coordinates relative to this tile's origin (exact small integers)
    const int lx = (warp & 1) * 8 + (grp & 1) * 4 + (lane & 3);
    const int ly = (warp >> 1) * 4 + (grp >> 1) * 2 + ((lane >> 2) & 1);
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < width && py < height;
    const float fpx = (float)lx, fpy = (float)ly;
    const int mbit = 4 * warp + (grp & 1) + 2 * (grp >> 1);   // this lane's group bit

    uint2 rg = ranges[tile];
    if (ctr && ctr->skip) rg = make_uint2(0u, 0u);  // pairs exceed the buffers: background only
    const uint32_t begin = rg.x, end = rg.y;

    float T = 1.0f, cr = 0.f, cg = 0.f, cb = 0.f;
    bool done = !inside;
    uint32_t fetched = begin;
    const float a_min = 1.0f / 255.0f;

    // prefetch the first batch
    float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra, rc = ra;
    const bool gatherer = threadIdx.x < BATCH;
    if (gatherer && begin + threadIdx.x < end) {
        const uint32_t id = __ldg(ids + begin + threadIdx.x);
        ra = __ldg(rec + 3 * (size_t)id);
        rb = __ldg(rec + 3 * (size_t)id + 1);
        rc = __ldg(rec + 3 * (size_t)id + 2);
    }

    for (uint32_t b = begin; b < end; b += BATCH) {
        if (__syncthreads_count(done) == kBlendThreads) break;
        if (gatherer && b + threadIdx.x < end) {
            // move the centre from its first tile's frame into this tile's frame
            const uint32_t o = __float_as_uint(rc.w);
            const float u = ra.x + (float)(kTile * ((int)(o & 0xffffu) - tx));
            const float v = ra.y + (float)(kTile * ((int)(o >> 16) - ty));
            s_a[threadIdx.x] = make_float4(u, v, ra.z, ra.w);
            s_b[threadIdx.x] = make_float4(rb.x, rb.y, rc.x, rc.y);
            s_c[threadIdx.x] = rc.z;
            s_m[threadIdx.x] = group_mask(u, v, rb.z, rb.w);
        }
        fetched = min(end, b + BATCH);
        __syncthreads();
        // prefetch the next batch while this one is blended
        const uint32_t jn = b + BATCH + threadIdx.x;
        if (gatherer && jn < end) {
            const uint32_t id = __ldg(ids + jn);
            ra = __ldg(rec + 3 * (size_t)id);
            rb = __ldg(rec + 3 * (size_t)id + 1);
            rc = __ldg(rec + 3 * (size_t)id + 2);
        }
        const int cnt = (int)min((uint32_t)BATCH, end - b);
        if (__all_sync(0xffffffffu, done)) continue;
#pragma unroll 1
        for (int g = 0; g * 32 < cnt; ++g) {
            // candidates g*32 .. g*32+31: one ballot per group of this warp
            const int sl = g * 32 + lane;
            const uint32_t gm = sl < cnt ? (s_m[sl] >> (4 * warp)) : 0u;
            const uint32_t m0 = __ballot_sync(0xffffffffu, gm & 1u);
            const uint32_t m1 = __ballot_sync(0xffffffffu, gm & 2u);
            const uint32_t m2 = __ballot_sync(0xffffffffu, gm & 4u);
            const uint32_t m3 = __ballot_sync(0xffffffffu, gm & 8u);
            const int gb = mbit - 4 * warp;
            uint32_t m = gb == 0 ? m0 : gb == 1 ? m1 : gb == 2 ? m2 : m3;
            // the four groups walk their own lists in lockstep; lanes whose list
            // is exhausted (or whose pixel has stopped) carry weight 0
            const int iters = (int)__reduce_max_sync(0xffffffffu, (uint32_t)__popc(m));
#pragma unroll 1
            for (int k = 0; k < iters; k += 2) {
                const bool act0 = m != 0u;
                const int s0 = g * 32 + (act0 ? __ffs(m) - 1 : 0);
                m &= m - 1;
                const bool act1 = m != 0u;
                const int s1 = g * 32 + (act1 ? __ffs(m) - 1 : 0);
                m &= m - 1;
                const float4 a0 = s_a[s0], b0 = s_b[s0];
                const float4 a1 = s_a[s1], b1 = s_b[s1];
                float dx = fpx - a0.x, dy = fpy - a0.y;
                const float p0 = fmaf(dx, fmaf(a0.z, dx, a0.w * dy), b0.x * dy * dy);
                dx = fpx - a1.x;
                dy = fpy - a1.y;
                const float p1 = fmaf(dx, fmaf(a1.z, dx, a1.w * dy), b1.x * dy * dy);
                const float al0 = fminf(0.99f, exp2_approx(fminf(p0, 0.0f) + b0.y));
                const float al1 = fminf(0.99f, exp2_approx(fminf(p1, 0.0f) + b1.y));
                {
                    const float nT = T * (1.0f - al0);
                    const bool take = act0 && !done && al0 >= a_min;
                    const bool stop = take && nT < 1e-4f;
                    const bool add = take && !stop;
                    const float w = add ? al0 * T : 0.0f;
                    cr = fmaf(b0.z, w, cr);
                    cg = fmaf(b0.w, w, cg);
                    cb = fmaf(s_c[s0], w, cb);
                    T = add ? nT : T;
                    done = done || stop;
                }
                {
                    const float nT = T * (1.0f - al1);
                    const bool take = act1 && !done && al1 >= a_min;
                    const bool stop = take && nT < 1e-4f;
                    const bool add = take && !stop;
                    const float w = add ? al1 * T : 0.0f;
                    cr = fmaf(b1.z, w, cr);
                    cg = fmaf(b1.w, w, cg);
                    cb = fmaf(s_c[s1], w, cb);
                    T = add ? nT : T;
                    done = done || stop;
                }
            }
            if (__all_sync(0xffffffffu, done)) break;
        }
    }
    if (inside) {
        const size_t p = (size_t)py * width + px;
        image[3 * p + 0] = cr + T * bg0;
        image[3 * p + 1] = cg + T * bg1;
        image[3 * p + 2] = cb + T * bg2;
        if (final_T) final_T[p] = T;
    }
    if (threadIdx.x == 0 && ctr) atomicAdd(&ctr->pairs_read, (unsigned long long)(fetched - begin));
}

int launch_blend(const uint2* ranges, const uint32_t* order, const uint32_t* ids, const float4* rec,
                 const DevCamera& cam, const float bg[3], float* image, float* final_T,
                 DevCounters* counters, int batch, cudaStream_t st) {
    const int tiles = cam.tiles_x * cam.tiles_y;
    if (batch == 128)
        blend_kernel<128><<<tiles, kBlendThreads, 0, st>>>(ranges, order, ids, rec, cam.width,
                                                           cam.height, cam.tiles_x, bg[0], bg[1],
                                                           bg[2], image, final_T, counters);
    else
        blend_kernel<256><<<tiles, kBlendThreads, 0, st>>>(ranges, order, ids, rec, cam.width,
                                                           cam.height, cam.tiles_x, bg[0], bg[1],
                                                           bg[2], image, final_T, counters);
    return 1;
}

}  // namespace recogs
