// Per-tile front-to-back alpha blending (Eq. 3 of ReCoGS, arXiv 2511.18441,
// Sec. 3.1) with HWC output (Sec. 4.2).
//
// One CTA of 256 threads per 16x16 tile, one thread per pixel. Warps own
// 8x4 pixel sub-tiles (2 across, 4 down), so a warp's pixels are compact
// and a small Gaussian touches few warps. Each batch of up to 256 sorted
// Gaussians is staged in shared memory by one coalesced gather; each warp
// then ballots which staged Gaussians' alpha >= 1/255 boxes meet its
// sub-tile and walks only those, in depth order. Pixels stop at the
// transmittance cut-off; a warp stops when all of its pixels have, and the
// CTA stops fetching batches when every pixel has.
#include "recogs_internal.cuh"

namespace recogs {

__global__ void __launch_bounds__(kBlendThreads)
    blend_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids,
                 const float4* __restrict__ rec, int width, int height, int tiles_x, float bg0,
                 float bg1, float bg2, float* __restrict__ image, float* __restrict__ final_T,
                 unsigned long long* __restrict__ pairs_read) {
    __shared__ float4 s_g0[kBlendThreads];   // (u, v, A, B), centre in this tile's frame
    __shared__ float4 s_g1[kBlendThreads];   // (C, sigma, ex, ey)
    __shared__ float4 s_c[kBlendThreads];    // (r, g, b, -)

    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // pixel coordinates relative to this tile's origin (exact small integers)
    const int lx0 = (warp & 1) * 8, ly0 = (warp >> 1) * 4;
    const int lx = lx0 + (lane & 7), ly = ly0 + (lane >> 3);
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < width && py < height;
    const float fpx = (float)lx, fpy = (float)ly;
    // the warp's pixel-centre box
    const float bx0 = (float)lx0, bx1 = (float)(lx0 + 7), by0 = (float)ly0, by1 = (float)(ly0 + 3);

    const uint2 rg = ranges[tile];
    const uint32_t begin = rg.x, end = rg.y;

    float T = 1.0f, cr = 0.f, cg = 0.f, cb = 0.f;
    bool done = !inside;
    uint32_t fetched = begin;
    const float a_min = 1.0f / 255.0f;

    for (uint32_t b = begin; b < end; b += kBlendThreads) {
        if (__syncthreads_count(done) == kBlendThreads) break;
        const uint32_t j = b + threadIdx.x;
        if (j < end) {
            const uint32_t id = __ldg(ids + j);
            float4 g0 = __ldg(rec + 3 * (size_t)id);
            const float4 g1 = __ldg(rec + 3 * (size_t)id + 1);
            const float4 c = __ldg(rec + 3 * (size_t)id + 2);
            // move the centre from its first tile's frame into this tile's frame
            const uint32_t o = __float_as_uint(c.w);
            g0.x += (float)(kTile * ((int)(o & 0xffffu) - tx));
            g0.y += (float)(kTile * ((int)(o >> 16) - ty));
            s_g0[threadIdx.x] = g0;
            s_g1[threadIdx.x] = g1;
            s_c[threadIdx.x] = c;
        }
        fetched = min(end, b + kBlendThreads);
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBlendThreads, end - b);
        if (__all_sync(0xffffffffu, done)) continue;
        // which staged Gaussians can reach this warp's pixels: their
        // alpha >= 1/255 box, slightly widened so that rounding never drops a
        // pixel the per-pixel test would keep
        uint32_t hit[kBlendThreads / 32];
#pragma unroll
        for (int g = 0; g < kBlendThreads / 32; ++g) {
            const int s = g * 32 + lane;
            bool h = false;
            if (s < cnt) {
                const float4 g0 = s_g0[s];
                const float4 g1 = s_g1[s];
                const float ex = g1.z * 1.0001f + 0.01f, ey = g1.w * 1.0001f + 0.01f;
                const float dx = g0.x - fminf(fmaxf(g0.x, bx0), bx1);
                const float dy = g0.y - fminf(fmaxf(g0.y, by0), by1);
                h = fabsf(dx) <= ex && fabsf(dy) <= ey;
            }
            hit[g] = __ballot_sync(0xffffffffu, h);
        }
        bool warp_done = false;
#pragma unroll
        for (int g = 0; g < kBlendThreads / 32; ++g) {
            uint32_t m = warp_done ? 0u : hit[g];
            while (m) {
                const int s = g * 32 + __ffs(m) - 1;
                m &= m - 1;
                if (!done) {
                    const float4 g0 = s_g0[s];
                    const float4 g1 = s_g1[s];
                    const float dx = fpx - g0.x, dy = fpy - g0.y;
                    float power = -0.5f * (g0.z * dx * dx + g1.x * dy * dy) - g0.w * dx * dy;
                    power = fminf(power, 0.0f);
                    const float alpha = fminf(0.99f, g1.y * __expf(power));
                    if (alpha >= a_min) {
                        const float nT = T * (1.0f - alpha);
                        if (nT < 1e-4f) {
                            done = true;
                        } else {
                            const float4 c = s_c[s];
                            const float w = alpha * T;
                            cr = fmaf(c.x, w, cr);
                            cg = fmaf(c.y, w, cg);
                            cb = fmaf(c.z, w, cb);
                            T = nT;
                        }
                    }
                }
                if (__all_sync(0xffffffffu, done)) {
                    warp_done = true;
                    m = 0u;
                }
            }
        }
    }
    if (inside) {
        const size_t p = (size_t)py * width + px;
        image[3 * p + 0] = cr + T * bg0;
        image[3 * p + 1] = cg + T * bg1;
        image[3 * p + 2] = cb + T * bg2;
        if (final_T) final_T[p] = T;
    }
    if (threadIdx.x == 0 && pairs_read) atomicAdd(pairs_read, (unsigned long long)(fetched - begin));
}

int launch_blend(const uint2* ranges, const uint32_t* ids, const float4* rec, const DevCamera& cam,
                 const float bg[3], float* image, float* final_T, DevCounters* counters,
                 cudaStream_t st) {
    const int tiles = cam.tiles_x * cam.tiles_y;
    blend_kernel<<<tiles, kBlendThreads, 0, st>>>(ranges, ids, rec, cam.width, cam.height,
                                                  cam.tiles_x, bg[0], bg[1], bg[2], image, final_T,
                                                  counters ? &counters->pairs_read : nullptr);
    return 1;
}

}  // namespace recogs
