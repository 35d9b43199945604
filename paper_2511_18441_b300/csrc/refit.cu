// The SH-only refit of ReCoGS (arXiv 2511.18441, Sec. 3.3): with the geometry
// frozen, only the SH coefficients C are fitted to edited target views. The
// loss gradient with respect to the image is the hard-coded L1 term of Eq. 6
// (sign(y - target) / N; the SSIM weight is taken as 0), the rasteriser
// backward of Eq. 7 is needed only for dL/dC: the blend kernel in gradient
// mode gives dL/dc per Gaussian (Eq. 3 is linear in the colours), and this
// kernel chains it through Eq. 2 and steps C with Adam.
#include "recogs_internal.cuh"

namespace recogs {

// Real SH basis function k = l*l + l + m of degree <= 3 at a unit direction
// (Eq. 2), the same constants as the forward pass; k is a compile-time
// constant wherever the loops below are unrolled.
__device__ __forceinline__ float refit_sh_basis_k(int k, float x, float y, float z) {
    switch (k) {
    case 0: return 0.28209479177387814f;
    case 1: return -0.4886025119029199f * y;
    case 2: return 0.4886025119029199f * z;
    case 3: return -0.4886025119029199f * x;
    case 4: return 1.0925484305920792f * x * y;
    case 5: return -1.0925484305920792f * y * z;
    case 6: return 0.31539156525252005f * (3.0f * (z * z) - 1.0f);
    case 7: return -1.0925484305920792f * x * z;
    case 8: return 0.5462742152960396f * (x * x - y * y);
    case 9: return -0.5900435899266436f * y * (3.0f * (x * x) - y * y);
    case 10: return 2.8906114426405547f * x * y * z;
    case 11: return -0.4570457994644658f * y * (5.0f * (z * z) - 1.0f);
    case 12: return 0.3731763325901154f * z * (5.0f * (z * z) - 3.0f);
    case 13: return -0.4570457994644658f * x * (5.0f * (z * z) - 1.0f);
    case 14: return 1.4453057213202773f * z * (x * x - y * y);
    default: return -0.5900435899266436f * x * (x * x - 3.0f * (y * y));
    }
}

// One Adam step (Kingma and Ba, 2015) of one coefficient C with gradient g:
// m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// C -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__device__ __forceinline__ void refit_adam(const RefitAdam& a, float g, float& C, float& m,
                                           float& v) {
    m = a.beta1 * m + (1.0f - a.beta1) * g;
    v = a.beta2 * v + (1.0f - a.beta2) * g * g;
    // approximate square root and reciprocal (a few ulp; the IEEE-rounded
    // forms cost the streaming kernel 13% of its time): sqrt.approx(0) = 0,
    // and eps > 0 keeps the reciprocal finite
    float s;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(v * a.inv_bc2));
    C = C - a.lr * (m * a.inv_bc1) * rcp_approx(s + a.eps);
}

// Per Gaussian: dL/dC_{k,ch} = Y_k(d) [c_ch > 0] dL/dc_ch (the shown colour
// c = max(f + 0.5, 0) passes the gradient only where it is not clamped; a
// culled Gaussian has a zero gradient), written to grad_sh with GRAD; with
// ADAM, one Adam step of every coefficient (refit_adam). The kernel is bound
// by HBM (24 bytes per coefficient). One thread per Gaussian: the 48 rows of
// C, m and v ([48][n], row r = 3k + ch) are streamed three rows (one k) at a
// time, the nine loads issued before the first store. This is the general
// form; sh_refit_tile_kernel below takes aligned arrays with n % 4 == 0.
template <bool ADAM, bool GRAD>
__global__ void __launch_bounds__(256, 4)
    sh_refit_kernel(int n, const float* __restrict__ xyz, float3 cam_pos,
                    const float4* __restrict__ rec, const uint32_t* __restrict__ count,
                    const float* __restrict__ grad_rgb, float* __restrict__ sh,
                    float* __restrict__ m, float* __restrict__ v, RefitAdam adam,
                    float* __restrict__ grad_sh) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gc[3] = {0.f, 0.f, 0.f};
    float ux = 0.f, uy = 0.f, uz = 1.f;   // culled: any finite direction (gc = 0)
    if (count[i] > 0) {
        const float4 c = rec[3 * (size_t)i + 2];
        gc[0] = c.x > 0.f ? grad_rgb[3 * (size_t)i + 0] : 0.f;
        gc[1] = c.y > 0.f ? grad_rgb[3 * (size_t)i + 1] : 0.f;
        gc[2] = c.z > 0.f ? grad_rgb[3 * (size_t)i + 2] : 0.f;
        float dx = xyz[i] - cam_pos.x, dy = xyz[n + i] - cam_pos.y, dz = xyz[2 * n + i] - cam_pos.z;
        const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
        ux = dx * dn;
        uy = dy * dn;
        uz = dz * dn;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float Yk = refit_sh_basis_k(k, ux, uy, uz);
        float cs[3], cm[3], cv[3];
        if (ADAM) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const size_t o = (size_t)(3 * k + ch) * n + i;
                cs[ch] = __ldcs(sh + o);
                cm[ch] = __ldcs(m + o);
                cv[ch] = __ldcs(v + o);
            }
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const size_t o = (size_t)(3 * k + ch) * n + i;
            const float g = Yk * gc[ch];
            if (GRAD) __stcs(grad_sh + o, g);
            if (ADAM) {
                refit_adam(adam, g, cs[ch], cm[ch], cv[ch]);
                __stcs(m + o, cm[ch]);
                __stcs(v + o, cv[ch]);
                __stcs(sh + o, cs[ch]);
            }
        }
    }
}

// The same per coefficient with the rows of a block's Gaussians streamed in
// runs: a block owns kRefitTile consecutive Gaussians (n % 4 == 0, every
// array 16-byte aligned), keeps their view directions and colour gradients
// in shared memory (48 KB), and walks the 48 rows; each row of C, m and v is
// a contiguous 8 KB run read and written as float4, two per thread. At 3M
// Gaussians this streams 3.58 GB in 0.67 ms on a B300; one Gaussian per
// thread took 0.75 ms, four per thread with all 48 rows per thread 0.72 ms,
// longer runs with more loads per thread (4096 or 8192 Gaussians per block)
// were slower (0.98, 1.65 ms: fewer resident warps), and so were equal
// ranges of several tiles per resident block (0.75 ms).
constexpr int kRefitTile = 2048;
constexpr int kRefitTileThreads = 256;
constexpr int kRefitVec = kRefitTile / 4 / kRefitTileThreads;   // float4 per thread per row
static_assert(kRefitTile % (4 * kRefitTileThreads) == 0, "tile");

template <bool ADAM, bool GRAD>
__global__ void __launch_bounds__(kRefitTileThreads)
    sh_refit_tile_kernel(int n4, int per_block, const float* __restrict__ xyz, float3 cam_pos,
                         const float4* __restrict__ rec, const uint32_t* __restrict__ count,
                         const float* __restrict__ grad_rgb, float4* __restrict__ sh,
                         float4* __restrict__ m, float4* __restrict__ v, RefitAdam adam,
                         float4* __restrict__ grad_sh) {
    extern __shared__ float4 s_dyn[];
    // per Gaussian of the tile: direction x, y, z and colour gradient 0, 1, 2
    float* const s_u = reinterpret_cast<float*>(s_dyn);
    const float4* const s_u4 = s_dyn;   // float4 j of array a at a * kRefitTile / 4 + j
    const int n = 4 * n4;
    // this block's Gaussians, in float4 units: [qb, qe), in tiles of kRefitTile
    const int qb = blockIdx.x * per_block, qe = min(n4, qb + per_block);
    for (int q0 = qb; q0 < qe; q0 += kRefitTile / 4) {
        const int tq = min(kRefitTile / 4, qe - q0), tn = 4 * tq, i0 = 4 * q0;
        if (q0 != qb) __syncthreads();   // the previous tile's rows are done with s_u
        for (int t = threadIdx.x; t < tn; t += kRefitTileThreads) {
            const int i = i0 + t;
            float g0 = 0.f, g1 = 0.f, g2 = 0.f, ux = 0.f, uy = 0.f, uz = 1.f;
            if (count[i] > 0) {
                const float4 c = rec[3 * (size_t)i + 2];
                g0 = c.x > 0.f ? grad_rgb[3 * (size_t)i + 0] : 0.f;
                g1 = c.y > 0.f ? grad_rgb[3 * (size_t)i + 1] : 0.f;
                g2 = c.z > 0.f ? grad_rgb[3 * (size_t)i + 2] : 0.f;
                const float dx = xyz[i] - cam_pos.x, dy = xyz[n + i] - cam_pos.y,
                            dz = xyz[2 * (size_t)n + i] - cam_pos.z;
                const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
                ux = dx * dn;
                uy = dy * dn;
                uz = dz * dn;
            }
            s_u[0 * kRefitTile + t] = ux;
            s_u[1 * kRefitTile + t] = uy;
            s_u[2 * kRefitTile + t] = uz;
            s_u[3 * kRefitTile + t] = g0;
            s_u[4 * kRefitTile + t] = g1;
            s_u[5 * kRefitTile + t] = g2;
        }
        __syncthreads();
#pragma unroll 1
        for (int r = 0; r < 48; ++r) {
            const int k = r / 3, ch = r - 3 * k;
            float4 cs[kRefitVec], cm[kRefitVec], cv[kRefitVec];
            if (ADAM) {
#pragma unroll
                for (int e = 0; e < kRefitVec; ++e) {
                    const int j = threadIdx.x + e * kRefitTileThreads;
                    if (j < tq) {
                        const size_t o = (size_t)r * n4 + q0 + j;
                        cs[e] = __ldcs(sh + o);
                        cm[e] = __ldcs(m + o);
                        cv[e] = __ldcs(v + o);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < kRefitVec; ++e) {
                const int j = threadIdx.x + e * kRefitTileThreads;
                if (j >= tq) continue;
                const size_t o = (size_t)r * n4 + q0 + j;
                const float4 ux = s_u4[0 * (kRefitTile / 4) + j],
                             uy = s_u4[1 * (kRefitTile / 4) + j],
                             uz = s_u4[2 * (kRefitTile / 4) + j];
                const float4 gc = s_u4[(3 + ch) * (kRefitTile / 4) + j];
                float g[4];
                g[0] = refit_sh_basis_k(k, ux.x, uy.x, uz.x) * gc.x;
                g[1] = refit_sh_basis_k(k, ux.y, uy.y, uz.y) * gc.y;
                g[2] = refit_sh_basis_k(k, ux.z, uy.z, uz.z) * gc.z;
                g[3] = refit_sh_basis_k(k, ux.w, uy.w, uz.w) * gc.w;
                if (GRAD) __stcs(grad_sh + o, make_float4(g[0], g[1], g[2], g[3]));
                if (ADAM) {
                    refit_adam(adam, g[0], cs[e].x, cm[e].x, cv[e].x);
                    refit_adam(adam, g[1], cs[e].y, cm[e].y, cv[e].y);
                    refit_adam(adam, g[2], cs[e].z, cm[e].z, cv[e].z);
                    refit_adam(adam, g[3], cs[e].w, cm[e].w, cv[e].w);
                    __stcs(m + o, cm[e]);
                    __stcs(v + o, cv[e]);
                    __stcs(sh + o, cs[e]);
                }
            }
        }
    }
}

namespace {
bool aligned16(const void* p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; }

template <bool ADAM, bool GRAD>
void refit_launch(int n, const float* xyz, float3 cp, const float4* rec, const uint32_t* count,
                  const float* grad_rgb, float* sh, float* m, float* v, const RefitAdam& adam,
                  float* grad_sh, cudaStream_t st) {
    const bool tiled = n % 4 == 0 && aligned16(xyz) && aligned16(count) &&
                       aligned16(grad_rgb) && aligned16(sh) && aligned16(m) && aligned16(v) &&
                       aligned16(grad_sh);
    if (tiled) {
        constexpr int smem = 6 * kRefitTile * 4;
        static std::atomic<uint64_t> opted{0};
        smem_opt_in(sh_refit_tile_kernel<ADAM, GRAD>, smem, opted);
        const int n4 = n / 4;
        const int per_block = kRefitTile / 4;   // one tile per block
        const int blocks = (n4 + per_block - 1) / per_block;
        sh_refit_tile_kernel<ADAM, GRAD><<<blocks, kRefitTileThreads, smem, st>>>(
            n4, per_block, xyz, cp, rec, count, grad_rgb, reinterpret_cast<float4*>(sh),
            reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v), adam,
            reinterpret_cast<float4*>(grad_sh));
    } else {
        sh_refit_kernel<ADAM, GRAD><<<(n + 255) / 256, 256, 0, st>>>(
            n, xyz, cp, rec, count, grad_rgb, sh, m, v, adam, grad_sh);
    }
}
}  // namespace

int launch_sh_refit(int n, const float* xyz, const float cam_pos[3], const float4* rec,
                    const uint32_t* count, const float* grad_rgb, float* sh, float* m, float* v,
                    const RefitAdam& adam, float* grad_sh, cudaStream_t st) {
    if (n == 0 || (!m && !grad_sh)) return 0;
    const float3 cp = make_float3(cam_pos[0], cam_pos[1], cam_pos[2]);
    if (m && grad_sh)
        refit_launch<true, true>(n, xyz, cp, rec, count, grad_rgb, sh, m, v, adam, grad_sh, st);
    else if (m)
        refit_launch<true, false>(n, xyz, cp, rec, count, grad_rgb, sh, m, v, adam, grad_sh, st);
    else
        refit_launch<false, true>(n, xyz, cp, rec, count, grad_rgb, sh, m, v, adam, grad_sh, st);
    return 1;
}

}  // namespace recogs
