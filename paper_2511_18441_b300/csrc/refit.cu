// The SH-only refit of ReCoGS (arXiv 2511.18441, Sec. 3.3): with the geometry
// frozen, only the SH coefficients C are fitted to edited target views. The
// loss gradient with respect to the image is the hard-coded L1 term of Eq. 6
// (sign(y - target) / N; the SSIM weight is taken as 0), the rasteriser
// backward of Eq. 7 is needed only for dL/dC: the blend kernel in gradient
// mode gives dL/dc per Gaussian (Eq. 3 is linear in the colours), and this
// kernel chains it through Eq. 2 and steps C with Adam.
#include "recogs_internal.cuh"

namespace recogs {

// Real SH basis of degree 3 at a unit direction (Eq. 2), k = l*l + l + m,
// the same constants as the forward pass.
__device__ __forceinline__ void refit_sh_basis(float x, float y, float z, float* Y) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = 0.28209479177387814f;
    Y[1] = -0.4886025119029199f * y;
    Y[2] = 0.4886025119029199f * z;
    Y[3] = -0.4886025119029199f * x;
    Y[4] = 1.0925484305920792f * x * y;
    Y[5] = -1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (3.0f * zz - 1.0f);
    Y[7] = -1.0925484305920792f * x * z;
    Y[8] = 0.5462742152960396f * (xx - yy);
    Y[9] = -0.5900435899266436f * y * (3.0f * xx - yy);
    Y[10] = 2.8906114426405547f * x * y * z;
    Y[11] = -0.4570457994644658f * y * (5.0f * zz - 1.0f);
    Y[12] = 0.3731763325901154f * z * (5.0f * zz - 3.0f);
    Y[13] = -0.4570457994644658f * x * (5.0f * zz - 1.0f);
    Y[14] = 1.4453057213202773f * z * (xx - yy);
    Y[15] = -0.5900435899266436f * x * (xx - 3.0f * yy);
}

// Per Gaussian: dL/dC_{k,ch} = Y_k(d) [c_ch > 0] dL/dc_ch (the shown colour
// c = max(f + 0.5, 0) passes the gradient only where it is not clamped; a
// culled Gaussian has a zero gradient), written to grad_sh if given; with
// m and v, one Adam step (Kingma and Ba, 2015) of every coefficient:
// m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// C -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__global__ void __launch_bounds__(256)
    sh_refit_kernel(int n, const float* __restrict__ xyz, float3 cam_pos,
                    const float4* __restrict__ rec, const uint32_t* __restrict__ count,
                    const float* __restrict__ grad_rgb, float* __restrict__ sh,
                    float* __restrict__ m, float* __restrict__ v, RefitAdam adam,
                    float* __restrict__ grad_sh) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gc[3] = {0.f, 0.f, 0.f};
    float Y[16];
    if (count[i] > 0) {
        const float4 c = rec[3 * (size_t)i + 2];
        gc[0] = c.x > 0.f ? grad_rgb[3 * (size_t)i + 0] : 0.f;
        gc[1] = c.y > 0.f ? grad_rgb[3 * (size_t)i + 1] : 0.f;
        gc[2] = c.z > 0.f ? grad_rgb[3 * (size_t)i + 2] : 0.f;
        float dx = xyz[i] - cam_pos.x, dy = xyz[n + i] - cam_pos.y, dz = xyz[2 * n + i] - cam_pos.z;
        const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
        refit_sh_basis(dx * dn, dy * dn, dz * dn, Y);
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) Y[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const size_t o = (size_t)(3 * k + ch) * n + i;
            const float g = Y[k] * gc[ch];
            if (grad_sh) grad_sh[o] = g;
            if (m) {
                const float mm = adam.beta1 * m[o] + (1.0f - adam.beta1) * g;
                const float vv = adam.beta2 * v[o] + (1.0f - adam.beta2) * g * g;
                m[o] = mm;
                v[o] = vv;
                sh[o] -= adam.lr * (mm * adam.inv_bc1) / (sqrtf(vv * adam.inv_bc2) + adam.eps);
            }
        }
    }
}

int launch_sh_refit(int n, const float* xyz, const float cam_pos[3], const float4* rec,
                    const uint32_t* count, const float* grad_rgb, float* sh, float* m, float* v,
                    const RefitAdam& adam, float* grad_sh, cudaStream_t st) {
    if (n == 0) return 0;
    sh_refit_kernel<<<(n + 255) / 256, 256, 0, st>>>(
        n, xyz, make_float3(cam_pos[0], cam_pos[1], cam_pos[2]), rec, count, grad_rgb, sh, m, v,
        adam, grad_sh);
    return 1;
}

}  // namespace recogs
