// Fourth-order divergence with caller-supplied coefficients d_ijkl
// (Eq. gen4thPDE_Model): (P u) = sum_ij d_ij [ sum_kl d_ijkl u_kl ], with the
// Hessian stencils of Sec. 3.3 and the boundary rule of the solver: u
// mirrored, T_xx and T_yy mirrored, T_xy and T_yx odd across each border.
// Any field d expresses a member of the paper's unifying framework (FOEED,
// You-Kaveh, Hajiaboli, Li et al.); it need not be symmetric.
#include <cuda_runtime.h>

#include "dispatch.h"
#include "foeed_device.cuh"

namespace foeed {

namespace {

constexpr int FW = 32, FH = 16;

template <typename T>
__global__ void __launch_bounds__(256) apply_field_kernel(const T *__restrict__ u, const T *__restrict__ d,
                                                          T *__restrict__ pu, int w, int h, long pitch)
{
    constexpr int UW = FW + 4, UH = FH + 4;  // u on tile +- 2
    constexpr int QW = FW + 2, QH = FH + 2;  // T on tile +- 1
    __shared__ T su[UH * UW];
    __shared__ T st[4][QH * QW];
    const int x0 = blockIdx.x * FW, y0 = blockIdx.y * FH;
    for (int i = threadIdx.x; i < UW * UH; i += 256) {
        int r = i / UW, c = i - r * UW;
        su[i] = u[(long)mirror_idx(y0 - 2 + r, h) * pitch + mirror_idx(x0 - 2 + c, w)];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < QW * QH; i += 256) {
        int r = i / QW, c = i - r * QW;
        const int px = x0 - 1 + c, py = y0 - 1 + r;
        if (px > w || py > h) continue;  // never read: outputs stop at w - 1, h - 1
        const int mx = mirror_idx(px, w), my = mirror_idx(py, h);
        // odd components flip sign once per reflection
        const int fx = px < 0 || px >= w, fy = py < 0 || py >= h;
        const T sgn = (fx ^ fy) ? T(-1) : T(1);
        // Hessian of u at the mirrored pixel (inside the loaded window)
        const T *u0 = su + (my - (y0 - 2)) * UW + (mx - (x0 - 2));
        const T hxx = (u0[-1] + u0[1]) - T(2) * u0[0];
        const T hyy = (u0[-UW] + u0[UW]) - T(2) * u0[0];
        const T hxy = ((u0[UW + 1] + u0[-UW - 1]) - (u0[UW - 1] + u0[-UW + 1])) / T(4);
        const T H[4] = {hxx, hxy, hxy, hyy};
        const T *dp = d + ((long)my * pitch + mx) * 16;
#pragma unroll
        for (int ij = 0; ij < 4; ++ij) {
            T s = T(0);
#pragma unroll
            for (int kl = 0; kl < 4; ++kl) s += dp[ij * 4 + kl] * H[kl];
            st[ij][i] = (ij == 1 || ij == 2) ? sgn * s : s;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < FW * FH; i += 256) {
        int r = i / FW, c = i - r * FW;
        const int gx = x0 + c, gy = y0 + r;
        if (gx >= w || gy >= h) continue;
        const int k = (r + 1) * QW + (c + 1);
        const T dxx = (st[0][k - 1] + st[0][k + 1]) - T(2) * st[0][k];
        const T dxy = ((st[1][k + QW + 1] + st[1][k - QW - 1]) - (st[1][k + QW - 1] + st[1][k - QW + 1])) / T(4);
        const T dyx = ((st[2][k + QW + 1] + st[2][k - QW - 1]) - (st[2][k + QW - 1] + st[2][k - QW + 1])) / T(4);
        const T dyy = (st[3][k - QW] + st[3][k + QW]) - T(2) * st[3][k];
        pu[(long)gy * pitch + gx] = ((dxx + dxy) + dyx) + dyy;
    }
}

}  // namespace

cudaError_t apply_field(const void *u, const void *d, void *pu, int w, int h, long pitch, bool f64, cudaStream_t s)
{
    dim3 grid((w + FW - 1) / FW, (h + FH - 1) / FH);
    if (f64)
        apply_field_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double *>(u), static_cast<const double *>(d),
                                                        static_cast<double *>(pu), w, h, pitch);
    else
        apply_field_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float *>(u), static_cast<const float *>(d),
                                                       static_cast<float *>(pu), w, h, pitch);
    return cudaGetLastError();
}

}  // namespace foeed
