// Backward (adjoint) kernels of one masked FOEED FSI step, for the gradient of
// a loss of the reconstruction with respect to the stored grey values.
//
// Step: u^{k+1} = M u^k + (1-M)(a (u^k - tau F(u^k)) + (1-a) p),  F(x) = P(x) x,
// p = u^{k-1} (u^k at the first step of a cycle). Given g = dL/du^{k+1}:
//   v = (1-M) g
//   J_F(x)^T v = P(x) v + G D^T q,   q = d/d(grad u_sigma) of  H(v) : D(grad u_sigma) : H(x)
//   dL/du^k += M g + a v - a tau J_F(x)^T v,   dL/dp += (1-a) v
// P is symmetric (outer operator = transpose of the inner one), so its
// transpose is P itself; G (mirrored Gaussian) is symmetric; D^T = -D_odd
// (central difference with odd ghosts).
//
// B1 computes P(x) v and q on a tile (the forward stages on x, plus the
// Hessian of v); B2 applies -D_odd to q, the Gaussian, and the recursion.
#pragma once

#include "foeed_device.cuh"

namespace foeed {

template <typename T>
struct AdjArgs {
    const T *x;          // state u^k (internal pitch)
    const T *g;          // dL/du^{k+1}
    const uint8_t *mask; // internal 0/1 mask
    T *pv;               // out (B1): P(x) v
    T *qx, *qy;          // out (B1) / in (B2)
    T *gout;             // out (B2): dL/du^k (may alias g)
    T *pend;             // in/out (B2): pending dL/du^k from the next step's u^{k-1} use
    int w, h;
    long pitch;
    T alpha, tau;
    T l2;                // lambda^2
    T inv_l2;            // 1 / lambda^2
    T wts[2 * kRMax + 1];
    int first_of_cycle;  // 1: this step's p is u^k itself
};

// Tiles of TW x 16 pixels: 64 wide in FP32, 32 wide in FP64 (shared memory).
constexpr int kAdjTH = 16;
template <typename T>
constexpr int adj_tile_w() { return sizeof(T) == sizeof(float) ? 64 : 32; }

// FP32 approximations (MUFU) used by the FP32 kernels; FP64 keeps IEEE operations.
__device__ __forceinline__ float adj_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float adj_rsqrt(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float adj_sqrt(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Asynchronous global -> shared copies (cp.async) of 16 bytes, of one element, of 4 bytes.
__device__ __forceinline__ uint32_t adj_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void adj_cp16(uint32_t d, const void *s)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(s) : "memory");
}
template <typename T>
__device__ __forceinline__ void adj_cp_elem(uint32_t d, const T *s)
{
    if (sizeof(T) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(s) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(s) : "memory");
}
__device__ __forceinline__ void adj_cp4(uint32_t d, const void *s)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(s) : "memory");
}
__device__ __forceinline__ void adj_cp_wait()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Eight consecutive floats from shared memory (two float4 loads; s is 16-byte aligned).
__device__ __forceinline__ void ld_8f(const float *s, float *o)
{
    const float4 a = *reinterpret_cast<const float4 *>(s);
    const float4 b = *reinterpret_cast<const float4 *>(s + 4);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
// B1 in FP64 (the FP32 path is adj_b1_fast below): P(x) v and q at every pixel
// of a TW x 16 tile.
template <typename T, int R, int TW>
__global__ void __launch_bounds__(256) adj_b1_kernel(const AdjArgs<T> a)
{
    constexpr int TH = kAdjTH;
    constexpr int HL = R + 2;
    constexpr int E = 16 / (int)sizeof(T);            // elements per 16 bytes
    constexpr int XW = TW + 16, XH = TH + 2 * HL;     // x window: cols x0-8 .. x0+TW+7
    constexpr int XOFF = 8 - HL;                      // window column of x0 - HL
    constexpr int VW = TW + 8, VH = TH + 4;           // g and mask windows: cols x0-4 .. x0+TW+3, rows tile +- 2
    constexpr int VOFF = 2;                           // window column of x0 - 2
    constexpr int SW = TW + 4, SH = TH + 4;           // u_sigma on tile +- 2
    constexpr int QW = TW + 2, QH = TH + 2;           // tile +- 1
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sxw = reinterpret_cast<T *>(smem_raw);
    T *sv = sxw + XW * XH;     // g, then v = (1 - M) g
    T *sxp = sv + VW * VH;     // x pass: XH rows x SW columns
    T *ss = sxp + XH * SW;     // u_sigma
    T *tw = ss + SW * SH;      // T_w = D : H(v), 3 planes on tile +- 1
    unsigned char *smk = reinterpret_cast<unsigned char *>(tw + 3 * QW * QH);  // mask window
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const int w = a.w, h = a.h;
    const long pitch = a.pitch;
    // Windows copied asynchronously: 16-byte copies where all their columns lie
    // inside the image, otherwise element copies of the mirrored pixels.
    {
        const bool xin = x0 - 8 >= 0 && x0 + TW + 8 <= w;
        const bool vin = x0 - 4 >= 0 && x0 + TW + 4 <= w;
        const uint32_t bx = adj_smem(sxw), bv = adj_smem(sv), bm = adj_smem(smk);
        for (int i = tid; i < XH * (XW / E); i += 256) {
            const int r = i / (XW / E), q = i - r * (XW / E);
            const T *row = a.x + (long)mirror_idx(y0 - HL + r, h) * pitch;
            const int gx = x0 - 8 + E * q;
            const uint32_t d = bx + (uint32_t)sizeof(T) * (r * XW + E * q);
            if (xin) {
                adj_cp16(d, row + gx);
            } else {
                for (int j = 0; j < E; ++j) adj_cp_elem(d + (uint32_t)sizeof(T) * j, row + mirror_idx(gx + j, w));
            }
        }
        for (int i = tid; i < VH * (VW / E); i += 256) {
            const int r = i / (VW / E), q = i - r * (VW / E);
            const T *row = a.g + (long)mirror_idx(y0 - 2 + r, h) * pitch;
            const int gx = x0 - 4 + E * q;
            const uint32_t d = bv + (uint32_t)sizeof(T) * (r * VW + E * q);
            if (vin) {
                adj_cp16(d, row + gx);
            } else {
                for (int j = 0; j < E; ++j) adj_cp_elem(d + (uint32_t)sizeof(T) * j, row + mirror_idx(gx + j, w));
            }
        }
        for (int i = tid; i < VH * (VW / 4); i += 256) {
            const int r = i / (VW / 4), q = i - r * (VW / 4);
            const uint8_t *row = a.mask + (long)mirror_idx(y0 - 2 + r, h) * pitch;
            const int gx = x0 - 4 + 4 * q;
            if (vin) {
                adj_cp4(bm + (uint32_t)(r * VW + 4 * q), row + gx);
            } else {
                for (int j = 0; j < 4; ++j) smk[r * VW + 4 * q + j] = row[mirror_idx(gx + j, w)];
            }
        }
        adj_cp_wait();
    }
    __syncthreads();
    for (int i = tid; i < VW * VH; i += 256)  // v = (1 - M) g
        if (smk[i]) sv[i] = T(0);
    for (int i = tid; i < XH * SW; i += 256) {  // Gaussian x pass
        int r = i / SW, c = i - r * SW;
        const T *row = sxw + r * XW + c + XOFF;
        T acc = T(0);
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) acc += a.wts[t] * row[t];
        sxp[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < SW * SH; i += 256) {  // Gaussian y pass
        int r = i / SW, c = i - r * SW;
        const T *col = sxp + r * SW + c;
        T acc = T(0);
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) acc += a.wts[t] * col[t * SW];
        ss[i] = acc;
    }
    __syncthreads();
    constexpr int PL = QW * QH;
    const T l2 = a.l2;
    for (int i = tid; i < PL; i += 256) {
        int r = i / QW, c = i - r * QW;  // tile (r-1, c-1)
        const T *s0 = ss + (r + 1) * SW + (c + 1);
        const T gx = (s0[1] - s0[-1]) * T(0.5), gy = (s0[SW] - s0[-SW]) * T(0.5);
        const T rho2 = gx * gx + gy * gy;
        T C, S;
        const T sq = sqrt(T(1) + rho2 / l2);  // 1 / mu1
        const T mu1 = T(1) / sq;
        const T mu3 = sqrt(mu1);
        if (rho2 == T(0)) { C = T(1); S = T(0); }
        else { C = (gx * gx - gy * gy) / rho2; S = T(2) * gx * gy / rho2; }
        const T *x0p = sxw + (r + 1 + R) * XW + (c + 1 + R + XOFF);
        const T *v0 = sv + (r + 1) * VW + (c + 1 + VOFF);
        const T hxx = (x0p[-1] + x0p[1]) - T(2) * x0p[0];
        const T hyy = (x0p[-XW] + x0p[XW]) - T(2) * x0p[0];
        const T hxy = ((x0p[XW + 1] + x0p[-XW - 1]) - (x0p[XW - 1] + x0p[-XW + 1])) * T(0.25);
        const T wxx = (v0[-1] + v0[1]) - T(2) * v0[0];
        const T wyy = (v0[-VW] + v0[VW]) - T(2) * v0[0];
        const T wxy = ((v0[VW + 1] + v0[-VW - 1]) - (v0[VW - 1] + v0[-VW + 1])) * T(0.25);
        // rotated frame (double angle C = cos 2t, S = sin 2t)
        const T Ah = (hxx + hyy) * T(0.5), Bh = (hxx - hyy) * T(0.5);
        const T Aw = (wxx + wyy) * T(0.5), Bw = (wxx - wyy) * T(0.5);
        const T h11 = Ah + C * Bh + S * hxy, h22 = Ah - C * Bh - S * hxy, h12 = C * hxy - S * Bh;
        const T w11 = Aw + C * Bw + S * wxy, w22 = Aw - C * Bw - S * wxy, w12 = C * wxy - S * Bw;
        // T_w = D : W  (the frozen-tensor part applies P(x) to v)
        {
            const T pp = mu1 * w11, qq = w22, rr = mu3 * w12;
            const T hs = (pp + qq) * T(0.5), hd = (pp - qq) * T(0.5);
            tw[i] = hs + C * hd - S * rr;
            tw[PL + i] = S * hd + C * rr;
            tw[2 * PL + i] = hs - C * hd + S * rr;
        }
        // q = d s / d g for s = W : D(g) : H = W:H + (mu1-1) w11 h11 + 2 (mu3-1) w12 h12
        if (r >= 1 && r <= TH && c >= 1 && c <= TW) {
            const int gxp = x0 + c - 1, gyp = y0 + r - 1;
            if (gxp < w && gyp < h) {
                // d mu1 / d rho^2, d mu3 / d rho^2, (1 - mu1) / rho^2, (1 - mu3) / rho^2
                const T dmu1 = -mu1 * mu1 * mu1 / (T(2) * l2);
                const T dmu3 = dmu1 / (T(2) * mu3);
                const T rs = sqrt(sq);
                const T c1 = T(1) / (l2 * sq * (sq + T(1)));
                const T c3 = T(1) / (l2 * (sq + T(1)) * rs * (rs + T(1)));
                const T srho = dmu1 * w11 * h11 + T(2) * dmu3 * w12 * h12;  // d s / d rho^2
                const T th = -c1 * T(2) * (w12 * h11 + w11 * h12) - T(2) * c3 * (-(w11 - w22) * h12 - w12 * (h11 - h22));
                const long gi = (long)gyp * pitch + gxp;
                a.qx[gi] = T(2) * gx * srho - gy * th;
                a.qy[gi] = T(2) * gy * srho + gx * th;
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < TW * TH; i += 256) {  // P(x) v: outer divergence of T_w
        int r = i / TW, c = i - r * TW;
        int gxp = x0 + c, gyp = y0 + r;
        if (gxp >= w || gyp >= h) continue;
        const int k = (r + 1) * QW + (c + 1);
        const T *txx = tw, *txy = tw + PL, *tyy = tw + 2 * PL;
        const T dxx = (txx[k - 1] + txx[k + 1]) - T(2) * txx[k];
        const T dyy = (tyy[k - QW] + tyy[k + QW]) - T(2) * tyy[k];
        const T dxy = ((txy[k + QW + 1] + txy[k - QW - 1]) - (txy[k + QW - 1] + txy[k - QW + 1])) * T(0.5);
        a.pv[(long)gyp * pitch + gxp] = (dxx + dyy) + dxy;
    }
}

// -D_odd q at pixel (x, y): the transpose of the central-difference gradient
// (q_x odd across the left/right border, q_y across the top/bottom border).
template <typename T>
__device__ __forceinline__ T adj_divq(const AdjArgs<T> &a, int x, int y)
{
    const long row = (long)y * a.pitch;
    const T xr = x + 1 < a.w ? a.qx[row + x + 1] : -a.qx[row + x];
    const T xl = x - 1 >= 0 ? a.qx[row + x - 1] : -a.qx[row + x];
    const T yd = y + 1 < a.h ? a.qy[row + a.pitch + x] : -a.qy[row + x];
    const T yu = y - 1 >= 0 ? a.qy[row - a.pitch + x] : -a.qy[row + x];
    return -((xr - xl) + (yd - yu)) * T(0.5);
}

// B2 in FP64 (the FP32 path is adj_b2_fast below): z = G (-D_odd q), then the
// step's adjoint recursion at every pixel of a tile.
template <typename T, int R, int TW>
__global__ void __launch_bounds__(256) adj_b2_kernel(const AdjArgs<T> a)
{
    constexpr int TH = kAdjTH;
    constexpr int RW = TW + 2 * R, RH = TH + 2 * R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sr = reinterpret_cast<T *>(smem_raw);  // -D_odd q on tile +- R (mirrored outside the image)
    T *sxp = sr + RW * RH;                    // x pass: RH rows x TW columns
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    for (int i = tid; i < RW * RH; i += 256) {
        int r = i / RW, c = i - r * RW;
        sr[i] = adj_divq(a, mirror_idx(x0 - R + c, a.w), mirror_idx(y0 - R + r, a.h));
    }
    __syncthreads();
    for (int i = tid; i < RH * TW; i += 256) {
        int r = i / TW, c = i - r * TW;
        const T *row = sr + r * RW + c;
        T acc = T(0);
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) acc += a.wts[t] * row[t];
        sxp[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < TW * TH; i += 256) {
        int r = i / TW, c = i - r * TW;
        int gxp = x0 + c, gyp = y0 + r;
        if (gxp >= a.w || gyp >= a.h) continue;
        const T *col = sxp + r * TW + c;
        T z = T(0);
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) z += a.wts[t] * col[t * TW];
        const long gi = (long)gyp * a.pitch + gxp;
        const T gv = a.g[gi];
        const bool known = a.mask[gi] != 0;
        const T v = known ? T(0) : gv;
        const T jt = a.pv[gi] + z;  // J_F(x)^T v
        const T dcur = (known ? gv : T(0)) + a.alpha * v - a.alpha * a.tau * jt;
        const T dprev = (T(1) - a.alpha) * v;
        const T pe = a.pend[gi];
        if (a.first_of_cycle) {
            a.gout[gi] = pe + dcur + dprev;
            a.pend[gi] = T(0);
        } else {
            a.gout[gi] = pe + dcur;
            a.pend[gi] = dprev;
        }
    }
}

// ---------------------------------------------------------------------------
// B1 for FP32, register-blocked like the forward step kernel: 64 x 16 tiles,
// 256 threads; the windows are copied with one fixed float4 column per thread,
// the x pass produces 8 outputs per item, the y pass 2 rows per item, and the
// tensor stage 4 consecutive positions per item from float4 shared loads.

// Two-lane FP32 arithmetic: a - b as fma(b, -1, a) (one rounding, as a subtraction);
// an aligned register pair of a float array.
__device__ __forceinline__ float2 adj_sub2(const float2 a, const float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 adj_pr(const float *v, const int i) { return make_float2(v[i], v[i + 1]); }

// The adjoint arithmetic of two positions (the algebra of adj_b1_kernel), in
// two-lane FP32 instructions with the MUFU approximations lane by lane:
// T_w = D : W and q = d/d(grad u_sigma) of W : D : H, formed for both lanes.
// In the rotated frame of grad u_sigma (C = cos 2theta, S = sin 2theta), with
// sq = 1/mu1, mu3 = sqrt(mu1) (so sqrt(sq) = 1/mu3 = mu3 sq = rs):
//   T_w = (mu1 w11 v1 v1^T + w22 v2 v2^T) + mu3 w12 (v1 v2^T + v2 v1^T)
//   srho = dmu1 w11 h11 + 2 dmu3 w12 h12, th = 2 (c3 e3 - c1 e1),
//   e1 = w12 h11 + w11 h12, e3 = (w11 - w22) h12 + w12 (h11 - h22),
//   q = 2 srho grad u_sigma + th grad u_sigma^perp,
// where the two reciprocals c1 = 1/(A sq), c3 = 1/(A B) (A = l2 (sq + 1),
// B = rs (rs + 1)) share one: c1 = B / (A sq B), c3 = sq / (A sq B).
__device__ __forceinline__ void adj_position_f32x2(const float2 gx, const float2 gy, const float2 hxx,
                                                   const float2 hyy, const float2 hxy, const float2 wxx,
                                                   const float2 wyy, const float2 wxy, const float inv_l2,
                                                   const float l2, float2 &txx, float2 &txy, float2 &tyy,
                                                   float2 &qx, float2 &qy)
{
    const float2 half = make_float2(0.5f, 0.5f), m1 = make_float2(-1.f, -1.f);
    const float2 gx2 = __fmul2_rn(gx, gx), gy2 = __fmul2_rn(gy, gy);
    const float2 rho2 = __fadd2_rn(gx2, gy2);
    const float2 t = __ffma2_rn(rho2, make_float2(inv_l2, inv_l2), make_float2(1.f, 1.f));
    const float2 mu1 = make_float2(adj_rsqrt(t.x), adj_rsqrt(t.y));
    const float2 sq = __fmul2_rn(t, mu1);  // 1 / mu1
    const float2 mu3 = make_float2(adj_sqrt(mu1.x), adj_sqrt(mu1.y));
    const float2 inv = make_float2(adj_rcp(rho2.x), adj_rcp(rho2.y));
    float2 C = __fmul2_rn(adj_sub2(gx2, gy2), inv);
    float2 S = __fmul2_rn(__fmul2_rn(__fadd2_rn(gx, gx), gy), inv);
    if (rho2.x == 0.f) { C.x = 1.f; S.x = 0.f; }
    if (rho2.y == 0.f) { C.y = 1.f; S.y = 0.f; }
    const float2 nC = __fmul2_rn(C, m1), nS = __fmul2_rn(S, m1);
    const float2 Ah = __fmul2_rn(__fadd2_rn(hxx, hyy), half), Bh = __fmul2_rn(adj_sub2(hxx, hyy), half);
    const float2 Aw = __fmul2_rn(__fadd2_rn(wxx, wyy), half), Bw = __fmul2_rn(adj_sub2(wxx, wyy), half);
    const float2 h11 = __ffma2_rn(S, hxy, __ffma2_rn(C, Bh, Ah));
    const float2 h22 = __ffma2_rn(nS, hxy, __ffma2_rn(nC, Bh, Ah));
    const float2 h12 = __ffma2_rn(nS, Bh, __fmul2_rn(C, hxy));
    const float2 w11 = __ffma2_rn(S, wxy, __ffma2_rn(C, Bw, Aw));
    const float2 w22 = __ffma2_rn(nS, wxy, __ffma2_rn(nC, Bw, Aw));
    const float2 w12 = __ffma2_rn(nS, Bw, __fmul2_rn(C, wxy));
    const float2 pp = __fmul2_rn(mu1, w11), rr = __fmul2_rn(mu3, w12);
    const float2 hs = __fmul2_rn(__fadd2_rn(pp, w22), half), hd = __fmul2_rn(adj_sub2(pp, w22), half);
    txx = __ffma2_rn(nS, rr, __ffma2_rn(C, hd, hs));
    txy = __ffma2_rn(S, hd, __fmul2_rn(C, rr));
    tyy = __ffma2_rn(S, rr, __ffma2_rn(nC, hd, hs));
    const float2 dmu1 = __fmul2_rn(__fmul2_rn(__fmul2_rn(mu1, mu1), mu1), make_float2(-0.5f * inv_l2, -0.5f * inv_l2));
    const float2 rs = __fmul2_rn(mu3, sq);
    const float2 dmu3 = __fmul2_rn(__fmul2_rn(dmu1, half), rs);
    const float2 A = __ffma2_rn(make_float2(l2, l2), sq, make_float2(l2, l2)), B = __ffma2_rn(rs, rs, rs);
    const float2 den = __fmul2_rn(__fmul2_rn(A, sq), B);
    const float2 rAB = make_float2(adj_rcp(den.x), adj_rcp(den.y));
    const float2 c1 = __fmul2_rn(B, rAB), c3 = __fmul2_rn(sq, rAB);
    const float2 srho = __ffma2_rn(__fmul2_rn(__fadd2_rn(dmu3, dmu3), w12), h12, __fmul2_rn(__fmul2_rn(dmu1, w11), h11));
    const float2 e1 = __ffma2_rn(w12, h11, __fmul2_rn(w11, h12));
    const float2 e3 = __ffma2_rn(adj_sub2(w11, w22), h12, __fmul2_rn(w12, adj_sub2(h11, h22)));
    const float2 th = __fmul2_rn(adj_sub2(__fmul2_rn(c3, e3), __fmul2_rn(c1, e1)), make_float2(2.f, 2.f));
    qx = adj_sub2(__fmul2_rn(__fadd2_rn(gx, gx), srho), __fmul2_rn(gy, th));
    qy = __ffma2_rn(gx, th, __fmul2_rn(__fadd2_rn(gy, gy), srho));
}

template <int R>
struct AdjFast {
    static constexpr int TW = 64, TH = kAdjTH, HL = R + 2;
    static constexpr int XS = 84, XH = TH + 2 * HL;  // x window: cols x0-8 .. x0+71 (80 loaded), stride 21 float4
    static constexpr int VS = 76, VH = TH + 4;       // v window: cols x0-4 .. x0+67 (72 loaded), rows tile +- 2
    static constexpr int MS = 72;                   // mask window stride (bytes)
    static constexpr int PS = 76;                   // x pass: cols x0-2 .. x0+69 (72 computed), XH rows
    static constexpr int SS = 76, SH = TH + 4;      // u_sigma: cols x0-2 .. x0+65 (68), rows tile +- 2
    static constexpr int QS = 68, QH = TH + 2;      // T_w planes: positions tile +- 1, cols x0-1 .. x0+66
    static constexpr int PQ = (PS * XH > 3 * QS * QH) ? PS * XH : 3 * QS * QH;  // x pass and T_w share
    static constexpr int ELEMS = XS * XH + VS * VH + PQ + SS * SH + (MS * VH) / 4;
    static constexpr size_t SMEM = sizeof(float) * ELEMS;
};

template <int R>
__global__ void __launch_bounds__(256, 3) adj_b1_fast(const AdjArgs<float> a)
{
    using G = AdjFast<R>;
    constexpr int TW = G::TW, TH = G::TH, HL = G::HL;
    extern __shared__ __align__(16) float sm[];
    float *sxw = sm;                       // x window
    float *sv = sxw + G::XS * G::XH;       // g, then v = (1 - M) g
    float *sxp = sv + G::VS * G::VH;       // x pass; then the T_w planes
    float *tw = sxp;
    float *ss = sxp + G::PQ;               // u_sigma
    unsigned char *smk = reinterpret_cast<unsigned char *>(ss + G::SS * G::SH);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const int w = a.w, h = a.h;
    const long pitch = a.pitch;

    // ---- windows: thread tid owns one float4 (or 4-byte) column and strided rows ----
    {
        if (tid < 240) {  // x: 20 float4 columns, 12 rows per pass
            const int q = tid % 20, r0 = tid / 20, gx = x0 - 8 + 4 * q;
            const bool xin = gx >= 0 && gx + 4 <= w;  // this column lies inside the image
            uint32_t d = adj_smem(sxw) + 4u * (uint32_t)(r0 * G::XS + 4 * q);
            for (int r = r0; r < G::XH; r += 12, d += 4u * 12 * G::XS) {
                const float *row = a.x + (long)mirror_idx(y0 - HL + r, h) * pitch;
                if (xin) adj_cp16(d, row + gx);
                else
                    for (int j = 0; j < 4; ++j) adj_cp_elem(d + 4u * j, row + mirror_idx(gx + j, w));
            }
        }
        if (tid < 252) {  // g: 18 float4 columns, 14 rows per pass; mask: 18 four-byte columns
            const int q = tid % 18, r0 = tid / 18, gx = x0 - 4 + 4 * q;
            const bool vin = gx >= 0 && gx + 4 <= w;
            uint32_t d = adj_smem(sv) + 4u * (uint32_t)(r0 * G::VS + 4 * q);
            uint32_t dm = adj_smem(smk) + (uint32_t)(r0 * G::MS + 4 * q);
            for (int r = r0; r < G::VH; r += 14, d += 4u * 14 * G::VS, dm += 14 * G::MS) {
                const long ro = (long)mirror_idx(y0 - 2 + r, h) * pitch;
                if (vin) {
                    adj_cp16(d, a.g + ro + gx);
                    adj_cp4(dm, a.mask + ro + gx);
                } else {
                    for (int j = 0; j < 4; ++j) {
                        const int c = mirror_idx(gx + j, w);
                        adj_cp_elem(d + 4u * j, a.g + ro + c);
                        smk[(r * G::MS + 4 * q) + j] = a.mask[ro + c];
                    }
                }
            }
        }
        adj_cp_wait();
    }
    __syncthreads();
    // v = (1 - M) g, one float4 per item
    for (int i = tid; i < G::VH * 18; i += 256) {
        const int r = i / 18, q = i - r * 18;
        float4 *p = reinterpret_cast<float4 *>(sv + r * G::VS + 4 * q);
        const uint32_t m = *reinterpret_cast<const uint32_t *>(smk + r * G::MS + 4 * q);
        if (m) {
            float4 v = *p;
            if (m & 0xffu) v.x = 0.f;
            if (m & 0xff00u) v.y = 0.f;
            if (m & 0xff0000u) v.z = 0.f;
            if (m & 0xff000000u) v.w = 0.f;
            *p = v;
        }
    }
    // ---- x pass: sxp (row i, col c <-> global x0-2+c) <- x window cols c+6-R .. c+6+R; 8 outputs per item ----
    {
        float wt[2 * R + 1];
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) wt[t] = a.wts[t];
        for (int i = tid; i < G::XH * 9; i += 256) {
            const int g = i / G::XH, r = i - g * G::XH;  // consecutive lanes on consecutive rows
            const float *src = sxw + r * G::XS + 8 * g;
            float v[20];
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const float4 f = *reinterpret_cast<const float4 *>(src + 4 * j);
                v[4 * j] = f.x; v[4 * j + 1] = f.y; v[4 * j + 2] = f.z; v[4 * j + 3] = f.w;
            }
            float o[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int t = -R; t <= R; ++t) acc = fmaf(wt[t + R], v[6 + k + t], acc);
                o[k] = acc;
            }
            float *dst = sxp + r * G::PS + 8 * g;
            *reinterpret_cast<float4 *>(dst) = make_float4(o[0], o[1], o[2], o[3]);
            *reinterpret_cast<float4 *>(dst + 4) = make_float4(o[4], o[5], o[6], o[7]);
        }
    }
    __syncthreads();
    // ---- y pass: ss row i (global y0-2+i) <- sxp rows i .. i+2R; 2 rows x 4 columns per item ----
    {
        float wt[2 * R + 1];
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) wt[t] = a.wts[t];
        constexpr int NS = G::SH / 2;
        for (int i = tid; i < NS * 17; i += 256) {
            const bool main = i < NS * 16;
            const int s = main ? (i >> 4) : i - NS * 16, q = main ? (i & 15) : 16;
            const float *src = sxp + (2 * s) * G::PS + 4 * q;
            float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0;
#pragma unroll
            for (int j = 0; j < 2 * R + 2; ++j) {
                const float4 f = *reinterpret_cast<const float4 *>(src + j * G::PS);
                if (j <= 2 * R) {
                    const float c = wt[j];
                    o0.x = fmaf(c, f.x, o0.x); o0.y = fmaf(c, f.y, o0.y); o0.z = fmaf(c, f.z, o0.z); o0.w = fmaf(c, f.w, o0.w);
                }
                if (j >= 1) {
                    const float c = wt[j - 1];
                    o1.x = fmaf(c, f.x, o1.x); o1.y = fmaf(c, f.y, o1.y); o1.z = fmaf(c, f.z, o1.z); o1.w = fmaf(c, f.w, o1.w);
                }
            }
            *reinterpret_cast<float4 *>(ss + (2 * s) * G::SS + 4 * q) = o0;
            *reinterpret_cast<float4 *>(ss + (2 * s + 1) * G::SS + 4 * q) = o1;
        }
    }
    __syncthreads();
    // ---- T_w and q at positions (r, c), r = 0 .. TH+1, c = 0 .. 67 <-> global (y0-1+r, x0-1+c);
    // one row of four positions per item ----
    constexpr int PL = G::QS * G::QH;
    {
        const float l2 = a.l2, inv_l2 = a.inv_l2;
        for (int i = tid; i < G::QH * 17; i += 256) {
            const bool main = i < G::QH * 16;
            const int q = main ? (i & 15) : 16, r = main ? (i >> 4) : i - G::QH * 16;
            float su[8], sc[8], sd[8], xu[8], xc[8], xd[8], vu[8], vc[8], vd[8];
            // u_sigma rows r .. r+2, cols 4q .. 4q+7 (position 4q+k at index k+1)
            const float *sp = ss + r * G::SS + 4 * q;
            // x rows (r-1+HL) -1 .. +1, cols 4q+4 .. 4q+11 of the window (position at index k+3)
            const float *xp = sxw + (r - 2 + HL) * G::XS + 4 * q + 4;
            // v rows r .. r+2, cols 4q .. 4q+7 of the v window (position at index k+3)
            const float *vp = sv + r * G::VS + 4 * q;
            ld_8f(sp, su); ld_8f(sp + G::SS, sc); ld_8f(sp + 2 * G::SS, sd);
            ld_8f(xp, xu); ld_8f(xp + G::XS, xc); ld_8f(xp + 2 * G::XS, xd);
            ld_8f(vp, vu); ld_8f(vp + G::VS, vc); ld_8f(vp + 2 * G::VS, vd);
            float o0[4], o1[4], o2[4];
            const int gyp = y0 + r - 1;
            const float2 half = make_float2(0.5f, 0.5f), quarter = make_float2(0.25f, 0.25f);
#pragma unroll
            for (int k = 0; k < 4; k += 2) {
                // positions k, k+1: x differences and cross terms from aligned pairs, the
                // y differences and centre terms lane by lane
                const float2 gx = __fmul2_rn(adj_sub2(adj_pr(sc, k + 2), adj_pr(sc, k)), half);
                const float2 gy = make_float2((sd[k + 1] - su[k + 1]) * 0.5f, (sd[k + 2] - su[k + 2]) * 0.5f);
                const float2 sxh = __fadd2_rn(adj_pr(xc, k + 2), adj_pr(xc, k + 4));
                const float2 hxx = make_float2(fmaf(-2.f, xc[k + 3], sxh.x), fmaf(-2.f, xc[k + 4], sxh.y));
                const float2 hyy = make_float2(fmaf(-2.f, xc[k + 3], xu[k + 3] + xd[k + 3]),
                                               fmaf(-2.f, xc[k + 4], xu[k + 4] + xd[k + 4]));
                const float2 hxy = __fmul2_rn(adj_sub2(__fadd2_rn(adj_pr(xd, k + 4), adj_pr(xu, k + 2)),
                                                       __fadd2_rn(adj_pr(xd, k + 2), adj_pr(xu, k + 4))),
                                              quarter);
                const float2 swv = __fadd2_rn(adj_pr(vc, k + 2), adj_pr(vc, k + 4));
                const float2 wxx = make_float2(fmaf(-2.f, vc[k + 3], swv.x), fmaf(-2.f, vc[k + 4], swv.y));
                const float2 wyy = make_float2(fmaf(-2.f, vc[k + 3], vu[k + 3] + vd[k + 3]),
                                               fmaf(-2.f, vc[k + 4], vu[k + 4] + vd[k + 4]));
                const float2 wxy = __fmul2_rn(adj_sub2(__fadd2_rn(adj_pr(vd, k + 4), adj_pr(vu, k + 2)),
                                                       __fadd2_rn(adj_pr(vd, k + 2), adj_pr(vu, k + 4))),
                                              quarter);
                float2 t0, t1, t2, qx, qy;
                adj_position_f32x2(gx, gy, hxx, hyy, hxy, wxx, wyy, wxy, inv_l2, l2, t0, t1, t2, qx, qy);
                o0[k] = t0.x; o0[k + 1] = t0.y;
                o1[k] = t1.x; o1[k + 1] = t1.y;
                o2[k] = t2.x; o2[k + 1] = t2.y;
                const bool rin = r >= 1 && r <= TH && gyp < h;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int c = 4 * q + k + j, gxp = x0 + c - 1;
                    if (rin && c >= 1 && c <= TW && gxp < w) {
                        const long gi = (long)gyp * pitch + gxp;
                        a.qx[gi] = j ? qx.y : qx.x;
                        a.qy[gi] = j ? qy.y : qy.x;
                    }
                }
            }
            float *dst = tw + r * G::QS + 4 * q;
            *reinterpret_cast<float4 *>(dst) = make_float4(o0[0], o0[1], o0[2], o0[3]);
            *reinterpret_cast<float4 *>(dst + PL) = make_float4(o1[0], o1[1], o1[2], o1[3]);
            *reinterpret_cast<float4 *>(dst + 2 * PL) = make_float4(o2[0], o2[1], o2[2], o2[3]);
        }
    }
    __syncthreads();
    // ---- P(x) v: outer divergence of T_w at the tile's pixels, 4 per thread ----
    {
        const int qe = tid & 15, ty = tid >> 4;  // output row ty, cols 4qe .. 4qe+3 <-> positions (ty+1, 4qe+1+k)
        const int gyp = y0 + ty, gxp = x0 + 4 * qe;
        if (gyp < h && gxp < w) {
            float xx[8], yu[8], yc[8], yd[8], du[8], dd[8];
            const float *t0 = tw + (ty + 1) * G::QS + 4 * qe;
            ld_8f(t0, xx);
            ld_8f(t0 + 2 * PL - G::QS, yu); ld_8f(t0 + 2 * PL, yc); ld_8f(t0 + 2 * PL + G::QS, yd);
            ld_8f(t0 + PL - G::QS, du); ld_8f(t0 + PL + G::QS, dd);
            float o[4];
#pragma unroll
            for (int k = 0; k < 4; k += 2) {  // pixel pairs, as in the forward output stage
                const int c = 1 + k;
                const float2 sxx = __fadd2_rn(adj_pr(xx, c - 1), adj_pr(xx, c + 1));
                const float2 dxx = make_float2(fmaf(-2.f, xx[c], sxx.x), fmaf(-2.f, xx[c + 1], sxx.y));
                const float2 dyy = make_float2(fmaf(-2.f, yc[c], yu[c] + yd[c]), fmaf(-2.f, yc[c + 1], yu[c + 1] + yd[c + 1]));
                const float2 dxy = __fmul2_rn(adj_sub2(__fadd2_rn(adj_pr(dd, c + 1), adj_pr(du, c - 1)),
                                                       __fadd2_rn(adj_pr(dd, c - 1), adj_pr(du, c + 1))),
                                              make_float2(0.5f, 0.5f));
                const float2 pv = __fadd2_rn(__fadd2_rn(dxx, dyy), dxy);
                o[k] = pv.x;
                o[k + 1] = pv.y;
            }
            const long gi = (long)gyp * pitch + gxp;
            if (gxp + 3 < w) {
                *reinterpret_cast<float4 *>(a.pv + gi) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
                for (int k = 0; k < 4; ++k)
                    if (gxp + k < w) a.pv[gi + k] = o[k];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// B2 for FP32, register-blocked like B1: 64 x 16 tiles, 256 threads.
//   windows  q_x, q_y rows tile-R-1 .. tile+TH+R, columns tile-12 .. tile+75 (interior
//            tiles, 16-byte cp.async with one fixed float4 column per thread)
//   D        -D_odd q on rows tile-R .. tile+TH+R-1, four columns per item from float4
//            loads (border tiles: per position, with the odd ghosts); column d <-> tile-8+d
//   x pass   Gaussian along rows of D, 8 outputs per item from six float4 loads
//   y pass   z = Gaussian along columns, four pixels per thread, then the step's
//            adjoint recursion with float4 global loads and stores
// The x-pass output aliases the q windows, which are dead once D is formed.
template <int R>
struct AdjB2Fast {
    static constexpr int TW = 64, TH = kAdjTH;
    static constexpr int QR = TH + 2 * R + 2, QC = 88;  // q windows
    static constexpr int DH = TH + 2 * R, DS = 84;       // D: 80 columns used, 21 float4 per row
    static constexpr int XS = 68;                        // x pass: 64 columns, 17 float4 per row
    static_assert(DH * XS <= 2 * QR * QC, "x pass fits in the q windows");
    static constexpr int ELEMS = 2 * QR * QC + DH * DS;
    static constexpr size_t SMEM = sizeof(float) * ELEMS;
};

template <int R>
__global__ void __launch_bounds__(256) adj_b2_fast(const AdjArgs<float> a)
{
    using G = AdjB2Fast<R>;
    constexpr int TW = G::TW, TH = G::TH;
    extern __shared__ __align__(16) float sm[];
    float *sqx = sm, *sqy = sm + G::QR * G::QC;  // q windows
    float *sd = sm + 2 * G::QR * G::QC;           // -D_odd q
    float *sx = sm;                               // x pass (after D)
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const int w = a.w, h = a.h;
    const long pitch = a.pitch;
    // D columns 8-R .. 71+R (tile-R .. tile+63+R) are the ones the x pass reads
    constexpr int M0 = (8 - R) / 4, M1 = (71 + R) / 4, NM = M1 - M0 + 1;
    const bool inner = x0 - 12 >= 0 && x0 + 76 <= w && y0 - R - 1 >= 0 && y0 + TH + R + 1 <= h;
    if (inner) {
        if (tid < 242) {  // 22 float4 columns, 11 rows per pass
            const int q = tid % 22, r0 = tid / 22;
            const long go = (long)(y0 - R - 1 + r0) * pitch + (x0 - 12 + 4 * q);
            uint32_t dx = adj_smem(sqx + r0 * G::QC + 4 * q), dy = adj_smem(sqy + r0 * G::QC + 4 * q);
            for (int r = r0; r < G::QR; r += 11, dx += 4u * 11 * G::QC, dy += 4u * 11 * G::QC) {
                const long o = go + (long)(r - r0) * pitch;
                adj_cp16(dx, a.qx + o);
                adj_cp16(dy, a.qy + o);
            }
        }
        adj_cp_wait();
        __syncthreads();
        // D column d <-> q window column d+4; position group m: D columns 4m .. 4m+3
        for (int i = tid; i < G::DH * NM; i += 256) {
            const int r = i / NM, m = M0 + (i - r * NM);
            const float *px = sqx + (r + 1) * G::QC + 4 * m;  // q_x columns 4m .. 4m+8 <-> x[0..8]
            float x[9];
            {
                const float4 f0 = *reinterpret_cast<const float4 *>(px);
                const float4 f1 = *reinterpret_cast<const float4 *>(px + 4);
                x[0] = f0.x; x[1] = f0.y; x[2] = f0.z; x[3] = f0.w; x[4] = f1.x; x[5] = f1.y; x[6] = f1.z; x[7] = f1.w;
                x[8] = px[8];
            }
            const float4 yu = *reinterpret_cast<const float4 *>(sqy + r * G::QC + 4 * m + 4);
            const float4 yd = *reinterpret_cast<const float4 *>(sqy + (r + 2) * G::QC + 4 * m + 4);
            float4 o;
            o.x = -((x[5] - x[3]) + (yd.x - yu.x)) * 0.5f;
            o.y = -((x[6] - x[4]) + (yd.y - yu.y)) * 0.5f;
            o.z = -((x[7] - x[5]) + (yd.z - yu.z)) * 0.5f;
            o.w = -((x[8] - x[6]) + (yd.w - yu.w)) * 0.5f;
            *reinterpret_cast<float4 *>(sd + r * G::DS + 4 * m) = o;
        }
    } else {
        constexpr int DW = TW + 2 * R;
        for (int i = tid; i < G::DH * DW; i += 256) {
            const int r = i / DW, c = i - r * DW;  // tile column c - R
            sd[r * G::DS + c + 8 - R] = adj_divq(a, mirror_idx(x0 - R + c, w), mirror_idx(y0 - R + r, h));
        }
    }
    __syncthreads();
    float wt[2 * R + 1];
#pragma unroll
    for (int t = 0; t <= 2 * R; ++t) wt[t] = a.wts[t];
    // x pass: sx row r, column c (tile column c) <- D columns c+8-R .. c+8+R
    for (int i = tid; i < G::DH * 8; i += 256) {
        const int r = i >> 3, g = i & 7;
        const float *src = sd + r * G::DS + 8 * g;
        float v[24];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const float4 f = *reinterpret_cast<const float4 *>(src + 4 * j);
            v[4 * j] = f.x; v[4 * j + 1] = f.y; v[4 * j + 2] = f.z; v[4 * j + 3] = f.w;
        }
        float o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * R; ++t) acc = fmaf(wt[t], v[k + 8 - R + t], acc);
            o[k] = acc;
        }
        float *dst = sx + r * G::XS + 8 * g;
        *reinterpret_cast<float4 *>(dst) = make_float4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<float4 *>(dst + 4) = make_float4(o[4], o[5], o[6], o[7]);
    }
    __syncthreads();
    // y pass and the recursion: row ty, pixels 4qe .. 4qe+3
    {
        const int qe = tid & 15, ty = tid >> 4;
        const int gy = y0 + ty, gx = x0 + 4 * qe;
        if (gy < h && gx < w) {
            float z[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int t = 0; t <= 2 * R; ++t) {
                const float4 f = *reinterpret_cast<const float4 *>(sx + (ty + t) * G::XS + 4 * qe);
                z[0] = fmaf(wt[t], f.x, z[0]);
                z[1] = fmaf(wt[t], f.y, z[1]);
                z[2] = fmaf(wt[t], f.z, z[2]);
                z[3] = fmaf(wt[t], f.w, z[3]);
            }
            const long gi = (long)gy * pitch + gx;
            const bool full = gx + 3 < w;
            float gv[4], pv[4], pe[4];
            uint32_t mk = 0;
            if (full) {
                const float4 g4 = *reinterpret_cast<const float4 *>(a.g + gi);
                const float4 p4 = *reinterpret_cast<const float4 *>(a.pv + gi);
                const float4 e4 = *reinterpret_cast<const float4 *>(a.pend + gi);
                mk = *reinterpret_cast<const uint32_t *>(a.mask + gi);
                gv[0] = g4.x; gv[1] = g4.y; gv[2] = g4.z; gv[3] = g4.w;
                pv[0] = p4.x; pv[1] = p4.y; pv[2] = p4.z; pv[3] = p4.w;
                pe[0] = e4.x; pe[1] = e4.y; pe[2] = e4.z; pe[3] = e4.w;
            } else {
                for (int k = 0; k < 4; ++k) {
                    const bool in = gx + k < w;
                    gv[k] = in ? a.g[gi + k] : 0.f;
                    pv[k] = in ? a.pv[gi + k] : 0.f;
                    pe[k] = in ? a.pend[gi + k] : 0.f;
                    if (in && a.mask[gi + k]) mk |= 0xffu << (8 * k);
                }
            }
            float go[4], pn[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool known = ((mk >> (8 * k)) & 0xffu) != 0;
                const float v = known ? 0.f : gv[k];
                const float jt = pv[k] + z[k];  // J_F(x)^T v
                const float dcur = (known ? gv[k] : 0.f) + a.alpha * v - a.alpha * a.tau * jt;
                const float dprev = (1.f - a.alpha) * v;
                if (a.first_of_cycle) {
                    go[k] = pe[k] + dcur + dprev;
                    pn[k] = 0.f;
                } else {
                    go[k] = pe[k] + dcur;
                    pn[k] = dprev;
                }
            }
            if (full) {
                *reinterpret_cast<float4 *>(a.gout + gi) = make_float4(go[0], go[1], go[2], go[3]);
                *reinterpret_cast<float4 *>(a.pend + gi) = make_float4(pn[0], pn[1], pn[2], pn[3]);
            } else {
                for (int k = 0; k < 4; ++k)
                    if (gx + k < w) {
                        a.gout[gi + k] = go[k];
                        a.pend[gi + k] = pn[k];
                    }
            }
        }
    }
}

template <typename T, int R>
struct AdjSmem {
    static constexpr int HL = R + 2, TW = adj_tile_w<T>(), TH = kAdjTH;
    static constexpr size_t B1 = sizeof(T) * ((TW + 16) * (TH + 2 * HL) + (TW + 8) * (TH + 4) +
                                              (TH + 2 * HL) * (TW + 4) + (TW + 4) * (TH + 4) + 3 * (TW + 2) * (TH + 2)) +
                                 (size_t)(TW + 8) * (TH + 4);
    static constexpr size_t B2 = sizeof(T) * ((TW + 2 * R) * (TH + 2 * R) + (TH + 2 * R) * TW);
};

template <typename T, int R>
cudaError_t launch_adjoint_step(const AdjArgs<T> *ap, cudaStream_t s)
{
    using SM = AdjSmem<T, R>;
    constexpr int TW = SM::TW, TH = SM::TH;
    if constexpr (sizeof(T) == sizeof(float)) {  // the register-blocked FP32 kernels
        if (!ap) {
            cudaError_t e =
                cudaFuncSetAttribute(adj_b1_fast<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AdjFast<R>::SMEM);
            if (e != cudaSuccess) return e;
            return cudaFuncSetAttribute(adj_b2_fast<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)AdjB2Fast<R>::SMEM);
        }
        dim3 grid((ap->w + TW - 1) / TW, (ap->h + TH - 1) / TH);
        adj_b1_fast<R><<<grid, 256, AdjFast<R>::SMEM, s>>>(*ap);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        adj_b2_fast<R><<<grid, 256, AdjB2Fast<R>::SMEM, s>>>(*ap);
        return cudaGetLastError();
    } else {
        if (!ap) {
            cudaError_t e =
                cudaFuncSetAttribute(adj_b1_kernel<T, R, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::B1);
            if (e != cudaSuccess) return e;
            return cudaFuncSetAttribute(adj_b2_kernel<T, R, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)SM::B2);
        }
        dim3 grid((ap->w + TW - 1) / TW, (ap->h + TH - 1) / TH);
        adj_b1_kernel<T, R, TW><<<grid, 256, SM::B1, s>>>(*ap);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        adj_b2_kernel<T, R, TW><<<grid, 256, SM::B2, s>>>(*ap);
        return cudaGetLastError();
    }
}

}  // namespace foeed
