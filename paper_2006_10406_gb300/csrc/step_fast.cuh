// Register-blocked FP32 fused FSI step (FOEED with Charbonnier g and
// mu3 = sqrt(mu1), or EED with Charbonnier g): the hot kernel of the solver.
//
// One CTA of 256 threads owns a 64 x 32 output tile. Every stage works on
// groups of four consecutive pixels of one row (float4 in shared memory), so
// shared-memory traffic is vectorised and no index needs a division:
//   A  u^k window, rows tile-(R+2) .. tile+31+(R+2), columns tile-8 .. tile+75
//      (float4 global loads for interior columns, mirrored scalar loads at the
//      image border)
//   B  Gaussian x pass, columns tile-2 .. tile+69, every window row
//   C  Gaussian y pass, 3 rows per thread, columns tile-2 .. tile+69
//   D  gradient, mu1/mu3, Hessian and T (FOEED) or the EED fluxes on tile+-1
//   E  outer divergence, masked FSI update, optional cycle residual, float4 store
// Requirements (checked on the host): row pitch a multiple of 4 elements and
// 16-byte aligned image and mask pointers.
#pragma once

#include "foeed_device.cuh"

namespace foeed {

__device__ __forceinline__ float rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_fast(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_fast(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int R, bool EED>
struct FastTile {
    static constexpr int TW = 64, TH = 32;
    static constexpr int HL = R + 2;
    static constexpr int SU_W = 84, SU_H = TH + 2 * HL;  // u: columns tile-8 .. tile+75
    // Row strides are an odd number of float4 so that the column-major stages
    // (consecutive lanes on consecutive rows) are free of bank conflicts.
    static constexpr int SX_W = 76, SX_H = SU_H;         // x pass: columns tile-2 .. tile+69 (+4 pad)
    static constexpr int SS_W = 76, SS_H = TH + 4;       // u_sigma: rows tile-2 .. tile+33
    static constexpr int ST_W = 68, ST_H = TH + 2;       // T: rows/cols tile-1 .. (cols to tile+66)
    static constexpr int NT = EED ? 4 : 3;
    // the T planes reuse the x-pass buffer, which is dead after stage C
    static constexpr int SXT = (SX_W * SX_H > NT * ST_W * ST_H) ? SX_W * SX_H : NT * ST_W * ST_H;
    static constexpr int ELEMS = SU_W * SU_H + SXT + SS_W * SS_H;
    static constexpr size_t SMEM = sizeof(float) * ELEMS;
};

// The image one tile belongs to: its buffers for this step and its geometry.
struct TileImg {
    const float *uprev, *ucur;
    float *unext;
    const uint8_t *mask;  // may be null
    const float *c0;      // cycle start (residual steps)
    int w, h;
    long pitch;
    float c4;             // 1/(4 lambda^2)
};

// One 64 x 32 tile of one FSI step (stages A..E) of image im; p supplies the
// Gaussian taps, alpha, tau and whether this step accumulates the cycle
// residual (added to rnum/rden).
template <int R, bool EED, typename U>
__device__ __forceinline__ void fast_tile(const StepArgs<float> &p, const TileImg &im, const int x0, const int y0,
                                          float *sm, double &rnum, double &rden)
{
    using G = FastTile<R, EED>;
    float *su = sm;
    float *sx = su + G::SU_W * G::SU_H;
    float *st = sx;  // aliases sx: written in stage D, after the last read of sx in stage C
    float *ss = sx + G::SXT;
    const U alpha = sizeof(U) == sizeof(float) ? U(p.alpha_t) : U(p.alpha);
    const U tau = sizeof(U) == sizeof(float) ? U(p.tau_t) : U(p.tau);

    const int tid = threadIdx.x;
    const int w = im.w, h = im.h;
    const long pitch = im.pitch;

    // ---- A: u window, copied global -> shared asynchronously (cp.async) ----
    {
        const float *__restrict__ uc = im.ucur;
        const bool xin = (x0 - 8 >= 0) && (x0 + 76 <= w);
        const bool yin = (y0 - G::HL >= 0) && (y0 + G::TH + G::HL <= h);
        constexpr int NQ = G::SU_W / 4;  // 21 float4 per row
        const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(su);
        for (int i = tid; i < G::SU_H * NQ; i += 256) {
            int r = i / NQ, q = i - r * NQ;
            int gy = yin ? y0 - G::HL + r : mirror_idx(y0 - G::HL + r, h);
            const float *row = uc + (long)gy * pitch;
            int gx = x0 - 8 + 4 * q;
            uint32_t sa = sbase + 4u * (uint32_t)(r * G::SU_W + 4 * q);
            if (xin) {
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(row + gx) : "memory");
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa + 4u * j),
                                 "l"(row + mirror_idx(gx + j, w))
                                 : "memory");
            }
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();

    // ---- B: Gaussian x pass; out column tile-2+4q+k <- su index 4q+6+k+t ----
    {
        float wt[2 * R + 1];
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) wt[t] = p.wts[t];
        constexpr int NQ = 18;  // output groups per row (columns tile-2 .. tile+69)
        for (int i = tid; i < G::SX_H * NQ; i += 256) {
            int q = i / G::SX_H, r = i - q * G::SX_H;  // consecutive lanes on consecutive rows
            const float *src = su + r * G::SU_W + 4 * q;
            float v[16];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float4 a = *reinterpret_cast<const float4 *>(src + 4 * j);
                v[4 * j] = a.x; v[4 * j + 1] = a.y; v[4 * j + 2] = a.z; v[4 * j + 3] = a.w;
            }
            float o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int t = -R; t <= R; ++t) acc = fmaf(wt[t + R], v[6 + k + t], acc);
                o[k] = acc;
            }
            *reinterpret_cast<float4 *>(sx + r * G::SX_W + 4 * q) = make_float4(o[0], o[1], o[2], o[3]);
        }
    }
    __syncthreads();

    // ---- C: Gaussian y pass, 3 output rows per item; ss row y+2 <- sx rows y+2 .. y+2+2R ----
    {
        float wt[2 * R + 1];
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) wt[t] = p.wts[t];
        constexpr int NQ = 18;                // groups per row
        constexpr int NS = G::SS_H / 3;       // 12 strips
        static_assert(G::SS_H % 3 == 0, "strip height");
        for (int i = tid; i < NS * NQ; i += 256) {
            int q = i / NS, s = i - q * NS;
            const float *src = sx + (3 * s) * G::SX_W + 4 * q;
            float2 acc[3][2];
#pragma unroll
            for (int v = 0; v < 3; ++v) acc[v][0] = acc[v][1] = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 2 * R + 3; ++j) {
                float4 a = *reinterpret_cast<const float4 *>(src + j * G::SX_W);
                const float2 lo = make_float2(a.x, a.y), hi = make_float2(a.z, a.w);
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const int t = j - v;  // tap index 0..2R
                    if (t >= 0 && t <= 2 * R) {
                        const float2 ww = make_float2(wt[t], wt[t]);
                        acc[v][0] = __ffma2_rn(ww, lo, acc[v][0]);
                        acc[v][1] = __ffma2_rn(ww, hi, acc[v][1]);
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < 3; ++v)
                *reinterpret_cast<float4 *>(ss + (3 * s + v) * G::SS_W + 4 * q) =
                    make_float4(acc[v][0].x, acc[v][0].y, acc[v][1].x, acc[v][1].y);
        }
    }
    __syncthreads();

    // ---- D: on tile+-1 (T row r <-> tile row r-1, T col 4q+k <-> tile col 4q+k-1) ----
    constexpr int PL = G::ST_W * G::ST_H;
    {
        const float c4 = im.c4;
        constexpr int NQ = G::ST_W / 4;  // 17
        for (int i = tid; i < G::ST_H * NQ; i += 256) {
            int q = i / G::ST_H, r = i - q * G::ST_H;
            // u_sigma: tile (y, x) <-> ss (y+2, x+2); this group: ss row r+1, cols 4q+1 .. 4q+4
            const float *sm0 = ss + (r + 1) * G::SS_W + 4 * q;
            float sc[8], sup[8], sdn[8];
            {
                float4 a = *reinterpret_cast<const float4 *>(sm0);
                float4 b = *reinterpret_cast<const float4 *>(sm0 + 4);
                sc[0] = a.x; sc[1] = a.y; sc[2] = a.z; sc[3] = a.w; sc[4] = b.x; sc[5] = b.y; sc[6] = b.z; sc[7] = b.w;
                a = *reinterpret_cast<const float4 *>(sm0 - G::SS_W);
                b = *reinterpret_cast<const float4 *>(sm0 - G::SS_W + 4);
                sup[0] = a.x; sup[1] = a.y; sup[2] = a.z; sup[3] = a.w; sup[4] = b.x; sup[5] = b.y; sup[6] = b.z; sup[7] = b.w;
                a = *reinterpret_cast<const float4 *>(sm0 + G::SS_W);
                b = *reinterpret_cast<const float4 *>(sm0 + G::SS_W + 4);
                sdn[0] = a.x; sdn[1] = a.y; sdn[2] = a.z; sdn[3] = a.w; sdn[4] = b.x; sdn[5] = b.y; sdn[6] = b.z; sdn[7] = b.w;
            }
            // u: tile (y, x) <-> su (y+HL, x+8); this group: su row r-1+HL, cols 4q+7 .. 4q+10
            const float *um0 = su + (r - 1 + G::HL) * G::SU_W + 4 * q + 4;
            float uc[8], uu[8], ud[8];
            {
                float4 a = *reinterpret_cast<const float4 *>(um0);
                float4 b = *reinterpret_cast<const float4 *>(um0 + 4);
                uc[0] = a.x; uc[1] = a.y; uc[2] = a.z; uc[3] = a.w; uc[4] = b.x; uc[5] = b.y; uc[6] = b.z; uc[7] = b.w;
                a = *reinterpret_cast<const float4 *>(um0 - G::SU_W);
                b = *reinterpret_cast<const float4 *>(um0 - G::SU_W + 4);
                uu[0] = a.x; uu[1] = a.y; uu[2] = a.z; uu[3] = a.w; uu[4] = b.x; uu[5] = b.y; uu[6] = b.z; uu[7] = b.w;
                a = *reinterpret_cast<const float4 *>(um0 + G::SU_W);
                b = *reinterpret_cast<const float4 *>(um0 + G::SU_W + 4);
                ud[0] = a.x; ud[1] = a.y; ud[2] = a.z; ud[3] = a.w; ud[4] = b.x; ud[5] = b.y; ud[6] = b.z; ud[7] = b.w;
            }
            float o0[4], o1[4], o2[4], o3[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // ss index of this pixel within sc: 1+k ; su index within uc: 3+k
                float dx = sc[2 + k] - sc[k];
                float dy = sdn[1 + k] - sup[1 + k];
                // A zero gradient gets v1 = (1, 0): the tiny offset leaves every
                // representable non-negligible dx unchanged.
                float dxe = dx + 1e-18f;
                float dxe2 = dxe * dxe;
                float sq = fmaf(dy, dy, dxe2);          // 4 lambda1
                float mu1 = rsqrt_fast(fmaf(sq, c4, 1.f));
                float inv = rcp_fast(sq);
                float C = fmaf(-dy, dy, dxe2) * inv;    // cos 2theta
                float S = 2.f * dxe * dy * inv;         // sin 2theta
                const float ucv = uc[3 + k];
                if (!EED) {
                    float mu3 = sqrt_fast(mu1);
                    float hxx = (uc[2 + k] + uc[4 + k]) - 2.f * ucv;
                    float hyy = (uu[3 + k] + ud[3 + k]) - 2.f * ucv;
                    float hxy = ((ud[4 + k] + uu[2 + k]) - (ud[2 + k] + uu[4 + k])) * 0.25f;
                    float A = (hxx + hyy) * 0.5f, B = (hxx - hyy) * 0.5f;
                    float X = fmaf(C, B, S * hxy);
                    float h11 = A + X, h22 = A - X;
                    float h12 = fmaf(C, hxy, -S * B);
                    float pp = mu1 * h11, rr = mu3 * h12;
                    float hs = (pp + h22) * 0.5f, hd = (pp - h22) * 0.5f;
                    float Y = fmaf(C, hd, -S * rr);
                    o0[k] = hs + Y;                 // T_xx
                    o1[k] = fmaf(S, hd, C * rr);    // T_xy
                    o2[k] = hs - Y;                 // T_yy
                } else {
                    float m1 = mu1 - 1.f, m2 = mu1 + 1.f;
                    float a = fmaf(C, m1, m2) * 0.5f;
                    float cc = fmaf(-C, m1, m2) * 0.5f;
                    float b = S * m1 * 0.5f;
                    o0[k] = a;
                    o1[k] = cc;
                    o2[k] = b * ((ud[3 + k] - uu[3 + k]) * 0.5f);  // b * d_y u
                    o3[k] = b * ((uc[4 + k] - uc[2 + k]) * 0.5f);  // b * d_x u
                }
            }
            float *dst = st + r * G::ST_W + 4 * q;
            *reinterpret_cast<float4 *>(dst) = make_float4(o0[0], o0[1], o0[2], o0[3]);
            *reinterpret_cast<float4 *>(dst + PL) = make_float4(o1[0], o1[1], o1[2], o1[3]);
            *reinterpret_cast<float4 *>(dst + 2 * PL) = make_float4(o2[0], o2[1], o2[2], o2[3]);
            if (EED) *reinterpret_cast<float4 *>(dst + 3 * PL) = make_float4(o3[0], o3[1], o3[2], o3[3]);
        }
    }
    // Each thread owns exactly two output groups in stage E (row i/16, group i%16
    // for i = tid, tid+256). Their u^{k-1} and mask loads are issued here, before
    // the barrier, so that their latency overlaps the wait.
    constexpr int NQE = G::TW / 4;  // 16 groups per row
    static_assert(G::TH * NQE == 512, "two output groups per thread");
    float4 pre_up[2];
    uint32_t pre_mk[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int i = tid + 256 * e, r = i / NQE, q = i - r * NQE;
        const int gy = y0 + r, gx = x0 + 4 * q;
        pre_up[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        pre_mk[e] = 0u;
        if (gy < h && gx < w) {
            const long gi = (long)gy * pitch + gx;
            if (gx + 3 < w) {
                pre_up[e] = __ldg(reinterpret_cast<const float4 *>(im.uprev + gi));
                if (im.mask) pre_mk[e] = __ldg(reinterpret_cast<const unsigned int *>(im.mask + gi));
            } else {
                float *pu = reinterpret_cast<float *>(&pre_up[e]);
                for (int k = 0; k < 4; ++k)
                    if (gx + k < w) {
                        pu[k] = im.uprev[gi + k];
                        if (im.mask) pre_mk[e] |= uint32_t(im.mask[gi + k] != 0) << (8 * k);
                    }
            }
        }
    }
    __syncthreads();

    // ---- E: output rows tile+r, columns tile+4q .. 4q+3 (T index (r+1, 4q+1+k)) ----
    {
        constexpr int NQ = NQE;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int i = tid + 256 * e;
            int r = i / NQ, q = i - r * NQ;
            int gy = y0 + r, gx = x0 + 4 * q;
            if (gy >= h || gx >= w) continue;
            const float *t0 = st + (r + 1) * G::ST_W + 4 * q;
            float Pu[4];
            const float *um = su + (r + G::HL) * G::SU_W + 4 * q + 8;  // u^k at this group
            float4 ucv4 = *reinterpret_cast<const float4 *>(um);
            float ucv[4] = {ucv4.x, ucv4.y, ucv4.z, ucv4.w};
            if (!EED) {
                float xx[8], yu[8], yc[8], yd[8], du[8], dd[8];
                auto ld8 = [](const float *s, float *o) {
                    float4 a = *reinterpret_cast<const float4 *>(s);
                    float4 b = *reinterpret_cast<const float4 *>(s + 4);
                    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
                };
                ld8(t0, xx);
                ld8(t0 + 2 * PL - G::ST_W, yu);
                ld8(t0 + 2 * PL, yc);
                ld8(t0 + 2 * PL + G::ST_W, yd);
                ld8(t0 + PL - G::ST_W, du);
                ld8(t0 + PL + G::ST_W, dd);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int c = 1 + k;
                    float dxx = (xx[c - 1] + xx[c + 1]) - 2.f * xx[c];
                    float dyy = (yu[c] + yd[c]) - 2.f * yc[c];
                    float dxy = ((dd[c + 1] + du[c - 1]) - (dd[c - 1] + du[c + 1])) * 0.5f;
                    Pu[k] = (dxx + dyy) + dxy;
                }
            } else {
                float ac[8], cu[8], cc[8], cd[8], qxr[8], qyu[8], qyd[8], uu[8], ud[8], ucx[8];
                auto ld8 = [](const float *s, float *o) {
                    float4 a = *reinterpret_cast<const float4 *>(s);
                    float4 b = *reinterpret_cast<const float4 *>(s + 4);
                    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
                };
                ld8(t0, ac);
                ld8(t0 + PL - G::ST_W, cu);
                ld8(t0 + PL, cc);
                ld8(t0 + PL + G::ST_W, cd);
                ld8(t0 + 2 * PL, qxr);
                ld8(t0 + 3 * PL - G::ST_W, qyu);
                ld8(t0 + 3 * PL + G::ST_W, qyd);
                // u neighbours: su cols 4q+7 .. 4q+12 <-> ucx[3..8]; load su cols 4q+4 .. 4q+11 and 4q+12
                ld8(um - 4, ucx);
                float ur = um[4];
                {
                    float4 a = *reinterpret_cast<const float4 *>(um - G::SU_W);
                    uu[0] = a.x; uu[1] = a.y; uu[2] = a.z; uu[3] = a.w;
                    a = *reinterpret_cast<const float4 *>(um + G::SU_W);
                    ud[0] = a.x; ud[1] = a.y; ud[2] = a.z; ud[3] = a.w;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int c = 1 + k;
                    float u0 = ucv[k];
                    float ul = ucx[3 + k];
                    float urr = (k == 3) ? ur : ucx[5 + k];
                    float fx = ((ac[c] + ac[c + 1]) * (urr - u0) - (ac[c - 1] + ac[c]) * (u0 - ul)) * 0.5f;
                    float fy = ((cc[c] + cd[c]) * (ud[k] - u0) - (cu[c] + cc[c]) * (u0 - uu[k])) * 0.5f;
                    // plane 2 holds b * d_y u (differentiated in x), plane 3 b * d_x u (in y)
                    float mx = qxr[c + 1] - qxr[c - 1];
                    float my = qyd[c] - qyu[c];
                    Pu[k] = -((fx + fy) + (mx + my) * 0.5f);
                }
            }
            const long gi = (long)gy * pitch + gx;
            const bool full = gx + 3 < w;
            const float upv[4] = {pre_up[e].x, pre_up[e].y, pre_up[e].z, pre_up[e].w};
            float c0v[4] = {0.f, 0.f, 0.f, 0.f};
            if (p.residual) {
                if (full) {
                    float4 c = *reinterpret_cast<const float4 *>(im.c0 + gi);
                    c0v[0] = c.x; c0v[1] = c.y; c0v[2] = c.z; c0v[3] = c.w;
                } else {
                    for (int k = 0; k < 4; ++k)
                        if (gx + k < w) c0v[k] = im.c0[gi + k];
                }
            }
            float un[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if ((pre_mk[e] >> (8 * k)) & 0xffu) {
                    un[k] = ucv[k];
                } else {
                    U up = U(upv[k]);
                    U ex = U(ucv[k]) - tau * U(Pu[k]);
                    un[k] = float(up + alpha * (ex - up));
                }
            }
            if (p.residual) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (gx + k < w) {
                        double d = double(un[k]) - double(c0v[k]);
                        rnum += d * d;
                        rden += double(un[k]) * double(un[k]);
                    }
            }
            if (full) {
                *reinterpret_cast<float4 *>(im.unext + gi) = make_float4(un[0], un[1], un[2], un[3]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (gx + k < w) im.unext[gi + k] = un[k];
            }
        }
    }

}

// Cycle residual of one image: the last of its nblocks tiles to finish sums
// the per-tile partials in tile order and updates its control block.
__device__ __forceinline__ void finish_cycle_residual(double rnum, double rden, Ctl *ctl, double *partials,
                                                      int nblocks, int bid, double *red)
{
    if (grid_sum2_last(rnum, rden, partials, &ctl->ticket, nblocks, bid, red)) {
        double rel = rden > 0.0 ? sqrt(rnum) / sqrt(rden) : sqrt(rnum);
        ctl->last_num = rnum;
        ctl->last_den = rden;
        ctl->last_rel = rel;
        ctl->cycles += 1;
        if (!isfinite(rel)) { ctl->diverged = 1; ctl->done = 1; }
        else if (ctl->tol > 0.0 && rel < ctl->tol) ctl->done = 1;
    }
}

// One FSI step over one image, one CTA per 64 x 32 tile.
template <int R, bool EED, typename U>
__global__ void __launch_bounds__(256) fsi_step_fast(const StepArgs<float> p)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ double red[64];
    // Programmatic dependent launch: wait until the previous step's grid has
    // completed and its writes are visible (a no-op for an ordinary launch),
    // then let the next step's CTAs be scheduled as SM slots free up.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (p.check_done && p.ctl->done) return;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const TileImg im{p.uprev, p.ucur, p.unext, p.mask, p.c0, p.w, p.h, p.pitch, p.c4};
    double rnum = 0.0, rden = 0.0;
    fast_tile<R, EED, U>(p, im, blockIdx.x * FastTile<R, EED>::TW, blockIdx.y * FastTile<R, EED>::TH, sm, rnum, rden);
    if (p.residual)
        finish_cycle_residual(rnum, rden, p.ctl, p.partials, gridDim.x * gridDim.y,
                              blockIdx.y * gridDim.x + blockIdx.x, red);
}

// ---------------------------------------------------------------------------
// Batched FOEED or EED: one launch per FSI step over the tiles of many images.

template <int R, bool EED, typename U>
__global__ void __launch_bounds__(256) fsi_batch_step_fast(const StepArgs<float> p, const BatchArgs b)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ double red[64];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int2 tl = b.tiles[blockIdx.x];
    const BatchInst I = b.inst[tl.x];
    if (I.ctl->done) return;  // this image has converged (or diverged)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    TileImg im;
    switch (b.role) {
    case kRoleFirst: im.uprev = I.C; im.ucur = I.C; im.unext = I.A; break;
    case kRoleSecond: im.uprev = I.C; im.ucur = I.A; im.unext = I.B; break;
    case kRoleEven: im.uprev = I.A; im.ucur = I.B; im.unext = I.A; break;
    default: im.uprev = I.B; im.ucur = I.A; im.unext = I.B; break;
    }
    if (b.last) im.unext = I.C;
    im.mask = I.mask;
    im.c0 = I.C;
    im.w = I.w;
    im.h = I.h;
    im.pitch = I.pitch;
    im.c4 = I.c4;
    const int ty = tl.y / I.ntx, tx = tl.y - ty * I.ntx;
    double rnum = 0.0, rden = 0.0;
    fast_tile<R, EED, U>(p, im, tx * FastTile<R, EED>::TW, ty * FastTile<R, EED>::TH, sm, rnum, rden);
    if (b.last) finish_cycle_residual(rnum, rden, I.ctl, I.partials, I.ntx * I.nty, tl.y, red);
}

template <int R, bool EED, typename U>
cudaError_t launch_fsi_batch_step_fast(const StepArgs<float> *ap, const BatchArgs *bp, int ntiles, cudaStream_t s)
{
    using G = FastTile<R, EED>;
    auto kern = fsi_batch_step_fast<R, EED, U>;
    if (!ap) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (!ap->pdl) {
        kern<<<ntiles, 256, G::SMEM, s>>>(*ap, *bp);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ntiles);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, *ap, *bp);
}

template <int R, bool EED, typename U>
cudaError_t launch_fsi_step_fast(const StepArgs<float> *ap, cudaStream_t s)
{
    using G = FastTile<R, EED>;
    auto kern = fsi_step_fast<R, EED, U>;
    if (!ap) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    dim3 grid((ap->w + G::TW - 1) / G::TW, (ap->h + G::TH - 1) / G::TH);
    return launch_step_kernel(kern, grid, 256, G::SMEM, s, *ap);
}

}  // namespace foeed
