// Register-blocked FP32 fused FSI step (FOEED with Charbonnier g and
// mu3 = sqrt(mu1), or EED with Charbonnier g): the hot kernel of the solver.
//
// One CTA of 256 threads owns a 64 x 32 output tile (64 x 16 for small images;
// for single FOEED images the autotuner also tries 64 x 64 tiles of 512 threads
// and 64 x 8 tiles of 128). Every stage works on groups of four consecutive
// pixels of one row (float4 in shared memory), and each thread keeps a small
// block of rows or columns in registers so that a shared-memory value is
// loaded once for several outputs (the row ranges below are those of a 64 x 32
// tile):
//   A  u^k window, rows tile-(R+2) .. tile+31+(R+2), columns tile-8 .. tile+75
//      (cp.async 16-byte copies for interior columns, mirrored 4-byte copies at
//      the image border)
//   B  Gaussian x pass, 8 outputs per item, columns tile-2 .. tile+69, every window row
//   C  Gaussian y pass, 6 rows per item, columns tile-2 .. tile+65
//   D  gradient, mu1/mu3, Hessian and T (FOEED) or the EED tensor D on tile+-1,
//      segments of three (or two) rows per item sharing their u_sigma and u rows
//   E  outer divergence, masked FSI update, optional cycle residual, float4 store;
//      two rows per thread sharing two T_yy rows
// A 128-bit shared-memory access is served in quarter-warp phases of 8 lanes,
// each phase conflict-free only if its 8 lanes touch 8 different float4 bank
// groups. Hence odd float4 row strides for the stages whose lanes walk down
// rows, and lanes along 16 column groups (of the 17 a row holds) for the
// stages whose items span several rows; the 17th group's items come last.
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

// Error-free transformations in FP32 arithmetic: a + b = s + e exactly with
// s = fl(a + b) (Knuth's TwoSum, six operations, no ordering of a and b needed),
// and a * b = p + e exactly with p = fl(a * b) (the FMA form of TwoProduct in
// Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput.
// 26(6), 2005).
__device__ __forceinline__ void two_sum(const float a, const float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(const float a, const float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// The masked FSI update u^{k-1} + alpha ((u^k - tau P u^k) - u^{k-1}) (Sec. 3.3)
// of float operands, with alpha and tau given as two-word values (hi + lo),
// carried in two-float arithmetic and rounded to float once: every
// intermediate is held to about 2^-44 of the operands' size, so the result is
// the float nearest the exact update, as an evaluation in double gives, except
// where that value lies that close to a rounding boundary.
__device__ __forceinline__ float fsi_update_ff(const float up, const float u, const float P, const float a_hi,
                                               const float a_lo, const float t_hi, const float t_lo)
{
    float th, tl, eh, el, dh, dl, qh, ql, sh, sl;
    two_prod(t_hi, P, th, tl);
    tl = __fmaf_rn(t_lo, P, tl);   // tau P = th + tl
    two_sum(u, -th, eh, el);
    el = __fsub_rn(el, tl);        // u - tau P = eh + el
    two_sum(eh, -up, dh, dl);
    dl = __fadd_rn(dl, el);        // (u - tau P) - u^{k-1} = dh + dl
    two_prod(a_hi, dh, qh, ql);
    ql = __fmaf_rn(a_hi, dl, ql);
    ql = __fmaf_rn(a_lo, dh, ql);  // alpha ((u - tau P) - u^{k-1}) = qh + ql
    two_sum(up, qh, sh, sl);
    return __fadd_rn(sh, __fadd_rn(sl, ql));
}

// Two-lane FP32 arithmetic (one instruction for two pixels; each lane rounds
// exactly as the scalar operation does). a - b is fma(b, -1, a): one rounding
// of the exact difference, the same value as a plain subtraction.
__device__ __forceinline__ float2 sub2(const float2 a, const float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 pr(const float *v, const int i) { return make_float2(v[i], v[i + 1]); }

// Eight consecutive floats from shared memory (two float4 loads; s is 16-byte aligned).
__device__ __forceinline__ void ld8(const float *s, float *o)
{
    const float4 a = *reinterpret_cast<const float4 *>(s);
    const float4 b = *reinterpret_cast<const float4 *>(s + 4);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}

// One row of four T groups of stage D. sup/sc/sdn: u_sigma rows above/at/below
// (cols 4q .. 4q+7 of ss: this group's pixels are 1..4), uu/uc/ud: u rows (cols
// 4q+4 .. 4q+11 of su: pixels 3..6). FOEED writes T_xx, T_xy, T_yy to planes
// 0..2; EED writes the entries a, c, b of D = [[a, b], [b, c]] to planes 0..2.
template <bool EED>
__device__ __forceinline__ void tensor_row(const float *sup, const float *sc, const float *sdn, const float *uu,
                                           const float *uc, const float *ud, const float c4, float *dst, const int PL)
{
    float o0[4], o1[4], o2[4];
    if (!EED) {
        // FOEED, per pixel (dx, dy: central differences of u_sigma times 2; u_c: centre):
        //   qq = dy^2 + 1e-18, pp = dx^2, pq = dx dy, s2 = pp + qq, d = pp - qq
        //   mu1 = 1 / sqrt(1 + s2 c4), mu3 = sqrt(mu1), k1 = (mu1 - 1)/s2^2, k3 = (mu3 - 1)/s2^2
        //   hxx, hyy, hxy: the Hessian of u
        //   e1 = g^T H g = 2 pq hxy + pp hxx + qq hyy, e3 = g^T H g_perp = pq (hyy - hxx) + d hxy
        //   T_xx = hxx + k1 e1 pp - k3 e3 2pq, T_xy = hxy + k1 e1 pq + k3 e3 d,
        //   T_yy = hyy + k1 e1 qq + k3 e3 2pq
        // The offset in qq keeps 1/s2^2 finite for a zero gradient (where mu1 = mu3 = 1
        // and the corrections vanish); it is below the rounding of any dy^2 > 1e-11.
        // Evaluated in pixel pairs (k, k+1) with two-lane instructions: the operands of
        // the x differences and of the cross term sit in aligned register pairs of the
        // float4 loads; the y difference and the centre terms are formed lane by lane.
        // Each product with a negated factor is an exact sign flip of the scalar one.
        const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
        for (int k = 0; k < 4; k += 2) {
            const float2 dx = sub2(pr(sc, 2 + k), pr(sc, k));
            const float2 dy = make_float2(__fsub_rn(sdn[1 + k], sup[1 + k]), __fsub_rn(sdn[2 + k], sup[2 + k]));
            const float2 qq = __ffma2_rn(dy, dy, make_float2(1e-18f, 1e-18f));
            const float2 pp = __fmul2_rn(dx, dx);
            const float2 pq = __fmul2_rn(dx, dy);
            const float2 s2 = __fadd2_rn(pp, qq);
            const float2 t = __ffma2_rn(s2, make_float2(c4, c4), make_float2(1.f, 1.f));
            const float2 mu1 = make_float2(rsqrt_fast(t.x), rsqrt_fast(t.y));
            const float2 inv = make_float2(rcp_fast(s2.x), rcp_fast(s2.y));
            const float2 inv2 = __fmul2_rn(inv, inv);
            const float2 ninv2 = __fmul2_rn(inv2, m1);
            const float2 k1 = __ffma2_rn(mu1, inv2, ninv2);
            const float2 mu3 = make_float2(sqrt_fast(mu1.x), sqrt_fast(mu1.y));
            const float2 k3 = __ffma2_rn(mu3, inv2, ninv2);
            const float2 sxx = __fadd2_rn(pr(uc, 2 + k), pr(uc, 4 + k));
            const float2 hxx = make_float2(__fmaf_rn(-2.f, uc[3 + k], sxx.x), __fmaf_rn(-2.f, uc[4 + k], sxx.y));
            const float2 hyy = make_float2(__fmaf_rn(-2.f, uc[3 + k], __fadd_rn(uu[3 + k], ud[3 + k])),
                                           __fmaf_rn(-2.f, uc[4 + k], __fadd_rn(uu[4 + k], ud[4 + k])));
            const float2 hxy = __fmul2_rn(sub2(__fadd2_rn(pr(ud, 4 + k), pr(uu, 2 + k)),
                                               __fadd2_rn(pr(ud, 2 + k), pr(uu, 4 + k))),
                                          make_float2(0.25f, 0.25f));
            const float2 d = sub2(pp, qq);
            const float2 pq2 = __fadd2_rn(pq, pq);
            const float2 e1 = __ffma2_rn(pq2, hxy, __ffma2_rn(pp, hxx, __fmul2_rn(qq, hyy)));
            const float2 e3 = __ffma2_rn(pq, sub2(hyy, hxx), __fmul2_rn(d, hxy));
            const float2 a = __fmul2_rn(k1, e1);
            const float2 b = __fmul2_rn(k3, e3);
            const float2 txx = __ffma2_rn(a, pp, __ffma2_rn(b, __fmul2_rn(pq2, m1), hxx));
            const float2 txy = __ffma2_rn(a, pq, __ffma2_rn(b, d, hxy));
            const float2 tyy = __ffma2_rn(a, qq, __ffma2_rn(b, pq2, hyy));
            o0[k] = txx.x; o0[k + 1] = txx.y;
            o1[k] = txy.x; o1[k + 1] = txy.y;
            o2[k] = tyy.x; o2[k + 1] = tyy.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dx = __fsub_rn(sc[2 + k], sc[k]);
            const float dy = __fsub_rn(sdn[1 + k], sup[1 + k]);
            // A zero gradient gets v1 = (1, 0): the tiny offset leaves every
            // representable non-negligible dx unchanged.
            float dxe = dx + 1e-18f;
            float dxe2 = dxe * dxe;
            float sq = fmaf(dy, dy, dxe2);          // 4 lambda1
            float mu1 = rsqrt_fast(fmaf(sq, c4, 1.f));
            float inv = rcp_fast(sq);
            float C = fmaf(-dy, dy, dxe2) * inv;    // cos 2theta
            float S = 2.f * dxe * dy * inv;         // sin 2theta
            float m1 = mu1 - 1.f, m2 = mu1 + 1.f;
            float a = fmaf(C, m1, m2) * 0.5f;
            float cc = fmaf(-C, m1, m2) * 0.5f;
            float b = S * m1 * 0.5f;
            o0[k] = a;
            o1[k] = cc;
            o2[k] = b;
        }
    }
    *reinterpret_cast<float4 *>(dst) = make_float4(o0[0], o0[1], o0[2], o0[3]);
    *reinterpret_cast<float4 *>(dst + PL) = make_float4(o1[0], o1[1], o1[2], o1[3]);
    *reinterpret_cast<float4 *>(dst + 2 * PL) = make_float4(o2[0], o2[1], o2[2], o2[3]);
}

// Tile geometry: 64 x TH output pixels, TH = 32 (large images) or 16 (images
// with fewer tiles than the GPU has SMs: more, shorter CTAs per step); for
// single FOEED images also TH = 64 (512 threads) and TH = 8 (128 threads).
template <int R, bool EED, int TH_ = 32>
struct FastTile {
    static constexpr int TW = 64, TH = TH_;
    static_assert(TH == 64 || TH == 32 || TH == 16 || TH == 8, "tile height");
    static constexpr int NTHR = TH == 64 ? 512 : (TH == 8 ? 128 : 256);  // threads per CTA
    // CTAs per SM the register allocation is bounded for: the 54 KB of shared
    // memory of a 64 x 32 tile fit four 256-thread CTAs (64 registers each)
    static constexpr int MINB = 1024 / NTHR;
    static constexpr int HL = R + 2;
    static constexpr int SU_W = 84, SU_H = TH + 2 * HL;  // u: columns tile-8 .. tile+75
    // Row strides are an odd number of float4 so that the column-major stages
    // (consecutive lanes on consecutive rows) are free of bank conflicts.
    static constexpr int SX_W = 76, SX_H = SU_H;         // x pass: columns tile-2 .. tile+69 (+4 pad)
    static constexpr int SS_W = 76, SS_H = TH + 4;       // u_sigma: rows tile-2 .. tile+33
    static constexpr int ST_W = 68, ST_H = TH + 2;       // T: rows/cols tile-1 .. (cols to tile+66)
    static constexpr int NT = 3;  // T planes
    // the T planes reuse the x-pass buffer, which is dead after stage C
    static constexpr int SXT = (SX_W * SX_H > NT * ST_W * ST_H) ? SX_W * SX_H : NT * ST_W * ST_H;
    static constexpr int ELEMS = SU_W * SU_H + SXT + SS_W * SS_H;
    static constexpr size_t SMEM = sizeof(float) * ELEMS;
    // y pass: strips of RS rows; tensor stage: N3 segments of 3 rows, then N2 of 2
    static constexpr int RS = SS_H % 6 == 0 ? 6 : (SS_H % 5 == 0 ? 5 : 4);
    static_assert(SS_H % RS == 0, "strip height");
    static constexpr int N2 = ST_H % 3 == 0 ? 0 : (ST_H % 3 == 1 ? 2 : 1);
    static constexpr int N3 = (ST_H - 2 * N2) / 3;
    // output stage: ER rows per thread (16 four-pixel groups per row, 256 threads)
    static constexpr int ER = TH * (TW / 4) / NTHR;
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

// One 64 x TH tile of one FSI step (stages A..E) of image im; p supplies the
// Gaussian taps, alpha, tau and whether this step accumulates the cycle
// residual (added to rnum/rden).
template <int R, bool EED, typename U, int TH = 32>
__device__ __forceinline__ void fast_tile(const StepArgs<float> &p, const TileImg &im, const int x0, const int y0,
                                          float *sm, double &rnum, double &rden)
{
    using G = FastTile<R, EED, TH>;
    float *su = sm;
    float *sx = su + G::SU_W * G::SU_H;
    float *st = sx;  // aliases sx: written in stage D, after the last read of sx in stage C
    float *ss = sx + G::SXT;
    const float alpha = p.alpha_t, tau = p.tau_t;

    const int tid = threadIdx.x;
    const int w = im.w, h = im.h;
    const long pitch = im.pitch;

    // ---- A: u window, copied global -> shared asynchronously (cp.async). Thread tid < 21 RP
    // owns the float4 column q = tid % 21 and the rows r0 = tid / 21, r0 + RP, ... (RP = 12
    // with 256 threads); interior tiles copy 16 bytes per row with no index arithmetic
    // beyond a pointer increment ----
    {
        const float *__restrict__ uc = im.ucur;
        const bool xin = (x0 - 8 >= 0) && (x0 + 76 <= w);
        const bool yin = (y0 - G::HL >= 0) && (y0 + G::TH + G::HL <= h);
        constexpr int NQ = G::SU_W / 4;                // 21 float4 per row
        constexpr int RP = G::NTHR / NQ;                 // rows per pass (12; 24 / 6 with 512 / 128 threads)
        constexpr int NP = (G::SU_H + RP - 1) / RP;    // passes
        if (tid < RP * NQ) {
            const int q = tid % NQ, r0 = tid / NQ;
            const int gx = x0 - 8 + 4 * q;
            uint32_t sa = (uint32_t)__cvta_generic_to_shared(su) + 4u * (uint32_t)(r0 * G::SU_W + 4 * q);
            if (xin && yin) {
                const float *src = uc + (long)(y0 - G::HL + r0) * pitch + gx;
                const long step = (long)RP * pitch;
#pragma unroll
                for (int k = 0; k < NP; ++k)
                    if (r0 + RP * k < G::SU_H)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa + 4u * RP * G::SU_W * k),
                                     "l"(src + step * k)
                                     : "memory");
            } else {
                // border tiles: rows are mirrored; a float4 column inside the image is still
                // one 16-byte copy, only columns reaching past the border go element-wise
                const bool cin = gx >= 0 && gx + 4 <= w;
                for (int r = r0; r < G::SU_H; r += RP, sa += 4u * RP * G::SU_W) {
                    const float *row = uc + (long)mirror_idx(y0 - G::HL + r, h) * pitch;
                    if (cin) {
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(row + gx) : "memory");
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa + 4u * j),
                                         "l"(row + mirror_idx(gx + j, w))
                                         : "memory");
                    }
                }
            }
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();

    // ---- B: Gaussian x pass, 8 outputs per item; out column tile-2+8g+k <- su index 8g+6+k+t ----
    {
        float wt[2 * R + 1];
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) wt[t] = p.wts[t];
        constexpr int NG = 9;  // 8-wide output groups per row (columns tile-2 .. tile+69)
        for (int i = tid; i < G::SX_H * NG; i += G::NTHR) {
            const int g = i / G::SX_H, r = i - g * G::SX_H;  // consecutive lanes on consecutive rows
            const float *src = su + r * G::SU_W + 8 * g;
            float v[20];
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                float4 a = *reinterpret_cast<const float4 *>(src + 4 * j);
                v[4 * j] = a.x; v[4 * j + 1] = a.y; v[4 * j + 2] = a.z; v[4 * j + 3] = a.w;
            }
            float o[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int t = -R; t <= R; ++t) acc = fmaf(wt[t + R], v[6 + k + t], acc);
                o[k] = acc;
            }
            float *dst = sx + r * G::SX_W + 8 * g;
            *reinterpret_cast<float4 *>(dst) = make_float4(o[0], o[1], o[2], o[3]);
            *reinterpret_cast<float4 *>(dst + 4) = make_float4(o[4], o[5], o[6], o[7]);
        }
    }
    __syncthreads();

    // ---- C: Gaussian y pass, RS output rows per item; ss row y <- sx rows y .. y+2R ----
    {
        float wt[2 * R + 1];
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) wt[t] = p.wts[t];
        constexpr int RS = G::RS;          // output rows per item
        constexpr int NQ = 17;             // groups per row (columns tile-2 .. tile+65)
        constexpr int NS = G::SS_H / RS;   // strips
        static_assert(NQ == 17, "16 column groups plus one");
        for (int i = tid; i < NS * NQ; i += G::NTHR) {
            // lanes along the first 16 column groups of a strip (conflict-free quarter
            // warps); the strips of the 17th group come last
            const bool main = i < NS * 16;
            const int s = main ? (i >> 4) : i - NS * 16, q = main ? (i & 15) : 16;
            const float *src = sx + (RS * s) * G::SX_W + 4 * q;
            float2 acc[RS][2];
#pragma unroll
            for (int v = 0; v < RS; ++v) acc[v][0] = acc[v][1] = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 2 * R + RS; ++j) {
                float4 a = *reinterpret_cast<const float4 *>(src + j * G::SX_W);
                const float2 lo = make_float2(a.x, a.y), hi = make_float2(a.z, a.w);
#pragma unroll
                for (int v = 0; v < RS; ++v) {
                    const int t = j - v;  // tap index 0..2R
                    if (t >= 0 && t <= 2 * R) {
                        const float2 ww = make_float2(wt[t], wt[t]);
                        acc[v][0] = __ffma2_rn(ww, lo, acc[v][0]);
                        acc[v][1] = __ffma2_rn(ww, hi, acc[v][1]);
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < RS; ++v)
                *reinterpret_cast<float4 *>(ss + (RS * s + v) * G::SS_W + 4 * q) =
                    make_float4(acc[v][0].x, acc[v][0].y, acc[v][1].x, acc[v][1].y);
        }
    }
    __syncthreads();

    // ---- D: on tile+-1 (T row r <-> tile row r-1, T col 4q+k <-> tile col 4q+k-1), two T rows
    // per item: the three u_sigma and u rows of the first are loaded once, the second adds one of each
    constexpr int PL = G::ST_W * G::ST_H;
    {
        const float c4 = im.c4;
        constexpr int NQ = G::ST_W / 4;  // 17
        static_assert(NQ == 17, "16 column groups plus one");
        constexpr int NSEG = G::N3 + G::N2;  // TH 32: ten segments of 3 rows, two of 2; TH 16: six of 3
        for (int i = tid; i < NSEG * NQ; i += G::NTHR) {
            // lanes along the first 16 column groups of a segment (conflict-free quarter
            // warps); the segments of the 17th group come last
            const bool main = i < NSEG * 16;
            const int q = main ? (i & 15) : 16, sg = main ? (i >> 4) : i - NSEG * 16;
            const int r0 = sg < G::N3 ? 3 * sg : 3 * G::N3 + 2 * (sg - G::N3);
            // T row r: u_sigma rows r .. r+2 of ss (cols 4q .. 4q+7), u rows r-2+HL .. r+HL of su (cols 4q+4 .. 4q+11)
            const float *sm0 = ss + r0 * G::SS_W + 4 * q;
            const float *um0 = su + (r0 - 2 + G::HL) * G::SU_W + 4 * q + 4;
            float sa[8], sb[8], sc[8], ua[8], ub[8], uc[8];
            ld8(sm0, sa);
            ld8(sm0 + G::SS_W, sb);
            ld8(sm0 + 2 * G::SS_W, sc);
            ld8(um0, ua);
            ld8(um0 + G::SU_W, ub);
            ld8(um0 + 2 * G::SU_W, uc);
            tensor_row<EED>(sa, sb, sc, ua, ub, uc, c4, st + r0 * G::ST_W + 4 * q, PL);
            ld8(sm0 + 3 * G::SS_W, sa);
            ld8(um0 + 3 * G::SU_W, ua);
            tensor_row<EED>(sb, sc, sa, ub, uc, ua, c4, st + (r0 + 1) * G::ST_W + 4 * q, PL);
            if (sg < G::N3) {
                ld8(sm0 + 4 * G::SS_W, sb);
                ld8(um0 + 4 * G::SU_W, ub);
                tensor_row<EED>(sc, sa, sb, uc, ua, ub, c4, st + (r0 + 2) * G::ST_W + 4 * q, PL);
            }
        }
    }
    // Each thread owns the output groups (rows ER*(tid/16) .. ER*(tid/16)+ER-1, group
    // tid%16) of stage E. Their u^{k-1} and mask loads are issued here, before the
    // barrier, so that their latency overlaps the wait.
    constexpr int NQE = G::TW / 4;  // 16 groups per row
    constexpr int ER = G::ER;       // rows per thread
    static_assert(G::TH * NQE == G::NTHR * ER, "whole output groups per thread");
    const int qe = tid % NQE, re = ER * (tid / NQE);
    float4 pre_up[ER];
    uint32_t pre_mk[ER];
#pragma unroll
    for (int e = 0; e < ER; ++e) {
        const int gy = y0 + re + e, gx = x0 + 4 * qe;
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

    // ---- E: output rows tile+re .. tile+re+ER-1, columns tile+4qe .. 4qe+3 (T index (r+1, 4qe+1+k)) ----
    {
        const int q = qe;
        // FOEED: T_xx row, T_yy rows r .. r+2 and T_xy rows r, r+2 (T rows) of output row r-1;
        // the second output row reuses two of the T_yy rows
        float xx[8], ya[8], yb[8], yc[8], da[8], db[8];
        // EED: plane-1 rows r .. r+2 (the second output row reuses two); the row below's
        // u values, which are the second output row's own
        float cu[8], cc[8], cd[8], ud4[4];
#pragma unroll
        for (int e = 0; e < ER; ++e) {
            const int r = re + e;
            const int gy = y0 + r, gx = x0 + 4 * q;
            if (gy >= h || gx >= w) continue;
            const float *t0 = st + (r + 1) * G::ST_W + 4 * q;
            float Pu[4];
            const float *um = su + (r + G::HL) * G::SU_W + 4 * q + 8;  // u^k at this group
            float ucv[4];
            if (EED && e == 1) {
#pragma unroll
                for (int k = 0; k < 4; ++k) ucv[k] = ud4[k];
            } else {
                const float4 ucv4 = *reinterpret_cast<const float4 *>(um);
                ucv[0] = ucv4.x; ucv[1] = ucv4.y; ucv[2] = ucv4.z; ucv[3] = ucv4.w;
            }
            if (!EED) {
                if (e == 0) {
                    ld8(t0 + 2 * PL - G::ST_W, ya);
                    ld8(t0 + 2 * PL, yb);
                } else {
#pragma unroll
                    for (int k = 0; k < 8; ++k) { ya[k] = yb[k]; yb[k] = yc[k]; }
                }
                ld8(t0, xx);
                ld8(t0 + 2 * PL + G::ST_W, yc);
                ld8(t0 + PL - G::ST_W, da);
                ld8(t0 + PL + G::ST_W, db);
                // per pixel c (T index 1 + k): Pu = (dxx + dyy) + dxy with
                //   dxx = (xx[c-1] + xx[c+1]) - 2 xx[c], dyy = (ya[c] + yc[c]) - 2 yb[c],
                //   dxy = ((db[c+1] + da[c-1]) - (db[c-1] + da[c+1])) / 2,
                // in pixel pairs: the x neighbours and the cross term in two-lane instructions
#pragma unroll
                for (int k = 0; k < 4; k += 2) {
                    const int c = 1 + k;
                    const float2 sxx = __fadd2_rn(pr(xx, c - 1), pr(xx, c + 1));
                    const float2 dxx = make_float2(__fmaf_rn(-2.f, xx[c], sxx.x), __fmaf_rn(-2.f, xx[c + 1], sxx.y));
                    const float2 dyy = make_float2(__fmaf_rn(-2.f, yb[c], __fadd_rn(ya[c], yc[c])),
                                                   __fmaf_rn(-2.f, yb[c + 1], __fadd_rn(ya[c + 1], yc[c + 1])));
                    const float2 dxy = __fmul2_rn(sub2(__fadd2_rn(pr(db, c + 1), pr(da, c - 1)),
                                                       __fadd2_rn(pr(db, c - 1), pr(da, c + 1))),
                                                  make_float2(0.5f, 0.5f));
                    const float2 P2 = __fadd2_rn(__fadd2_rn(dxx, dyy), dxy);
                    Pu[k] = P2.x;
                    Pu[k + 1] = P2.y;
                }
            } else {
                // a (plane 0) on this row, c (plane 1) and b (plane 2) on T rows r .. r+2;
                // u rows tile row-1 .. row+1 at su cols 4q+4 .. 4q+12 (xa/xc/xb[j] <-> col 4q+4+j,
                // pixel k at j = 4 + k). The products b d_y u (differentiated in x) and b d_x u
                // (in y) are formed here at the neighbour positions, as rounded products of
                // the same operands in the same order as a stored plane of them would hold.
                float ac[8], bm[8], bu[8], bd[8], xa[9], xc[9], xb[9];
                ld8(t0, ac);
                if (e == 0) {
                    ld8(t0 + PL - G::ST_W, cu);
                    ld8(t0 + PL, cc);
                } else {
#pragma unroll
                    for (int k = 0; k < 8; ++k) { cu[k] = cc[k]; cc[k] = cd[k]; }
                }
                ld8(t0 + PL + G::ST_W, cd);
                ld8(t0 + 2 * PL, bm);
                ld8(t0 + 2 * PL - G::ST_W, bu);
                ld8(t0 + 2 * PL + G::ST_W, bd);
                ld8(um - 4 - G::SU_W, xa);
                xa[8] = um[4 - G::SU_W];
                ld8(um - 4, xc);
                xc[8] = um[4];
                ld8(um - 4 + G::SU_W, xb);
                xb[8] = um[4 + G::SU_W];
#pragma unroll
                for (int k = 0; k < 4; ++k) ud4[k] = xb[4 + k];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int c = 1 + k, j = 4 + k;
                    const float u0 = ucv[k];
                    // the fluxes as explicit fma(a, b, -round(c d)): the same bits in every instantiation
                    float fx = fmaf(ac[c] + ac[c + 1], xc[j + 1] - u0, -__fmul_rn(ac[c - 1] + ac[c], u0 - xc[j - 1])) * 0.5f;
                    float fy = fmaf(cc[c] + cd[c], xb[j] - u0, -__fmul_rn(cu[c] + cc[c], u0 - xa[j])) * 0.5f;
                    // b d_y u at (row, col +- 1), b d_x u at (row +- 1, col)
                    const float pr_ = __fmul_rn(bm[c + 1], __fmul_rn(__fsub_rn(xb[j + 1], xa[j + 1]), 0.5f));
                    const float pl_ = __fmul_rn(bm[c - 1], __fmul_rn(__fsub_rn(xb[j - 1], xa[j - 1]), 0.5f));
                    const float pd_ = __fmul_rn(bd[c], __fmul_rn(__fsub_rn(xb[j + 1], xb[j - 1]), 0.5f));
                    const float pu_ = __fmul_rn(bu[c], __fmul_rn(__fsub_rn(xa[j + 1], xa[j - 1]), 0.5f));
                    float mx = __fsub_rn(pr_, pl_);
                    float my = __fsub_rn(pd_, pu_);
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
            if (sizeof(U) == sizeof(double)) {  // the extended-precision update
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    un[k] = fsi_update_ff(upv[k], ucv[k], Pu[k], p.alpha_t, p.alpha_lo, p.tau_t, p.tau_lo);
            } else {
                // per pixel: e = u^k - tau P u^k, u^{k+1} = u^{k-1} + alpha (e - u^{k-1}), in pixel pairs
#pragma unroll
                for (int k = 0; k < 4; k += 2) {
                    const float2 up = pr(upv, k);
                    const float2 ex = __ffma2_rn(make_float2(-tau, -tau), pr(Pu, k), pr(ucv, k));
                    const float2 nu = __ffma2_rn(make_float2(alpha, alpha), sub2(ex, up), up);
                    un[k] = nu.x;
                    un[k + 1] = nu.y;
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if ((pre_mk[e] >> (8 * k)) & 0xffu) un[k] = ucv[k];  // known pixels keep u^k
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

// The size rule used when no tile height is given (the launches that are not
// autotuned): images with fewer 64 x 32 tiles than this run on 64 x 16 tiles,
// as they fill less than a wave of the GPU and a step's time is then the
// latency of one tile.
constexpr long long kFastSmallTiles = 304;

// One FSI step over one image, one CTA per 64 x TH tile.
template <int R, bool EED, typename U, int TH>
__global__ void __launch_bounds__(FastTile<R, EED, TH>::NTHR, FastTile<R, EED, TH>::MINB) fsi_step_fast(const StepArgs<float> p)
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
    fast_tile<R, EED, U, TH>(p, im, blockIdx.x * FastTile<R, EED, TH>::TW, blockIdx.y * TH, sm, rnum, rden);
    if (p.residual)
        finish_cycle_residual(rnum, rden, p.ctl, p.partials, gridDim.x * gridDim.y,
                              blockIdx.y * gridDim.x + blockIdx.x, red);
}

// ---------------------------------------------------------------------------
// Batched FOEED or EED: one launch per FSI step over the tiles of many images.

template <int R, bool EED, typename U>
__global__ void __launch_bounds__(256, FastTile<R, EED>::MINB) fsi_batch_step_fast(const StepArgs<float> p, const BatchArgs b)
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
    if (I.th == 16)
        fast_tile<R, EED, U, 16>(p, im, tx * 64, ty * 16, sm, rnum, rden);
    else
        fast_tile<R, EED, U, 32>(p, im, tx * 64, ty * 32, sm, rnum, rden);
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
    using G32 = FastTile<R, EED, 32>;
    using G16 = FastTile<R, EED, 16>;
    auto k32 = fsi_step_fast<R, EED, U, 32>;
    auto k16 = fsi_step_fast<R, EED, U, 16>;
    if (!ap) {
        cudaError_t e = cudaFuncSetAttribute(k32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G32::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G16::SMEM);
        if constexpr (!EED) {
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(fsi_step_fast<R, EED, U, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)FastTile<R, EED, 64>::SMEM);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(fsi_step_fast<R, EED, U, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)FastTile<R, EED, 8>::SMEM);
        }
        return e;
    }
    const int ntx = (ap->w + 63) / 64;
    if constexpr (!EED) {
        // 64 x 64 tiles, 512 threads, two CTAs per SM (FOEED only: a candidate of
        // the autotuner that measured slower at every size, not instantiated for EED)
        if (ap->tile_h == 64) {
            using G64 = FastTile<R, EED, 64>;
            dim3 grid(ntx, (ap->h + 63) / 64);
            return launch_step_kernel(fsi_step_fast<R, EED, U, 64>, grid, G64::NTHR, G64::SMEM, s, *ap);
        }
        // 64 x 8 tiles, 128 threads, up to eight CTAs per SM (FOEED only: a
        // candidate of the autotuner for images under one wave of tiles)
        if (ap->tile_h == 8) {
            using G8 = FastTile<R, EED, 8>;
            dim3 grid(ntx, (ap->h + 7) / 8);
            return launch_step_kernel(fsi_step_fast<R, EED, U, 8>, grid, G8::NTHR, G8::SMEM, s, *ap);
        }
    }
    const bool h16 = ap->tile_h == 16 || (ap->tile_h != 32 && (long long)ntx * ((ap->h + 31) / 32) < kFastSmallTiles);
    if (h16) {
        dim3 grid(ntx, (ap->h + 15) / 16);
        return launch_step_kernel(k16, grid, 256, G16::SMEM, s, *ap);
    }
    dim3 grid(ntx, (ap->h + 31) / 32);
    return launch_step_kernel(k32, grid, 256, G32::SMEM, s, *ap);
}

}  // namespace foeed
