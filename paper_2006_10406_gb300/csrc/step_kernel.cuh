// Fused explicit FSI step for FOEED (Eq. genModel) and EED (Eq. EEDModel).
// T = storage / stencil type (float or double), U = type of the FSI update
// (double for the mixed-precision mode), R = Gaussian radius, TW x TH tile.
#pragma once

#include "foeed_device.cuh"

namespace foeed {

template <int R, int TW, int TH, bool EED>
struct Tile {
    static constexpr int HL = R + 2;           // u halo
    static constexpr int SU_W = TW + 2 * HL;   // u tile
    static constexpr int SU_H = TH + 2 * HL;
    static constexpr int SX_W = TW + 4;        // x-smoothed rows (all u rows, tile+-2 columns)
    static constexpr int SX_H = SU_H;
    static constexpr int SS_W = TW + 4;        // u_sigma on tile+-2
    static constexpr int SS_H = TH + 4;
    static constexpr int ST_W = TW + 2;        // tensor products on tile+-1
    static constexpr int ST_H = TH + 2;
    static constexpr int NT = EED ? 4 : 3;     // FOEED: Txx, Txy, Tyy; EED: a, c, qx, qy
    static constexpr int ELEMS = SU_W * SU_H + SX_W * SX_H + SS_W * SS_H + NT * ST_W * ST_H;
};

template <typename T, typename U, int R, int TW, int TH, bool EED>
__global__ void __launch_bounds__(kThreads) fsi_step_kernel(const StepArgs<T> p)
{
    using G = Tile<R, TW, TH, EED>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *su = reinterpret_cast<T *>(smem_raw);
    T *sx = su + G::SU_W * G::SU_H;
    T *ss = sx + G::SX_W * G::SX_H;
    T *st = ss + G::SS_W * G::SS_H;
    __shared__ double red[64];

    // Programmatic dependent launch: wait until the previous step's grid has
    // completed and its writes are visible (a no-op for an ordinary launch),
    // then let the next step's CTAs be scheduled as SM slots free up.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (p.check_done && p.ctl->done) return;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // alpha and tau in the update type: the pre-rounded copies when U == T
    const U alpha = sizeof(U) == sizeof(T) ? U(p.alpha_t) : U(p.alpha);
    const U tau = sizeof(U) == sizeof(T) ? U(p.tau_t) : U(p.tau);

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const int w = p.w, h = p.h;
    const long pitch = p.pitch;

    // ---- A: u^k tile + halo, mirrored at the border (Eq. smoothingModel) ----
    {
        const bool interior = (x0 - G::HL >= 0) && (x0 + TW + G::HL <= w) && (y0 - G::HL >= 0) &&
                              (y0 + TH + G::HL <= h);
        const T *__restrict__ uc = p.ucur;
        for (int i = tid; i < G::SU_W * G::SU_H; i += kThreads) {
            int r = i / G::SU_W, c = i - r * G::SU_W;
            int gy = y0 - G::HL + r, gx = x0 - G::HL + c;
            if (!interior) { gy = mirror_idx(gy, h); gx = mirror_idx(gx, w); }
            su[i] = uc[(long)gy * pitch + gx];
        }
    }
    __syncthreads();

    // ---- B: Gaussian x pass (taps -R..R) ----
    for (int i = tid; i < G::SX_W * G::SX_H; i += kThreads) {
        int r = i / G::SX_W, c = i - r * G::SX_W;
        const T *row = su + r * G::SU_W + c;  // output column c <-> u columns c .. c + 2R
        T acc = T(0);
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) acc += p.wts[t] * row[t];
        sx[i] = acc;
    }
    __syncthreads();

    // ---- C: Gaussian y pass -> u_sigma on tile+-2 ----
    for (int i = tid; i < G::SS_W * G::SS_H; i += kThreads) {
        int r = i / G::SS_W, c = i - r * G::SS_W;
        const T *col = sx + r * G::SX_W + c;
        T acc = T(0);
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) acc += p.wts[t] * col[t * G::SX_W];
        ss[i] = acc;
    }
    __syncthreads();

    // ---- D: tensor and inner derivatives on tile+-1 ----
    const T l2 = p.l2;
    const T inv_l2 = p.inv_l2;
    constexpr int PL = G::ST_W * G::ST_H;
    for (int i = tid; i < PL; i += kThreads) {
        int r = i / G::ST_W, c = i - r * G::ST_W;
        // u_sigma around this pixel: ss row r+1, col c+1
        const T *s0 = ss + (r + 1) * G::SS_W + (c + 1);
        T dx = s0[1] - s0[-1];                  // 2 d_x u_sigma
        T dy = s0[G::SS_W] - s0[-G::SS_W];      // 2 d_y u_sigma
        T sq = dx * dx + dy * dy;               // 4 lambda1
        T mu1 = diffusivity<T>(p.g_kind, sq * T(0.25), inv_l2, l2);
        T C, S;
        if (sq == T(0)) { C = T(1); S = T(0); }   // v1 := (1, 0) for a zero gradient
        else { T inv = T(1) / sq; C = (dx * dx - dy * dy) * inv; S = T(2) * dx * dy * inv; }
        const T *u0 = su + (r + 1 + R) * G::SU_W + (c + 1 + R);
        T uc = u0[0];
        if (!EED) {
            T hxx = (u0[-1] + u0[1]) - T(2) * uc;
            T hyy = (u0[-G::SU_W] + u0[G::SU_W]) - T(2) * uc;
            T hxy = ((u0[G::SU_W + 1] + u0[-G::SU_W - 1]) - (u0[G::SU_W - 1] + u0[-G::SU_W + 1])) * T(0.25);
            T mu3 = mu3_of<T>(p.mu3_mode, mu1);
            // rotated frame: h11 = v1'Hv1, h22 = v2'Hv2, h12 = v1'Hv2 (Eq. E3, Eq. foad_diff_direc)
            T A = (hxx + hyy) * T(0.5), B = (hxx - hyy) * T(0.5);
            T h11 = A + C * B + S * hxy;
            T h22 = A - C * B - S * hxy;
            T h12 = C * hxy - S * B;
            T pp = mu1 * h11, qq = h22, rr = mu3 * h12;
            // T = pp v1v1' + qq v2v2' + rr (v1v2' + v2v1')
            T half_sum = (pp + qq) * T(0.5), half_dif = (pp - qq) * T(0.5);
            st[i] = half_sum + C * half_dif - S * rr;            // T_xx
            st[PL + i] = S * half_dif + C * rr;                  // T_xy
            st[2 * PL + i] = half_sum - C * half_dif + S * rr;   // T_yy
        } else {
            // D = mu1 v1v1' + v2v2' = [[a, b], [b, c]]
            T a = ((mu1 + T(1)) + C * (mu1 - T(1))) * T(0.5);
            T cc = ((mu1 + T(1)) - C * (mu1 - T(1))) * T(0.5);
            T b = S * (mu1 - T(1)) * T(0.5);
            st[i] = a;
            st[PL + i] = cc;
            st[2 * PL + i] = b * ((u0[G::SU_W] - u0[-G::SU_W]) * T(0.5));  // b * d_y u
            st[3 * PL + i] = b * ((u0[1] - u0[-1]) * T(0.5));               // b * d_x u
        }
    }
    __syncthreads();

    // ---- E: outer divergence, masked FSI update, residual ----
    double rnum = 0.0, rden = 0.0;
    for (int i = tid; i < TW * TH; i += kThreads) {
        int r = i / TW, c = i - r * TW;
        int gx = x0 + c, gy = y0 + r;
        if (gx >= w || gy >= h) continue;
        const int k = (r + 1) * G::ST_W + (c + 1);
        const T *u0 = su + (r + G::HL) * G::SU_W + (c + G::HL);
        T uc = u0[0];
        T Pu;
        if (!EED) {
            const T *txx = st, *txy = st + PL, *tyy = st + 2 * PL;
            T dxx = (txx[k - 1] + txx[k + 1]) - T(2) * txx[k];
            T dyy = (tyy[k - G::ST_W] + tyy[k + G::ST_W]) - T(2) * tyy[k];
            T dxy = ((txy[k + G::ST_W + 1] + txy[k - G::ST_W - 1]) - (txy[k + G::ST_W - 1] + txy[k - G::ST_W + 1])) * T(0.5);
            Pu = (dxx + dyy) + dxy;  // d_xx T_xx + (d_xy + d_yx) T_xy + d_yy T_yy
        } else {
            const T *sa = st, *sc = st + PL, *qx = st + 2 * PL, *qy = st + 3 * PL;
            T fx = ((sa[k] + sa[k + 1]) * (u0[1] - uc) - (sa[k - 1] + sa[k]) * (uc - u0[-1])) * T(0.5);
            T fy = ((sc[k] + sc[k + G::ST_W]) * (u0[G::SU_W] - uc) - (sc[k - G::ST_W] + sc[k]) * (uc - u0[-G::SU_W])) * T(0.5);
            T mx = (qx[k + 1] - qx[k - 1]) * T(0.5);
            T my = (qy[k + G::ST_W] - qy[k - G::ST_W]) * T(0.5);
            Pu = -((fx + fy) + (mx + my));
        }
        const long gi = (long)gy * pitch + gx;
        T un;
        if (p.mask && p.mask[gi]) {
            un = uc;
        } else {
            U up = U(p.uprev[gi]);
            U ex = U(uc) - tau * U(Pu);  // (I - tau P) u^k
            un = T(up + alpha * (ex - up));
        }
        if (p.residual) {
            double d = double(un) - double(p.c0[gi]);
            rnum += d * d;
            rden += double(un) * double(un);
        }
        p.unext[gi] = un;
    }

    if (p.residual) {
        const int nblocks = gridDim.x * gridDim.y;
        const int bid = blockIdx.y * gridDim.x + blockIdx.x;
        if (grid_sum2_last(rnum, rden, p.partials, &p.ctl->ticket, nblocks, bid, red)) {
            Ctl *ctl = p.ctl;
            double rel = rden > 0.0 ? sqrt(rnum) / sqrt(rden) : sqrt(rnum);
            ctl->last_num = rnum;
            ctl->last_den = rden;
            ctl->last_rel = rel;
            ctl->cycles += 1;
            if (!isfinite(rel)) { ctl->diverged = 1; ctl->done = 1; }
            else if (ctl->tol > 0.0 && rel < ctl->tol) ctl->done = 1;
        }
    }
}

// Launches one step; with a == nullptr it only sets the kernel's shared-memory
// attribute (done before any stream capture).
template <typename T, typename U, int R, int TW, int TH, bool EED>
cudaError_t launch_fsi_step(const StepArgs<T> *ap, cudaStream_t s)
{
    using G = Tile<R, TW, TH, EED>;
    constexpr size_t smem = sizeof(T) * G::ELEMS;
    auto kern = fsi_step_kernel<T, U, R, TW, TH, EED>;
    if (!ap) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const StepArgs<T> &a = *ap;
    dim3 grid((a.w + TW - 1) / TW, (a.h + TH - 1) / TH);
    return launch_step_kernel(kern, grid, kThreads, smem, s, a);
}

}  // namespace foeed
