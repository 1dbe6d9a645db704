/*
 * FP64 CPU oracle for FOEED and EED sparse-mask inpainting with FSI
 * (Jumakulyyev & Schultz, "Fourth-Order Anisotropic Diffusion for Inpainting
 * and Image Compression", arXiv 2006.10406).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow reference against
 * which the CUDA path is checked. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product library never does.
 * It shares no code, header or table with the CUDA path.
 *
 * Style: plain scalar loops in IEEE double, compiled without FMA contraction
 * (-ffp-contract=off), fixed summation orders as written below. Every function
 * follows the passage of the paper it cites. Where the paper is silent or its
 * text is garbled, the reading taken is stated at the function.
 *
 * Grid convention: image of w columns (x, fastest) and h rows (y), row-major,
 * u[y*w + x], pixel size dx = dy = 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

/* Number of host threads the row loops may use (OpenMP builds only). */
void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* Boundary: homogeneous Neumann condition (Eq. smoothingModel, Sec. 2.1),
 * discretised as a half-sample mirror: index -1 maps to 0, -2 to 1, n to n-1.
 * Indices further out keep reflecting (period 2n), so tiny images work. */
static long mirror(long i, long n)
{
    long p = 2 * n;
    i %= p;
    if (i < 0) i += p;
    return i < n ? i : p - 1 - i;
}

/* Number of mirror reflections between i and the image: the sign of an odd
 * ghost value is (-1)^reflections. */
static int reflections_parity(long i, long n)
{
    long q = i >= 0 ? i / n : -((-i + n - 1) / n);
    return (int)(q & 1);
}

/* ------------------------------------------------------------------------ */
/* Gaussian pre-smoothing u_sigma = K_sigma * u (Sec. 2.2, Eq. CharDiff text;
 * Sec. 3.1, Eq. faod_diffTensor). The paper gives no discretisation; the
 * reading taken: sampled exp(-t^2/(2 sigma^2)), truncated at R = ceil(3 sigma),
 * normalised to sum 1. sigma <= 0 means no smoothing (R = 0, weight 1).
 * Writes 2R+1 weights (w[0] belongs to offset -R) and returns R. */
int orc_gauss_weights(double sigma, double *wts, int max_taps)
{
    int R = sigma > 0.0 ? (int)ceil(3.0 * sigma) : 0;
    if (2 * R + 1 > max_taps) return -1;
    double sum = 0.0;
    for (int t = -R; t <= R; ++t) {
        double v = sigma > 0.0 ? exp(-((double)t * (double)t) / (2.0 * sigma * sigma)) : 1.0;
        wts[t + R] = v;
        sum += v;
    }
    for (int t = 0; t < 2 * R + 1; ++t) wts[t] /= sum;
    return R;
}

/* Separable Gaussian: x pass then y pass, taps -R..R in order, mirrored ghosts. */
void orc_presmooth(const double *u, int w, int h, double sigma, double *us)
{
    double wts[257];
    int R = orc_gauss_weights(sigma, wts, 257);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)w * h);
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double s = 0.0;
            for (int t = -R; t <= R; ++t) s += wts[t + R] * u[(size_t)y * w + mirror(x + t, w)];
            tmp[(size_t)y * w + x] = s;
        }
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double s = 0.0;
            for (int t = -R; t <= R; ++t) s += wts[t + R] * tmp[(size_t)mirror(y + t, h) * w + x];
            us[(size_t)y * w + x] = s;
        }
    free(tmp);
}

/* Regularised gradient grad(u_sigma) by central differences with mirrored
 * ghosts (Sec. 3.1, text after Eq. foad_diffTensor_entries; the stencil is
 * not printed, central differences are the reading taken). */
void orc_gradient(const double *us, int w, int h, double *gx, double *gy)
{
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            gx[p] = (us[(size_t)y * w + mirror(x + 1, w)] - us[(size_t)y * w + mirror(x - 1, w)]) / 2.0;
            gy[p] = (us[(size_t)mirror(y + 1, h) * w + x] - us[(size_t)mirror(y - 1, h) * w + x]) / 2.0;
        }
}

/* ------------------------------------------------------------------------ */
/* Diffusivities g(s^2), s = |grad u_sigma|.
 *   0 Charbonnier      1/sqrt(1 + s^2/lambda^2)          (Eq. CharDiff)
 *   1 Perona-Malik     1/(1 + s^2/lambda^2)               (Table 6)
 *   2 Perona-Malik 2   exp(-s^2/lambda^2)                 (Table 6)
 *   3 Aubert           (s/lambda)^2 / (s^2+lambda^2)^2    (Table 6, as printed)
 *   4 Geman-Reynolds   2 lambda^2 / (s^2+lambda^2)^2      (Table 6, as printed)
 * The last two are taken literally from the table; they are not bounded by 1. */
double orc_diffusivity(int kind, double s2, double lambda)
{
    double l2 = lambda * lambda;
    switch (kind) {
    case 0: return 1.0 / sqrt(1.0 + s2 / l2);
    case 1: return 1.0 / (1.0 + s2 / l2);
    case 2: return exp(-s2 / l2);
    case 3: return (s2 / l2) / ((s2 + l2) * (s2 + l2));
    case 4: return 2.0 * l2 / ((s2 + l2) * (s2 + l2));
    default: return NAN;
    }
}

/* mu_3 choices (Sec. 3.1, Table 1): 0 geometric mean sqrt(mu1 mu2) (the
 * paper's choice for all experiments), 1 arithmetic mean (mu1+mu2)/2,
 * 2 maximum mu3 = 1. */
static double mu3_of(int mode, double mu1, double mu2)
{
    switch (mode) {
    case 1: return (mu1 + mu2) / 2.0;
    case 2: return 1.0;
    default: return sqrt(mu1 * mu2);
    }
}

/* Eigenvector v1 of the structure tensor J = grad u_s grad u_s^T (Sec. 3.1):
 * v1 = grad/|grad|, v2 = grad^perp/|grad| = (-v1y, v1x). The paper leaves v1
 * undefined for a zero gradient; then mu1 = mu2 = mu3 = 1 (Charbonnier), the
 * tensor is the identity on symmetric matrices for any v1, and (1,0) is taken. */
static void eigvec(double gx, double gy, double *v1x, double *v1y)
{
    double l1 = gx * gx + gy * gy;
    if (l1 == 0.0) { *v1x = 1.0; *v1y = 0.0; return; }
    double n = sqrt(l1);
    *v1x = gx / n;
    *v1y = gy / n;
}

/* Literal fourth-order diffusion tensor d_ijkl (Eq. faod_diffTensor and
 * Eq. foad_diffTensor_entries): D = sum_r mu_r E_r (x) E_r with
 *   mu1 = g(lambda1), E1 = v1 v1^T;  mu2 = 1, E2 = v2 v2^T;
 *   mu3 per mode,     E3 = (v1 v2^T + v2 v1^T)/sqrt 2;
 *   mu4 = 0,          E4 = (v1 v2^T - v2 v1^T)/sqrt 2,
 * lambda1 = |grad u_sigma|^2. Output index d[((i*2+j)*2+k)*2+l], i,j,k,l in
 * {0 = x, 1 = y}. mu_out (optional) receives mu1..mu4. */
void orc_foeed_tensor(double gx, double gy, double lambda, int g_kind, int mu3_mode,
                      double d[16], double mu_out[4])
{
    double v1[2], v2[2];
    eigvec(gx, gy, &v1[0], &v1[1]);
    v2[0] = -v1[1];
    v2[1] = v1[0];
    double l1 = gx * gx + gy * gy;
    double mu[4];
    mu[0] = orc_diffusivity(g_kind, l1, lambda);
    mu[1] = 1.0;
    mu[2] = mu3_of(mu3_mode, mu[0], mu[1]);
    mu[3] = 0.0;
    double r2 = 1.0 / sqrt(2.0);
    double E[4][2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            E[0][i][j] = v1[i] * v1[j];
            E[1][i][j] = v2[i] * v2[j];
            E[2][i][j] = r2 * (v1[i] * v2[j] + v2[i] * v1[j]);
            E[3][i][j] = r2 * (v1[i] * v2[j] - v2[i] * v1[j]);
        }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 2; ++l) {
                    double s = 0.0;
                    for (int r = 0; r < 4; ++r) s += mu[r] * E[r][i][j] * E[r][k][l];
                    d[((i * 2 + j) * 2 + k) * 2 + l] = s;
                }
    if (mu_out)
        for (int r = 0; r < 4; ++r) mu_out[r] = mu[r];
}

/* Tensor field for a whole image: d[p*16 + ...] from u (pre-smoothing,
 * gradient, literal tensor), Sec. 3.1. */
void orc_foeed_tensor_field(const double *u, int w, int h, double sigma, double lambda,
                            int g_kind, int mu3_mode, double *d)
{
    size_t n = (size_t)w * h;
    double *us = (double *)malloc(sizeof(double) * n);
    double *gx = (double *)malloc(sizeof(double) * n);
    double *gy = (double *)malloc(sizeof(double) * n);
    orc_presmooth(u, w, h, sigma, us);
    orc_gradient(us, w, h, gx, gy);
#pragma omp parallel for num_threads(g_threads)
    for (long p = 0; p < (long)n; ++p) orc_foeed_tensor(gx[p], gy[p], lambda, g_kind, mu3_mode, d + p * 16, NULL);
    free(us);
    free(gx);
    free(gy);
}

/* Inner Hessian H(u) by the finite differences of Sec. 3.3 with mirrored
 * ghosts. The printed u_xy stencil has four plus signs, which is not a
 * derivative; the reading taken is the standard
 * (u[i+1,j+1] + u[i-1,j-1] - u[i-1,j+1] - u[i+1,j-1]) / 4, and u_yx = u_xy. */
void orc_hessian(const double *u, int w, int h, double *hxx, double *hxy, double *hyy)
{
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            long xm = mirror(x - 1, w), xp = mirror(x + 1, w);
            long ym = mirror(y - 1, h), yp = mirror(y + 1, h);
            hxx[p] = u[(size_t)y * w + xm] - 2.0 * u[p] + u[(size_t)y * w + xp];
            hyy[p] = u[(size_t)ym * w + x] - 2.0 * u[p] + u[(size_t)yp * w + x];
            hxy[p] = (u[(size_t)yp * w + xp] + u[(size_t)ym * w + xm] - u[(size_t)yp * w + xm] -
                      u[(size_t)ym * w + xp]) / 4.0;
        }
}

/* Fourth-order operator for a given tensor field (Eq. ts-fourth-order-diffusion,
 * Eq. double-dot, Eq. genModel):
 *   T_ij = sum_kl d_ijkl H_kl,   (P u) = sum_ij d_ij T_ij
 * over the four outer pairs xx, xy, yx, yy, so that du/dt = -(P u).
 * Outer differences use the same stencils as the inner ones. The paper states
 * no boundary rule for the outer derivatives; the reading taken: T_xx, T_yy
 * get even (mirror) ghosts and the mixed components T_xy, T_yx get odd ghosts
 * across each edge (the sign flips once per reflection). This makes the outer
 * operator the transpose of the inner one, so P is symmetric as the FSI
 * analysis of Sec. 3.3 requires. */
void orc_apply_P_field(const double *u, const double *d, int w, int h, double *Pu)
{
    size_t n = (size_t)w * h;
    double *H[3], *T[4];
    for (int c = 0; c < 3; ++c) H[c] = (double *)malloc(sizeof(double) * n);
    for (int c = 0; c < 4; ++c) T[c] = (double *)malloc(sizeof(double) * n);
    orc_hessian(u, w, h, H[0], H[1], H[2]);
#pragma omp parallel for num_threads(g_threads)
    for (long p = 0; p < (long)n; ++p) {
        double Hm[2][2] = {{H[0][p], H[1][p]}, {H[1][p], H[2][p]}};
        const double *dp = d + p * 16;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double s = 0.0;
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 2; ++l) s += dp[((i * 2 + j) * 2 + k) * 2 + l] * Hm[k][l];
                T[i * 2 + j][p] = s;
            }
    }
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            /* ghost access: T value at (x+ox, y+oy), with the parity rule above */
#define TG(c, ox, oy)                                                                              \
    ((((c) == 1 || (c) == 2) &&                                                                    \
      (reflections_parity(x + (ox), w) ^ reflections_parity(y + (oy), h)))                         \
         ? -T[c][(size_t)mirror(y + (oy), h) * w + mirror(x + (ox), w)]                            \
         : T[c][(size_t)mirror(y + (oy), h) * w + mirror(x + (ox), w)])
            double dxx = TG(0, -1, 0) - 2.0 * TG(0, 0, 0) + TG(0, 1, 0);
            double dxy = (TG(1, 1, 1) + TG(1, -1, -1) - TG(1, -1, 1) - TG(1, 1, -1)) / 4.0;
            double dyx = (TG(2, 1, 1) + TG(2, -1, -1) - TG(2, -1, 1) - TG(2, 1, -1)) / 4.0;
            double dyy = TG(3, 0, -1) - 2.0 * TG(3, 0, 0) + TG(3, 0, 1);
#undef TG
            Pu[(size_t)y * w + x] = dxx + dxy + dyx + dyy;
        }
    for (int c = 0; c < 3; ++c) free(H[c]);
    for (int c = 0; c < 4; ++c) free(T[c]);
}

/* FOEED operator P(u) u (Eq. genModel): tensor field from u, then the
 * fourth-order divergence above. */
void orc_foeed_operator(const double *u, int w, int h, double sigma, double lambda, int g_kind,
                        int mu3_mode, double *Pu)
{
    size_t n = (size_t)w * h;
    double *d = (double *)malloc(sizeof(double) * 16 * n);
    orc_foeed_tensor_field(u, w, h, sigma, lambda, g_kind, mu3_mode, d);
    orc_apply_P_field(u, d, w, h, Pu);
    free(d);
}

/* ------------------------------------------------------------------------ */
/* Second-order EED (Eq. EEDModel, Eq. diffTensor_EED): du/dt = div(D grad u),
 * D = g(|grad u_s|^2) v1 v1^T + 1 v2 v2^T = [[a, b], [b, c]].
 * Tensor field for a whole image, abc[p*3 + {0,1,2}] = (a, b, c). */
void orc_eed_tensor_field(const double *u, int w, int h, double sigma, double lambda, int g_kind,
                          double *abc)
{
    size_t n = (size_t)w * h;
    double *us = (double *)malloc(sizeof(double) * n);
    double *gx = (double *)malloc(sizeof(double) * n);
    double *gy = (double *)malloc(sizeof(double) * n);
    orc_presmooth(u, w, h, sigma, us);
    orc_gradient(us, w, h, gx, gy);
#pragma omp parallel for num_threads(g_threads)
    for (long p = 0; p < (long)n; ++p) {
        double v1x, v1y;
        eigvec(gx[p], gy[p], &v1x, &v1y);
        double v2x = -v1y, v2y = v1x;
        double mu1 = orc_diffusivity(g_kind, gx[p] * gx[p] + gy[p] * gy[p], lambda);
        abc[p * 3 + 0] = mu1 * v1x * v1x + 1.0 * v2x * v2x;
        abc[p * 3 + 1] = mu1 * v1x * v1y + 1.0 * v2x * v2y;
        abc[p * 3 + 2] = mu1 * v1y * v1y + 1.0 * v2y * v2y;
    }
    free(us);
    free(gx);
    free(gy);
}

/* EED operator for a given tensor field: (P u) = -div(D grad u). The paper
 * prints no EED discretisation; the reading taken is the standard symmetric
 * central scheme:
 *   d_x(a d_x u) at i: [(a_i + a_{i+1})(u_{i+1} - u_i) - (a_{i-1} + a_i)(u_i - u_{i-1})] / 2
 *   d_x(b d_y u):      central difference in x of q = b * (central y-difference of u)
 *   d_y(b d_x u), d_y(c d_y u) likewise.
 * Ghosts: u, a, c even; the products q are odd across the edge normal to their
 * outer derivative, which makes the mixed part the transpose of itself. */
void orc_apply_eed_field(const double *u, const double *abc, int w, int h, double *Pu)
{
    size_t n = (size_t)w * h;
    double *qx = (double *)malloc(sizeof(double) * n); /* b * d_y u, differentiated in x */
    double *qy = (double *)malloc(sizeof(double) * n); /* b * d_x u, differentiated in y */
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            double uy = (u[(size_t)mirror(y + 1, h) * w + x] - u[(size_t)mirror(y - 1, h) * w + x]) / 2.0;
            double ux = (u[(size_t)y * w + mirror(x + 1, w)] - u[(size_t)y * w + mirror(x - 1, w)]) / 2.0;
            qx[p] = abc[p * 3 + 1] * uy;
            qy[p] = abc[p * 3 + 1] * ux;
        }
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            size_t pxm = (size_t)y * w + mirror(x - 1, w), pxp = (size_t)y * w + mirror(x + 1, w);
            size_t pym = (size_t)mirror(y - 1, h) * w + x, pyp = (size_t)mirror(y + 1, h) * w + x;
            double a = abc[p * 3 + 0], c = abc[p * 3 + 2];
            double fx = ((a + abc[pxp * 3 + 0]) * (u[pxp] - u[p]) - (abc[pxm * 3 + 0] + a) * (u[p] - u[pxm])) / 2.0;
            double fy = ((c + abc[pyp * 3 + 2]) * (u[pyp] - u[p]) - (abc[pym * 3 + 2] + c) * (u[p] - u[pym])) / 2.0;
            double sxp = reflections_parity(x + 1, w) ? -1.0 : 1.0;
            double sxm = reflections_parity(x - 1, w) ? -1.0 : 1.0;
            double syp = reflections_parity(y + 1, h) ? -1.0 : 1.0;
            double sym = reflections_parity(y - 1, h) ? -1.0 : 1.0;
            double mx = (sxp * qx[pxp] - sxm * qx[pxm]) / 2.0;
            double my = (syp * qy[pyp] - sym * qy[pym]) / 2.0;
            Pu[p] = -(fx + mx + my + fy);
        }
    free(qx);
    free(qy);
}

void orc_eed_operator(const double *u, int w, int h, double sigma, double lambda, int g_kind, double *Pu)
{
    size_t n = (size_t)w * h;
    double *abc = (double *)malloc(sizeof(double) * 3 * n);
    orc_eed_tensor_field(u, w, h, sigma, lambda, g_kind, abc);
    orc_apply_eed_field(u, abc, w, h, Pu);
    free(abc);
}

/* ------------------------------------------------------------------------ */
/* FSI extrapolation weight alpha_k = (4k + 2)/(2k + 3), k = 0..n-1 (Sec. 3.3). */
double orc_fsi_alpha(int k) { return (4.0 * k + 2.0) / (2.0 * k + 3.0); }

/* One masked FSI step (Sec. 3.3, FSI equation; Dirichlet data Eq. inpaintingModel):
 * unknown pixels: u^{k+1} = alpha (u^k - tau P(u^k) u^k) + (1 - alpha) u^{k-1};
 * known pixels (mask != 0): u^{k+1} = u^k. method 0 = FOEED, 1 = EED.
 * mask may be NULL (pure smoothing, no Dirichlet pixels). unext must not alias
 * uprev or ucur. */
void orc_fsi_step(int method, const double *uprev, const double *ucur, const uint8_t *mask, int w,
                  int h, double alpha, double tau, double sigma, double lambda, int g_kind,
                  int mu3_mode, double *unext)
{
    size_t n = (size_t)w * h;
    double *Pu = (double *)malloc(sizeof(double) * n);
    if (method == 0) orc_foeed_operator(ucur, w, h, sigma, lambda, g_kind, mu3_mode, Pu);
    else orc_eed_operator(ucur, w, h, sigma, lambda, g_kind, Pu);
    for (size_t p = 0; p < n; ++p) {
        if (mask && mask[p]) unext[p] = ucur[p];
        else unext[p] = alpha * (ucur[p] - tau * Pu[p]) + (1.0 - alpha) * uprev[p];
    }
    free(Pu);
}

/* Full inpainting solve (Eq. inpaintingModel with Eq. genModel or
 * Eq. EEDModel; time integration by FSI cycles, Sec. 3.3).
 *   f:    known grey values (read at mask != 0 only)
 *   u:    in/out image; on entry only read when init_mode == 1
 *   init_mode 0: unknown pixels start at the mean of f over the known set
 *                (the paper is silent on initialisation; 0 if no pixel is known)
 *   init_mode 1: unknown pixels start at the given u
 *   tau <= 0 selects the paper's step sizes: 0.05 (FOEED), 0.25 (EED).
 *   Each cycle m: u^{m,-1} := u^{m,0}; n steps; u^{m+1,0} := u^{m,n}.
 *   tol > 0: stop after the first cycle with |u^{m,n} - u^{m,0}|_2 / |u^{m,n}|_2 < tol
 *            (relative form of the paper's absolute test); tol == 0 runs
 *            exactly max_cycles cycles.
 * out[0] = cycles run, out[1] = last relative change, out[2] = converged flag.
 * Returns 0 ok, 3 not converged (tol > 0 only), 4 diverged (non-finite). */
int orc_inpaint(int method, const double *f, const uint8_t *mask, double *u, int w, int h,
                double sigma, double lambda, double tau, int cycle_len, int max_cycles, double tol,
                int g_kind, int mu3_mode, int init_mode, double out[3])
{
    size_t n = (size_t)w * h;
    if (tau <= 0.0) tau = method == 0 ? 0.05 : 0.25;
    if (init_mode == 0) {
        double s = 0.0;
        long cnt = 0;
        for (size_t p = 0; p < n; ++p)
            if (mask[p]) { s += f[p]; ++cnt; }
        double mean = cnt ? s / (double)cnt : 0.0;
        for (size_t p = 0; p < n; ++p) u[p] = mask[p] ? f[p] : mean;
    } else {
        for (size_t p = 0; p < n; ++p)
            if (mask[p]) u[p] = f[p];
    }
    double *u0 = (double *)malloc(sizeof(double) * n);
    double *um = (double *)malloc(sizeof(double) * n);
    double *un = (double *)malloc(sizeof(double) * n);
    int status = 0, cycles = 0, converged = 0;
    double rel = 0.0;
    for (int m = 0; m < max_cycles; ++m) {
        memcpy(u0, u, sizeof(double) * n);
        memcpy(um, u, sizeof(double) * n); /* u^{m,-1} := u^{m,0} */
        for (int k = 0; k < cycle_len; ++k) {
            orc_fsi_step(method, um, u, mask, w, h, orc_fsi_alpha(k), tau, sigma, lambda, g_kind,
                         mu3_mode, un);
            memcpy(um, u, sizeof(double) * n);
            memcpy(u, un, sizeof(double) * n);
        }
        double num = 0.0, den = 0.0;
        for (size_t p = 0; p < n; ++p) {
            double dlt = u[p] - u0[p];
            num += dlt * dlt;
            den += u[p] * u[p];
        }
        rel = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
        cycles = m + 1;
        if (!isfinite(rel)) { status = 4; break; }
        if (tol > 0.0 && rel < tol) { converged = 1; break; }
    }
    if (status == 0 && tol > 0.0 && !converged) status = 3;
    free(u0);
    free(um);
    free(un);
    out[0] = cycles;
    out[1] = rel;
    out[2] = converged;
    return status;
}

/* Error metrics of Sec. 3.2 over all w*h pixels: out[0] = MSE, out[1] = AAE. */
void orc_errors(const double *u, const double *v, long n, double out[2])
{
    double se = 0.0, ae = 0.0;
    for (long p = 0; p < n; ++p) {
        double dd = u[p] - v[p];
        se += dd * dd;
        ae += fabs(dd);
    }
    out[0] = se / (double)n;
    out[1] = ae / (double)n;
}

/* ------------------------------------------------------------------------ */
/* Adjoint (vector-Jacobian product) of the FOEED inpainting solve, for tonal
 * optimisation of the stored grey values. The paper has no adjoint; this is
 * the exact derivative of the discrete solve above (Charbonnier diffusivity),
 * written out step by step in its plainest form: every transpose is applied
 * by scattering the forward stencil's weights, and the tensor derivative is
 * taken from the literal spectral sum d = sum_r mu_r E_r (x) E_r. */

/* d d_ijkl / d g_m for the Charbonnier tensor at gradient g = (gx, gy):
 * dd[m*16 + ((i*2+j)*2+k)*2+l]. */
void orc_foeed_tensor_grad(double gx, double gy, double lambda, int mu3_mode, double dd[32])
{
    double v1[2], v2[2], dv1[2][2], dv2[2][2]; /* dv1[m][i] = d v1_i / d g_m */
    eigvec(gx, gy, &v1[0], &v1[1]);
    v2[0] = -v1[1];
    v2[1] = v1[0];
    double rho2 = gx * gx + gy * gy;
    double rho = sqrt(rho2);
    for (int m = 0; m < 2; ++m)
        for (int i = 0; i < 2; ++i)
            dv1[m][i] = rho > 0.0 ? ((i == m ? 1.0 : 0.0) - v1[i] * v1[m]) / rho : 0.0;
    for (int m = 0; m < 2; ++m) {
        dv2[m][0] = -dv1[m][1];
        dv2[m][1] = dv1[m][0];
    }
    double mu1 = orc_diffusivity(0, rho2, lambda);
    double mu3 = mu3_of(mu3_mode, mu1, 1.0);
    double g[2] = {gx, gy};
    double dmu[4][2];
    for (int m = 0; m < 2; ++m) {
        /* mu1 = (1 + rho^2/lambda^2)^(-1/2): d mu1 / d g_m = -mu1^3 g_m / lambda^2 */
        dmu[0][m] = -mu1 * mu1 * mu1 * g[m] / (lambda * lambda);
        dmu[1][m] = 0.0;
        dmu[2][m] = mu3_mode == 0 ? dmu[0][m] / (2.0 * mu3) : (mu3_mode == 1 ? dmu[0][m] / 2.0 : 0.0);
        dmu[3][m] = 0.0;
    }
    double mu[4] = {mu1, 1.0, mu3, 0.0};
    double r2 = 1.0 / sqrt(2.0);
    double E[4][2][2], dE[2][4][2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            E[0][i][j] = v1[i] * v1[j];
            E[1][i][j] = v2[i] * v2[j];
            E[2][i][j] = r2 * (v1[i] * v2[j] + v2[i] * v1[j]);
            E[3][i][j] = r2 * (v1[i] * v2[j] - v2[i] * v1[j]);
            for (int m = 0; m < 2; ++m) {
                dE[m][0][i][j] = dv1[m][i] * v1[j] + v1[i] * dv1[m][j];
                dE[m][1][i][j] = dv2[m][i] * v2[j] + v2[i] * dv2[m][j];
                dE[m][2][i][j] = r2 * (dv1[m][i] * v2[j] + v1[i] * dv2[m][j] + dv2[m][i] * v1[j] + v2[i] * dv1[m][j]);
                dE[m][3][i][j] = r2 * (dv1[m][i] * v2[j] + v1[i] * dv2[m][j] - dv2[m][i] * v1[j] - v2[i] * dv1[m][j]);
            }
        }
    for (int m = 0; m < 2; ++m)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 2; ++l) {
                        double s = 0.0;
                        for (int r = 0; r < 4; ++r)
                            s += dmu[r][m] * E[r][i][j] * E[r][k][l] +
                                 mu[r] * (dE[m][r][i][j] * E[r][k][l] + E[r][i][j] * dE[m][r][k][l]);
                        dd[m * 16 + ((i * 2 + j) * 2 + k) * 2 + l] = s;
                    }
}

/* Transpose of the separable mirrored Gaussian, applied by scattering. */
static void presmooth_T(const double *ubar_s, int w, int h, double sigma, double *ubar)
{
    double wts[257];
    int R = orc_gauss_weights(sigma, wts, 257);
    size_t n = (size_t)w * h;
    double *tmp = (double *)calloc(n, sizeof(double));
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            for (int t = -R; t <= R; ++t) tmp[(size_t)mirror(y + t, h) * w + x] += wts[t + R] * ubar_s[(size_t)y * w + x];
    memset(ubar, 0, sizeof(double) * n);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            for (int t = -R; t <= R; ++t) ubar[(size_t)y * w + mirror(x + t, w)] += wts[t + R] * tmp[(size_t)y * w + x];
    free(tmp);
}

/* J_F(x)^T v for F(x) = P(x) x (FOEED operator, Charbonnier): the frozen-tensor
 * part P(x)^T v = P(x) v (P is symmetric), plus the tensor's dependence on x
 * through the pre-smoothed gradient: q_m = sum_ijkl (H(v))_ij (H(x))_kl
 * d d_ijkl / d g_m, pulled back through the central-difference gradient and
 * the Gaussian by their transposes. */
void orc_foeed_vjp_F(const double *x, const double *v, int w, int h, double sigma, double lambda, int mu3_mode,
                     double *out)
{
    size_t n = (size_t)w * h;
    double *d = (double *)malloc(sizeof(double) * 16 * n);
    double *us = (double *)malloc(sizeof(double) * n);
    double *gx = (double *)malloc(sizeof(double) * n);
    double *gy = (double *)malloc(sizeof(double) * n);
    double *Hx[3], *Hv[3];
    for (int c = 0; c < 3; ++c) {
        Hx[c] = (double *)malloc(sizeof(double) * n);
        Hv[c] = (double *)malloc(sizeof(double) * n);
    }
    double *r = (double *)calloc(n, sizeof(double));
    double *z = (double *)malloc(sizeof(double) * n);
    orc_presmooth(x, w, h, sigma, us);
    orc_gradient(us, w, h, gx, gy);
    for (size_t p = 0; p < n; ++p) orc_foeed_tensor(gx[p], gy[p], lambda, 0, mu3_mode, d + p * 16, NULL);
    orc_apply_P_field(v, d, w, h, out); /* P(x) v */
    orc_hessian(x, w, h, Hx[0], Hx[1], Hx[2]);
    orc_hessian(v, w, h, Hv[0], Hv[1], Hv[2]);
    for (int y = 0; y < h; ++y)
        for (int xx = 0; xx < w; ++xx) {
            size_t p = (size_t)y * w + xx;
            double dd[32];
            orc_foeed_tensor_grad(gx[p], gy[p], lambda, mu3_mode, dd);
            double W[2][2] = {{Hv[0][p], Hv[1][p]}, {Hv[1][p], Hv[2][p]}};
            double H[2][2] = {{Hx[0][p], Hx[1][p]}, {Hx[1][p], Hx[2][p]}};
            double q[2] = {0.0, 0.0};
            for (int m = 0; m < 2; ++m)
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j)
                        for (int k = 0; k < 2; ++k)
                            for (int l = 0; l < 2; ++l) q[m] += W[i][j] * H[k][l] * dd[m * 16 + ((i * 2 + j) * 2 + k) * 2 + l];
            /* transpose of gx = (us[x+1] - us[x-1])/2, gy likewise, by scattering */
            r[(size_t)y * w + mirror(xx + 1, w)] += 0.5 * q[0];
            r[(size_t)y * w + mirror(xx - 1, w)] -= 0.5 * q[0];
            r[(size_t)mirror(y + 1, h) * w + xx] += 0.5 * q[1];
            r[(size_t)mirror(y - 1, h) * w + xx] -= 0.5 * q[1];
        }
    presmooth_T(r, w, h, sigma, z);
    for (size_t p = 0; p < n; ++p) out[p] += z[p];
    free(d); free(us); free(gx); free(gy);
    for (int c = 0; c < 3; ++c) { free(Hx[c]); free(Hv[c]); }
    free(r); free(z);
}

/* Gradient of a scalar loss L(u_final) with respect to the stored grey values
 * f on the known set, through the whole FOEED FSI solve (init_mode 0: unknown
 * pixels start at the mean of f over K; tol = 0, fixed cycles).
 *   grad_u: dL/du_final;  grad_f: dL/df on K, 0 elsewhere;  u_final optional.
 * Forward states are all kept (small images). Returns 0, or 1 for bad input.
 * Reverse recursion for step u^{k+1} = M u^k + (1-M)(a (u^k - tau F(u^k)) + (1-a) p),
 * p = u^{k-1} (or u^k at the first step of a cycle):
 *   du^k   += M g + a (1-M) g - a tau J_F(u^k)^T ((1-M) g)
 *   dp     += (1-a) (1-M) g */
int orc_inpaint_vjp(const double *f, const uint8_t *mask, const double *grad_u, double *grad_f, double *u_final,
                    int w, int h, double sigma, double lambda, double tau, int cycle_len, int cycles, int mu3_mode)
{
    if (cycle_len < 1 || cycles < 1) return 1;
    size_t n = (size_t)w * h;
    long S = (long)cycle_len * cycles;
    if (tau <= 0.0) tau = 0.05;
    double *X = (double *)malloc(sizeof(double) * n * (size_t)(S + 1)); /* x_0 .. x_S */
    double s = 0.0;
    long cnt = 0;
    for (size_t p = 0; p < n; ++p)
        if (mask[p]) { s += f[p]; ++cnt; }
    double mean = cnt ? s / (double)cnt : 0.0;
    for (size_t p = 0; p < n; ++p) X[p] = mask[p] ? f[p] : mean;
    for (long st = 0; st < S; ++st) {
        int k = (int)(st % cycle_len);
        const double *cur = X + (size_t)st * n;
        const double *prev = k == 0 ? cur : X + (size_t)(st - 1) * n;
        orc_fsi_step(0, prev, cur, mask, w, h, orc_fsi_alpha(k), tau, sigma, lambda, 0, mu3_mode,
                     X + (size_t)(st + 1) * n);
    }
    if (u_final) memcpy(u_final, X + (size_t)S * n, sizeof(double) * n);
    double *g = (double *)malloc(sizeof(double) * n);    /* dL/dx_{s+1}, complete */
    double *pend = (double *)calloc(n, sizeof(double));  /* pending dL/dx_s from step s+1 */
    double *vv = (double *)malloc(sizeof(double) * n);
    double *jt = (double *)malloc(sizeof(double) * n);
    memcpy(g, grad_u, sizeof(double) * n);
    for (long st = S - 1; st >= 0; --st) {
        int k = (int)(st % cycle_len);
        double a = orc_fsi_alpha(k);
        const double *cur = X + (size_t)st * n;
        for (size_t p = 0; p < n; ++p) vv[p] = mask[p] ? 0.0 : g[p];
        orc_foeed_vjp_F(cur, vv, w, h, sigma, lambda, mu3_mode, jt);
        for (size_t p = 0; p < n; ++p) {
            double m = mask[p] ? 1.0 : 0.0;
            double dcur = m * g[p] + a * vv[p] - a * tau * jt[p];
            double dprev = (1.0 - a) * vv[p];
            if (k == 0) {
                g[p] = pend[p] + dcur + dprev;
                pend[p] = 0.0;
            } else {
                g[p] = pend[p] + dcur;
                pend[p] = dprev;
            }
        }
    }
    /* x_0 = M f + (1 - M) mean(f_K) */
    double su = 0.0;
    for (size_t p = 0; p < n; ++p)
        if (!mask[p]) su += g[p];
    for (size_t p = 0; p < n; ++p) grad_f[p] = mask[p] ? g[p] + (cnt ? su / (double)cnt : 0.0) : 0.0;
    free(X); free(g); free(pend); free(vv); free(jt);
    return 0;
}
