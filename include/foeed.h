/*
 * foeed.h - C ABI of the GB300 FOEED / EED inpainting library.
 *
 * Method: Jumakulyyev & Schultz, "Fourth-Order Anisotropic Diffusion for
 * Inpainting and Image Compression" (arXiv 2006.10406).
 *
 * Problem (Sec. 2.1, Eq. inpaintingModel): given grey values f on a set K of
 * known pixels (the mask), evolve
 *     du/dt = -P(u) u   on the unknown pixels,   u = f on K,
 * with reflecting (homogeneous Neumann) image borders, to a steady state.
 *   FOEED: P(u)u = sum_ij d_ij [D(J(u_sigma)) : H(u)]_ij   (Eq. genModel), with
 *          the fourth-order tensor D of Eq. faod_diffTensor / foad_diffTensor_entries.
 *   EED:   P(u)u = -div(D grad u), D = g v1 v1^T + v2 v2^T   (Eq. EEDModel, diffTensor_EED).
 * Time integration: FSI cycles of length n (Sec. 3.3),
 *     u^{m,k+1} = alpha_k (u^{m,k} - tau P(u^{m,k}) u^{m,k}) + (1 - alpha_k) u^{m,k-1},
 *     alpha_k = (4k+2)/(2k+3),  u^{m,-1} = u^{m,0},  u^{m+1,0} = u^{m,n}.
 *
 * Conventions for every entry point:
 *   - Images are w columns (x, fastest) by h rows (y), row-major, with a row
 *     pitch given in ELEMENTS (pitch >= w). The uint8 mask uses the same pitch,
 *     counted in bytes. Nonzero mask = known pixel.
 *   - All data pointers are DEVICE pointers owned by the caller. The library
 *     never allocates device memory: scratch comes from the caller's workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Errors are returned as foeed_status codes; nothing aborts or throws across
 *     the ABI. foeed_last_error() gives a thread-local message for the last
 *     failing call on the calling thread.
 *   - Host threads: calls from different threads are independent (each thread
 *     keeps its own cache of captured FSI-cycle graphs and its own capture
 *     stream); calls that share a workspace must not overlap on the GPU.
 *   - dtype selects the storage and arithmetic type of the images: FOEED_F32
 *     (stencils in float, all reductions in double) or FOEED_F64 (double throughout).
 *     The mixed-precision FOEED_F32_F64U keeps images and stencils in float but
 *     evaluates the FSI extrapolation update u^{k-1} + alpha ((u^k - tau P u^k) -
 *     u^{k-1}) in extended precision and rounds it to float once: in two-float
 *     arithmetic (pairs of floats, error-free sums and FMA products) in the
 *     register-blocked kernel, in double in the generic one.
 */
#ifndef FOEED_H
#define FOEED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FOEED_OK = 0,
    FOEED_ERR_ARG = 1,           /* invalid argument (sizes, pointers, parameters, workspace too small) */
    FOEED_ERR_CUDA = 2,          /* a CUDA runtime call failed; see foeed_last_error() */
    FOEED_ERR_NOT_CONVERGED = 3, /* tol > 0 and max_cycles reached first; result is still written */
    FOEED_ERR_DIVERGED = 4,      /* a cycle produced a non-finite change; result is written as is */
    FOEED_ERR_TIMEOUT = 5        /* reserved for bounded device waits */
} foeed_status;

typedef enum { FOEED_F32 = 0, FOEED_F64 = 1, FOEED_F32_F64U = 2 } foeed_dtype;

/* Diffusivity g(s^2), s = |grad u_sigma| (Eq. CharDiff; Table 6). */
typedef enum {
    FOEED_G_CHARBONNIER = 0,   /* 1/sqrt(1 + s^2/lambda^2) (paper default) */
    FOEED_G_PERONA_MALIK = 1,  /* 1/(1 + s^2/lambda^2) */
    FOEED_G_PERONA_MALIK2 = 2, /* exp(-s^2/lambda^2) */
    FOEED_G_AUBERT = 3,        /* (s/lambda)^2/(s^2+lambda^2)^2, as printed in Table 6 */
    FOEED_G_GEMAN_REYNOLDS = 4 /* 2 lambda^2/(s^2+lambda^2)^2, as printed in Table 6 */
} foeed_diffusivity;

/* Eigenvalue mu_3 of the mixed eigentensor E3 (Sec. 3.1, Table 1). */
typedef enum {
    FOEED_MU3_GEOMETRIC = 0,  /* sqrt(mu1 mu2) = sqrt(g): the paper's choice */
    FOEED_MU3_ARITHMETIC = 1, /* (mu1 + mu2)/2 */
    FOEED_MU3_ONE = 2         /* max(mu1, mu2) = 1 */
} foeed_mu3_mode;

typedef struct {
    double lambda;    /* contrast parameter of g (> 0) */
    double sigma;     /* Gaussian pre-smoothing scale (>= 0; radius ceil(3 sigma) <= 6) */
    double tau;       /* explicit step size; <= 0 selects 0.05 (FOEED) or 0.25 (EED), Sec. 3.1 */
    int cycle_len;    /* FSI cycle length n >= 1 */
    int max_cycles;   /* number of cycles (tol == 0) or cycle cap (tol > 0), >= 1 */
    double tol;       /* > 0: stop after the first cycle with |u^{m,n}-u^{m,0}|_2/|u^{m,n}|_2 < tol */
    int diffusivity;  /* foeed_diffusivity */
    int mu3_mode;     /* foeed_mu3_mode (FOEED only) */
    int init_mode;    /* 0: unknown pixels start at the mean of f over K; 1: at u_inout */
    int check_every;  /* tol > 0: cycles between host polls of the device stop flag (<= 0: 8) */
} foeed_params;

typedef struct {
    int cycles_run;         /* cycles executed (the stop test is exact per cycle) */
    double last_rel_change; /* |u^{m,n}-u^{m,0}|_2 / |u^{m,n}|_2 of the last cycle run */
    int converged;          /* 1 if tol > 0 and the stop test passed */
    float ms;               /* device time of the solve (CUDA events), milliseconds */
} foeed_report;

/* Bytes of device workspace foeed_inpaint / eed_inpaint need for a w x h image;
 * 0 for an invalid size or dtype. */
size_t foeed_workspace_bytes(int w, int h, foeed_dtype dtype);

/*
 * Full inpainting solve by FOEED (Eq. genModel) with FSI cycles (Sec. 3.3).
 *   f        [h x pitch] known grey values, read only where mask != 0
 *   mask     [h x pitch] uint8, nonzero = known pixel (Dirichlet data, Eq. inpaintingModel)
 *   u_inout  [h x pitch] result; read on entry only if init_mode == 1
 *   workspace: device buffer of at least foeed_workspace_bytes(w, h, dtype)
 *              bytes, 256-byte aligned; contents on entry are ignored.
 *   report   may be NULL.
 * Stream-ordered on `stream`; returns after the result is written (the call
 * synchronises `stream` once at the end, and every check_every cycles when tol > 0).
 * On return the known pixels of u_inout equal f bitwise.
 * u_inout may alias f.
 */
foeed_status foeed_inpaint(const void *f, const uint8_t *mask, void *u_inout, int w, int h,
                           long pitch, foeed_dtype dtype, const foeed_params *params,
                           void *workspace, size_t workspace_bytes, void *stream,
                           foeed_report *report);

/* Same as foeed_inpaint with second-order EED (Eq. EEDModel, Eq. diffTensor_EED).
 * mu3_mode is ignored; tau <= 0 selects 0.25. */
foeed_status eed_inpaint(const void *f, const uint8_t *mask, void *u_inout, int w, int h,
                         long pitch, foeed_dtype dtype, const foeed_params *params,
                         void *workspace, size_t workspace_bytes, void *stream,
                         foeed_report *report);

/*
 * One masked FSI step of FOEED (Sec. 3.3, FSI equation):
 *   unknown: u_next = alpha (u_cur - tau P(u_cur) u_cur) + (1 - alpha) u_prev
 *   known:   u_next = u_cur (bitwise)
 * Uses params->lambda, sigma, tau (<= 0: 0.05), diffusivity, mu3_mode.
 * u_next may alias u_prev but not u_cur. mask may be NULL (no known pixels:
 * the smoothing variant). Asynchronous on `stream`; no workspace.
 */
foeed_status foeed_step(const void *u_prev, const void *u_cur, void *u_next, const uint8_t *mask,
                        int w, int h, long pitch, foeed_dtype dtype, double alpha,
                        const foeed_params *params, void *stream);

/* One masked FSI step of EED; same contract as foeed_step (tau <= 0: 0.25). */
foeed_status eed_step(const void *u_prev, const void *u_cur, void *u_next, const uint8_t *mask,
                      int w, int h, long pitch, foeed_dtype dtype, double alpha,
                      const foeed_params *params, void *stream);

/* One image of a batched solve: device pointers and sizes as for foeed_inpaint,
 * with its own contrast parameter lambda. */
typedef struct {
    const void *f;         /* [h x pitch] known grey values */
    const uint8_t *mask;   /* [h x pitch] nonzero = known pixel */
    void *u_inout;         /* [h x pitch] result (read on entry if init_mode == 1) */
    int w, h;
    long pitch;            /* elements (bytes for the mask) */
    double lambda;         /* contrast parameter of this image (> 0) */
} foeed_instance;

/* Workspace bytes foeed_inpaint_batch needs for these images. */
size_t foeed_batch_workspace_bytes(const foeed_instance *inst, int count, foeed_dtype dtype);

/*
 * Many FOEED inpainting problems of uneven sizes solved together: every FSI
 * step is one kernel launch over the tiles of all images (a work list of
 * (image, tile) pairs), one FSI cycle is one captured CUDA graph, each image
 * keeps its own lambda, mask, buffers, cycle residual and stop flag. Each
 * image's result equals foeed_inpaint on that image alone (the same tile
 * arithmetic). Supports FOEED_F32 / FOEED_F32_F64U with the Charbonnier
 * diffusivity and mu3 = sqrt(mu1) (the paper's configuration), cycle_len >= 2;
 * params->lambda is ignored (each image has its own). inst is a host array;
 * reports (count entries) may be NULL. Returns the first non-OK status of any
 * image (FOEED_ERR_NOT_CONVERGED / FOEED_ERR_DIVERGED), else FOEED_OK.
 */
foeed_status foeed_inpaint_batch(const foeed_instance *inst, int count, foeed_dtype dtype,
                                 const foeed_params *params, void *workspace, size_t workspace_bytes,
                                 void *stream, foeed_report *reports);

/* The batched solve with second-order EED (Eq. EEDModel); same contract and
 * workspace as foeed_inpaint_batch, tau <= 0 selects 0.25, mu3_mode ignored.
 * The channel-wise colour reconstructions of Sec. 5 are batches of this form:
 * one instance per channel, all sharing the mask. */
foeed_status eed_inpaint_batch(const foeed_instance *inst, int count, foeed_dtype dtype,
                               const foeed_params *params, void *workspace, size_t workspace_bytes,
                               void *stream, foeed_report *reports);

/* Workspace bytes foeed_inpaint_vjp needs (checkpoint every `checkpoint_every` steps). */
size_t foeed_vjp_workspace_bytes(int w, int h, foeed_dtype dtype, const foeed_params *params,
                                 int checkpoint_every);

/*
 * Gradient of a scalar loss of the FOEED reconstruction with respect to the
 * stored grey values (tonal optimisation). The paper has no adjoint; this is
 * the exact derivative of the discrete solve of foeed_inpaint: the forward
 * FSI solve is re-run with a checkpoint of (u^k, u^{k-1}) every
 * checkpoint_every steps, then each segment is recomputed from its checkpoint
 * (checkpoint_every = 1: the forward steps write every state u^0 .. u^S into the
 * workspace, (S + 1) images, and nothing is recomputed or copied)
 * and traversed backwards with the adjoint step kernels.
 *   grad_u  [h x pitch] dL/du_final (device)
 *   grad_f  [h x pitch] out: dL/df on the known pixels, 0 elsewhere; includes
 *           the path through the mean initialisation of the unknown pixels
 *   u_out   [h x pitch] out (may be NULL): the reconstruction u_final
 * Requirements: FOEED_F32 or FOEED_F64, Charbonnier diffusivity, mu3 =
 * sqrt(mu1), init_mode 0, tol 0 (a fixed number of cycles). Synchronises
 * `stream` at the end.
 */
foeed_status foeed_inpaint_vjp(const void *f, const uint8_t *mask, const void *grad_u, void *grad_f, void *u_out,
                               int w, int h, long pitch, foeed_dtype dtype, const foeed_params *params,
                               int checkpoint_every, void *workspace, size_t workspace_bytes, void *stream);

/*
 * The paper's unifying fourth-order operator (Eq. gen4thPDE_Model) with
 * caller-supplied coefficients: Pu = sum_ij d_ij [ sum_kl d_ijkl u_kl ], so that
 * du/dt = -Pu. FOEED (Eq. genModel), You-Kaveh, Hajiaboli and Li et al.
 * (Sec. 3.2) are particular fields d.
 *   u   [h x pitch] image;  Pu [h x pitch] output (must not alias u)
 *   d   [h x pitch x 16] coefficients, d[(y*pitch + x)*16 + ((i*2+j)*2+k)*2+l],
 *       index 0 = x, 1 = y; need not be symmetric.
 * Stencils of Sec. 3.3; u mirrored at the border, T_xx and T_yy mirrored,
 * T_xy and T_yx odd across each border. FOEED_F32 or FOEED_F64.
 * Asynchronous on `stream`.
 */
foeed_status foeed_apply_tensor_field(const void *u, const void *d, void *Pu, int w, int h, long pitch,
                                      foeed_dtype dtype, void *stream);

/* Bytes of workspace foeed_errors needs for a w x h image. */
size_t foeed_errors_workspace_bytes(int w, int h);

/*
 * Error metrics of Sec. 3.2 over all w*h pixels, reduced in double:
 *   out[0] = MSE, out[1] = AAE, out[2] = PSNR in dB for a peak of 1
 *   (10 log10(1/MSE); +inf when MSE == 0; not in the paper).
 * u and v are device images of the given dtype (FOEED_F32_F64U reads float).
 * Synchronises `stream`; out is a host pointer to 3 doubles.
 */
foeed_status foeed_errors(const void *u, const void *v, int w, int h, long pitch, foeed_dtype dtype,
                          void *workspace, size_t workspace_bytes, void *stream, double *out);

/*
 * FOEED solve for callers that cannot allocate device memory (no cudaMalloc,
 * no workspace of their own): code living inside another framework's memory
 * arena, plug-ins that must not touch the device heap, or latency-critical
 * paths where an allocation may block or fail. The paper has no counterpart;
 * this is a deployment variant of foeed_inpaint.
 *   Same arguments and result as foeed_inpaint, without the workspace: the
 *   scratch lives in one static device array of FOEED_STATIC_SCRATCH_BYTES
 *   (64 MiB) that every device loading the library keeps until the process
 *   exits. Images whose foeed_workspace_bytes(w, h, dtype) exceed it are
 *   rejected with FOEED_ERR_ARG (square images up to 2269 x 2269 in FP32,
 *   1632 x 1632 in FP64).
 *   The call allocates nothing: no cudaMalloc / cudaFree, no graph, no event;
 *   it launches the step kernels one by one on `stream`.
 *   The array is part of the library's device module: the module is loaded,
 *   and the 64 MiB taken from the device, by the first call into this library
 *   on that device (any entry point; under CUDA's lazy module loading that can
 *   be this one), so make a first call at set-up, outside any memory budget
 *   that must not change. The first call of this entry point on a device also
 *   looks up the array's device address (cudaGetSymbolAddress) with that device
 *   current; make that first call before any stream capture. Later calls take
 *   no device memory. All calls on a device share the one array and
 *   it keeps the previous call's contents (the solve re-initialises what it
 *   reads), so calls that overlap on the GPU (other streams, other threads)
 *   race: serialise them. report->ms is host wall time of the call.
 */
#define FOEED_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
size_t foeed_static_scratch_bytes(void);
foeed_status foeed_inpaint_static(const void *f, const uint8_t *mask, void *u_inout, int w, int h,
                                  long pitch, foeed_dtype dtype, const foeed_params *params, void *stream,
                                  foeed_report *report);

/*
 * Tile shapes of the register-blocked FP32 step kernels (FOEED_F32 and
 * FOEED_F32_F64U with the Charbonnier diffusivity and, for FOEED, mu3 =
 * sqrt(mu1); not in the paper, whose implementation is sequential). Each CTA
 * computes a 64 x 32 or a 64 x 16 block of output pixels, or, for a single
 * FOEED image, a 64 x 64 block (512 threads) or a 64 x 8 block (128 threads).
 * The shapes give bitwise the same results: only the time differs.
 *   FOEED_TILES_AUTO (default): the solvers time the candidates and keep the
 *     fastest, once per (device, image size, method, Gaussian radius, precision)
 *     for a single image, and once per (device, list of image sizes, method,
 *     radius, precision) for a batch, where the candidate plans are 64 x 32 tiles
 *     for every image, 64 x 16 for every image, and 64 x 16 for the images below
 *     a tile count (a few thresholds from the batch's own sizes). The timing runs
 *     inside the first solve of its kind (a few step launches into workspace
 *     buffers that the solve overwrites) and is cached for the process; single
 *     FOEED images also try 64 x 64 and 64 x 8 tiles.
 *   FOEED_TILES_H64 / FOEED_TILES_H32 / FOEED_TILES_H16 / FOEED_TILES_H8: that
 *     tile height for every image (64 and 8 only for single-image FOEED;
 *     elsewhere 64 means 32 and 8 means 16).
 * The policy applies to the calling host thread's later calls: foeed_inpaint,
 * eed_inpaint and the batched solvers tune as above; foeed_step, eed_step,
 * foeed_inpaint_static and the forward steps of foeed_inpaint_vjp, which do
 * not time anything, use a fixed policy when one is set and otherwise 64 x 16
 * tiles for images of fewer than 304 tiles of 64 x 32 (two per SM of a GB300)
 * and 64 x 32 tiles above. FOEED_ERR_ARG for an unknown policy.
 */
typedef enum {
    FOEED_TILES_AUTO = 0,
    FOEED_TILES_H8 = 8,  /* 64 x 8 tiles of 128 threads: single-image FOEED only (else 64 x 16) */
    FOEED_TILES_H16 = 16,
    FOEED_TILES_H32 = 32,
    FOEED_TILES_H64 = 64 /* 64 x 64 tiles of 512 threads: single-image FOEED only (else 64 x 32) */
} foeed_tile_policy;
foeed_status foeed_set_tile_policy(int policy);

/* The tile plan of the last foeed_inpaint / eed_inpaint / batched solve on the
 * calling thread. Times are microseconds per FSI step measured by the autotuner
 * (0 when it did not run for that solve, e.g. a cached or fixed choice). */
typedef struct {
    int tile_h;      /* single image: 64, 32, 16 or 8 (0: the generic kernel ran); batch: 0 */
    int images;      /* images in the solve */
    int images_h16;  /* images solved on 64 x 16 tiles */
    int tuned;       /* 1 if the autotuner timed the candidates for this solve */
    float us_h32;    /* time of the plan with 64 x 32 tiles for every image */
    float us_h16;    /* time of the plan with 64 x 16 tiles for every image */
    float us_chosen; /* time of the plan chosen */
    float us_h64;    /* single FOEED image: time with 64 x 64 tiles (0 otherwise) */
    float us_h8;     /* single FOEED image: time with 64 x 8 tiles (0 otherwise) */
} foeed_tile_plan;
foeed_status foeed_last_tile_plan(foeed_tile_plan *out);

/* Message describing the last failure on the calling thread ("" if none). */
const char *foeed_last_error(void);

/* Library version string. */
const char *foeed_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FOEED_H */
