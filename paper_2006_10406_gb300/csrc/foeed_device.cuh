// Device-side building blocks of the FOEED / EED step kernels (sm_103a).
//
// One fused kernel per explicit FSI step. Each CTA owns a TW x TH output tile
// and stages everything in shared memory:
//   A  u^k tile with a halo of R+2 pixels (mirrored at the image border)
//   B  Gaussian x pass on rows tile+-(R+2), columns tile+-2
//   C  Gaussian y pass on tile+-2                          -> u_sigma
//   D  per pixel of tile+-1: grad u_sigma, mu1/mu3, Hessian, T = D:H (FOEED)
//      or the EED fluxes
//   E  per output pixel: outer divergence, masked FSI update, optional cycle
//      residual (double), stores u^{k+1}
// Computing the tensor at ghost positions from the mirror-extended u yields
// exactly the parity ghosts of the outer operator (T_xx, T_yy even, T_xy odd
// per reflected axis), so the border needs no special case after stage A.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace foeed {

constexpr int kRMax = 6;  // Gaussian radius ceil(3 sigma) <= 6, i.e. sigma <= 2
constexpr int kThreads = 256;

// Device control block at the start of the workspace.
struct Ctl {
    unsigned int ticket;  // arrival counter of the last-block reduction
    int done;             // stop flag: converged (tol > 0) or diverged
    int cycles;           // completed FSI cycles
    int diverged;
    double tol;
    double last_num;      // sum (u^{m,n} - u^{m,0})^2 of the last cycle
    double last_den;      // sum (u^{m,n})^2
    double last_rel;
    double mean;          // mean of f over the known pixels
    long long known;      // number of known pixels
    double err[3];        // foeed_errors results
};

template <typename T>
struct StepArgs {
    const T *uprev;
    const T *ucur;
    T *unext;
    const uint8_t *mask;  // may be null
    const T *c0;          // cycle start u^{m,0} (residual mode), may alias unext
    int w, h;
    long pitch;   // elements, shared by images and (in bytes) the mask
    double alpha; // FSI extrapolation weight
    double tau;
    double lambda;
    // the same constants pre-rounded to T on the host (no per-thread FP64 work)
    T alpha_t, tau_t;
    T alpha_lo, tau_lo;  // alpha - alpha_t, tau - tau_t: alpha and tau as two-word values (hi + lo)
    T l2, inv_l2;  // lambda^2, 1/lambda^2
    T c4;          // 1/(4 lambda^2): lambda1/lambda^2 = |2 grad u_sigma|^2 * c4
    int g_kind, mu3_mode;
    T wts[2 * kRMax + 1];
    Ctl *ctl;            // null outside an inpaint solve
    double *partials;    // per-block residual partials
    int residual;        // 1: accumulate the cycle residual and finalise it
    int check_done;      // 1: return at once when ctl->done is set
    int pdl;             // host only: launch with programmatic dependency on the previous kernel
    int tile_h;          // host only: register-blocked FP32 kernel's tile height (16, 32; 0: size rule)
};

// Launches kern over grid with the arguments a, as an ordinary launch or, when
// a.pdl is set, with programmatic stream serialisation (the kernel waits for
// its predecessor with griddepcontrol.wait).
template <typename Kern, typename Args>
cudaError_t launch_step_kernel(Kern kern, dim3 grid, int threads, size_t smem, cudaStream_t s, const Args &a)
{
    if (!a.pdl) {
        kern<<<grid, threads, smem, s>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// One image of a batched solve (entry of a device table).
struct BatchInst {
    float *C, *A, *B;     // the image's cycle buffers (internal pitch)
    const uint8_t *mask;  // internal 0/1 mask
    int w, h;
    long pitch;
    float c4;             // 1/(4 lambda^2) of this image
    int th;               // its tile height (32 or 16)
    int ntx, nty;         // its 64 x th tile grid
    Ctl *ctl;             // its control block (cycle residual, stop flag)
    double *partials;     // its per-tile residual partials
};

// Buffer roles of one step of a cycle of length n >= 2 (the rotation of the
// single-image solver): step 0 (C,C)->A, step 1 (C,A)->B, even k >= 2
// (A,B)->A, odd k >= 3 (B,A)->B; the last step writes C instead.
enum BatchRole { kRoleFirst = 0, kRoleSecond = 1, kRoleEven = 2, kRoleOdd = 3 };

struct BatchArgs {
    const BatchInst *inst;
    const int2 *tiles;  // per CTA: (image, tile index within the image)
    int role;
    int last;           // last step of the cycle (writes C, accumulates the residual)
};

__device__ __forceinline__ int mirror_idx(int i, int n)
{
    if ((unsigned)i < (unsigned)n) return i;
    int p = 2 * n;
    i %= p;
    if (i < 0) i += p;
    return i < n ? i : p - 1 - i;
}

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }
__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }

// g(lambda1) for lambda1 = |grad u_sigma|^2 (Eq. CharDiff, Table 6); r = lambda1/lambda^2.
template <typename T>
__device__ __forceinline__ T diffusivity(int kind, T l1, T inv_l2, T l2)
{
    T r = l1 * inv_l2;
    switch (kind) {
    case 1: return T(1) / (T(1) + r);
    case 2: return exp_t(-r);
    case 3: return r / ((l1 + l2) * (l1 + l2));
    case 4: return T(2) * l2 / ((l1 + l2) * (l1 + l2));
    default: return rsqrt_t(T(1) + r);
    }
}

template <typename T>
__device__ __forceinline__ T mu3_of(int mode, T mu1)
{
    switch (mode) {
    case 1: return (mu1 + T(1)) * T(0.5);
    case 2: return T(1);
    default: return sqrt_t(mu1);
    }
}

// Warp + block reduction of two doubles; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double &a, double &b, double *sh /* >= 2*32 */)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[2 * wid] = a; sh[2 * wid + 1] = b; }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = lane < nw ? sh[2 * lane] : 0.0;
        b = lane < nw ? sh[2 * lane + 1] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// Deterministic grid reduction: each block stores its partial pair; the last
// block to arrive sums all partials in block order. Returns true in thread 0
// of the last block, with the totals in a, b.
__device__ __forceinline__ bool grid_sum2_last(double &a, double &b, double *partials, unsigned int *ticket,
                                               int nblocks, int bid, double *sh)
{
    __shared__ bool s_last;
    block_sum2(a, b, sh);
    if (threadIdx.x == 0) {
        partials[2 * bid] = a;
        partials[2 * bid + 1] = b;
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        s_last = (t == (unsigned)nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    // the last block: fixed-order sum, strided per thread then a fixed tree
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        sa += ((volatile double *)partials)[2 * i];
        sb += ((volatile double *)partials)[2 * i + 1];
    }
    __syncthreads();
    block_sum2(sa, sb, sh);
    a = sa;
    b = sb;
    if (threadIdx.x == 0) *ticket = 0u;
    return threadIdx.x == 0;
}

}  // namespace foeed
