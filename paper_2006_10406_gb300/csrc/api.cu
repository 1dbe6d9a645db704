// C ABI of the FOEED / EED inpainting library (declared in include/foeed.h).
//
// Host side of the solver: argument checks, workspace layout, the
// initialisation / copy / metric kernels, and the FSI cycle driver. One FSI
// cycle (n fused step kernels, the last one with the cycle residual) is
// captured once into a CUDA graph and replayed; a device stop flag makes
// every later kernel return at once after convergence, so the host only polls
// every few cycles.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <climits>
#include <map>
#include <mutex>
#include <vector>

#include "adjoint.cuh"
#include "dispatch.h"
#include "foeed.h"

using namespace foeed;

namespace {

thread_local char g_err[512] = "";

foeed_status fail(foeed_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(FOEED_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t elem_size(foeed_dtype d) { return d == FOEED_F64 ? 8 : 4; }

// Internal row pitch (elements): rows start on 128-byte boundaries.
long internal_pitch(int w, foeed_dtype d) { return (long)align_up((size_t)w, d == FOEED_F64 ? 16 : 32); }

int tile_w(foeed_dtype d) { return d == FOEED_F64 ? kTileW64 : kTileW32; }
int tile_h(foeed_dtype d) { return d == FOEED_F64 ? kTileH64 : kTileH32; }

constexpr int kRedThreads = 256;
constexpr int kRedBlocksMax = 1024;

// Reduction partials one step or reduction can write: one per CTA of the
// largest grid (FP32: the fast kernels' 64 x 8 tiles, the smallest they use).
constexpr int kFastMinTileH = 8;
long long max_blocks(int w, int h, foeed_dtype d)
{
    const int th = d == FOEED_F64 ? tile_h(d) : kFastMinTileH;
    long long step = (long long)((w + tile_w(d) - 1) / tile_w(d)) * ((h + th - 1) / th);
    return step > kRedBlocksMax ? step : kRedBlocksMax;
}

struct Layout {
    size_t ctl, partials, bufC, bufA, bufB, mask, total;
    long P;
};

Layout layout(int w, int h, foeed_dtype d)
{
    Layout L;
    L.P = internal_pitch(w, d);
    size_t img = align_up((size_t)h * L.P * elem_size(d), kAlign);
    size_t off = 0;
    L.ctl = off; off += align_up(sizeof(Ctl), kAlign);
    L.partials = off; off += align_up(sizeof(double) * 2 * (size_t)max_blocks(w, h, d), kAlign);
    L.bufC = off; off += img;
    L.bufA = off; off += img;
    L.bufB = off; off += img;
    L.mask = off; off += align_up((size_t)h * L.P, kAlign);
    L.total = off;
    return L;
}

// ---------------------------------------------------------------------------
// Set-up, copy and metric kernels (grid-stride over pixels).

// Internal mask copy (0/1) and the sums of f over the known set.
template <typename T>
__global__ void prep_kernel(const T *__restrict__ f, const uint8_t *__restrict__ mask, uint8_t *__restrict__ mi,
                            int w, int h, long pitch, long P, Ctl *ctl, double *partials)
{
    __shared__ double red[64];
    double s = 0.0, cnt = 0.0;
    const long n = (long)w * h;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        long y = i / w, x = i - y * w;
        uint8_t k = mask[y * pitch + x] != 0;
        mi[y * P + x] = k;
        if (k) { s += double(f[y * pitch + x]); cnt += 1.0; }
    }
    if (grid_sum2_last(s, cnt, partials, &ctl->ticket, gridDim.x, blockIdx.x, red)) {
        ctl->known = (long long)cnt;
        ctl->mean = cnt > 0.0 ? s / cnt : 0.0;
    }
}

// u^{0,0}: known pixels take f, unknown pixels the mean (mode 0) or u_inout (mode 1).
template <typename T>
__global__ void init_kernel(const T *__restrict__ f, const uint8_t *__restrict__ mi, const T *__restrict__ uin,
                            T *__restrict__ C, int w, int h, long pitch, long P, int init_mode, const Ctl *ctl)
{
    const long n = (long)w * h;
    const T mean = T(ctl->mean);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        long y = i / w, x = i - y * w;
        T v;
        if (mi[y * P + x]) v = f[y * pitch + x];
        else v = init_mode == 0 ? mean : uin[y * pitch + x];
        C[y * P + x] = v;
    }
}

template <typename T>
__global__ void copy_out_kernel(const T *__restrict__ src, T *__restrict__ dst, int w, int h, long P, long pitch)
{
    const long n = (long)w * h;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        long y = i / w, x = i - y * w;
        dst[y * pitch + x] = src[y * P + x];
    }
}

template <typename T>
__global__ void errors_kernel(const T *__restrict__ u, const T *__restrict__ v, int w, int h, long pitch,
                              Ctl *ctl, double *partials)
{
    __shared__ double red[64];
    double se = 0.0, ae = 0.0;
    const long n = (long)w * h;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        long y = i / w, x = i - y * w;
        double d = double(u[y * pitch + x]) - double(v[y * pitch + x]);
        se += d * d;
        ae += fabs(d);
    }
    if (grid_sum2_last(se, ae, partials, &ctl->ticket, gridDim.x, blockIdx.x, red)) {
        double mse = se / double(n), aae = ae / double(n);
        ctl->err[0] = mse;
        ctl->err[1] = aae;
        ctl->err[2] = mse > 0.0 ? 10.0 * log10(1.0 / mse) : INFINITY;
    }
}

int grid_for(long n)
{
    long b = (n + kRedThreads - 1) / kRedThreads;
    if (b < 1) b = 1;
    return (int)(b > kRedBlocksMax ? kRedBlocksMax : b);
}

// ---------------------------------------------------------------------------
// Parameter checks and the step launch shared by every entry point.

int gauss_radius(double sigma) { return sigma > 0.0 ? (int)std::ceil(3.0 * sigma) : 0; }

// Sampled, truncated, normalised Gaussian taps (pre-smoothing of Sec. 2.2).
template <typename T>
void gauss_taps(double sigma, T *out)
{
    int R = gauss_radius(sigma);
    double wv[2 * kRMax + 1], sum = 0.0;
    for (int t = -R; t <= R; ++t) {
        double v = sigma > 0.0 ? std::exp(-double(t) * t / (2.0 * sigma * sigma)) : 1.0;
        wv[t + R] = v;
        sum += v;
    }
    for (int t = 0; t <= 2 * R; ++t) out[t] = T(wv[t] / sum);
    for (int t = 2 * R + 1; t < 2 * kRMax + 1; ++t) out[t] = T(0);
}

foeed_status check_params(const foeed_params *p, bool need_cycles)
{
    if (!p) return fail(FOEED_ERR_ARG, "params is NULL");
    if (!(p->lambda > 0.0) || !std::isfinite(p->lambda)) return fail(FOEED_ERR_ARG, "lambda must be > 0");
    if (!(p->sigma >= 0.0) || gauss_radius(p->sigma) > kRMax)
        return fail(FOEED_ERR_ARG, "sigma must be in [0, 2] (Gaussian radius ceil(3 sigma) <= %d)", kRMax);
    if (!std::isfinite(p->tau)) return fail(FOEED_ERR_ARG, "tau must be finite");
    if (p->diffusivity < 0 || p->diffusivity > 4) return fail(FOEED_ERR_ARG, "unknown diffusivity %d", p->diffusivity);
    if (p->mu3_mode < 0 || p->mu3_mode > 2) return fail(FOEED_ERR_ARG, "unknown mu3_mode %d", p->mu3_mode);
    if (need_cycles) {
        if (p->cycle_len < 1) return fail(FOEED_ERR_ARG, "cycle_len must be >= 1");
        if (p->max_cycles < 1) return fail(FOEED_ERR_ARG, "max_cycles must be >= 1");
        if (!(p->tol >= 0.0)) return fail(FOEED_ERR_ARG, "tol must be >= 0");
        if (p->init_mode != 0 && p->init_mode != 1) return fail(FOEED_ERR_ARG, "init_mode must be 0 or 1");
    }
    return FOEED_OK;
}

foeed_status check_image(int w, int h, long pitch, foeed_dtype d)
{
    if (w < 1 || h < 1) return fail(FOEED_ERR_ARG, "image size %d x %d must be >= 1 x 1", w, h);
    if ((long long)w * h > (1LL << 31) - 1) return fail(FOEED_ERR_ARG, "image too large");
    if (pitch < w) return fail(FOEED_ERR_ARG, "pitch %ld < width %d", pitch, w);
    if (d != FOEED_F32 && d != FOEED_F64 && d != FOEED_F32_F64U) return fail(FOEED_ERR_ARG, "unknown dtype %d", (int)d);
    return FOEED_OK;
}

double default_tau(bool eed, double tau) { return tau > 0.0 ? tau : (eed ? 0.25 : 0.05); }

// Two timing events, destroyed on every return path.
struct EventPair {
    cudaEvent_t e[2] = {nullptr, nullptr};
    cudaError_t create()
    {
        cudaError_t err = cudaEventCreate(&e[0]);
        return err == cudaSuccess ? cudaEventCreate(&e[1]) : err;
    }
    ~EventPair()
    {
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
};

// Independent per-image launches of a batch (set-up, copy-out) spread over a
// few side streams forked from the caller's stream and joined back to it. The
// streams are created once per device and kept for the process.
constexpr int kSideStreams = 4;
cudaError_t side_streams(cudaStream_t *out)
{
    static std::mutex mu;
    static std::map<int, std::vector<cudaStream_t>> pool;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    std::vector<cudaStream_t> &v = pool[dev];
    while ((int)v.size() < kSideStreams) {
        cudaStream_t st = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return e;
        v.push_back(st);
    }
    for (int k = 0; k < kSideStreams; ++k) out[k] = v[k];
    return cudaSuccess;
}

struct Fork {
    cudaStream_t st[kSideStreams] = {};
    cudaEvent_t ev[kSideStreams + 1] = {};
    // the side streams wait for everything queued on s so far
    cudaError_t open(cudaStream_t s)
    {
        cudaError_t e = side_streams(st);
        for (int k = 0; k <= kSideStreams && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev[kSideStreams], s);
        for (int k = 0; k < kSideStreams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(st[k], ev[kSideStreams], 0);
        return e;
    }
    cudaStream_t operator[](int i) const { return st[i % kSideStreams]; }
    // s waits for everything queued on the side streams
    cudaError_t join(cudaStream_t s)
    {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < kSideStreams && e == cudaSuccess; ++k) e = cudaEventRecord(ev[k], st[k]);
        for (int k = 0; k < kSideStreams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(s, ev[k], 0);
        return e;
    }
    ~Fork()
    {
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
    }
};

struct StepCall {
    const void *uprev, *ucur, *c0;
    void *unext;
    const uint8_t *mask;
    int w, h;
    long pitch;
    double alpha, tau;
    Ctl *ctl;
    double *partials;
    int residual, check_done;
    int pdl;     // launch with a programmatic dependency on the previous kernel
    int tile_h;  // register-blocked FP32 kernel: tile height 16 or 32 (0: size rule)
};

template <typename T>
StepArgs<T> make_args(const StepCall &c, const foeed_params &p)
{
    StepArgs<T> a;
    a.uprev = static_cast<const T *>(c.uprev);
    a.ucur = static_cast<const T *>(c.ucur);
    a.unext = static_cast<T *>(c.unext);
    a.mask = c.mask;
    a.c0 = static_cast<const T *>(c.c0);
    a.w = c.w;
    a.h = c.h;
    a.pitch = c.pitch;
    a.alpha = c.alpha;
    a.tau = c.tau;
    a.lambda = p.lambda;
    a.alpha_t = T(c.alpha);
    a.tau_t = T(c.tau);
    a.alpha_lo = T(c.alpha - double(a.alpha_t));
    a.tau_lo = T(c.tau - double(a.tau_t));
    a.l2 = T(p.lambda * p.lambda);
    a.inv_l2 = T(1.0 / (p.lambda * p.lambda));
    a.c4 = T(0.25 / (p.lambda * p.lambda));
    a.g_kind = p.diffusivity;
    a.mu3_mode = p.mu3_mode;
    gauss_taps<T>(p.sigma, a.wts);
    a.ctl = c.ctl;
    a.partials = c.partials;
    a.residual = c.residual;
    a.check_done = c.check_done;
    a.pdl = c.pdl;
    a.tile_h = c.tile_h;
    return a;
}

// The register-blocked FP32 kernel covers the paper's configuration
// (Charbonnier g; mu3 = sqrt(mu1) for FOEED); other variants use the generic one.
bool fast_params(bool eed, const foeed_params &p) { return p.diffusivity == 0 && (eed || p.mu3_mode == 0); }

bool aligned16(const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

bool fast_eligible(bool eed, const StepCall &c, const foeed_params &p)
{
    if (!fast_params(eed, p) || c.pitch % 4 != 0) return false;
    if (!aligned16(c.uprev) || !aligned16(c.ucur) || !aligned16(c.unext)) return false;
    if (c.mask && !aligned16(c.mask)) return false;
    if (c.residual && !aligned16(c.c0)) return false;
    return true;
}

// c == nullptr: only prepare the kernel (shared-memory attribute), no launch.
cudaError_t launch_step(bool eed, foeed_dtype d, const StepCall *c, const foeed_params &p, cudaStream_t s)
{
    int R = gauss_radius(p.sigma);
    if (d == FOEED_F64) {
        StepArgs<double> a;
        if (c) a = make_args<double>(*c, p);
        return eed ? step_eed_f64(c ? &a : nullptr, R, s) : step_foeed_f64(c ? &a : nullptr, R, s);
    }
    StepArgs<float> a;
    if (c) a = make_args<float>(*c, p);
    bool f64u = d == FOEED_F32_F64U;
    if (c ? fast_eligible(eed, *c, p) : fast_params(eed, p)) {
        cudaError_t e = eed ? step_fast_eed_f32(c ? &a : nullptr, R, f64u, s)
                            : step_fast_foeed_f32(c ? &a : nullptr, R, f64u, s);
        if (c || e != cudaSuccess) return e;  // when preparing, also prepare the generic kernel
    }
    return eed ? step_eed_f32(c ? &a : nullptr, R, f64u, s) : step_foeed_f32(c ? &a : nullptr, R, f64u, s);
}

// ---------------------------------------------------------------------------
// Tile-shape autotuner of the register-blocked FP32 kernels (64 x 32 or 64 x 16
// output tiles; both give the same bits, only the time differs).

// Per host thread: the stream FSI cycles (and the autotuner's timing graphs) are captured on.
thread_local cudaStream_t g_capture_stream[64] = {};

cudaError_t capture_stream(int dev, cudaStream_t *out)
{
    cudaStream_t &cs = g_capture_stream[dev & 63];
    if (!cs) {
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    *out = cs;
    return cudaSuccess;
}

thread_local int g_tile_policy = FOEED_TILES_AUTO;
thread_local foeed_tile_plan g_last_plan = {};

// The tile height a fixed policy gives one image: 64 x 64 and 64 x 8 tiles exist
// for FOEED only, so EED takes 64 x 32 under FOEED_TILES_H64 and 64 x 16 under
// FOEED_TILES_H8.
int fixed_tile_h(bool eed)
{
    if (eed && g_tile_policy == FOEED_TILES_H64) return FOEED_TILES_H32;
    if (eed && g_tile_policy == FOEED_TILES_H8) return FOEED_TILES_H16;
    return g_tile_policy;
}

struct TuneKey {
    int dev, eed, R, f64u, w, h, count, pad;
    unsigned long long sizes;  // FNV-1a hash of a batch's image sizes (0 for one image)
    bool operator<(const TuneKey &o) const { return std::memcmp(this, &o, sizeof(TuneKey)) < 0; }
};

struct TuneVal {
    int choice;  // single image: tile height; batch: tile-count threshold of the 64 x 16 images
    float us_h32, us_h16, us_h64, us_h8, us_chosen;
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

bool tune_lookup(const TuneKey &k, TuneVal *v)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(k);
    if (it == g_tune.end()) return false;
    *v = it->second;
    return true;
}

void tune_store(const TuneKey &k, const TuneVal &v)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[k] = v;
}

// Mean microseconds of `reps` back-to-back calls of launch() on s after one
// untimed call; < 0 if a launch or an event fails.
template <typename F>
float time_launches(F launch, cudaStream_t s, int reps)
{
    EventPair ev;
    if (ev.create() != cudaSuccess) return -1.f;
    if (launch() != cudaSuccess) return -1.f;
    if (cudaEventRecord(ev.e[0], s) != cudaSuccess) return -1.f;
    for (int i = 0; i < reps; ++i)
        if (launch() != cudaSuccess) return -1.f;
    if (cudaEventRecord(ev.e[1], s) != cudaSuccess || cudaEventSynchronize(ev.e[1]) != cudaSuccess) return -1.f;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]) != cudaSuccess) return -1.f;
    return 1000.f * ms / reps;
}

constexpr int kTuneReps = 3;
constexpr int kTuneRounds = 2;
constexpr int kTuneSteps = 8;

// Tile height of a single-image solve whose initial image is already in buffer C
// of the workspace: the thread's fixed policy, the cached choice for this
// (device, size, method, radius, precision), or the faster of 64 x 32 and 64 x 16
// tiles, timed on one step C -> A (buffer A is overwritten by the solve's first
// step). 0 when the generic kernel runs.
foeed_status choose_tile_h(bool eed, foeed_dtype d, const foeed_params &p, int w, int h, const Layout &L, char *ws,
                           cudaStream_t s, int *tile_h)
{
    g_last_plan = foeed_tile_plan{};
    g_last_plan.images = 1;
    *tile_h = 0;
    if (d == FOEED_F64 || !fast_params(eed, p)) return FOEED_OK;
    if (g_tile_policy != FOEED_TILES_AUTO) {
        *tile_h = fixed_tile_h(eed);
    } else {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        TuneKey k;
        std::memset(&k, 0, sizeof(k));
        k.dev = dev; k.eed = eed; k.R = gauss_radius(p.sigma); k.f64u = d == FOEED_F32_F64U; k.w = w; k.h = h;
        k.count = 1;
        TuneVal v;
        if (tune_lookup(k, &v)) {
            *tile_h = v.choice;
        } else {
            // Each candidate runs as the solve runs it: kTuneSteps chained step
            // launches (programmatic dependent launch) in one captured graph, all
            // C -> A. Small images take less time per step than a host launch, so
            // timing plain launches would measure the host.
            StepCall c{};
            c.uprev = ws + L.bufC; c.ucur = ws + L.bufC; c.unext = ws + L.bufA;
            c.mask = reinterpret_cast<const uint8_t *>(ws + L.mask);
            c.w = w; c.h = h; c.pitch = L.P; c.alpha = 1.0; c.tau = default_tau(eed, p.tau);
            CK(launch_step(eed, d, nullptr, p, s));
            cudaStream_t cs = nullptr;
            CK(capture_stream(dev, &cs));
            // candidates: 64 x 32 and 64 x 16 tiles, and 64 x 64 and 64 x 8 for FOEED
            constexpr int kCand = 4;
            const int th[kCand] = {32, 16, 64, 8};
            const int ncand = eed ? 2 : kCand;
            cudaGraphExec_t ex[kCand] = {nullptr, nullptr, nullptr, nullptr};
            struct ExecGuard {
                cudaGraphExec_t *e;
                ~ExecGuard()
                {
                    for (int i = 0; i < kCand; ++i)
                        if (e[i]) cudaGraphExecDestroy(e[i]);
                }
            } guard{ex};
            for (int i = 0; i < ncand; ++i) {
                CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
                cudaError_t err = cudaSuccess;
                for (int k = 0; k < kTuneSteps && err == cudaSuccess; ++k) {
                    c.tile_h = th[i];
                    c.pdl = k > 0;
                    err = launch_step(eed, d, &c, p, cs);
                }
                cudaGraph_t graph = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
                if (err == cudaSuccess) err = e2;
                if (err == cudaSuccess) err = cudaGraphInstantiate(&ex[i], graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (err != cudaSuccess) return fail(FOEED_ERR_CUDA, "capturing the tile-shape timing: %s",
                                                    cudaGetErrorString(err));
            }
            float us[kCand] = {-1.f, -1.f, -1.f, -1.f};
            // the candidates alternate over kTuneRounds rounds and each keeps its
            // fastest time, so a clock still ramping up favours none
            for (int round = 0; round < kTuneRounds; ++round)
                for (int i = 0; i < ncand; ++i) {
                    const float t = time_launches([&] { return cudaGraphLaunch(ex[i], s); }, s, 2) / kTuneSteps;
                    if (t < 0.f)
                        return fail(FOEED_ERR_CUDA, "timing the tile shapes: %s", cudaGetErrorString(cudaGetLastError()));
                    if (us[i] < 0.f || t < us[i]) us[i] = t;
                }
            int best = 0;
            for (int i = 1; i < ncand; ++i)
                if (us[i] < us[best]) best = i;
            v.choice = th[best];
            v.us_h32 = us[0];
            v.us_h16 = us[1];
            v.us_h64 = ncand > 2 ? us[2] : 0.f;
            v.us_h8 = ncand > 3 ? us[3] : 0.f;
            v.us_chosen = us[best];
            tune_store(k, v);
            g_last_plan.tuned = 1;
            g_last_plan.us_h32 = v.us_h32;
            g_last_plan.us_h16 = v.us_h16;
            g_last_plan.us_h64 = v.us_h64;
            g_last_plan.us_h8 = v.us_h8;
            g_last_plan.us_chosen = v.us_chosen;
            *tile_h = v.choice;
        }
    }
    g_last_plan.tile_h = *tile_h;
    g_last_plan.images_h16 = *tile_h == 16;
    return FOEED_OK;
}

// ---------------------------------------------------------------------------
// Cycle graphs: one captured FSI cycle per (method, sizes, params, buffers).

struct GraphKey {
    int eed, dtype, w, h, n, g, mu3, dev, tile_h, pad;
    double lambda, sigma, tau;
    const void *base;
    long pitch;
    bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    unsigned long long stamp = 0;
};

// Per host thread: a graph handed out by the cache is launched after this
// function returns, so no other thread may evict it; a thread evicts only its
// own graphs, whose launches have completed (every solve synchronises its
// stream before it returns).
constexpr int kCache = 4;
thread_local GraphEntry g_cache[kCache];
thread_local unsigned long long g_clock = 0;

foeed_status capture_cycle(bool eed, foeed_dtype d, const foeed_params &p, int w, int h, const Layout &L,
                           char *ws, int dev, int tile_h, cudaGraphExec_t *out)
{
    cudaStream_t cs = nullptr;
    CK(capture_stream(dev, &cs));
    void *C = ws + L.bufC, *A = ws + L.bufA, *B = ws + L.bufB;
    void *buf[2] = {A, B};
    const uint8_t *mi = reinterpret_cast<const uint8_t *>(ws + L.mask);
    Ctl *ctl = reinterpret_cast<Ctl *>(ws + L.ctl);
    double *partials = reinterpret_cast<double *>(ws + L.partials);
    const int n = p.cycle_len;
    const double tau = default_tau(eed, p.tau);
    const size_t img_bytes = (size_t)h * L.P * elem_size(d);

    CK(launch_step(eed, d, nullptr, p, cs));
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < n && err == cudaSuccess; ++k) {
        StepCall c{};
        c.w = w; c.h = h; c.pitch = L.P; c.mask = mi;
        c.alpha = (4.0 * k + 2.0) / (2.0 * k + 3.0);
        c.tau = tau;
        c.ctl = ctl; c.partials = partials; c.check_done = 1;
        c.tile_h = tile_h;
        const bool last = (k == n - 1);
        if (k == 0) { c.uprev = C; c.ucur = C; c.unext = A; }
        else if (k == 1) { c.uprev = C; c.ucur = A; c.unext = last ? C : B; }
        else { c.uprev = buf[k % 2]; c.ucur = buf[(k + 1) % 2]; c.unext = last ? C : buf[k % 2]; }
        if (last) { c.residual = 1; c.c0 = C; }
        c.pdl = k > 0 ? 1 : 0;  // successive steps overlap launch and tail (programmatic dependency)
        err = launch_step(eed, d, &c, p, cs);
        if (err == cudaSuccess && last && n == 1) err = cudaMemcpyAsync(C, A, img_bytes, cudaMemcpyDeviceToDevice, cs);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (err != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(FOEED_ERR_CUDA, "capturing the FSI cycle: %s", cudaGetErrorString(err));
    }
    if (e2 != cudaSuccess) return fail(FOEED_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e2));
    cudaError_t e3 = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) return fail(FOEED_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e3));
    return FOEED_OK;
}

foeed_status get_cycle_graph(bool eed, foeed_dtype d, const foeed_params &p, int w, int h, const Layout &L,
                             char *ws, int tile_h, cudaGraphExec_t *out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.eed = eed; key.dtype = d; key.w = w; key.h = h; key.n = p.cycle_len;
    key.g = p.diffusivity; key.mu3 = eed ? 0 : p.mu3_mode; key.dev = dev;
    key.lambda = p.lambda; key.sigma = p.sigma; key.tau = default_tau(eed, p.tau);
    key.base = ws; key.pitch = L.P; key.tile_h = tile_h;
    int victim = 0;
    for (int i = 0; i < kCache; ++i) {
        if (g_cache[i].exec && g_cache[i].key == key) {
            g_cache[i].stamp = ++g_clock;
            *out = g_cache[i].exec;
            return FOEED_OK;
        }
        if (g_cache[i].stamp < g_cache[victim].stamp) victim = i;
    }
    cudaGraphExec_t exec = nullptr;
    foeed_status st = capture_cycle(eed, d, p, w, h, L, ws, dev, tile_h, &exec);
    if (st != FOEED_OK) return st;
    if (g_cache[victim].exec) cudaGraphExecDestroy(g_cache[victim].exec);
    g_cache[victim].key = key;
    g_cache[victim].exec = exec;
    g_cache[victim].stamp = ++g_clock;
    *out = exec;
    return FOEED_OK;
}

template <typename T>
cudaError_t launch_prep(const void *f, const uint8_t *mask, void *u_inout, int w, int h, long pitch, const Layout &L,
                        char *ws, int init_mode, cudaStream_t s)
{
    Ctl *ctl = reinterpret_cast<Ctl *>(ws + L.ctl);
    double *partials = reinterpret_cast<double *>(ws + L.partials);
    uint8_t *mi = reinterpret_cast<uint8_t *>(ws + L.mask);
    int g = grid_for((long)w * h);
    prep_kernel<T><<<g, kRedThreads, 0, s>>>(static_cast<const T *>(f), mask, mi, w, h, pitch, L.P, ctl, partials);
    init_kernel<T><<<g, kRedThreads, 0, s>>>(static_cast<const T *>(f), mi, static_cast<const T *>(u_inout),
                                             reinterpret_cast<T *>(ws + L.bufC), w, h, pitch, L.P, init_mode, ctl);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copy_out(const Layout &L, char *ws, void *u_inout, int w, int h, long pitch, cudaStream_t s)
{
    copy_out_kernel<T><<<grid_for((long)w * h), kRedThreads, 0, s>>>(reinterpret_cast<const T *>(ws + L.bufC),
                                                                      static_cast<T *>(u_inout), w, h, L.P, pitch);
    return cudaGetLastError();
}

foeed_status inpaint(bool eed, const void *f, const uint8_t *mask, void *u_inout, int w, int h, long pitch,
                     foeed_dtype d, const foeed_params *params, void *workspace, size_t ws_bytes, void *stream,
                     foeed_report *report)
{
    foeed_status st = check_image(w, h, pitch, d);
    if (st) return st;
    if ((st = check_params(params, true))) return st;
    if (!f || !mask || !u_inout || !workspace) return fail(FOEED_ERR_ARG, "NULL data or workspace pointer");
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return fail(FOEED_ERR_ARG, "workspace must be 256-byte aligned");
    Layout L = layout(w, h, d);
    if (ws_bytes < L.total) return fail(FOEED_ERR_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
    const foeed_params &p = *params;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    Ctl *dctl = reinterpret_cast<Ctl *>(ws + L.ctl);

    Ctl h0;
    std::memset(&h0, 0, sizeof(h0));
    h0.tol = p.tol;
    CK(cudaMemcpyAsync(dctl, &h0, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    EventPair evs;
    CK(evs.create());
    cudaEvent_t ev0 = evs.e[0], ev1 = evs.e[1];
    CK(cudaEventRecord(ev0, s));
    CK(d == FOEED_F64 ? launch_prep<double>(f, mask, u_inout, w, h, pitch, L, ws, p.init_mode, s)
                      : launch_prep<float>(f, mask, u_inout, w, h, pitch, L, ws, p.init_mode, s));
    int tile_h = 0;
    if ((st = choose_tile_h(eed, d, p, w, h, L, ws, s, &tile_h))) return st;
    cudaGraphExec_t exec = nullptr;
    if ((st = get_cycle_graph(eed, d, p, w, h, L, ws, tile_h, &exec))) return st;
    const int every = p.check_every > 0 ? p.check_every : 8;
    Ctl hc;
    std::memset(&hc, 0, sizeof(hc));
    for (int m = 0; m < p.max_cycles; ++m) {
        CK(cudaGraphLaunch(exec, s));
        if (p.tol > 0.0 && ((m + 1) % every == 0) && m + 1 < p.max_cycles) {
            CK(cudaMemcpyAsync(&hc, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (hc.done) break;
        }
    }
    CK(d == FOEED_F64 ? launch_copy_out<double>(L, ws, u_inout, w, h, pitch, s)
                      : launch_copy_out<float>(L, ws, u_inout, w, h, pitch, s));
    CK(cudaEventRecord(ev1, s));
    CK(cudaMemcpyAsync(&hc, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev0, ev1));
    if (report) {
        report->cycles_run = hc.cycles;
        report->last_rel_change = hc.last_rel;
        report->converged = (p.tol > 0.0 && hc.done && !hc.diverged) ? 1 : 0;
        report->ms = ms;
    }
    if (hc.diverged) return fail(FOEED_ERR_DIVERGED, "cycle %d produced a non-finite change", hc.cycles);
    if (p.tol > 0.0 && !hc.done)
        return fail(FOEED_ERR_NOT_CONVERGED, "relative change %.3e after %d cycles is not below tol %.3e",
                    hc.last_rel, hc.cycles, p.tol);
    g_err[0] = 0;
    return FOEED_OK;
}

foeed_status step(bool eed, const void *u_prev, const void *u_cur, void *u_next, const uint8_t *mask, int w, int h,
                  long pitch, foeed_dtype d, double alpha, const foeed_params *params, void *stream)
{
    foeed_status st = check_image(w, h, pitch, d);
    if (st) return st;
    if ((st = check_params(params, false))) return st;
    if (!u_prev || !u_cur || !u_next) return fail(FOEED_ERR_ARG, "NULL image pointer");
    if (u_next == u_cur) return fail(FOEED_ERR_ARG, "u_next must not alias u_cur");
    if (!std::isfinite(alpha)) return fail(FOEED_ERR_ARG, "alpha must be finite");
    StepCall c{};
    c.uprev = u_prev; c.ucur = u_cur; c.unext = u_next; c.mask = mask;
    c.w = w; c.h = h; c.pitch = pitch; c.alpha = alpha;
    c.tau = default_tau(eed, params->tau);
    c.c0 = nullptr; c.ctl = nullptr; c.partials = nullptr; c.residual = 0; c.check_done = 0;
    c.tile_h = fixed_tile_h(eed);
    CK(launch_step(eed, d, nullptr, *params, static_cast<cudaStream_t>(stream)));
    CK(launch_step(eed, d, &c, *params, static_cast<cudaStream_t>(stream)));
    return FOEED_OK;
}

}  // namespace

extern "C" {

size_t foeed_workspace_bytes(int w, int h, foeed_dtype dtype)
{
    if (w < 1 || h < 1 || (long long)w * h > (1LL << 31) - 1) return 0;
    if (dtype != FOEED_F32 && dtype != FOEED_F64 && dtype != FOEED_F32_F64U) return 0;
    return layout(w, h, dtype).total;
}

foeed_status foeed_inpaint(const void *f, const uint8_t *mask, void *u_inout, int w, int h, long pitch,
                           foeed_dtype dtype, const foeed_params *params, void *workspace, size_t workspace_bytes,
                           void *stream, foeed_report *report)
{
    return inpaint(false, f, mask, u_inout, w, h, pitch, dtype, params, workspace, workspace_bytes, stream, report);
}

foeed_status eed_inpaint(const void *f, const uint8_t *mask, void *u_inout, int w, int h, long pitch,
                         foeed_dtype dtype, const foeed_params *params, void *workspace, size_t workspace_bytes,
                         void *stream, foeed_report *report)
{
    return inpaint(true, f, mask, u_inout, w, h, pitch, dtype, params, workspace, workspace_bytes, stream, report);
}

foeed_status foeed_step(const void *u_prev, const void *u_cur, void *u_next, const uint8_t *mask, int w, int h,
                        long pitch, foeed_dtype dtype, double alpha, const foeed_params *params, void *stream)
{
    return step(false, u_prev, u_cur, u_next, mask, w, h, pitch, dtype, alpha, params, stream);
}

foeed_status eed_step(const void *u_prev, const void *u_cur, void *u_next, const uint8_t *mask, int w, int h,
                      long pitch, foeed_dtype dtype, double alpha, const foeed_params *params, void *stream)
{
    return step(true, u_prev, u_cur, u_next, mask, w, h, pitch, dtype, alpha, params, stream);
}

size_t foeed_errors_workspace_bytes(int w, int h)
{
    (void)w;
    (void)h;
    return align_up(sizeof(Ctl), kAlign) + align_up(sizeof(double) * 2 * kRedBlocksMax, kAlign);
}

foeed_status foeed_errors(const void *u, const void *v, int w, int h, long pitch, foeed_dtype dtype, void *workspace,
                          size_t workspace_bytes, void *stream, double *out)
{
    foeed_status st = check_image(w, h, pitch, dtype);
    if (st) return st;
    if (!u || !v || !workspace || !out) return fail(FOEED_ERR_ARG, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return fail(FOEED_ERR_ARG, "workspace must be 256-byte aligned");
    if (workspace_bytes < foeed_errors_workspace_bytes(w, h)) return fail(FOEED_ERR_ARG, "workspace too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    Ctl *ctl = reinterpret_cast<Ctl *>(ws);
    double *partials = reinterpret_cast<double *>(ws + align_up(sizeof(Ctl), kAlign));
    CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    int g = grid_for((long)w * h);
    if (dtype == FOEED_F64)
        errors_kernel<double><<<g, kRedThreads, 0, s>>>(static_cast<const double *>(u), static_cast<const double *>(v),
                                                        w, h, pitch, ctl, partials);
    else
        errors_kernel<float><<<g, kRedThreads, 0, s>>>(static_cast<const float *>(u), static_cast<const float *>(v), w,
                                                       h, pitch, ctl, partials);
    CK(cudaGetLastError());
    Ctl hc;
    CK(cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    out[0] = hc.err[0];
    out[1] = hc.err[1];
    out[2] = hc.err[2];
    return FOEED_OK;
}

foeed_status foeed_apply_tensor_field(const void *u, const void *d, void *Pu, int w, int h, long pitch,
                                      foeed_dtype dtype, void *stream)
{
    foeed_status st = check_image(w, h, pitch, dtype);
    if (st) return st;
    if (dtype == FOEED_F32_F64U) return fail(FOEED_ERR_ARG, "use FOEED_F32 or FOEED_F64");
    if (!u || !d || !Pu) return fail(FOEED_ERR_ARG, "NULL pointer");
    if (Pu == u) return fail(FOEED_ERR_ARG, "Pu must not alias u");
    CK(apply_field(u, d, Pu, w, h, pitch, dtype == FOEED_F64, static_cast<cudaStream_t>(stream)));
    return FOEED_OK;
}

foeed_status foeed_set_tile_policy(int policy)
{
    if (policy != FOEED_TILES_AUTO && policy != FOEED_TILES_H8 && policy != FOEED_TILES_H16 &&
        policy != FOEED_TILES_H32 && policy != FOEED_TILES_H64)
        return fail(FOEED_ERR_ARG, "unknown tile policy %d", policy);
    g_tile_policy = policy;
    return FOEED_OK;
}

foeed_status foeed_last_tile_plan(foeed_tile_plan *out)
{
    if (!out) return fail(FOEED_ERR_ARG, "NULL pointer");
    *out = g_last_plan;
    return FOEED_OK;
}

const char *foeed_last_error(void) { return g_err; }

const char *foeed_version(void) { return "foeed-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Adjoint of the solve (gradient with respect to the stored grey values).

namespace {

struct VjpLayout {
    Layout base;          // control block, partials, C/A/B, mask of the forward solve
    size_t img;           // bytes of one internal image
    size_t cp, seg, g, pend, pv, qx, qy, total;
    int ncp, K;
};

VjpLayout vjp_layout(int w, int h, foeed_dtype d, const foeed_params &p, int K)
{
    VjpLayout V;
    V.base = layout(w, h, d);
    V.img = align_up((size_t)h * V.base.P * elem_size(d), kAlign);
    const long S = (long)p.cycle_len * p.max_cycles;
    V.K = K;
    V.ncp = (int)((S + K - 1) / K);
    size_t off = V.base.total;
    if (K == 1) {
        // every state u^0 .. u^S, written by the forward steps themselves
        V.cp = off; off += V.img * (size_t)(S + 1);
        V.seg = off;
    } else {
        V.cp = off; off += V.img * 2 * (size_t)V.ncp;  // (u^s, u^{s-1}) at s = 0, K, 2K, ...
        V.seg = off; off += V.img * (size_t)K;           // states of one segment
    }
    V.g = off; off += V.img;
    V.pend = off; off += V.img;
    V.pv = off; off += V.img;
    V.qx = off; off += V.img;
    V.qy = off; off += V.img;
    V.total = off;
    return V;
}

foeed_status check_vjp(const foeed_params *params, foeed_dtype d, int K)
{
    foeed_status st;
    if ((st = check_params(params, true))) return st;
    if (d != FOEED_F32 && d != FOEED_F64) return fail(FOEED_ERR_ARG, "the adjoint runs FOEED_F32 or FOEED_F64");
    if (params->diffusivity != 0 || params->mu3_mode != 0)
        return fail(FOEED_ERR_ARG, "the adjoint needs the Charbonnier diffusivity and mu3 = sqrt(mu1)");
    if (params->tol != 0.0) return fail(FOEED_ERR_ARG, "the adjoint differentiates a fixed number of cycles (tol = 0)");
    if (params->init_mode != 0) return fail(FOEED_ERR_ARG, "the adjoint needs init_mode 0");
    if (K < 1) return fail(FOEED_ERR_ARG, "checkpoint_every must be >= 1");
    return FOEED_OK;
}

template <typename T>
__global__ void pitch_copy_kernel(const T *__restrict__ src, long sp, T *__restrict__ dst, long dp, int w, int h)
{
    const long n = (long)w * h;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        long y = i / w, x = i - y * w;
        dst[y * dp + x] = src[y * sp + x];
    }
}

// Sum of the adjoint over the unknown pixels (the mean initialisation path).
template <typename T>
__global__ void unknown_sum_kernel(const T *__restrict__ g, const uint8_t *__restrict__ mi, int w, int h, long P,
                                   Ctl *ctl, double *partials)
{
    __shared__ double red[64];
    double s = 0.0, c = 0.0;
    const long n = (long)w * h;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        long y = i / w, x = i - y * w;
        if (!mi[y * P + x]) { s += double(g[y * P + x]); c += 1.0; }
    }
    if (grid_sum2_last(s, c, partials, &ctl->ticket, gridDim.x, blockIdx.x, red)) ctl->err[0] = s;
}

// grad_f = M g + (sum over unknown pixels of g) / |K| on the known pixels.
template <typename T>
__global__ void grad_f_kernel(const T *__restrict__ g, const uint8_t *__restrict__ mi, int w, int h, long P,
                              T *__restrict__ gf, long pitch, const Ctl *ctl)
{
    const long n = (long)w * h;
    const double add = ctl->known > 0 ? ctl->err[0] / double(ctl->known) : 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        long y = i / w, x = i - y * w;
        gf[y * pitch + x] = mi[y * P + x] ? T(double(g[y * P + x]) + add) : T(0);
    }
}

template <typename T>
cudaError_t launch_adjoint(const AdjArgs<T> *a, int R, cudaStream_t s);
template <>
cudaError_t launch_adjoint<float>(const AdjArgs<float> *a, int R, cudaStream_t s) { return adjoint_step_f32(a, R, s); }
template <>
cudaError_t launch_adjoint<double>(const AdjArgs<double> *a, int R, cudaStream_t s) { return adjoint_step_f64(a, R, s); }

template <typename T>
foeed_status run_vjp(const void *f, const uint8_t *mask, const void *grad_u, void *grad_f, void *u_out, int w, int h,
                     long pitch, foeed_dtype d, const foeed_params &p, int K, char *ws, const VjpLayout &V,
                     cudaStream_t s)
{
    const Layout &L = V.base;
    const long P = L.P;
    Ctl *ctl = reinterpret_cast<Ctl *>(ws + L.ctl);
    double *partials = reinterpret_cast<double *>(ws + L.partials);
    const uint8_t *mi = reinterpret_cast<const uint8_t *>(ws + L.mask);
    T *buf[3] = {reinterpret_cast<T *>(ws + L.bufC), reinterpret_cast<T *>(ws + L.bufA),
                 reinterpret_cast<T *>(ws + L.bufB)};
    auto img = [&](size_t off, size_t i) { return reinterpret_cast<T *>(ws + off + V.img * i); };
    const int n = p.cycle_len;
    const long S = (long)n * p.max_cycles;
    const double tau = default_tau(false, p.tau);
    const int R = gauss_radius(p.sigma);
    const size_t ibytes = (size_t)h * P * sizeof(T);
    const int g1 = grid_for((long)w * h);

    Ctl h0;
    std::memset(&h0, 0, sizeof(h0));
    CK(cudaMemcpyAsync(ctl, &h0, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(launch_step(false, d, nullptr, p, s));
    CK(launch_adjoint<T>(nullptr, R, s));
    CK(launch_prep<T>(f, mask, nullptr, w, h, pitch, L, ws, 0, s));  // C = u^{0,0}

    auto fwd_step = [&](const T *prev, const T *cur, T *next, long st) -> cudaError_t {
        StepCall c{};
        const int k = (int)(st % n);
        c.uprev = prev; c.ucur = cur; c.unext = next; c.mask = mi;
        c.w = w; c.h = h; c.pitch = P;
        c.alpha = (4.0 * k + 2.0) / (2.0 * k + 3.0);
        c.tau = tau;
        c.tile_h = g_tile_policy;
        return launch_step(false, d, &c, p, s);
    };

    if (K == 1) {
        // forward solve into the state history: step s reads u^s (and u^{s-1}, or u^s
        // again at the first step of a cycle) and writes u^{s+1}; nothing is copied
        T *hist = img(V.cp, 0);
        CK(cudaMemcpyAsync(hist, buf[0], ibytes, cudaMemcpyDeviceToDevice, s));
        for (long st = 0; st < S; ++st) {
            const int k = (int)(st % n);
            const T *cur = img(V.cp, st);
            CK(fwd_step(k == 0 ? cur : img(V.cp, st - 1), cur, img(V.cp, st + 1), st));
        }
        if (u_out)
            pitch_copy_kernel<T><<<g1, kRedThreads, 0, s>>>(img(V.cp, S), P, static_cast<T *>(u_out), pitch, w, h);
    }
    // forward solve with checkpoints of (u^s, u^{s-1}) every K steps
    int icur = 0, iprev = 0;
    for (long st = 0; st < S && K > 1; ++st) {
        const int k = (int)(st % n);
        if (k == 0) iprev = icur;
        if (st % K == 0) {
            CK(cudaMemcpyAsync(img(V.cp, 2 * (st / K)), buf[icur], ibytes, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(img(V.cp, 2 * (st / K) + 1), buf[iprev], ibytes, cudaMemcpyDeviceToDevice, s));
        }
        int inext = 0;
        while (inext == icur || inext == iprev) ++inext;
        CK(fwd_step(buf[iprev], buf[icur], buf[inext], st));
        iprev = icur;
        icur = inext;
    }
    if (u_out && K > 1)
        pitch_copy_kernel<T><<<g1, kRedThreads, 0, s>>>(buf[icur], P, static_cast<T *>(u_out), pitch, w, h);

    // backward: g = dL/du_final, then the segments in reverse
    T *g = img(V.g, 0), *pend = img(V.pend, 0);
    pitch_copy_kernel<T><<<g1, kRedThreads, 0, s>>>(static_cast<const T *>(grad_u), pitch, g, P, w, h);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(pend, 0, ibytes, s));
    AdjArgs<T> a{};
    a.g = g; a.gout = g; a.pend = pend; a.mask = mi;
    a.pv = img(V.pv, 0); a.qx = img(V.qx, 0); a.qy = img(V.qy, 0);
    a.w = w; a.h = h; a.pitch = P;
    a.tau = T(tau);
    a.l2 = T(p.lambda * p.lambda);
    a.inv_l2 = T(1.0 / (p.lambda * p.lambda));
    gauss_taps<T>(p.sigma, a.wts);
    for (long st = S - 1; st >= 0 && K == 1; --st) {  // every state is kept: no recomputation
        const int k = (int)(st % n);
        a.x = img(V.cp, st);
        a.alpha = T((4.0 * k + 2.0) / (2.0 * k + 3.0));
        a.first_of_cycle = k == 0;
        CK(launch_adjoint<T>(&a, R, s));
    }
    for (int seg = V.ncp - 1; seg >= 0 && K > 1; --seg) {
        const long s0 = (long)seg * K, s1 = std::min<long>(S, s0 + K);
        // states u^{s0} .. u^{s1-1} of this segment, recomputed from its checkpoint
        CK(cudaMemcpyAsync(img(V.seg, 0), img(V.cp, 2 * seg), ibytes, cudaMemcpyDeviceToDevice, s));
        for (long st = s0; st + 1 < s1; ++st) {
            const int k = (int)(st % n);
            const T *cur = img(V.seg, st - s0);
            const T *prev = k == 0 ? cur : (st == s0 ? img(V.cp, 2 * seg + 1) : img(V.seg, st - s0 - 1));
            CK(fwd_step(prev, cur, img(V.seg, st - s0 + 1), st));
        }
        for (long st = s1 - 1; st >= s0; --st) {
            const int k = (int)(st % n);
            a.x = img(V.seg, st - s0);
            const double al = (4.0 * k + 2.0) / (2.0 * k + 3.0);
            a.alpha = T(al);
            a.first_of_cycle = k == 0;
            CK(launch_adjoint<T>(&a, R, s));
        }
    }
    // grad_f = M g + mean-path term (the control block still holds |K| from the set-up)
    unknown_sum_kernel<T><<<g1, kRedThreads, 0, s>>>(g, mi, w, h, P, ctl, partials);
    CK(cudaGetLastError());
    grad_f_kernel<T><<<g1, kRedThreads, 0, s>>>(g, mi, w, h, P, static_cast<T *>(grad_f), pitch, ctl);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    (void)buf;
    return FOEED_OK;
}

}  // namespace

extern "C" size_t foeed_vjp_workspace_bytes(int w, int h, foeed_dtype dtype, const foeed_params *params,
                                            int checkpoint_every)
{
    if (w < 1 || h < 1 || !params || checkpoint_every < 1 || params->cycle_len < 1 || params->max_cycles < 1) return 0;
    return vjp_layout(w, h, dtype, *params, checkpoint_every).total;
}

extern "C" foeed_status foeed_inpaint_vjp(const void *f, const uint8_t *mask, const void *grad_u, void *grad_f,
                                          void *u_out, int w, int h, long pitch, foeed_dtype dtype,
                                          const foeed_params *params, int checkpoint_every, void *workspace,
                                          size_t workspace_bytes, void *stream)
{
    foeed_status st = check_image(w, h, pitch, dtype);
    if (st) return st;
    if ((st = check_vjp(params, dtype, checkpoint_every))) return st;
    if (!f || !mask || !grad_u || !grad_f || !workspace) return fail(FOEED_ERR_ARG, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return fail(FOEED_ERR_ARG, "workspace must be 256-byte aligned");
    const VjpLayout V = vjp_layout(w, h, dtype, *params, checkpoint_every);
    if (workspace_bytes < V.total) return fail(FOEED_ERR_ARG, "workspace too small: %zu < %zu bytes", workspace_bytes, V.total);
    char *ws = static_cast<char *>(workspace);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = dtype == FOEED_F64 ? run_vjp<double>(f, mask, grad_u, grad_f, u_out, w, h, pitch, dtype, *params,
                                              checkpoint_every, ws, V, s)
                            : run_vjp<float>(f, mask, grad_u, grad_f, u_out, w, h, pitch, dtype, *params,
                                             checkpoint_every, ws, V, s);
    if (st == FOEED_OK) g_err[0] = 0;
    return st;
}

// ---------------------------------------------------------------------------
// Batched solve: many images, one launch per FSI step over all their tiles.

namespace {

struct BatchPlan {
    std::vector<Layout> lay;
    std::vector<size_t> off;  // workspace offset of each image's region
    size_t inst_off, tiles_off, total;
    int ntiles;               // capacity of the tile list (every image on 64 x 16 tiles)
};

// Device tables of one tile plan of a batch: images with fewer than `thresh`
// 64 x 32 tiles run on 64 x 16 tiles, the others on 64 x 32 tiles (thresh 0:
// every image on 64 x 32; INT_MAX: every image on 64 x 16). hi / ht receive the
// image table and the (image, tile) work list.
void batch_tables(const foeed_instance *inst, int count, const BatchPlan &bp, char *ws, int thresh,
                  std::vector<BatchInst> &hi, std::vector<int2> &ht, int *images_h16)
{
    hi.resize(count);
    ht.clear();
    *images_h16 = 0;
    for (int i = 0; i < count; ++i) {
        const Layout &L = bp.lay[i];
        char *b = ws + bp.off[i];
        BatchInst &I = hi[i];
        I.C = reinterpret_cast<float *>(b + L.bufC);
        I.A = reinterpret_cast<float *>(b + L.bufA);
        I.B = reinterpret_cast<float *>(b + L.bufB);
        I.mask = reinterpret_cast<const uint8_t *>(b + L.mask);
        I.w = inst[i].w;
        I.h = inst[i].h;
        I.pitch = L.P;
        I.c4 = float(0.25 / (inst[i].lambda * inst[i].lambda));
        const long long n32 = (long long)((inst[i].w + 63) / 64) * ((inst[i].h + 31) / 32);
        I.th = n32 < thresh ? 16 : 32;
        *images_h16 += I.th == 16;
        I.ntx = (inst[i].w + 63) / 64;
        I.nty = (inst[i].h + I.th - 1) / I.th;
        I.ctl = reinterpret_cast<Ctl *>(b + L.ctl);
        I.partials = reinterpret_cast<double *>(b + L.partials);
        for (int k = 0; k < I.ntx * I.nty; ++k) ht.push_back(make_int2(i, k));
    }
}

foeed_status batch_plan(const foeed_instance *inst, int count, foeed_dtype d, BatchPlan *bp)
{
    if (!inst || count < 1) return fail(FOEED_ERR_ARG, "need at least one image");
    bp->lay.resize(count);
    bp->off.resize(count);
    size_t off = 0;
    bp->inst_off = off;
    off += align_up(sizeof(BatchInst) * (size_t)count, kAlign);
    long long ntiles = 0;
    for (int i = 0; i < count; ++i) {
        foeed_status st = check_image(inst[i].w, inst[i].h, inst[i].pitch, d);
        if (st) {
            char msg[sizeof(g_err)];
            std::snprintf(msg, sizeof(msg), "%s", g_err);
            return fail(st, "image %d: %s", i, msg);
        }
        ntiles += (long long)((inst[i].w + 63) / 64) * ((inst[i].h + 15) / 16);  // the most tiles any plan has
    }
    if (ntiles > (1LL << 30)) return fail(FOEED_ERR_ARG, "too many tiles");
    bp->ntiles = (int)ntiles;
    bp->tiles_off = off;
    off += align_up(sizeof(int2) * (size_t)ntiles, kAlign);
    for (int i = 0; i < count; ++i) {
        bp->lay[i] = layout(inst[i].w, inst[i].h, d);
        bp->off[i] = off;
        off += bp->lay[i].total;
    }
    bp->total = off;
    return FOEED_OK;
}

}  // namespace

extern "C" size_t foeed_batch_workspace_bytes(const foeed_instance *inst, int count, foeed_dtype dtype)
{
    BatchPlan bp;
    if (batch_plan(inst, count, dtype, &bp) != FOEED_OK) return 0;
    return bp.total;
}

static foeed_status inpaint_batch(bool eed, const foeed_instance *inst, int count, foeed_dtype dtype,
                                  const foeed_params *params, void *workspace, size_t workspace_bytes, void *stream,
                                  foeed_report *reports)
{
    auto batch_step = eed ? batch_step_fast_eed_f32 : batch_step_fast_foeed_f32;
    foeed_status st;
    if ((st = check_params(params, true))) return st;
    const foeed_params &p = *params;
    if (dtype != FOEED_F32 && dtype != FOEED_F32_F64U)
        return fail(FOEED_ERR_ARG, "the batched solver runs FOEED_F32 or FOEED_F32_F64U");
    if (!fast_params(eed, p))
        return fail(FOEED_ERR_ARG, "the batched solver needs the Charbonnier diffusivity and mu3 = sqrt(mu1)");
    if (p.cycle_len < 2) return fail(FOEED_ERR_ARG, "the batched solver needs cycle_len >= 2");
    BatchPlan bp;
    if ((st = batch_plan(inst, count, dtype, &bp))) return st;
    for (int i = 0; i < count; ++i) {
        if (!inst[i].f || !inst[i].mask || !inst[i].u_inout) return fail(FOEED_ERR_ARG, "image %d: NULL pointer", i);
        if (!(inst[i].lambda > 0.0) || !std::isfinite(inst[i].lambda))
            return fail(FOEED_ERR_ARG, "image %d: lambda must be > 0", i);
    }
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % kAlign)
        return fail(FOEED_ERR_ARG, "workspace must be a 256-byte aligned device pointer");
    if (workspace_bytes < bp.total)
        return fail(FOEED_ERR_ARG, "workspace too small: %zu < %zu bytes", workspace_bytes, bp.total);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    const bool f64u = dtype == FOEED_F32_F64U;
    const int R = gauss_radius(p.sigma);
    const double tau = default_tau(eed, p.tau);

    // per-image set-up: control block, internal mask, initial image
    Ctl h0;
    std::memset(&h0, 0, sizeof(h0));
    h0.tol = p.tol;
    EventPair evs;
    CK(evs.create());
    cudaEvent_t ev0 = evs.e[0], ev1 = evs.e[1];
    CK(cudaEventRecord(ev0, s));
    {
        Fork fk;
        CK(fk.open(s));
        for (int i = 0; i < count; ++i) {
            const Layout &L = bp.lay[i];
            CK(cudaMemcpyAsync(ws + bp.off[i] + L.ctl, &h0, sizeof(Ctl), cudaMemcpyHostToDevice, fk[i]));
            CK(launch_prep<float>(inst[i].f, inst[i].mask, inst[i].u_inout, inst[i].w, inst[i].h, inst[i].pitch,
                                  bp.lay[i], ws + bp.off[i], p.init_mode, fk[i]));
        }
        CK(fk.join(s));
    }

    // tile plan: the thread's fixed policy, the cached choice for this list of
    // sizes, or the fastest candidate plan timed on one step C -> A over all
    // images (buffer A is overwritten by the solve's first step)
    StepCall c{};
    c.w = 1; c.h = 1; c.pitch = 4;
    c.tau = tau;
    StepArgs<float> a = make_args<float>(c, p);
    CK(batch_step(nullptr, nullptr, 0, R, f64u, s));
    std::vector<BatchInst> hi;
    std::vector<int2> ht;
    int images_h16 = 0;
    BatchArgs bt;
    bt.inst = reinterpret_cast<const BatchInst *>(ws + bp.inst_off);
    bt.tiles = reinterpret_cast<const int2 *>(ws + bp.tiles_off);
    bt.role = kRoleFirst;
    bt.last = 0;
    auto upload = [&](int thresh) -> cudaError_t {
        batch_tables(inst, count, bp, ws, thresh, hi, ht, &images_h16);
        cudaError_t e = cudaMemcpyAsync(ws + bp.inst_off, hi.data(), sizeof(BatchInst) * count,
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ws + bp.tiles_off, ht.data(), sizeof(int2) * ht.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host tables are rebuilt for the next plan
        return e;
    };
    g_last_plan = foeed_tile_plan{};
    g_last_plan.images = count;
    // a batch has no 64 x 64 or 64 x 8 tiles: those policies mean 64 x 32 and 64 x 16 there
    int thresh = (g_tile_policy == FOEED_TILES_H16 || g_tile_policy == FOEED_TILES_H8) ? INT_MAX : 0;
    if (g_tile_policy == FOEED_TILES_AUTO) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        TuneKey k;
        std::memset(&k, 0, sizeof(k));
        k.dev = dev; k.eed = eed; k.R = R; k.f64u = f64u; k.count = count;
        unsigned long long hsh = 1469598103934665603ULL;
        std::vector<long long> n32(count);
        for (int i = 0; i < count; ++i) {
            hsh = (hsh ^ (unsigned)inst[i].w) * 1099511628211ULL;
            hsh = (hsh ^ (unsigned)inst[i].h) * 1099511628211ULL;
            n32[i] = (long long)((inst[i].w + 63) / 64) * ((inst[i].h + 31) / 32);
        }
        k.sizes = hsh;
        TuneVal v;
        if (tune_lookup(k, &v)) {
            thresh = v.choice;
        } else {
            // candidates: every image on 64 x 32, every image on 64 x 16, and the images
            // below each quartile of the batch's 64 x 32 tile counts on 64 x 16
            std::vector<long long> sorted = n32;
            std::sort(sorted.begin(), sorted.end());
            std::vector<int> cand = {0, INT_MAX};
            for (int qn = 1; qn <= 3; ++qn) {
                const long long t = sorted[(size_t)(count - 1) * qn / 4] + 1;
                if (t < INT_MAX && std::find(cand.begin(), cand.end(), (int)t) == cand.end()) cand.push_back((int)t);
            }
            std::vector<float> tc(cand.size(), -1.f);
            for (int round = 0; round < kTuneRounds; ++round)  // alternating, fastest of the rounds
                for (size_t ci = 0; ci < cand.size(); ++ci) {
                    CK(upload(cand[ci]));
                    const int nt = (int)ht.size();
                    const float us = time_launches([&] { return batch_step(&a, &bt, nt, R, f64u, s); }, s, kTuneReps);
                    if (us < 0.f)
                        return fail(FOEED_ERR_CUDA, "timing the tile plans: %s", cudaGetErrorString(cudaGetLastError()));
                    if (tc[ci] < 0.f || us < tc[ci]) tc[ci] = us;
                }
            float best = -1.f;
            v.us_h32 = v.us_h16 = v.us_h64 = v.us_h8 = 0.f;
            for (size_t ci = 0; ci < cand.size(); ++ci) {
                if (cand[ci] == 0) v.us_h32 = tc[ci];
                if (cand[ci] == INT_MAX) v.us_h16 = tc[ci];
                if (best < 0.f || tc[ci] < best) { best = tc[ci]; v.choice = cand[ci]; }
            }
            v.us_chosen = best;
            tune_store(k, v);
            g_last_plan.tuned = 1;
            g_last_plan.us_h32 = v.us_h32;
            g_last_plan.us_h16 = v.us_h16;
            g_last_plan.us_chosen = v.us_chosen;
            thresh = v.choice;
        }
    }
    CK(upload(thresh));
    g_last_plan.images_h16 = images_h16;
    const int ntiles = (int)ht.size();

    // one FSI cycle = n launches over the work list, captured once
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaStream_t cs = nullptr;
    CK(capture_stream(dev, &cs));
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    const int n = p.cycle_len;
    for (int k = 0; k < n && err == cudaSuccess; ++k) {
        BatchArgs b;
        b.inst = reinterpret_cast<const BatchInst *>(ws + bp.inst_off);
        b.tiles = reinterpret_cast<const int2 *>(ws + bp.tiles_off);
        b.role = k == 0 ? kRoleFirst : k == 1 ? kRoleSecond : (k % 2 == 0 ? kRoleEven : kRoleOdd);
        b.last = k == n - 1;
        a.alpha = (4.0 * k + 2.0) / (2.0 * k + 3.0);
        a.alpha_t = float(a.alpha);
        a.alpha_lo = float(a.alpha - double(a.alpha_t));
        a.residual = b.last;
        a.pdl = k > 0;
        err = batch_step(&a, &b, ntiles, R, f64u, cs);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (err != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(FOEED_ERR_CUDA, "capturing the batched cycle: %s",
                    cudaGetErrorString(err != cudaSuccess ? err : e2));
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) return fail(FOEED_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e3));

    const int every = p.check_every > 0 ? p.check_every : 8;
    std::vector<Ctl> hc(count);
    foeed_status result = FOEED_OK;
    for (int m = 0; m < p.max_cycles && err == cudaSuccess; ++m) {
        err = cudaGraphLaunch(exec, s);
        if (err == cudaSuccess && p.tol > 0.0 && ((m + 1) % every == 0) && m + 1 < p.max_cycles) {
            for (int i = 0; i < count && err == cudaSuccess; ++i)
                err = cudaMemcpyAsync(&hc[i], hi[i].ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
            if (err == cudaSuccess) err = cudaStreamSynchronize(s);
            bool all = true;
            for (int i = 0; i < count; ++i) all = all && hc[i].done;
            if (all) break;
        }
    }
    if (err == cudaSuccess) {
        Fork fk;
        err = fk.open(s);
        for (int i = 0; i < count && err == cudaSuccess; ++i)
            err = launch_copy_out<float>(bp.lay[i], ws + bp.off[i], inst[i].u_inout, inst[i].w, inst[i].h,
                                         inst[i].pitch, fk[i]);
        if (err == cudaSuccess) err = fk.join(s);
    }
    if (err == cudaSuccess) err = cudaEventRecord(ev1, s);
    for (int i = 0; i < count && err == cudaSuccess; ++i)
        err = cudaMemcpyAsync(&hc[i], hi[i].ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    cudaGraphExecDestroy(exec);
    if (err != cudaSuccess) return fail(FOEED_ERR_CUDA, "batched solve: %s", cudaGetErrorString(err));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev0, ev1));
    for (int i = 0; i < count; ++i) {
        if (reports) {
            reports[i].cycles_run = hc[i].cycles;
            reports[i].last_rel_change = hc[i].last_rel;
            reports[i].converged = (p.tol > 0.0 && hc[i].done && !hc[i].diverged) ? 1 : 0;
            reports[i].ms = ms;
        }
        if (result == FOEED_OK && hc[i].diverged)
            result = fail(FOEED_ERR_DIVERGED, "image %d: cycle %d produced a non-finite change", i, hc[i].cycles);
        else if (result == FOEED_OK && p.tol > 0.0 && !hc[i].done)
            result = fail(FOEED_ERR_NOT_CONVERGED, "image %d did not reach tol %.3e", i, p.tol);
    }
    if (result == FOEED_OK) g_err[0] = 0;
    return result;
}

extern "C" foeed_status foeed_inpaint_batch(const foeed_instance *inst, int count, foeed_dtype dtype,
                                            const foeed_params *params, void *workspace, size_t workspace_bytes,
                                            void *stream, foeed_report *reports)
{
    return inpaint_batch(false, inst, count, dtype, params, workspace, workspace_bytes, stream, reports);
}

extern "C" foeed_status eed_inpaint_batch(const foeed_instance *inst, int count, foeed_dtype dtype,
                                          const foeed_params *params, void *workspace, size_t workspace_bytes,
                                          void *stream, foeed_report *reports)
{
    return inpaint_batch(true, inst, count, dtype, params, workspace, workspace_bytes, stream, reports);
}

// ---------------------------------------------------------------------------
// Solver entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's allocator arena, plug-ins that may not touch the device heap, or
// real-time paths where an allocation could block or fail. For them,
// foeed_inpaint_static runs the FP32/FP64 FOEED solve with its scratch (the
// control block, reduction partials, three image buffers and the internal
// mask) in one file-scope device array of fixed size instead of a caller
// workspace. Every device that loads this library holds that array until the
// process exits. The solve uses plain stream-ordered kernel launches: no graph,
// no event, no allocation of any kind.

namespace {

__device__ __align__(256) unsigned char g_static_scratch[FOEED_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
unsigned char *g_static_ptr[64] = {};

// Device address of the static scratch on the current device, looked up once
// per device (host code only sees a host-side stand-in for the symbol).
foeed_status static_scratch(unsigned char **out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(FOEED_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return fail(FOEED_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_static_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_static_ptr[dev];
    return FOEED_OK;
}

}  // namespace

extern "C" size_t foeed_static_scratch_bytes(void) { return FOEED_STATIC_SCRATCH_BYTES; }

extern "C" foeed_status foeed_inpaint_static(const void *f, const uint8_t *mask, void *u_inout, int w, int h,
                                             long pitch, foeed_dtype dtype, const foeed_params *params,
                                             void *stream, foeed_report *report)
{
    foeed_status st = check_image(w, h, pitch, dtype);
    if (st) return st;
    if ((st = check_params(params, true))) return st;
    if (!f || !mask || !u_inout) return fail(FOEED_ERR_ARG, "NULL data pointer");
    const Layout L = layout(w, h, dtype);
    if (L.total > FOEED_STATIC_SCRATCH_BYTES)
        return fail(FOEED_ERR_ARG, "image needs %zu bytes of scratch, more than the static %zu bytes", L.total,
                    (size_t)FOEED_STATIC_SCRATCH_BYTES);
    unsigned char *base = nullptr;
    if ((st = static_scratch(&base))) return st;
    char *ws = reinterpret_cast<char *>(base);
    const foeed_params &p = *params;
    const bool eed = false;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ctl *dctl = reinterpret_cast<Ctl *>(ws + L.ctl);
    double *partials = reinterpret_cast<double *>(ws + L.partials);
    const uint8_t *mi = reinterpret_cast<const uint8_t *>(ws + L.mask);
    void *C = ws + L.bufC, *A = ws + L.bufA, *B = ws + L.bufB;
    void *buf[2] = {A, B};
    const int n = p.cycle_len;
    const double tau = default_tau(eed, p.tau);
    const size_t img_bytes = (size_t)h * L.P * elem_size(dtype);
    const auto t0 = std::chrono::steady_clock::now();

    // the control block must start from zero (ticket, flags, counters)
    Ctl h0;
    std::memset(&h0, 0, sizeof(h0));
    h0.tol = p.tol;
    CK(cudaMemcpyAsync(dctl, &h0, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(launch_step(eed, dtype, nullptr, p, s));
    CK(dtype == FOEED_F64 ? launch_prep<double>(f, mask, u_inout, w, h, pitch, L, ws, p.init_mode, s)
                          : launch_prep<float>(f, mask, u_inout, w, h, pitch, L, ws, p.init_mode, s));
    const int every = p.check_every > 0 ? p.check_every : 8;
    Ctl hc;
    std::memset(&hc, 0, sizeof(hc));
    for (int m = 0; m < p.max_cycles; ++m) {
        for (int k = 0; k < n; ++k) {  // the same buffer rotation as the captured cycle
            StepCall c{};
            c.w = w; c.h = h; c.pitch = L.P; c.mask = mi;
            c.alpha = (4.0 * k + 2.0) / (2.0 * k + 3.0);
            c.tau = tau;
            c.ctl = dctl; c.partials = partials; c.check_done = 1;
            c.tile_h = g_tile_policy;
            const bool last = (k == n - 1);
            if (k == 0) { c.uprev = C; c.ucur = C; c.unext = A; }
            else if (k == 1) { c.uprev = C; c.ucur = A; c.unext = last ? C : B; }
            else { c.uprev = buf[k % 2]; c.ucur = buf[(k + 1) % 2]; c.unext = last ? C : buf[k % 2]; }
            if (last) { c.residual = 1; c.c0 = C; }
            CK(launch_step(eed, dtype, &c, p, s));
            if (last && n == 1) CK(cudaMemcpyAsync(C, A, img_bytes, cudaMemcpyDeviceToDevice, s));
        }
        if (p.tol > 0.0 && ((m + 1) % every == 0) && m + 1 < p.max_cycles) {
            CK(cudaMemcpyAsync(&hc, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (hc.done) break;
        }
    }
    CK(dtype == FOEED_F64 ? launch_copy_out<double>(L, ws, u_inout, w, h, pitch, s)
                          : launch_copy_out<float>(L, ws, u_inout, w, h, pitch, s));
    CK(cudaMemcpyAsync(&hc, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const auto t1 = std::chrono::steady_clock::now();
    if (report) {
        report->cycles_run = hc.cycles;
        report->last_rel_change = hc.last_rel;
        report->converged = (p.tol > 0.0 && hc.done && !hc.diverged) ? 1 : 0;
        report->ms = std::chrono::duration<float, std::milli>(t1 - t0).count();
    }
    if (hc.diverged) return fail(FOEED_ERR_DIVERGED, "cycle %d produced a non-finite change", hc.cycles);
    if (p.tol > 0.0 && !hc.done)
        return fail(FOEED_ERR_NOT_CONVERGED, "relative change %.3e after %d cycles is not below tol %.3e",
                    hc.last_rel, hc.cycles, p.tol);
    g_err[0] = 0;
    return FOEED_OK;
}
