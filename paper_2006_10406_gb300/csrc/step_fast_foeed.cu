// Instantiations of the register-blocked FP32 step: FOEED (Charbonnier g).
#include "dispatch.h"
#include "step_fast.cuh"

namespace foeed {

template <typename U>
static cudaError_t run(const StepArgs<float> *a, int R, cudaStream_t s)
{
    switch (R) {
    case 0: return launch_fsi_step_fast<0, false, U>(a, s);
    case 1: return launch_fsi_step_fast<1, false, U>(a, s);
    case 2: return launch_fsi_step_fast<2, false, U>(a, s);
    case 3: return launch_fsi_step_fast<3, false, U>(a, s);
    case 4: return launch_fsi_step_fast<4, false, U>(a, s);
    case 5: return launch_fsi_step_fast<5, false, U>(a, s);
    case 6: return launch_fsi_step_fast<6, false, U>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t step_fast_foeed_f32(const StepArgs<float> *a, int R, bool f64_update, cudaStream_t s)
{
    return f64_update ? run<double>(a, R, s) : run<float>(a, R, s);
}

template <typename U>
static cudaError_t run_batch(const StepArgs<float> *a, const BatchArgs *b, int ntiles, int R, cudaStream_t s)
{
    switch (R) {
    case 0: return launch_fsi_batch_step_fast<0, false, U>(a, b, ntiles, s);
    case 1: return launch_fsi_batch_step_fast<1, false, U>(a, b, ntiles, s);
    case 2: return launch_fsi_batch_step_fast<2, false, U>(a, b, ntiles, s);
    case 3: return launch_fsi_batch_step_fast<3, false, U>(a, b, ntiles, s);
    case 4: return launch_fsi_batch_step_fast<4, false, U>(a, b, ntiles, s);
    case 5: return launch_fsi_batch_step_fast<5, false, U>(a, b, ntiles, s);
    case 6: return launch_fsi_batch_step_fast<6, false, U>(a, b, ntiles, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t batch_step_fast_foeed_f32(const StepArgs<float> *a, const BatchArgs *b, int ntiles, int R,
                                      bool f64_update, cudaStream_t s)
{
    return f64_update ? run_batch<double>(a, b, ntiles, R, s) : run_batch<float>(a, b, ntiles, R, s);
}

}  // namespace foeed
