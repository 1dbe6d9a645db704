// Instantiations of the fused FSI step: FOEED method, float storage.
#include "dispatch.h"
#include "step_kernel.cuh"

namespace foeed {

template <typename U>
static cudaError_t run(const StepArgs<float> *a, int R, cudaStream_t s)
{
    switch (R) {
    case 0: return launch_fsi_step<float, U, 0, kTileW32, kTileH32, false>(a, s);
    case 1: return launch_fsi_step<float, U, 1, kTileW32, kTileH32, false>(a, s);
    case 2: return launch_fsi_step<float, U, 2, kTileW32, kTileH32, false>(a, s);
    case 3: return launch_fsi_step<float, U, 3, kTileW32, kTileH32, false>(a, s);
    case 4: return launch_fsi_step<float, U, 4, kTileW32, kTileH32, false>(a, s);
    case 5: return launch_fsi_step<float, U, 5, kTileW32, kTileH32, false>(a, s);
    case 6: return launch_fsi_step<float, U, 6, kTileW32, kTileH32, false>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t step_foeed_f32(const StepArgs<float> *a, int R, bool f64_update, cudaStream_t s)
{
    return f64_update ? run<double>(a, R, s) : run<float>(a, R, s);
}

}  // namespace foeed
