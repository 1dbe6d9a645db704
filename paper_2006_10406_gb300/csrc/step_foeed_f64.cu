// Instantiations of the fused FSI step: FOEED method, double storage.
#include "dispatch.h"
#include "step_kernel.cuh"

namespace foeed {

cudaError_t step_foeed_f64(const StepArgs<double> *a, int R, cudaStream_t s)
{
    switch (R) {
    case 0: return launch_fsi_step<double, double, 0, kTileW64, kTileH64, false>(a, s);
    case 1: return launch_fsi_step<double, double, 1, kTileW64, kTileH64, false>(a, s);
    case 2: return launch_fsi_step<double, double, 2, kTileW64, kTileH64, false>(a, s);
    case 3: return launch_fsi_step<double, double, 3, kTileW64, kTileH64, false>(a, s);
    case 4: return launch_fsi_step<double, double, 4, kTileW64, kTileH64, false>(a, s);
    case 5: return launch_fsi_step<double, double, 5, kTileW64, kTileH64, false>(a, s);
    case 6: return launch_fsi_step<double, double, 6, kTileW64, kTileH64, false>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace foeed
