// Instantiations of the adjoint step kernels (B1 + B2) for float and double.
#include "adjoint.cuh"
#include "dispatch.h"

namespace foeed {

template <typename T>
static cudaError_t run(const AdjArgs<T> *a, int R, cudaStream_t s)
{
    switch (R) {
    case 0: return launch_adjoint_step<T, 0>(a, s);
    case 1: return launch_adjoint_step<T, 1>(a, s);
    case 2: return launch_adjoint_step<T, 2>(a, s);
    case 3: return launch_adjoint_step<T, 3>(a, s);
    case 4: return launch_adjoint_step<T, 4>(a, s);
    case 5: return launch_adjoint_step<T, 5>(a, s);
    case 6: return launch_adjoint_step<T, 6>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t adjoint_step_f32(const AdjArgs<float> *a, int R, cudaStream_t s) { return run<float>(a, R, s); }
cudaError_t adjoint_step_f64(const AdjArgs<double> *a, int R, cudaStream_t s) { return run<double>(a, R, s); }

}  // namespace foeed
