// Host-side entry points of the step kernels, one translation unit per
// (method, storage type) so they compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "foeed_device.cuh"

namespace foeed {

// Output tile of one CTA per storage type (columns x rows).
constexpr int kTileW32 = 64, kTileH32 = 16;
constexpr int kTileW64 = 32, kTileH64 = 16;

// Each launches one step on s; a == nullptr only prepares the kernel's attributes.
cudaError_t step_foeed_f32(const StepArgs<float> *a, int R, bool f64_update, cudaStream_t s);
cudaError_t step_foeed_f64(const StepArgs<double> *a, int R, cudaStream_t s);
cudaError_t step_eed_f32(const StepArgs<float> *a, int R, bool f64_update, cudaStream_t s);
cudaError_t step_eed_f64(const StepArgs<double> *a, int R, cudaStream_t s);

// Register-blocked FP32 kernels (64 x 32 tiles): Charbonnier g, FOEED with
// mu3 = sqrt(mu1); need a row pitch that is a multiple of 4 elements and
// 16-byte aligned image and mask pointers.
cudaError_t step_fast_foeed_f32(const StepArgs<float> *a, int R, bool f64_update, cudaStream_t s);
cudaError_t step_fast_eed_f32(const StepArgs<float> *a, int R, bool f64_update, cudaStream_t s);

// One FOEED step over the tiles of many images (batched solve); a == nullptr
// only prepares the kernel.
cudaError_t batch_step_fast_foeed_f32(const StepArgs<float> *a, const BatchArgs *b, int ntiles, int R,
                                      bool f64_update, cudaStream_t s);
cudaError_t batch_step_fast_eed_f32(const StepArgs<float> *a, const BatchArgs *b, int ntiles, int R,
                                    bool f64_update, cudaStream_t s);

// Backward of one masked FOEED FSI step (kernels B1 + B2, adjoint.cuh);
// a == nullptr only prepares the kernels.
template <typename T>
struct AdjArgs;
cudaError_t adjoint_step_f32(const AdjArgs<float> *a, int R, cudaStream_t s);
cudaError_t adjoint_step_f64(const AdjArgs<double> *a, int R, cudaStream_t s);

// Fourth-order divergence with a caller-supplied coefficient field (generic_field.cu).
cudaError_t apply_field(const void *u, const void *d, void *pu, int w, int h, long pitch, bool f64, cudaStream_t s);

}  // namespace foeed
