// Opacity-entropy loss kernels (dvr_entropy.cu), internal to the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dvr {

constexpr int kEntropyViews = 512;   // views per launch

struct EntropyViews {
    long long offset[kEntropyViews];  // first pixel of the view
    int pixels[kEntropyViews];        // width * height
    int n;
};

cudaError_t launch_entropy(const EntropyViews& v, const float* image, int channels, float scale, float* grad,
                           float* loss, double* stats, cudaStream_t stream);

}  // namespace dvr
