// Bandwidth probes (dvr_probe.cu), internal to the library.
#pragma once

#include <cuda_runtime.h>

namespace dvr {

cudaError_t launch_probe(int kind, void* buf, size_t bytes, int reps, float* sink, cudaStream_t stream);

}  // namespace dvr
