// Host-side launchers of the renderer's kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "dvr_device.cuh"

namespace dvr {

// Variants of the adjoint kernel (template parameters, Sec. 4.4). The API
// asks for kTFNone, kTFDelayed or kTFImmediate; "delayed" runs as
// kTFPrivate (per-lane shared-memory copies) when R <= kPrivateMaxR, else
// as kTFWarp (per-warp copies with shared atomics).
enum TFMode { kTFNone = 0, kTFDelayed = 1, kTFImmediate = 2, kTFPrivate = 3, kTFWarp = 4 };
constexpr int kPrivateMaxR = 32;

// How the adjoint recovers the accumulated opacity before each sample.
// kInvDepth: from the exactly carried optical depth (default).
// kInvAlpha32: Eq. inv-blend-forward as printed, A_i = (alpha - A_{i+1}) /
//   (alpha - 1), in binary32 from the binary32 image opacity (ablation).
// kInvAlpha64: the same, starting from the optical depth and dividing in
//   binary64 once A > 0.99 (ablation).
enum InvMode { kInvDepth = 0, kInvAlpha32 = 1, kInvAlpha64 = 2 };

cudaError_t launch_forward(const Params& p, int model, int vol_dtype, cudaStream_t stream);
cudaError_t launch_backward(const Params& p, int model, int vol_dtype, bool grad_volume,
                            int tf_mode, bool grad_position, int inv_mode, cudaStream_t stream);
cudaError_t launch_backward_cells(const Params& p, int model, int vol_dtype, bool grad_volume, int tf_mode,
                                  bool grad_position, cudaStream_t stream);
cudaError_t launch_backward_cells4(const Params& p, int model, int vol_dtype, bool grad_volume, int tf_mode,
                                   bool grad_position, cudaStream_t stream);
cudaError_t launch_backward_cells8(const Params& p, int model, int vol_dtype, bool grad_volume, int tf_mode,
                                   bool grad_position, cudaStream_t stream);
cudaError_t launch_make_cells(const void* data, int dtype, int nx, int ny, int nz, int brick, void* cells,
                              cudaStream_t stream);
cudaError_t launch_cells_to_vertices(const float* cg, int nx, int ny, int nz, int brick, float* grad,
                                     cudaStream_t stream);
cudaError_t launch_forward_color(const Params& p, int vol_dtype, cudaStream_t stream);
cudaError_t launch_backward_color(const Params& p, int vol_dtype, bool grad_volume, bool grad_position,
                                  cudaStream_t stream);
cudaError_t launch_tangent(const Params& p, int model, int vol_dtype, float* tangent, cudaStream_t stream);
cudaError_t launch_contract(const Params& p, int channels, const float* tangent, const float* grad_image,
                            float* grad_eye, cudaStream_t stream);
cudaError_t launch_volume_prior(const float* v, int nx, int ny, int nz, float scale, float* grad, float* loss,
                                cudaStream_t s);
cudaError_t launch_tf_prior(const float* tf, int R, float scale, float* grad, float* loss, cudaStream_t s);
cudaError_t launch_loss_l1(const float* x, const float* y, long long n, float scale, float* g, float* loss,
                           cudaStream_t s);
cudaError_t launch_resample(const float* src, int sx, int sy, int sz, float* dst, int dx, int dy, int dz,
                            cudaStream_t s);
cudaError_t launch_loss_l2(const float* image, const float* target, long long n, float scale,
                           float* grad_image, float* loss, cudaStream_t stream);
cudaError_t launch_orbit_eye(const float* params, int n, float* eye, cudaStream_t stream);
cudaError_t launch_orbit_eye_backward(const float* params, const float* grad_eye, int n,
                                      float* grad_params, cudaStream_t stream);

// Number of SMs and L2 size in bytes of the current device (cached per
// device; 0 bytes if unknown).
int sm_count();
long long l2_bytes();

}  // namespace dvr
