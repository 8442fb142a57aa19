// The adjoint march kernels that gather from the volume's cell layout
// (dvr_make_cells) with records in bricks of 8^3 cells: the variants of
// dvr_backward.cu with CB = 8, in a translation unit of their own.
#include "dvr_backward.cuh"

namespace dvr {

cudaError_t launch_backward_cells8(const Params& p, int model, int vol_dtype, bool grad_volume, int tf_mode,
                                   bool grad_position, cudaStream_t stream)
{
    return launch_backward_source<8>(p, model, vol_dtype, grad_volume, tf_mode, grad_position, kInvDepth,
                                     stream);
}

}  // namespace dvr
