// The adjoint march kernels that gather from the volume's cell layout
// (dvr_make_cells): the variants of dvr_backward.cu with CELLS set, in a
// translation unit of their own so that the two sets compile in parallel.
#include "dvr_backward.cuh"

namespace dvr {

cudaError_t launch_backward_cells(const Params& p, int model, int vol_dtype, bool grad_volume, int tf_mode,
                                  bool grad_position, cudaStream_t stream)
{
    return launch_backward_source<true>(p, model, vol_dtype, grad_volume, tf_mode, grad_position, kInvDepth,
                                        stream);
}

}  // namespace dvr
