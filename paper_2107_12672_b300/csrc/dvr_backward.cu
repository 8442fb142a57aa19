// Adjoint pass (Alg. 2) in memory that does not grow with the step count.
//
// Each thread re-sets up its ray exactly as the forward kernel did and
// marches it back to front. The state before sample i is not read from a
// record: the optical depth S_i = S_{i+1} - dt tau_i is recovered from the
// stored total (an unevaluated float pair, so the subtraction does not
// drift), and the transmittance 1 - A_i = exp(-S_i). This is the inversion
// of the blend of Sec. 4.4 (Eq. inv-blend-forward) carried out on the
// logarithm of the transmittance, where it neither cancels nor underflows.
// Only the accumulated opacity is needed by the adjoint of the blend; the
// colour adjoint is constant along the ray (Eq. adj-blend-forward). With
// T_i = 1 - A_i and T^_i the adjoint of T_i, the blend adjoint is carried
// scaled by the transmittance: the sample's weight (1 - A_i) alpha_i is
// T_i - T_{i+1}, U_i = T_i T^_i obeys U_i = U_{i+1} + (T_i - T_{i+1})
// rgb_i . C^, and tau^_i = dt (T_{i+1} rgb_i . C^ - U_{i+1}): Alg. 2's
// updates multiplied through by T_i, with no alpha and no division.
//
// Gradients (all "+=", Alg. 2):
//  - TF ("adjoint-delayed", Sec. 5.2): for R <= 32 every lane owns a copy
//    of the TF gradient in shared memory, laid out [row][channel][lane] so
//    that the per-sample updates are conflict-free plain adds; for larger R
//    each lane sums in registers while its samples stay in one TF segment
//    and adds the sums to a per-warp copy with shared atomics when the
//    segment changes. The copies are summed per block and added to global
//    memory once per block. The ablation "adjoint-immediate" adds every
//    sample's contribution to global memory directly;
//  - volume: the 8 corner contributions are summed in registers while the
//    ray stays in one cell and added to global memory with atomics when it
//    leaves the cell (Sec. 4.4: "on exit of the current cell");
//  - eye / step: x^_o, w^ summed in registers along the ray (Alg. 2 last
//    loop line), chained through f_camera per ray, warp-reduced, one atomic
//    per warp.
#include "dvr_backward.cuh"

namespace dvr {

cudaError_t launch_backward(const Params& p, int model, int vol_dtype, bool grad_volume,
                            int tf_mode, bool grad_position, int inv_mode, cudaStream_t stream)
{
    // with the cell layout (every volume of the launch has one), except for
    // the inversion ablations, which read the volume's array
    if (p.vol[0].cells && inv_mode == kInvDepth) {
        if (p.vol[0].cells_brick == 8)
            return launch_backward_cells8(p, model, vol_dtype, grad_volume, tf_mode, grad_position, stream);
        if (p.vol[0].cells_brick == 4)
            return launch_backward_cells4(p, model, vol_dtype, grad_volume, tf_mode, grad_position, stream);
        return launch_backward_cells(p, model, vol_dtype, grad_volume, tf_mode, grad_position, stream);
    }
    return launch_backward_source<0>(p, model, vol_dtype, grad_volume, tf_mode, grad_position, inv_mode, stream);
}

}  // namespace dvr
