// The H_phi f axis passes of the float launchers, in a translation unit of their
// own so that they compile in parallel with the rest (see passes_f32.cu).
#include "passes_impl.cuh"

namespace atkm {
#define ATKM_H_SIG (atkm_plan*, const Phys&, const double*, const double*, const double*, double*, int, cudaStream_t)
template cudaError_t h_pass_x<float> ATKM_H_SIG;
template cudaError_t h_pass_y<float> ATKM_H_SIG;
template cudaError_t h_pass_z<float> ATKM_H_SIG;
}  // namespace atkm
