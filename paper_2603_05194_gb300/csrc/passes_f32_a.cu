// The ATKM passes of the float launchers, in a translation unit of their own so
// that they compile in parallel with the rest (see passes_f32.cu).
#include "passes_impl.cuh"

namespace atkm {
#define ATKM_A_SIG (atkm_plan*, int, const double*, const double*, double*, cudaStream_t)
template cudaError_t atkm_pass_xf<float> ATKM_A_SIG;
template cudaError_t atkm_pass_yf<float> ATKM_A_SIG;
template cudaError_t atkm_pass_z<float> ATKM_A_SIG;
template cudaError_t atkm_pass_yi<float> ATKM_A_SIG;
template cudaError_t atkm_pass_xi<float> ATKM_A_SIG;
}  // namespace atkm
