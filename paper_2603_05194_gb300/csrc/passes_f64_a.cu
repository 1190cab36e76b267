// The ATKM passes of the double launchers, in a translation unit of their own so
// that they compile in parallel with the rest (see passes_f64.cu).
#include "passes_impl.cuh"

namespace atkm {
#define ATKM_A_SIG (atkm_plan*, int, const double*, const double*, double*, cudaStream_t)
template cudaError_t atkm_pass_xf<double> ATKM_A_SIG;
template cudaError_t atkm_pass_yf<double> ATKM_A_SIG;
template cudaError_t atkm_pass_z<double> ATKM_A_SIG;
template cudaError_t atkm_pass_yi<double> ATKM_A_SIG;
template cudaError_t atkm_pass_xi<double> ATKM_A_SIG;
}  // namespace atkm
