// Double-word instantiation of the ATKM x passes (see passes_df.cu).
#include "passes_impl.cuh"

namespace atkm {
template cudaError_t atkm_pass_xf<df>(atkm_plan*, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t atkm_pass_xi<df>(atkm_plan*, int, const double*, const double*, double*, cudaStream_t);
}  // namespace atkm
