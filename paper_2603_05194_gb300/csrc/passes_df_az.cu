// Double-word instantiation of the ATKM z pass (see passes_df.cu).
#include "passes_impl.cuh"

namespace atkm {
template cudaError_t atkm_pass_z<df>(atkm_plan*, int, const double*, const double*, double*, cudaStream_t);
}  // namespace atkm
