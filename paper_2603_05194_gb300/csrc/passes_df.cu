// Double-word (double-FP32) instantiation of the ATKM launcher (see
// passes_impl.cuh and df32.cuh).  Its passes are instantiated in translation
// units of their own (passes_df_ax/ay/az.cu) so that the double-word kernels
// compile in parallel.
#include "passes_impl.cuh"

namespace atkm {
#define ATKM_A_SIG (atkm_plan*, int, const double*, const double*, double*, cudaStream_t)
extern template cudaError_t atkm_pass_xf<df> ATKM_A_SIG;
extern template cudaError_t atkm_pass_yf<df> ATKM_A_SIG;
extern template cudaError_t atkm_pass_z<df> ATKM_A_SIG;
extern template cudaError_t atkm_pass_yi<df> ATKM_A_SIG;
extern template cudaError_t atkm_pass_xi<df> ATKM_A_SIG;
template cudaError_t launch_atkm<df> ATKM_A_SIG;
}  // namespace atkm
