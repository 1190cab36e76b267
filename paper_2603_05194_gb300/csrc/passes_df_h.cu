// Double-word instantiation of the H_phi f launcher.  Its three axis passes
// are instantiated in translation units of their own (passes_df_hx/hy/hz.cu)
// so that the double-word kernels compile in parallel.
#include "passes_impl.cuh"

namespace atkm {
#define ATKM_H_SIG (atkm_plan*, const Phys&, const double*, const double*, const double*, double*, int, cudaStream_t)
extern template cudaError_t h_pass_x<df> ATKM_H_SIG;
extern template cudaError_t h_pass_y<df> ATKM_H_SIG;
extern template cudaError_t h_pass_z<df> ATKM_H_SIG;
template cudaError_t launch_H<df> ATKM_H_SIG;
}  // namespace atkm
