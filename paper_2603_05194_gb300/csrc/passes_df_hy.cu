// Double-word instantiation of the y pass of H_phi f (see passes_df_h.cu).
#include "passes_impl.cuh"

namespace atkm {
template cudaError_t h_pass_y<df>(atkm_plan*, const Phys&, const double*, const double*, const double*, double*,
                                    int, cudaStream_t);
}  // namespace atkm
