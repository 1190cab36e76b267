// FP32 (complex64 workspace) instantiation of the spectral-operator launchers (see passes_impl.cuh).
#include "passes_impl.cuh"

namespace atkm {
template cudaError_t launch_atkm<float>(atkm_plan*, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_H<float>(atkm_plan*, const Phys&, const double*, const double*, const double*, double*,
                                      int, cudaStream_t);
template cudaError_t launch_precond<float>(atkm_plan*, const Phys&, const double*, const double*, const double*,
                                            const double*, double*, cudaStream_t);
}  // namespace atkm
