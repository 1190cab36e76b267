// FP64 instantiation of the spectral-operator launchers (see passes_impl.cuh).
#include "passes_impl.cuh"

namespace atkm {
template cudaError_t launch_atkm<double>(atkm_plan*, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_H<double>(atkm_plan*, const Phys&, const double*, const double*, const double*, double*,
                                      int, cudaStream_t);
template cudaError_t launch_precond<double>(atkm_plan*, const Phys&, const double*, const double*, const double*,
                                            const double*, double*, cudaStream_t);
template cudaError_t launch_cfft3<double>(atkm_plan*, double2*, int, cudaStream_t);
}  // namespace atkm
