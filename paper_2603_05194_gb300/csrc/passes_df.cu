// Double-word (double-FP32) instantiation of the spectral-operator launchers
// (see passes_impl.cuh and df32.cuh).
#include "passes_impl.cuh"

namespace atkm {
template cudaError_t launch_atkm<df>(atkm_plan*, int, const double*, const double*, double*, cudaStream_t);
}  // namespace atkm
