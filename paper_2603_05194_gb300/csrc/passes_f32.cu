// FP32 (complex64 workspace) instantiation of the spectral-operator launchers (see passes_impl.cuh).
#include "passes_impl.cuh"

namespace atkm {
// the ATKM and H passes are instantiated in passes_f32_a.cu and passes_f32_h.cu
#define ATKM_A_SIG (atkm_plan*, int, const double*, const double*, double*, cudaStream_t)
#define ATKM_H_SIG (atkm_plan*, const Phys&, const double*, const double*, const double*, double*, int, cudaStream_t)
extern template cudaError_t atkm_pass_xf<float> ATKM_A_SIG;
extern template cudaError_t atkm_pass_yf<float> ATKM_A_SIG;
extern template cudaError_t atkm_pass_z<float> ATKM_A_SIG;
extern template cudaError_t atkm_pass_yi<float> ATKM_A_SIG;
extern template cudaError_t atkm_pass_xi<float> ATKM_A_SIG;
extern template cudaError_t h_pass_x<float> ATKM_H_SIG;
extern template cudaError_t h_pass_y<float> ATKM_H_SIG;
extern template cudaError_t h_pass_z<float> ATKM_H_SIG;
template cudaError_t launch_atkm<float>(atkm_plan*, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_H<float>(atkm_plan*, const Phys&, const double*, const double*, const double*, double*,
                                      int, cudaStream_t);
template cudaError_t launch_precond<float>(atkm_plan*, const Phys&, const double*, const double*, const double*,
                                            const double*, double*, cudaStream_t);
}  // namespace atkm
