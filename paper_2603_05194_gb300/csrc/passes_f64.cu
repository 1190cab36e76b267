// FP64 instantiation of the spectral-operator launchers (see passes_impl.cuh).
#include "passes_impl.cuh"

namespace atkm {
// the ATKM and H passes are instantiated in passes_f64_a.cu and passes_f64_h.cu
#define ATKM_A_SIG (atkm_plan*, int, const double*, const double*, double*, cudaStream_t)
#define ATKM_H_SIG (atkm_plan*, const Phys&, const double*, const double*, const double*, double*, int, cudaStream_t)
extern template cudaError_t atkm_pass_xf<double> ATKM_A_SIG;
extern template cudaError_t atkm_pass_yf<double> ATKM_A_SIG;
extern template cudaError_t atkm_pass_z<double> ATKM_A_SIG;
extern template cudaError_t atkm_pass_yi<double> ATKM_A_SIG;
extern template cudaError_t atkm_pass_xi<double> ATKM_A_SIG;
extern template cudaError_t h_pass_x<double> ATKM_H_SIG;
extern template cudaError_t h_pass_y<double> ATKM_H_SIG;
extern template cudaError_t h_pass_z<double> ATKM_H_SIG;
template cudaError_t launch_atkm<double>(atkm_plan*, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_H<double>(atkm_plan*, const Phys&, const double*, const double*, const double*, double*,
                                      int, cudaStream_t);
template cudaError_t launch_precond<double>(atkm_plan*, const Phys&, const double*, const double*, const double*,
                                            const double*, double*, cudaStream_t);
template cudaError_t launch_cfft3<double>(atkm_plan*, double2*, int, cudaStream_t);
}  // namespace atkm
