// Fused step kernels: f32, complex matrix values.
#include "step_kernels.cuh"

namespace cfd {

template cfd_status launch_step_p<float, false>(int, int, int, const StepArgs<float> &, int, cudaStream_t);
template cfd_status launch_persistent_p<float, false>(int, int, const StepArgs<float> &, cplx_t<float> *, cplx_t<float> *,
                                                  cplx_t<float> *, int64_t, int, int, cudaStream_t);

}  // namespace cfd
