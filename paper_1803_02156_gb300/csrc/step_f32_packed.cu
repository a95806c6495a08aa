// Fused step kernels: f32, packed matrix values.
#include "step_kernels.cuh"

namespace cfd {

template cfd_status launch_step_p<float, true>(int, int, int, const StepArgs<float> &, int, cudaStream_t);
template cfd_status launch_persistent_p<float, true>(int, int, const StepArgs<float> &, cplx_t<float> *, cplx_t<float> *,
                                                  cplx_t<float> *, int64_t, int, int, cudaStream_t);

template cfd_status launch_persistent_staged<float>(int, int, const StepArgs<float> &, cplx_t<float> *, cplx_t<float> *, int,
                                                   int, cudaStream_t);

}  // namespace cfd
