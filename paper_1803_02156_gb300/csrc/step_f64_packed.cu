// Fused step kernels: f64, packed matrix values.
#include "step_kernels.cuh"

namespace cfd {

template cfd_status launch_step_p<double, true>(int, int, int, const StepArgs<double> &, int, cudaStream_t);
template cfd_status launch_persistent_p<double, true>(int, int, const StepArgs<double> &, cplx_t<double> *, cplx_t<double> *,
                                                  cplx_t<double> *, int64_t, int, int, cudaStream_t);

template cfd_status launch_persistent_staged<double>(int, int, const StepArgs<double> &, cplx_t<double> *, cplx_t<double> *, int,
                                                   int, cudaStream_t);

}  // namespace cfd
