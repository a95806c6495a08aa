// cfd_filter_noalloc: the ChebFD filter with its scratch memory in a static
// device array owned by the library, for callers that may not allocate.
//
// Who needs it: code that runs under a host application's device-memory
// budget or pool, where raw cudaMalloc calls are forbidden or all memory is
// already reserved by that pool, and latency-critical loops that cannot pay
// cudaMalloc's cost and its implicit device-wide synchronisation.  Such
// callers pass only their inputs and outputs; the work blocks, weights,
// per-step dot products and reduction partials live in cfd_noalloc_scratch.
#include "filter.cuh"

namespace cfd {
namespace {

// One copy per device that loads the library, held until process exit.
static __device__ __align__(256) unsigned char cfd_noalloc_scratch[CFD_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device.  In host code
// the symbol is only a host-side handle, so the kernels must be given this
// address instead.  Looked up on every call (no allocation, no stream work):
// a cached address would go stale if the module were loaded again in a new
// context (after cudaDeviceReset), and the kernels would then write through a
// dangling pointer.  The first lookup on a device may load the module, which
// is why the first call there must come before any stream capture.
cfd_status scratch_for_current_device(void **out) {
    int dev = -1;
    CFD_CUDA(cudaGetDevice(&dev));
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, cfd_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(CFD_ERR_CUDA, "cudaGetSymbolAddress(cfd_noalloc_scratch) failed on device %d: %s", dev,
                    cudaGetErrorString(e));
    *out = p;
    return CFD_OK;
}

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" {

cfd_status cfd_filter_noalloc(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r, int n_p,
                              cfd_block X, int n_b, double *moments, cudaStream_t stream) {
    clear_error();
    // the real argument errors first, then whether the problem fits
    CFD_TRY(check_filter_args(H, n_p, X, n_b, 0));
    size_t need = filter_workspace(H->n_rows, X.n_cols, n_b, n_p, H->prec, X.prec);
    if (need > (size_t)CFD_NOALLOC_SCRATCH_BYTES)
        return fail(CFD_ERR_ARG,
                    "cfd_filter_noalloc: this problem needs %zu bytes of scratch but the static scratch holds %zu "
                    "(N * n_b too large); use cfd_filter with a caller-provided workspace",
                    need, (size_t)CFD_NOALLOC_SCRATCH_BYTES);
    void *scratch = nullptr;
    CFD_TRY(scratch_for_current_device(&scratch));
    return filter_impl(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, 0, 0, scratch, (size_t)CFD_NOALLOC_SCRATCH_BYTES,
                       moments, stream);
}

cfd_status cfd_filter_noalloc_status(cudaStream_t stream) {
    clear_error();
    void *scratch = nullptr;
    CFD_TRY(scratch_for_current_device(&scratch));
    // the filter carves its status word from the start of the scratch
    return cfd_workspace_status(scratch, stream);
}

}  // extern "C"
