// ChebFD filter of a search space held in host memory (Algorithm 2's
// subspace blocking taken one level further: Sect. 5 notes that only the
// active n_b block and the two recurrence blocks need fast memory while the
// filter runs, so the n_s-wide search space can live in slower, larger
// memory).  On a Grace-Blackwell node the host memory sits behind the
// chip-to-chip link; two device block buffers are used in turn: while block b
// is filtered on the caller's stream, a copy stream writes block b - 1 back
// and brings block b + 1 in.  Blocks are column windows of the row-major
// host block.  Where the GPU can address the host block (page-locked memory,
// or any host memory on a system with pageable-memory access), a copy kernel
// moves the windows over the link with coalesced 16-byte loads and stores:
// every row of a window is one contiguous run of n_b complex values, which a
// pitched 2-D DMA copy moves as a separate small transfer per row (about
// 5 GB/s for 512-byte rows).  Otherwise pitched 2-D copies are used.

#include <algorithm>

#include "filter.cuh"

namespace cfd {

namespace {

size_t host_filter_workspace(int64_t N, int n_b, int n_p, int prec_H, int prec_X) {
    const size_t sX = prec_X == CFD_C128 ? 16 : 8;
    return round_up(filter_workspace(N, n_b, n_b, n_p, prec_H, prec_X), 256) + 2 * round_up((size_t)N * n_b * sX, 256);
}

// Stream and events of one call, released on every return path (destruction
// while work is pending is deferred by the runtime until that work is done).
struct CopyPipe {
    cudaStream_t copy = nullptr;
    cudaEvent_t start = nullptr, in[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr}, out = nullptr;
    ~CopyPipe() {
        for (cudaEvent_t e : {start, in[0], in[1], done[0], done[1], out})
            if (e) cudaEventDestroy(e);
        if (copy) cudaStreamDestroy(copy);
    }
    cfd_status create() {
        // the copies' CTAs are scheduled ahead of the filter's when SM slots free up
        int lo = 0, hi = 0;
        CFD_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CFD_CUDA(cudaStreamCreateWithPriority(&copy, cudaStreamNonBlocking, hi));
        for (cudaEvent_t *e : {&start, &in[0], &in[1], &done[0], &done[1], &out})
            CFD_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        return CFD_OK;
    }
};

// dst rows (stride ldd bytes) <- src rows (stride lds bytes), n_rows rows of
// width bytes (multiples of 16).  Each CTA moves one small span (four
// 16-byte moves per thread) and exits, so while the filter's full-wave step
// launches hold the SMs, copy CTAs still get the slots that free up between
// them (a few long-lived copy CTAs would hold their share of the copy back).
constexpr int kCopyThreads = 256;
constexpr int kCopyPerThread = 4;

__global__ void __launch_bounds__(kCopyThreads)
k_copy_rows(const char *src, int64_t lds, char *dst, int64_t ldd, int64_t n_rows, int width) {
    const int w16 = width >> 4;
    const int64_t total = n_rows * w16;
    const int64_t e0 = (int64_t)blockIdx.x * (kCopyThreads * kCopyPerThread) + threadIdx.x;
    uint4 v[kCopyPerThread];
#pragma unroll
    for (int u = 0; u < kCopyPerThread; ++u) {
        const int64_t f = e0 + u * kCopyThreads;
        if (f < total) v[u] = *reinterpret_cast<const uint4 *>(src + (f / w16) * lds + (f % w16) * 16);
    }
#pragma unroll
    for (int u = 0; u < kCopyPerThread; ++u) {
        const int64_t f = e0 + u * kCopyThreads;
        if (f < total) *reinterpret_cast<uint4 *>(dst + (f / w16) * ldd + (f % w16) * 16) = v[u];
    }
}

cfd_status copy_rows(const void *src, int64_t lds, void *dst, int64_t ldd, int64_t n_rows, size_t width,
                     cudaStream_t stream) {
    const int64_t total = n_rows * (int64_t)(width >> 4);
    const int64_t grid = (total + kCopyThreads * kCopyPerThread - 1) / (kCopyThreads * kCopyPerThread);
    if (grid == 0) return CFD_OK;
    if (grid > 2147483647LL) return fail(CFD_ERR_ARG, "block too large to copy (%lld rows)", (long long)n_rows);
    k_copy_rows<<<(unsigned)grid, kCopyThreads, 0, stream>>>(static_cast<const char *>(src), lds,
                                                             static_cast<char *>(dst), ldd, n_rows, (int)width);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

}  // namespace

}  // namespace cfd

using namespace cfd;

extern "C" size_t cfd_filter_host_workspace(int64_t N, int n_s, int n_b, int n_p, int prec_H, int prec_X) {
    (void)n_s;
    if (N < 1 || n_b < 1 || n_p < 2) return 0;
    return host_filter_workspace(N, n_b, n_p, prec_H & 0xff, prec_X & 0xff);
}

// blocked: X holds the search space block after block (block b, rows of n_b
// values, at X.ptr + b N n_b elements; X.ld == n_b), so a block moves as one
// contiguous copy; else X is row-major with row stride X.ld.
// How a block-after-block search space moves: 1 by the copy kernel on the
// high-priority copy stream (where the GPU can address the host block), 0 by
// DMA copies.  DMA copies between host and device measured about 200 GB/s on
// an idle GB300 and about 5 GB/s while kernels occupy the SMs.
#ifndef CFD_HOST_BLOCKED_KERNEL
#define CFD_HOST_BLOCKED_KERNEL 1
#endif
// Schedule of a block-after-block search space.  Overlapped: block b + 1
// comes in and b - 1 goes out on the copy stream while b is filtered with
// the gathered steps (several CTAs per SM leave room for the copy kernel).
// Serial: each block's DMA copies on the filter's own stream, before and
// after its filter, at the link's full rate, and the footprint-staged
// steps, next to which overlapped copies are starved.  At low degree the
// copies dominate and overlapping them pays; at high degree the faster
// steps do.  Degrees up to CFD_HOST_OVERLAP_MAX_NP take the overlapped
// schedule (measured on 200x200x100, 16 blocks: n_p = 5 and 20 overlapped
// 3.2 and 7.6 s against 6.3 and 8.8 s serial; n_p = 100 24.5 against 20.3 s).
#ifndef CFD_HOST_OVERLAP_MAX_NP
#define CFD_HOST_OVERLAP_MAX_NP 40
#endif

static cfd_status filter_host_impl(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                                   int n_p, cfd_block X, int n_b, void *work, size_t work_bytes, double *moments,
                                   int arith, bool blocked, cudaStream_t stream) {
    CFD_TRY(check_matrix(H));
    if (blocked) {
        if (X.ld != n_b) return fail(CFD_ERR_ARG, "a blocked search space has ld == n_b");
        cfd_block one = X;
        one.n_cols = n_b;
        CFD_TRY(validate_block(one, H->n_rows));
    } else {
        CFD_TRY(validate_block(X, H->n_rows));
    }
    if (n_b != 8 && n_b != 16 && n_b != 32 && n_b != 64) return fail(CFD_ERR_ARG, "n_b=%d not in {8,16,32,64}", n_b);
    if (X.n_cols % n_b) return fail(CFD_ERR_ARG, "n_b=%d does not divide n_s=%d", n_b, X.n_cols);
    if (n_p < 2) return fail(CFD_ERR_ARG, "n_p=%d < 2", n_p);
    if (!work) return fail(CFD_ERR_ARG, "work is NULL");
    if (!aligned16(work)) return fail(CFD_ERR_ARG, "work must be 16-byte aligned");
    cudaPointerAttributes pa;
    CFD_CUDA(cudaPointerGetAttributes(&pa, X.ptr));
    if (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged)
        return fail(CFD_ERR_ARG, "X must be host memory (use cfd_filter for device blocks)");
    // the host block's address as the GPU sees it, if it can address it
    char *host_dev = nullptr;
    if (pa.type == cudaMemoryTypeHost && pa.devicePointer) {
        host_dev = static_cast<char *>(pa.devicePointer);
    } else {
        int dev = 0, pageable = 0;
        CFD_CUDA(cudaGetDevice(&dev));
        CFD_CUDA(cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev));
        if (pageable) host_dev = static_cast<char *>(X.ptr);
    }
    const size_t need = host_filter_workspace(H->n_rows, n_b, n_p, H->prec, X.prec);
    if (work_bytes < need) return fail(CFD_ERR_OOM, "host filter workspace %zu < %zu bytes", work_bytes, need);

    const int64_t N = H->n_rows;
    const size_t sX = X.prec == CFD_C128 ? 16 : 8;
    const size_t fws = round_up(filter_workspace(N, n_b, n_b, n_p, H->prec, X.prec), 256);
    char *dbuf[2] = {static_cast<char *>(work) + fws,
                     static_cast<char *>(work) + fws + round_up((size_t)N * n_b * sX, 256)};
    const size_t hpitch = (size_t)X.ld * sX, width = (size_t)n_b * sX;
    const int n_blocks = X.n_cols / n_b;
    char *host = static_cast<char *>(X.ptr);

    const bool serial = blocked && n_p > CFD_HOST_OVERLAP_MAX_NP;
    if (serial) {
        const size_t block_bytes = (size_t)N * width;
        for (int b = 0; b < n_blocks; ++b) {
            CFD_CUDA(cudaMemcpyAsync(dbuf[0], host + (size_t)b * block_bytes, block_bytes, cudaMemcpyHostToDevice,
                                     stream));
            cfd_block D = X;
            D.ptr = dbuf[0];
            D.ld = n_b;
            D.n_cols = n_b;
            CFD_TRY(filter_impl_opts(H, lmin, lmax, lam_l, lam_r, n_p, D, n_b, 0, 0, 0, 0, work, fws,
                                     moments ? moments + (int64_t)b * n_b * 2 * n_p : nullptr, stream, 0, 0, arith));
            CFD_CUDA(cudaMemcpyAsync(host + (size_t)b * block_bytes, dbuf[0], block_bytes, cudaMemcpyDeviceToHost,
                                     stream));
        }
        return CFD_OK;
    }
    CopyPipe cp;
    CFD_TRY(cp.create());
    // the copy stream starts after the work already queued on `stream`
    CFD_CUDA(cudaEventRecord(cp.start, stream));
    CFD_CUDA(cudaStreamWaitEvent(cp.copy, cp.start, 0));
    const size_t block_bytes = (size_t)N * width;
    auto bring_in = [&](int b) -> cfd_status {
        if (blocked && CFD_HOST_BLOCKED_KERNEL && host_dev)
            CFD_TRY(copy_rows(host_dev + (size_t)b * block_bytes, (int64_t)width, dbuf[b & 1], (int64_t)width, N, width,
                              cp.copy));
        else if (blocked)
            CFD_CUDA(cudaMemcpyAsync(dbuf[b & 1], host + (size_t)b * block_bytes, block_bytes, cudaMemcpyHostToDevice,
                                     cp.copy));
        else if (host_dev)
            CFD_TRY(copy_rows(host_dev + (size_t)b * width, (int64_t)hpitch, dbuf[b & 1], (int64_t)width, N, width,
                              cp.copy));
        else
            CFD_CUDA(cudaMemcpy2DAsync(dbuf[b & 1], width, host + (size_t)b * width, hpitch, width, (size_t)N,
                                       cudaMemcpyHostToDevice, cp.copy));
        CFD_CUDA(cudaEventRecord(cp.in[b & 1], cp.copy));
        return CFD_OK;
    };
    CFD_TRY(bring_in(0));
    if (n_blocks > 1) CFD_TRY(bring_in(1));
    for (int b = 0; b < n_blocks; ++b) {
        CFD_CUDA(cudaStreamWaitEvent(stream, cp.in[b & 1], 0));
        cfd_block D = X;
        D.ptr = dbuf[b & 1];
        D.ld = n_b;
        D.n_cols = n_b;
        CFD_TRY(filter_impl_opts(H, lmin, lmax, lam_l, lam_r, n_p, D, n_b, 0, 0, 0, 0, work, fws,
                                 moments ? moments + (int64_t)b * n_b * 2 * n_p : nullptr, stream, 0, 0, arith, 0,
                                 -1));
        CFD_CUDA(cudaEventRecord(cp.done[b & 1], stream));
        // write block b back, then reuse its buffer for block b + 2
        CFD_CUDA(cudaStreamWaitEvent(cp.copy, cp.done[b & 1], 0));
        if (blocked && CFD_HOST_BLOCKED_KERNEL && host_dev)
            CFD_TRY(copy_rows(dbuf[b & 1], (int64_t)width, host_dev + (size_t)b * block_bytes, (int64_t)width, N, width,
                              cp.copy));
        else if (blocked)
            CFD_CUDA(cudaMemcpyAsync(host + (size_t)b * block_bytes, dbuf[b & 1], block_bytes, cudaMemcpyDeviceToHost,
                                     cp.copy));
        else if (host_dev)
            CFD_TRY(copy_rows(dbuf[b & 1], (int64_t)width, host_dev + (size_t)b * width, (int64_t)hpitch, N, width,
                              cp.copy));
        else
            CFD_CUDA(cudaMemcpy2DAsync(host + (size_t)b * width, hpitch, dbuf[b & 1], width, width, (size_t)N,
                                       cudaMemcpyDeviceToHost, cp.copy));
        if (b + 2 < n_blocks) CFD_TRY(bring_in(b + 2));
    }
    // later work on `stream` sees the whole search space written back
    CFD_CUDA(cudaEventRecord(cp.out, cp.copy));
    CFD_CUDA(cudaStreamWaitEvent(stream, cp.out, 0));
    return CFD_OK;
}

extern "C" cfd_status cfd_filter_host(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                                      int n_p, cfd_block X, int n_b, void *work, size_t work_bytes, double *moments,
                                      cudaStream_t stream) {
    clear_error();
    return filter_host_impl(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, work, work_bytes, moments, ARITH_NATIVE, false,
                            stream);
}

extern "C" cfd_status cfd_filter_host_ex(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                                         int n_p, cfd_block X, int n_b, void *work, size_t work_bytes,
                                         double *moments, const cfd_filter_opts *opts, cudaStream_t stream) {
    clear_error();
    if (opts && (opts->vpt || opts->grid_cap || opts->persistent || opts->staged || opts->gather ||
                 opts->fixed_chunk || opts->graph || opts->footprint))
        return fail(CFD_ERR_ARG, "cfd_filter_host_ex takes only the arith option");
    return filter_host_impl(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, work, work_bytes, moments,
                            opts ? opts->arith : ARITH_NATIVE, false, stream);
}

extern "C" cfd_status cfd_filter_host_blocked(const cfd_matrix *H, double lmin, double lmax, double lam_l,
                                              double lam_r, int n_p, cfd_block X, int n_b, void *work,
                                              size_t work_bytes, double *moments, const cfd_filter_opts *opts,
                                              cudaStream_t stream) {
    clear_error();
    if (opts && (opts->vpt || opts->grid_cap || opts->persistent || opts->staged || opts->gather ||
                 opts->fixed_chunk || opts->graph || opts->footprint))
        return fail(CFD_ERR_ARG, "cfd_filter_host_blocked takes only the arith option");
    return filter_host_impl(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, work, work_bytes, moments,
                            opts ? opts->arith : ARITH_NATIVE, true, stream);
}
