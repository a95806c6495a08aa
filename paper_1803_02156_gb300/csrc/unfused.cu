// Unfused ChebFD filter: the same recurrence as the fused chebfd_op, built
// from a minimum set of separate standard calls, one SpMMV and BLAS-1
// operations (axpby, dot) per step.  This is the "SpMMV + BLAS1" chain the
// paper compares its fused kernel against (Sect. 4, Fig. 2, "GHOST-nofuse").
// It exists for the fusion ablation: every kernel is as good as this library
// makes it (the SpMMV is the library's own SELL gather kernel), so the
// difference in time against cfd_filter is what the fusion saves.
//
// Per general step p (U = V_cur, W = V_prev, Y a third block):
//   Y = H U                      SpMMV
//   W = 2 alpha Y - W            axpby
//   W = W - 2 alpha beta U       axpy
//   X = X + g_p c_p W            axpy (weight read from device memory)
//   <U, U>, Re <W, U>            two dots (per-CTA partials + fixed-order fold)
// Block-vector traffic 14 N n_b s bytes per step instead of the fused 5.

#include <algorithm>

#include "filter.cuh"
#include "step_kernels.cuh"

namespace cfd {

namespace {

constexpr int BL_THREADS = 256;
constexpr int DOT_MAX_GRID = 1216;   // 8 CTAs x 152 SMs

// y = a x + b y over an n_rows x nb block (real scalars; a scalar whose
// device pointer is set is read from device memory, where the filter weights
// live).
template <typename T>
__global__ void __launch_bounds__(BL_THREADS)
k_axpby(int64_t n_rows, int nb, double a, const double *a_dev, const cplx_t<T> *x, int64_t ldx, double b,
        const double *b_dev, cplx_t<T> *y, int64_t ldy) {
    const T aa = (T)(a_dev ? __ldg(a_dev) : a), bb = (T)(b_dev ? __ldg(b_dev) : b);
    const int64_t n = n_rows * nb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / nb;
        const int j = (int)(e - i * nb);
        const cplx_t<T> xv = x[i * ldx + j];
        cplx_t<T> yv = y[i * ldy + j];
        yv.x = fma(aa, xv.x, bb * yv.x);
        yv.y = fma(aa, xv.y, bb * yv.y);
        y[i * ldy + j] = yv;
    }
}

// Per-CTA partial sums of Re <x_j, y_j> = sum_i Re(conj(x_ij) y_ij) for the
// nb columns; thread t keeps column t % nb (nb divides the CTA size).
template <typename T>
__global__ void __launch_bounds__(BL_THREADS)
k_dot_part(int64_t n_rows, int nb, const cplx_t<T> *x, int64_t ldx, const cplx_t<T> *y, int64_t ldy,
           double *partial) {
    __shared__ double red[BL_THREADS];
    const int j = threadIdx.x % nb;
    const int64_t rows_per_cta = BL_THREADS / nb;
    MomentAcc<T> s;
    for (int64_t i = blockIdx.x * rows_per_cta + threadIdx.x / nb; i < n_rows;
         i += (int64_t)gridDim.x * rows_per_cta) {
        const cplx_t<T> xv = x[i * ldx + j], yv = y[i * ldy + j];
        s.add2(xv.x, yv.x, xv.y, yv.y);
    }
    red[threadIdx.x] = s.value();
    __syncthreads();
    if (threadIdx.x < nb) {
        double t = 0.0;
        for (int k = threadIdx.x; k < BL_THREADS; k += nb) t += red[k];
        partial[(int64_t)blockIdx.x * nb + threadIdx.x] = t;
    }
}

// out[j * stride] = sum over CTAs of partial[cta][j], in a fixed order.
__global__ void k_dot_fold(const double *partial, int n_cta, int nb, double *out, int stride) {
    const int j = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < n_cta; b += 32) s += partial[(int64_t)b * nb + j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) out[(int64_t)j * stride] = s;
}

int blas_grid(int64_t n) { return (int)std::min<int64_t>((n + BL_THREADS - 1) / BL_THREADS, 152 * 16); }

template <typename T>
cfd_status axpby(int64_t n_rows, int nb, double a, const double *a_dev, const cplx_t<T> *x, int64_t ldx, double b,
                 const double *b_dev, cplx_t<T> *y, int64_t ldy, cudaStream_t s) {
    k_axpby<T><<<blas_grid(n_rows * nb), BL_THREADS, 0, s>>>(n_rows, nb, a, a_dev, x, ldx, b, b_dev, y, ldy);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

template <typename T>
cfd_status dot(int64_t n_rows, int nb, const cplx_t<T> *x, int64_t ldx, const cplx_t<T> *y, int64_t ldy,
               double *partial, double *out, int stride, cudaStream_t s) {
    const int64_t rows_per_cta = BL_THREADS / nb;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n_rows + rows_per_cta - 1) / rows_per_cta,
                                                                 DOT_MAX_GRID));
    k_dot_part<T><<<grid, BL_THREADS, 0, s>>>(n_rows, nb, x, ldx, y, ldy, partial);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    k_dot_fold<<<nb, 32, 0, s>>>(partial, grid, nb, out, stride);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

struct UnfusedScratch {
    FilterScratch f;
    void *y;
    double *dot_partial;
};

size_t unfused_workspace(int64_t N, int n_b, int n_p, int prec_H, int prec_X) {
    size_t sH = prec_H == CFD_C128 ? 16 : 8;
    return round_up(filter_workspace(N, 0, n_b, n_p, prec_H, prec_X) + (size_t)N * n_b * sH + 256 +
                        (size_t)DOT_MAX_GRID * n_b * sizeof(double) + 256,
                    256);
}

template <typename T>
cfd_status run_unfused(const cfd_matrix *H, double alpha, double beta, int n_p, int n_b, const cfd_block &X,
                       const UnfusedScratch &ws, double *moments, cudaStream_t stream) {
    using C = cplx_t<T>;
    const bool mixed = (X.prec != H->prec);
    const int64_t N = H->n_rows;
    // SpMMV Y = H vin: the library's SELL gather kernel as a plain SpMMV
    StepArgs<T> A;
    A.H = sell_view<T>(H);
    A.gc = ws.f.gc;
    A.partial = ws.f.partial;
    A.ticket = ws.f.ticket;
    A.a = 1.0;
    A.beta = 0.0;
    A.p = 1;
    A.dots = nullptr;
    A.x = nullptr;
    A.ldx = 0;
    A.status = ws.f.status;
    auto spmmv = [&](const C *vin, int64_t ldin, C *y) {
        A.vin = vin; A.ldin = ldin; A.w = y; A.ldw = n_b;
        return launch_step<T>(STEP_FIRST, n_b, default_vpt(H->prec, n_b), A, STEP_MAX_GRID, stream);
    };
    C *va = static_cast<C *>(ws.f.va), *vb = static_cast<C *>(ws.f.vb), *y = static_cast<C *>(ws.y);
    const size_t sX = X.prec == CFD_C128 ? 16 : 8;
    const int n_blocks = X.n_cols / n_b;
    for (int b = 0; b < n_blocks; ++b) {
        char *xsrc = static_cast<char *>(X.ptr) + (size_t)b * n_b * sX;
        C *xb;
        int64_t ldx;
        if (mixed) {
            CFD_TRY(launch_narrow(reinterpret_cast<const double2 *>(xsrc), X.ld, static_cast<float2 *>(ws.f.xn),
                                  n_b, N, n_b, stream));
            xb = static_cast<C *>(ws.f.xn);
            ldx = n_b;
        } else {
            xb = reinterpret_cast<C *>(xsrc);
            ldx = X.ld;
        }
        double *raw = ws.f.raw;
        // step 1: V1 = alpha H X - alpha beta X
        CFD_TRY(spmmv(xb, ldx, va));
        CFD_TRY(axpby<T>(N, n_b, -alpha * beta, nullptr, xb, ldx, alpha, nullptr, va, n_b, stream));
        if (moments) {
            CFD_TRY(dot<T>(N, n_b, xb, ldx, xb, ldx, ws.dot_partial, raw, 2, stream));
            CFD_TRY(dot<T>(N, n_b, va, n_b, xb, ldx, ws.dot_partial, raw + 1, 2, stream));
        }
        // step 2: V2 = 2 alpha H V1 - 2 alpha beta V1 - X; X = g0 c0 X + g1 c1 V1 + g2 c2 V2
        CFD_TRY(spmmv(va, n_b, vb));
        CFD_TRY(axpby<T>(N, n_b, -2.0 * alpha * beta, nullptr, va, n_b, 2.0 * alpha, nullptr, vb, n_b, stream));
        CFD_TRY(axpby<T>(N, n_b, -1.0, nullptr, xb, ldx, 1.0, nullptr, vb, n_b, stream));
        if (moments) {
            CFD_TRY(dot<T>(N, n_b, va, n_b, va, n_b, ws.dot_partial, raw + 2 * n_b, 2, stream));
            CFD_TRY(dot<T>(N, n_b, vb, n_b, va, n_b, ws.dot_partial, raw + 2 * n_b + 1, 2, stream));
        }
        // X = g1 c1 V1 + g0 c0 X, then X += g2 c2 V2
        CFD_TRY(axpby<T>(N, n_b, 0.0, ws.f.gc + 1, va, n_b, 0.0, ws.f.gc, xb, ldx, stream));
        CFD_TRY(axpby<T>(N, n_b, 0.0, ws.f.gc + 2, vb, n_b, 1.0, nullptr, xb, ldx, stream));
        // steps 3..n_p
        for (int p = 3; p <= n_p; ++p) {
            C *cur = (p & 1) ? vb : va;
            C *prev = (p & 1) ? va : vb;
            CFD_TRY(spmmv(cur, n_b, y));
            CFD_TRY(axpby<T>(N, n_b, 2.0 * alpha, nullptr, y, n_b, -1.0, nullptr, prev, n_b, stream));
            CFD_TRY(axpby<T>(N, n_b, -2.0 * alpha * beta, nullptr, cur, n_b, 1.0, nullptr, prev, n_b, stream));
            CFD_TRY(axpby<T>(N, n_b, 0.0, ws.f.gc + p, prev, n_b, 1.0, nullptr, xb, ldx, stream));
            if (moments) {
                double *d = raw + (int64_t)(p - 1) * 2 * n_b;
                CFD_TRY(dot<T>(N, n_b, cur, n_b, cur, n_b, ws.dot_partial, d, 2, stream));
                CFD_TRY(dot<T>(N, n_b, prev, n_b, cur, n_b, ws.dot_partial, d + 1, 2, stream));
            }
        }
        if (moments)
            CFD_TRY(launch_moments(raw, n_p, n_b, moments + (int64_t)b * n_b * 2 * n_p, 2 * n_p, ws.f.status, stream));
        if (mixed)
            CFD_TRY(launch_widen(static_cast<const float2 *>(ws.f.xn), n_b, reinterpret_cast<double2 *>(xsrc),
                                 X.ld, N, n_b, stream));
    }
    return CFD_OK;
}

}  // namespace

}  // namespace cfd

using namespace cfd;

extern "C" size_t cfd_filter_unfused_workspace(int64_t N, int n_s, int n_b, int n_p, int prec_H, int prec_X) {
    (void)n_s;
    if (N < 1 || n_b < 1 || n_p < 1) return 0;
    return unfused_workspace(N, n_b, n_p, prec_H & 0xff, prec_X & 0xff);
}

extern "C" cfd_status cfd_filter_unfused(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                                         int n_p, cfd_block X, int n_b, void *work, size_t work_bytes,
                                         double *moments, cudaStream_t stream) {
    clear_error();
    CFD_TRY(check_matrix(H));
    CFD_TRY(validate_block(X, H->n_rows));
    if (n_p < 2) return fail(CFD_ERR_ARG, "n_p=%d < 2", n_p);
    if (n_b != 8 && n_b != 16 && n_b != 32 && n_b != 64) return fail(CFD_ERR_ARG, "n_b=%d not in {8,16,32,64}", n_b);
    if (X.n_cols % n_b) return fail(CFD_ERR_ARG, "n_b=%d does not divide n_s=%d", n_b, X.n_cols);
    if (!(X.prec == H->prec || (H->prec == CFD_C64 && X.prec == CFD_C128)))
        return fail(CFD_ERR_ARG, "unsupported precision pair (matrix %d, block %d)", H->prec, X.prec);
    if (!(lmin < lmax) || !(lmin <= lam_l && lam_l < lam_r && lam_r <= lmax))
        return fail(CFD_ERR_ARG, "need lmin <= lam_l < lam_r <= lmax (got %g %g %g %g)", lmin, lam_l, lam_r, lmax);
    if (!work) return fail(CFD_ERR_ARG, "work is NULL");
    if (!aligned16(work)) return fail(CFD_ERR_ARG, "work must be 16-byte aligned");
    const size_t need = unfused_workspace(H->n_rows, n_b, n_p, H->prec, X.prec);
    if (work_bytes < need) return fail(CFD_ERR_OOM, "unfused filter workspace %zu < %zu bytes", work_bytes, need);
    const size_t sH = H->prec == CFD_C128 ? 16 : 8;
    Carve c(work, work_bytes);
    UnfusedScratch ws;
    ws.f.status = c.take<int>(64);
    ws.f.va = c.take<char>((size_t)H->n_rows * n_b * sH);
    ws.f.vb = c.take<char>((size_t)H->n_rows * n_b * sH);
    ws.f.xn = (H->prec != X.prec) ? c.take<char>((size_t)H->n_rows * n_b * 8) : nullptr;
    ws.f.gc = c.take<double>((size_t)n_p + 1);
    ws.f.raw = c.take<double>((size_t)n_p * n_b * 2);
    ws.f.partial = c.take<double>((size_t)STEP_MAX_GRID * 2 * n_b);
    ws.f.ticket = c.take<unsigned>(64);
    ws.f.grid_cap = STEP_MAX_GRID;
    ws.y = c.take<char>((size_t)H->n_rows * n_b * sH);
    ws.dot_partial = c.take<double>((size_t)DOT_MAX_GRID * n_b);
    if (c.off > work_bytes) return fail(CFD_ERR_INTERNAL, "unfused workspace carve overflow");
    CFD_CUDA(cudaMemsetAsync(ws.f.ticket, 0, sizeof(unsigned), stream));
    CFD_CUDA(cudaMemsetAsync(ws.f.status, 0, sizeof(int), stream));
    const double alpha = 2.0 / (lmax - lmin), beta = 0.5 * (lmax + lmin);
    CFD_TRY(launch_filter_coeffs(alpha, beta, lam_l, lam_r, n_p, ws.f.gc, stream));
    if (H->prec == CFD_C128) return run_unfused<double>(H, alpha, beta, n_p, n_b, X, ws, moments, stream);
    return run_unfused<float>(H, alpha, beta, n_p, n_b, X, ws, moments, stream);
}
