// The ChebFD polynomial filter (Algorithm 1, blocked as Algorithm 2): one
// fused SELL-C-sigma SpMMV kernel per recurrence step (the paper's
// chebfd_op), weights table, moment finalisation, precision conversion.
#include <algorithm>
#include <cstring>
#include <cooperative_groups.h>
#include <type_traits>

#include "filter.cuh"

namespace cg = cooperative_groups;

namespace cfd {

// ------------------------------------------------------------ weights --

// g_k c_k: Chebyshev coefficient of the window indicator times the Jackson
// kernel (M = n_p + 1 moments), on the axis scaled by alpha (x - beta).
__device__ double filter_weight(double alpha, double beta, double lam_l, double lam_r, int n_p, int k) {
    const double pi = 3.141592653589793238462643383279502884;
    double xl = fmin(fmax(alpha * (lam_l - beta), -1.0), 1.0);
    double xr = fmin(fmax(alpha * (lam_r - beta), -1.0), 1.0);
    double tl = acos(xl), tr = acos(xr);
    double c = (k == 0) ? (tl - tr) / pi : 2.0 * (sin(k * tl) - sin(k * tr)) / (k * pi);
    double M = n_p + 1.0;
    double q = pi / (M + 1.0);
    double g = ((M - k + 1.0) * cos(q * k) + sin(q * k) / tan(q)) / (M + 1.0);
    return g * c;
}

// gc[k] = g_k c_k, k = 0..n_p.
__global__ void k_filter_coeffs(double alpha, double beta, double lam_l, double lam_r, int n_p,
                                double *gc) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n_p) return;
    gc[k] = filter_weight(alpha, beta, lam_l, lam_r, n_p, k);
}

// Per realisation r of a batch, from win[r] = (lmin, lmax, lam_l, lam_r):
// rc[r] = {alpha, beta, g_0 c_0, ..., g_np c_np}, stride n_p + 3.
__global__ void k_batch_coeffs(const double *win, int R, int n_p, double *rc) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t ld = n_p + 3;
    if (e >= (int64_t)R * ld) return;
    int r = (int)(e / ld), k = (int)(e % ld);
    const double *w = win + 4 * r;
    double alpha = 2.0 / (w[1] - w[0]), beta = 0.5 * (w[1] + w[0]);
    double v;
    if (k == 0) v = alpha;
    else if (k == 1) v = beta;
    else v = filter_weight(alpha, beta, w[2], w[3], n_p, k - 2);
    rc[e] = v;
}

cfd_status launch_filter_coeffs(double alpha, double beta, double lam_l, double lam_r, int n_p,
                                double *gc, cudaStream_t stream) {
    k_filter_coeffs<<<(n_p + 1 + 127) / 128, 128, 0, stream>>>(alpha, beta, lam_l, lam_r, n_p, gc);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

// One thread per row position r of the padded SELL layout (chunk r >> log2C,
// row r & (C - 1) within it): its slots k < the chunk's length sit at
// chunk_ptr + k C + row.  The canonical row index i (through perm) tells the
// diagonal slot, the one whose column is i; rows past the end have none.
// Computed in fp64 and rounded once to the storage precision.
template <typename T, bool PACK>
__global__ void k_prepare_values(SellView<T> H, int64_t n_pos, double alpha, double beta, const int32_t *chunk_rid,
                                 const double *rcoef, int64_t rcoef_ld, void *out) {
    using C = cplx_t<T>;
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_pos) return;
    const int64_t ch = r >> H.log2C;
    const int64_t base = H.chunk_ptr[ch] + (r & ((1 << H.log2C) - 1));
    const int cl = H.chunk_len[ch];
    const int len = PACK ? (cl & 0xffff) + (cl >> 16) : cl;
    const int64_t i = r < H.n_rows ? (H.perm ? (int64_t)H.perm[r] : r) : -2;   // -2 never matches a column
    if (chunk_rid) {
        const double *rc = rcoef + (int64_t)chunk_rid[ch] * rcoef_ld;
        alpha = rc[0];
        beta = rc[1];
    }
    const double a2 = 2.0 * alpha;
    for (int k = 0; k < len; ++k) {
        const int64_t s = base + ((int64_t)k << H.log2C);
        const bool diag = H.col[s] == i;
        if constexpr (PACK) {
            const double h = (double)H.pval[s];
            static_cast<T *>(out)[s] = (T)(diag ? a2 * (h - beta) : a2 * h);
        } else {
            const C h = H.val[s];
            C v;
            v.x = (T)(diag ? a2 * ((double)h.x - beta) : a2 * (double)h.x);
            v.y = (T)(a2 * (double)h.y);
            static_cast<C *>(out)[s] = v;
        }
    }
}

template <typename T>
static cfd_status prepare_values_t(const cfd_matrix *H, double alpha, double beta, const int32_t *chunk_rid,
                                   const double *rcoef, int64_t rcoef_ld, void *out, size_t out_bytes,
                                   cudaStream_t stream) {
    const SellView<T> v = sell_view<T>(H);
    const size_t bytes = (size_t)H->n_slots * (v.packed ? sizeof(T) : sizeof(cplx_t<T>));
    if (bytes > out_bytes)
        return fail(CFD_ERR_ARG, "matrix stores %lld slots, more than the filter workspace prepares (%d per row)",
                    (long long)H->n_slots, kMaxRowSlots);
    const int64_t n_pos = H->n_chunks << v.log2C;
    if (n_pos == 0) return CFD_OK;
    const unsigned grid = (unsigned)((n_pos + 255) / 256);
    if (v.packed)
        k_prepare_values<T, true><<<grid, 256, 0, stream>>>(v, n_pos, alpha, beta, chunk_rid, rcoef, rcoef_ld, out);
    else
        k_prepare_values<T, false><<<grid, 256, 0, stream>>>(v, n_pos, alpha, beta, chunk_rid, rcoef, rcoef_ld, out);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

cfd_status launch_prepare_values(const cfd_matrix *H, double alpha, double beta, const int32_t *chunk_rid,
                                 const double *rcoef, int64_t rcoef_ld, void *out, size_t out_bytes,
                                 cudaStream_t stream) {
    if (H->prec == CFD_C128)
        return prepare_values_t<double>(H, alpha, beta, chunk_rid, rcoef, rcoef_ld, out, out_bytes, stream);
    return prepare_values_t<float>(H, alpha, beta, chunk_rid, rcoef, rcoef_ld, out, out_bytes, stream);
}

// ------------------------------------------------------ step dispatch --

// The step kernels are compiled in four translation units (fp64/fp32 x
// complex/packed values, step_*.cu); these pick the one for the matrix.
template <typename T>
cfd_status launch_step(int kind, int nb, int vpt, const StepArgs<T> &A, int grid_cap, cudaStream_t s) {
    if (A.H.packed) return launch_step_p<T, true>(kind, nb, vpt, A, grid_cap, s);
    return launch_step_p<T, false>(kind, nb, vpt, A, grid_cap, s);
}

template <typename T>
cfd_status launch_persistent(int nb, int vpt, const StepArgs<T> &A, cplx_t<T> *va, cplx_t<T> *vb, cplx_t<T> *xb,
                             int64_t ldx, int n_p, int grid_cap, cudaStream_t s) {
    if (A.H.packed) return launch_persistent_p<T, true>(nb, vpt, A, va, vb, xb, ldx, n_p, grid_cap, s);
    return launch_persistent_p<T, false>(nb, vpt, A, va, vb, xb, ldx, n_p, grid_cap, s);
}

template cfd_status launch_step<double>(int, int, int, const StepArgs<double> &, int, cudaStream_t);
template cfd_status launch_step<float>(int, int, int, const StepArgs<float> &, int, cudaStream_t);

// ------------------------------------------------- moments, conversion --

// raw[p-1][j][0] = <T_{p-1}x_j, T_{p-1}x_j>, raw[p-1][j][1] = Re <T_p x_j, T_{p-1}x_j>
// -> mu[j][m] = <x_j, T_m x_j>, m = 0..2 n_p - 1 (T_k T_l = (T_{k+l} + T_{|k-l|}) / 2).
__global__ void k_moments(const double *raw, int n_p, int nb, double *mu, int64_t ld_mu) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)nb * 2 * n_p) return;
    int j = (int)(e / (2 * n_p));
    int m = (int)(e % (2 * n_p));
    double mu0 = raw[2 * j + 0], mu1 = raw[2 * j + 1];
    double v;
    if (m == 0) v = mu0;
    else if (m == 1) v = mu1;
    else {
        int p = m / 2 + 1;
        const double *d = raw + (int64_t)(p - 1) * 2 * nb + 2 * j;
        v = (m & 1) ? 2.0 * d[1] - mu1 : 2.0 * d[0] - mu0;
    }
    mu[(int64_t)j * ld_mu + m] = v;
}

// Guard on the spectral bounds: with every eigenvalue of H~ in [-1, 1],
// |mu_m| = |sum_i |v_i^H x|^2 T_m(lambda~_i)| <= mu_0 for every m; an
// eigenvalue outside makes the moments grow like cosh(m arccosh |lambda~|).
// A moment above mu_0 by more than 1% (far beyond the rounding of either
// precision), or not finite, records CFD_ERR_BOUNDS in *status.
__global__ void k_check_moments(const double *mu, int nb, int n_mom, int64_t ld_mu, int *status) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)nb * n_mom) return;
    const int j = (int)(e / n_mom), m = (int)(e % n_mom);
    const double mu0 = mu[(int64_t)j * ld_mu], v = mu[(int64_t)j * ld_mu + m];
    if (!(fabs(v) <= 1.01 * fabs(mu0)))            // also true for NaN
        atomicCAS(status, 0, (int)CFD_ERR_BOUNDS);
}

cfd_status launch_moments(const double *raw, int n_p, int nb, double *mu, int64_t ld_mu, int *status,
                          cudaStream_t stream) {
    int64_t n = (int64_t)nb * 2 * n_p;
    k_moments<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(raw, n_p, nb, mu, ld_mu);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    if (status) {
        k_check_moments<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(mu, nb, 2 * n_p, ld_mu, status);
        CFD_COUNT_LAUNCH();
        CFD_LAUNCH_CHECK();
    }
    return CFD_OK;
}

// Round a strided complex-double block to a contiguous complex-float block
// (round to nearest) or widen it back.
__global__ void k_narrow(const double2 *src, int64_t lds, float2 *dst, int64_t ldd, int64_t n_rows,
                         int nb) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_rows * nb) return;
    int64_t i = e / nb;
    int j = (int)(e % nb);
    double2 z = src[i * lds + j];
    dst[i * ldd + j] = make_float2(__double2float_rn(z.x), __double2float_rn(z.y));
}

__global__ void k_widen(const float2 *src, int64_t lds, double2 *dst, int64_t ldd, int64_t n_rows,
                        int nb) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_rows * nb) return;
    int64_t i = e / nb;
    int j = (int)(e % nb);
    float2 z = src[i * lds + j];
    dst[i * ldd + j] = make_double2((double)z.x, (double)z.y);
}

cfd_status launch_narrow(const double2 *src, int64_t lds, float2 *dst, int64_t ldd, int64_t n_rows,
                         int nb, cudaStream_t stream) {
    int64_t n = n_rows * nb;
    k_narrow<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(src, lds, dst, ldd, n_rows, nb);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

cfd_status launch_widen(const float2 *src, int64_t lds, double2 *dst, int64_t ldd, int64_t n_rows,
                        int nb, cudaStream_t stream) {
    int64_t n = n_rows * nb;
    k_widen<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(src, lds, dst, ldd, n_rows, nb);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

// ------------------------------------------------------------- driver --

// Vectors per thread: two for fp32 (one 16-byte access); for fp64 two as well
// once n_b >= 16 (the per-slot index and value loads are shared by both
// vectors, which matters on GB300's issue-limited fp64 path).
// General steps stage their matrix chunks by TMA in both precisions: the
// fp32 steps are memory-latency bound, and the fp64 steps, bound by the
// FP64 pipe, keep it busier when no index or value load sits between a
// row's gathers (1.07 ms against 1.29 ms per step on the 64x64x32 lattice
// at n_b = 32).
bool default_staged(int prec) { (void)prec; return true; }

// Gathers in flight per row in the staged steps (STEP_GATHER_ALL or groups of four).
int default_gather(int prec) { (void)prec; return 4; }

int default_vpt(int prec, int n_b) {
    if (prec == CFD_C64) return 2;
    return n_b >= 16 ? 2 : 1;
}

// Bytes of prepared values for a matrix of N rows: kMaxRowSlots complex
// values per row, rows padded to whole chunks of the largest height (128).
static size_t prep_bytes(int64_t N, int prec_H) {
    return (size_t)kMaxRowSlots * (size_t)(N + 127) * (prec_H == CFD_C128 ? 16 : 8);
}

size_t filter_workspace(int64_t N, int n_s, int n_b, int n_p, int prec_H, int prec_X) {
    (void)n_s;
    size_t sH = prec_H == CFD_C128 ? 16 : 8;
    Carve c(nullptr, 0);
    c.take<int>(64);                                          // status word
    c.take<char>((size_t)N * n_b * sH);                      // V_a
    c.take<char>((size_t)N * n_b * sH);                      // V_b
    if (prec_H != prec_X) c.take<char>((size_t)N * n_b * 8); // narrowed X block
    c.take<char>(prep_bytes(N, prec_H));                      // prepared matrix values
    c.take<double>((size_t)n_p + 1);                          // weights
    c.take<double>((size_t)n_p * n_b * 2);                    // raw dots
    c.take<double>((size_t)STEP_MAX_GRID * 2 * n_b);       // CTA partials
    c.take<unsigned>(64);                                     // ticket
    if (n_b == 32) c.take<char>(footprint_bytes(N));          // chunk footprints
    return round_up(c.off, 256);
}

cfd_status validate_block(const cfd_block &X, int64_t n_rows) {
    if (!X.ptr) return fail(CFD_ERR_ARG, "block pointer is NULL");
    if (X.n_rows != n_rows) return fail(CFD_ERR_ARG, "block has %lld rows, matrix %lld",
                                        (long long)X.n_rows, (long long)n_rows);
    if (X.n_cols < 1 || X.ld < X.n_cols) return fail(CFD_ERR_ARG, "block ld/n_cols invalid");
    if (X.prec != CFD_C128 && X.prec != CFD_C64) return fail(CFD_ERR_ARG, "block precision invalid");
    size_t s = X.prec == CFD_C128 ? 16 : 8;
    if (!aligned16(X.ptr) || ((size_t)X.ld * s) % 16) return fail(CFD_ERR_ARG, "block must be 16-byte aligned with ld * scalar a multiple of 16 bytes");
    return CFD_OK;
}

template <typename T>
static cfd_status run_filter(const cfd_matrix *H, const FilterPlan &P, const cfd_block &X, const FilterScratch &ws,
                             double *moments, cudaStream_t stream) {
    using C = cplx_t<T>;
    const bool mixed = (X.prec != H->prec);
    const int n_b = P.n_b, n_p = P.n_p, vpt = P.vpt;
    StepArgs<T> A;
    A.H = sell_view<T>(H);
    A.gc = ws.gc;
    A.partial = ws.partial;
    A.ticket = ws.ticket;
    A.chunk_rid = P.chunk_rid;
    A.rcoef = P.rcoef;
    A.rcoef_ld = P.rcoef_ld;
    A.beta = P.beta;
    A.staged = P.staged;
    A.gather = P.gather;
    A.fixed_chunk = P.fixed_chunk;
    A.status = ws.status;
    const bool dw = std::is_same<T, double>::value && P.arith == ARITH_DW;
    // persistent general steps with the staged chunk loop (packed values);
    // the unstaged persistent kernel runs all steps in one launch
    const bool pstaged = P.persistent && P.staged && A.H.packed;
    if (dw) {
        // double-word general steps: 2 alpha (H - beta) as {hi, lo} float pairs
        CFD_TRY(launch_prepare_values_dw(H, P.alpha, P.beta, P.chunk_rid, P.rcoef, P.rcoef_ld, ws.prep,
                                         ws.prep_bytes, stream));
        A.prep_val = ws.prep;
    } else if (P.staged && (!P.persistent || pstaged)) {
        // the staged general steps read 2 alpha (H - beta), prepared once per call
        CFD_TRY(launch_prepare_values(H, P.alpha, P.beta, P.chunk_rid, P.rcoef, P.rcoef_ld, ws.prep, ws.prep_bytes,
                                      stream));
        A.prep_val = ws.prep;
    }
    // footprint-staged general steps (complex float, or double-word), with
    // the chunks' footprints found once per call
    FpView F;
    if (P.footprint >= 0 && !P.persistent && P.staged >= 1 && ws.fp && (dw || std::is_same<T, float>::value)) {
        int fmax = footprint_rows_cap(H, n_b, vpt, dw, P.footprint > 0);
        if (P.footprint > 0) fmax = std::min(fmax, P.footprint);
        if (fmax > 0) CFD_TRY(launch_footprint(H, P.chunk_rid, fmax, ws.fp, ws.fp_bytes, &F, stream));
    }
    C *va = static_cast<C *>(ws.va), *vb = static_cast<C *>(ws.vb);
    const int n_blocks = X.n_cols / n_b;
    const size_t sX = X.prec == CFD_C128 ? 16 : 8;
    for (int b = 0; b < n_blocks; ++b) {
        C *xb;
        int64_t ldx;
        char *xsrc = static_cast<char *>(X.ptr) + (size_t)b * n_b * sX;
        if (mixed) {
            CFD_TRY(launch_narrow(reinterpret_cast<const double2 *>(xsrc), X.ld, static_cast<float2 *>(ws.xn),
                                  n_b, X.n_rows, n_b, stream));
            xb = static_cast<C *>(ws.xn);
            ldx = n_b;
        } else {
            xb = reinterpret_cast<C *>(xsrc);
            ldx = X.ld;
        }
        if (pstaged) {
            // steps 1 and 2 as single launches, then steps 3..n_p in one
            // cooperative launch
            A.dots = nullptr;
            A.vin = xb; A.ldin = ldx; A.w = va; A.ldw = n_b; A.x = nullptr; A.ldx = 0; A.a = P.alpha; A.p = 1;
            CFD_TRY(launch_step<T>(STEP_FIRST, n_b, vpt, A, P.grid_cap, stream));
            A.vin = va; A.ldin = n_b; A.w = vb; A.ldw = n_b; A.x = xb; A.ldx = ldx; A.a = 2.0 * P.alpha; A.p = 2;
            CFD_TRY(launch_step<T>(STEP_SECOND, n_b, vpt, A, P.grid_cap, stream));
            if (n_p >= 3) CFD_TRY(launch_persistent_staged<T>(n_b, vpt, A, va, vb, n_p, P.grid_cap, stream));
        } else if (P.persistent) {
            // all n_p steps of this block in one cooperative launch
            A.a = P.alpha;
            A.dots = nullptr;
            CFD_TRY(launch_persistent<T>(n_b, vpt, A, va, vb, xb, ldx, n_p, P.grid_cap, stream));
        } else {
            // double-word steps (n_p >= 3): X_b to double-word form first; the
            // last general step writes it back as complex double
            const bool dws = dw && n_p >= 3;
            if (dws) CFD_TRY(launch_dw_convert(xb, ldx, X.n_rows, n_b, true, stream));
            // step 1: V1 = H~ X_b
            A.vin = xb; A.ldin = ldx; A.w = va; A.ldw = n_b; A.x = nullptr; A.ldx = 0;
            A.a = P.alpha; A.p = 1; A.dots = moments ? ws.raw : nullptr;
            if constexpr (std::is_same<T, double>::value) {
                if (dws) CFD_TRY(launch_step_dw(STEP_FIRST, n_b, vpt, A, false, P.grid_cap, stream));
            }
            if (!dws) CFD_TRY(launch_step<T>(STEP_FIRST, n_b, vpt, A, P.grid_cap, stream));
            // step 2: V2 = 2 H~ V1 - X_b, X_b = gc0 X_b + gc1 V1 + gc2 V2
            A.vin = va; A.ldin = n_b; A.w = vb; A.ldw = n_b; A.x = xb; A.ldx = ldx;
            A.a = 2.0 * P.alpha; A.p = 2; A.dots = moments ? ws.raw + 2 * n_b : nullptr;
            if constexpr (std::is_same<T, double>::value) {
                if (dws) CFD_TRY(launch_step_dw(STEP_SECOND, n_b, vpt, A, false, P.grid_cap, stream));
            }
            if (!dws) CFD_TRY(launch_step<T>(STEP_SECOND, n_b, vpt, A, P.grid_cap, stream));
            // steps 3..n_p: swap(V_prev, V_cur); V_prev = 2 H~ V_cur - V_prev; X_b += gc_p V_prev
            for (int p = 3; p <= n_p; ++p) {
                C *cur = (p & 1) ? vb : va;
                C *prev = (p & 1) ? va : vb;
                A.vin = cur; A.ldin = n_b; A.w = prev; A.ldw = n_b; A.p = p;
                A.dots = moments ? ws.raw + (int64_t)(p - 1) * 2 * n_b : nullptr;
                if constexpr (std::is_same<T, double>::value) {
                    if (dw && F.fmax > 0) {
                        CFD_TRY(launch_step_fp_dw(A, F, n_b, vpt, p == n_p, P.grid_cap, stream));
                        continue;
                    }
                    if (dw) {
                        CFD_TRY(launch_step_dw(STEP_GENERAL, n_b, vpt, A, p == n_p, P.grid_cap, stream));
                        continue;
                    }
                } else {
                    if (F.fmax > 0) {
                        CFD_TRY(launch_step_fp(A, F, n_b, vpt, P.grid_cap, stream));
                        continue;
                    }
                }
                CFD_TRY(launch_step<T>(STEP_GENERAL, n_b, vpt, A, P.grid_cap, stream));
            }
            if (moments)
                CFD_TRY(launch_moments(ws.raw, n_p, n_b, moments + (int64_t)b * n_b * 2 * n_p, 2 * n_p, ws.status,
                                       stream));
        }
        if (mixed)
            CFD_TRY(launch_widen(static_cast<const float2 *>(ws.xn), n_b, reinterpret_cast<double2 *>(xsrc),
                                 X.ld, X.n_rows, n_b, stream));
    }
    return CFD_OK;
}

cfd_status check_filter_args(const cfd_matrix *H, int n_p, const cfd_block &X, int n_b, int vpt) {
    CFD_TRY(check_matrix(H));
    CFD_TRY(validate_block(X, H->n_rows));
    if (n_p < 2) return fail(CFD_ERR_ARG, "n_p=%d < 2", n_p);
    if (n_b != 8 && n_b != 16 && n_b != 32 && n_b != 64) return fail(CFD_ERR_ARG, "n_b=%d not in {8,16,32,64}", n_b);
    if (X.n_cols % n_b) return fail(CFD_ERR_ARG, "n_b=%d does not divide n_s=%d", n_b, X.n_cols);
    if (!(X.prec == H->prec || (H->prec == CFD_C64 && X.prec == CFD_C128)))
        return fail(CFD_ERR_ARG, "unsupported precision pair (matrix %d, block %d)", H->prec, X.prec);
    if (vpt < 0 || vpt > 2 || (vpt == 1 && n_b > 32)) return fail(CFD_ERR_ARG, "vpt=%d invalid for n_b=%d", vpt, n_b);
    return CFD_OK;
}

static FilterScratch carve_filter(const cfd_matrix *H, const cfd_block &X, int n_b, int n_p, void *work,
                                  size_t work_bytes) {
    size_t sH = H->prec == CFD_C128 ? 16 : 8;
    Carve c(work, work_bytes);
    FilterScratch ws;
    ws.status = c.take<int>(64);
    ws.va = c.take<char>((size_t)H->n_rows * n_b * sH);
    ws.vb = c.take<char>((size_t)H->n_rows * n_b * sH);
    ws.xn = (H->prec != X.prec) ? c.take<char>((size_t)H->n_rows * n_b * 8) : nullptr;
    ws.prep_bytes = prep_bytes(H->n_rows, H->prec);
    ws.prep = c.take<char>(ws.prep_bytes);
    ws.gc = c.take<double>((size_t)n_p + 1);
    ws.raw = c.take<double>((size_t)n_p * n_b * 2);
    ws.partial = c.take<double>((size_t)STEP_MAX_GRID * 2 * n_b);
    ws.ticket = c.take<unsigned>(64);
    ws.fp_bytes = n_b == 32 ? footprint_bytes(H->n_rows) : 0;
    ws.fp = ws.fp_bytes ? c.take<char>(ws.fp_bytes) : nullptr;
    ws.grid_cap = STEP_MAX_GRID;
    return ws;
}

cfd_status filter_impl_opts(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r, int n_p,
                            const cfd_block &X, int n_b, int vpt, int grid_cap, int persistent, int staged,
                            void *work, size_t work_bytes, double *moments, cudaStream_t stream, int gather,
                            int fixed_chunk, int arith, int graph, int footprint) {
    CFD_TRY(check_filter_args(H, n_p, X, n_b, vpt));
    if (arith != ARITH_NATIVE && arith != ARITH_DW) return fail(CFD_ERR_ARG, "arith=%d not in {0, 1}", arith);
    if (arith == ARITH_DW) {
        if (H->prec != CFD_C128 || X.prec != CFD_C128)
            return fail(CFD_ERR_ARG, "double-word arithmetic is for complex-double matrices and blocks");
        if (!(H->flags & CFD_MATRIX_PACKED))
            return fail(CFD_ERR_ARG, "double-word arithmetic needs packed matrix values (CFD_PACK_RI)");
        if (persistent) return fail(CFD_ERR_ARG, "the persistent filter has no double-word variant");
    }
    if (graph != 0 && graph != 1) return fail(CFD_ERR_ARG, "graph=%d not in {0, 1}", graph);
    if (!(lmin < lmax) || !(lmin <= lam_l && lam_l < lam_r && lam_r <= lmax))
        return fail(CFD_ERR_ARG, "need lmin <= lam_l < lam_r <= lmax (got %g %g %g %g)", lmin, lam_l, lam_r, lmax);
    if (persistent && moments) return fail(CFD_ERR_ARG, "the persistent filter records no moments");
    if (!work) return fail(CFD_ERR_ARG, "work is NULL");
    size_t need = filter_workspace(H->n_rows, X.n_cols, n_b, n_p, H->prec, X.prec);
    if (work_bytes < need) return fail(CFD_ERR_OOM, "filter workspace %zu < %zu bytes", work_bytes, need);
    if (!aligned16(work)) return fail(CFD_ERR_ARG, "work must be 16-byte aligned");
    FilterScratch ws = carve_filter(H, X, n_b, n_p, work, work_bytes);
    FilterPlan P;
    P.n_b = n_b;
    P.n_p = n_p;
    P.vpt = vpt > 0 ? vpt : default_vpt(H->prec, n_b);
    P.grid_cap = std::min(grid_cap > 0 ? grid_cap : STEP_MAX_GRID, STEP_MAX_GRID);
    P.persistent = persistent != 0;
    P.staged = staged > 0 ? staged : (staged < 0 ? 0 : (int)default_staged(H->prec));
    P.gather = gather > 0 ? gather : default_gather(H->prec);
    P.fixed_chunk = fixed_chunk;
    P.arith = arith;
    P.footprint = footprint;
    P.alpha = 2.0 / (lmax - lmin);
    P.beta = 0.5 * (lmax + lmin);
    auto enqueue = [&](cudaStream_t s) -> cfd_status {
        CFD_CUDA(cudaMemsetAsync(ws.ticket, 0, sizeof(unsigned), s));
        CFD_CUDA(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
        CFD_TRY(launch_filter_coeffs(P.alpha, P.beta, lam_l, lam_r, n_p, ws.gc, s));
        if (H->prec == CFD_C128) return run_filter<double>(H, P, X, ws, moments, s);
        return run_filter<float>(H, P, X, ws, moments, s);
    };
    if (!graph) return enqueue(stream);
    // every argument that shapes the launch sequence or its parameters
    struct Key {
        cfd_matrix H;
        cfd_block X;
        double lmin, lmax, lam_l, lam_r;
        const void *work, *moments;
        size_t work_bytes;
        int n_p, n_b, vpt, grid_cap, persistent, staged, gather, fixed_chunk, arith, footprint, kind;
    } key;
    std::memset(&key, 0, sizeof(key));
    key.H = *H;
    key.X = X;
    key.lmin = lmin; key.lmax = lmax; key.lam_l = lam_l; key.lam_r = lam_r;
    key.work = work; key.moments = moments; key.work_bytes = work_bytes;
    key.n_p = n_p; key.n_b = n_b; key.vpt = P.vpt; key.grid_cap = P.grid_cap; key.persistent = persistent;
    key.staged = P.staged; key.gather = P.gather; key.fixed_chunk = fixed_chunk; key.arith = arith; key.footprint = footprint;
    key.kind = 1;
    return run_as_graph(&key, sizeof(key), stream, enqueue);
}

cfd_status filter_impl(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                       int n_p, const cfd_block &X, int n_b, int vpt, int grid_cap, void *work,
                       size_t work_bytes, double *moments, cudaStream_t stream) {
    return filter_impl_opts(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, vpt, grid_cap, 0, 0, work, work_bytes,
                            moments, stream, 0);
}

// Chebyshev moments of the columns of R without the filter accumulation
// (Algorithm 1 without line 12, the kernel polynomial method): the same fused
// steps with no X read or written, R left unchanged.
cfd_status kpm_impl(const cfd_matrix *H, double lmin, double lmax, int n_p, const cfd_block &R, int n_b,
                    void *work, size_t work_bytes, double *moments, cudaStream_t stream) {
    CFD_TRY(check_filter_args(H, n_p, R, n_b, 0));
    if (R.prec != H->prec) return fail(CFD_ERR_ARG, "moments need the block in the matrix precision");
    if (!(lmin < lmax)) return fail(CFD_ERR_ARG, "need lmin < lmax");
    if (!moments || !work) return fail(CFD_ERR_ARG, "moments or work is NULL");
    size_t need = filter_workspace(H->n_rows, R.n_cols, n_b, n_p, H->prec, R.prec);
    if (work_bytes < need) return fail(CFD_ERR_OOM, "workspace %zu < %zu bytes", work_bytes, need);
    FilterScratch ws = carve_filter(H, R, n_b, n_p, work, work_bytes);
    CFD_CUDA(cudaMemsetAsync(ws.ticket, 0, sizeof(unsigned), stream));
    CFD_CUDA(cudaMemsetAsync(ws.status, 0, sizeof(int), stream));
    const double alpha = 2.0 / (lmax - lmin), beta = 0.5 * (lmax + lmin);
    const int vpt = default_vpt(H->prec, n_b);
    const size_t s = H->prec == CFD_C128 ? 16 : 8;
    CFD_TRY(launch_filter_coeffs(alpha, beta, lmin, lmax, n_p, ws.gc, stream));   // weights unused
    const bool staged = default_staged(H->prec);
    if (staged)
        CFD_TRY(launch_prepare_values(H, alpha, beta, nullptr, nullptr, 0, ws.prep, ws.prep_bytes, stream));
    for (int b = 0; b < R.n_cols / n_b; ++b) {
        const void *rb = static_cast<const char *>(R.ptr) + (size_t)b * n_b * s;
        double *mu = moments + (int64_t)b * n_b * 2 * n_p;
        if (H->prec == CFD_C128) {
            StepArgs<double> A;
            A.H = sell_view<double>(H);
            A.gc = ws.gc; A.partial = ws.partial; A.ticket = ws.ticket; A.status = ws.status; A.beta = beta;
            A.staged = staged;
            A.gather = default_gather(H->prec);
            A.prep_val = staged ? ws.prep : nullptr;
            double2 *va = static_cast<double2 *>(ws.va), *vb = static_cast<double2 *>(ws.vb);
            A.vin = static_cast<const double2 *>(rb); A.ldin = R.ld; A.w = va; A.ldw = n_b; A.x = nullptr;
            A.a = alpha; A.p = 1; A.dots = ws.raw;
            CFD_TRY(launch_step<double>(STEP_FIRST, n_b, vpt, A, 0, stream));
            A.vin = va; A.ldin = n_b; A.w = vb; A.x0 = static_cast<const double2 *>(rb); A.ldx0 = R.ld;
            A.a = 2.0 * alpha; A.p = 2; A.dots = ws.raw + 2 * n_b;
            CFD_TRY(launch_step<double>(STEP_SECOND, n_b, vpt, A, 0, stream));
            for (int p = 3; p <= n_p; ++p) {
                A.vin = (p & 1) ? vb : va; A.w = (p & 1) ? va : vb; A.p = p;
                A.dots = ws.raw + (int64_t)(p - 1) * 2 * n_b;
                CFD_TRY(launch_step<double>(STEP_GENERAL, n_b, vpt, A, 0, stream));
            }
        } else {
            StepArgs<float> A;
            A.H = sell_view<float>(H);
            A.gc = ws.gc; A.partial = ws.partial; A.ticket = ws.ticket; A.status = ws.status; A.beta = beta;
            A.staged = staged;
            A.gather = default_gather(H->prec);
            A.prep_val = staged ? ws.prep : nullptr;
            float2 *va = static_cast<float2 *>(ws.va), *vb = static_cast<float2 *>(ws.vb);
            A.vin = static_cast<const float2 *>(rb); A.ldin = R.ld; A.w = va; A.ldw = n_b; A.x = nullptr;
            A.a = alpha; A.p = 1; A.dots = ws.raw;
            CFD_TRY(launch_step<float>(STEP_FIRST, n_b, vpt, A, 0, stream));
            A.vin = va; A.ldin = n_b; A.w = vb; A.x0 = static_cast<const float2 *>(rb); A.ldx0 = R.ld;
            A.a = 2.0 * alpha; A.p = 2; A.dots = ws.raw + 2 * n_b;
            CFD_TRY(launch_step<float>(STEP_SECOND, n_b, vpt, A, 0, stream));
            for (int p = 3; p <= n_p; ++p) {
                A.vin = (p & 1) ? vb : va; A.w = (p & 1) ? va : vb; A.p = p;
                A.dots = ws.raw + (int64_t)(p - 1) * 2 * n_b;
                CFD_TRY(launch_step<float>(STEP_GENERAL, n_b, vpt, A, 0, stream));
            }
        }
        CFD_TRY(launch_moments(ws.raw, n_p, n_b, mu, 2 * n_p, ws.status, stream));
    }
    return CFD_OK;
}

size_t batched_workspace(int64_t N, int R, int n_s, int n_b, int n_p, int prec_H, int prec_X) {
    return filter_workspace(N, n_s, n_b, n_p, prec_H, prec_X) + round_up((size_t)R * (n_p + 3) * sizeof(double), 256);
}

cfd_status filter_batched_impl(const cfd_matrix *H, const int32_t *chunk_rid, int R, const double *windows, int n_p,
                               const cfd_block &X, int n_b, int vpt, int persistent, void *work, size_t work_bytes,
                               cudaStream_t stream, int arith, int graph) {
    CFD_TRY(check_filter_args(H, n_p, X, n_b, vpt));
    if (!chunk_rid || !windows || R < 1) return fail(CFD_ERR_ARG, "batch description missing");
    if (!work) return fail(CFD_ERR_ARG, "work is NULL");
    if (arith != ARITH_NATIVE && arith != ARITH_DW) return fail(CFD_ERR_ARG, "arith=%d not in {0, 1}", arith);
    if (arith == ARITH_DW && (H->prec != CFD_C128 || X.prec != CFD_C128 || !(H->flags & CFD_MATRIX_PACKED) ||
                              persistent))
        return fail(CFD_ERR_ARG, "double-word arithmetic needs a packed complex-double batch and block, "
                                 "without the persistent launch");
    if (graph != 0 && graph != 1) return fail(CFD_ERR_ARG, "graph=%d not in {0, 1}", graph);
    size_t need = batched_workspace(H->n_rows, R, X.n_cols, n_b, n_p, H->prec, X.prec);
    if (work_bytes < need) return fail(CFD_ERR_OOM, "batched filter workspace %zu < %zu bytes", work_bytes, need);
    if (!aligned16(work)) return fail(CFD_ERR_ARG, "work must be 16-byte aligned");
    size_t base = filter_workspace(H->n_rows, X.n_cols, n_b, n_p, H->prec, X.prec);
    FilterScratch ws = carve_filter(H, X, n_b, n_p, work, base);
    double *rcoef = reinterpret_cast<double *>(static_cast<char *>(work) + base);
    int64_t ld = n_p + 3;
    FilterPlan P;
    P.n_b = n_b;
    P.n_p = n_p;
    P.vpt = vpt > 0 ? vpt : default_vpt(H->prec, n_b);
    P.grid_cap = STEP_MAX_GRID;
    P.persistent = persistent != 0;
    P.alpha = 0.0;
    P.beta = 0.0;
    P.chunk_rid = chunk_rid;
    P.rcoef = rcoef;
    P.rcoef_ld = ld;
    P.staged = (int)default_staged(H->prec);
    P.gather = default_gather(H->prec);
    P.arith = arith;
    auto enqueue = [&](cudaStream_t s) -> cfd_status {
        CFD_CUDA(cudaMemsetAsync(ws.ticket, 0, sizeof(unsigned), s));
        CFD_CUDA(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
        k_batch_coeffs<<<(unsigned)((R * ld + 127) / 128), 128, 0, s>>>(windows, R, n_p, rcoef);
        CFD_COUNT_LAUNCH();
        CFD_LAUNCH_CHECK();
        if (H->prec == CFD_C128) return run_filter<double>(H, P, X, ws, nullptr, s);
        return run_filter<float>(H, P, X, ws, nullptr, s);
    };
    if (!graph) return enqueue(stream);
    struct Key {
        cfd_matrix H;
        cfd_block X;
        const void *chunk_rid, *windows, *work;
        size_t work_bytes;
        int R, n_p, n_b, vpt, persistent, arith, kind;
    } key;
    std::memset(&key, 0, sizeof(key));
    key.H = *H;
    key.X = X;
    key.chunk_rid = chunk_rid; key.windows = windows; key.work = work; key.work_bytes = work_bytes;
    key.R = R; key.n_p = n_p; key.n_b = n_b; key.vpt = P.vpt; key.persistent = persistent; key.arith = arith;
    key.kind = 2;
    return run_as_graph(&key, sizeof(key), stream, enqueue);
}

}  // namespace cfd

using namespace cfd;

extern "C" {

cfd_status cfd_filter_coeffs(double lmin, double lmax, double lam_l, double lam_r, int n_p, double *gc,
                             cudaStream_t stream) {
    clear_error();
    if (!gc) return fail(CFD_ERR_ARG, "gc is NULL");
    if (!(lmin < lmax) || !(lmin <= lam_l && lam_l < lam_r && lam_r <= lmax))
        return fail(CFD_ERR_ARG, "need lmin <= lam_l < lam_r <= lmax");
    if (n_p < 2) return fail(CFD_ERR_ARG, "n_p < 2");
    return launch_filter_coeffs(2.0 / (lmax - lmin), 0.5 * (lmax + lmin), lam_l, lam_r, n_p, gc, stream);
}

size_t cfd_filter_workspace(int64_t N, int n_s, int n_b, int n_p, int prec_H, int prec_X) {
    if (N < 1 || n_b < 1 || n_p < 2) return 0;
    return filter_workspace(N, n_s, n_b, n_p, prec_H & 0xff, prec_X & 0xff);
}

cfd_status cfd_filter(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r, int n_p,
                      cfd_block X, int n_b, void *work, size_t work_bytes, double *moments,
                      cudaStream_t stream) {
    clear_error();
    return filter_impl(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, 0, 0, work, work_bytes, moments, stream);
}

cfd_status cfd_filter_ex(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r, int n_p,
                         cfd_block X, int n_b, void *work, size_t work_bytes, double *moments,
                         const cfd_filter_opts *opts, cudaStream_t stream) {
    clear_error();
    int vpt = opts ? opts->vpt : 0, cap = opts ? opts->grid_cap : 0, pers = opts ? opts->persistent : 0;
    int staged = opts ? opts->staged : 0;
    int gather = opts ? opts->gather : 0;
    int fixed_chunk = opts ? opts->fixed_chunk : 0;
    int arith = opts ? opts->arith : 0;
    int graph = opts ? opts->graph : 0;
    int footprint = opts ? opts->footprint : 0;
    if (cap < 0) return fail(CFD_ERR_ARG, "grid_cap < 0");
    if (footprint < -1) return fail(CFD_ERR_ARG, "footprint=%d < -1", footprint);
    if (staged < -1 || staged > 2) return fail(CFD_ERR_ARG, "staged=%d not in -1..2", staged);
    if (gather != 0 && gather != 4 && gather != 8 && gather != STEP_GATHER_ALL)
        return fail(CFD_ERR_ARG, "gather=%d not in {0, 4, 8, %d}", gather, STEP_GATHER_ALL);
    return filter_impl_opts(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, vpt, cap, pers, staged, work, work_bytes,
                            moments, stream, gather, fixed_chunk, arith, graph, footprint);
}

cfd_status cfd_kpm_moments(const cfd_matrix *H, double lmin, double lmax, int n_p, cfd_block R, int n_b, void *work,
                           size_t work_bytes, double *moments, cudaStream_t stream) {
    clear_error();
    return kpm_impl(H, lmin, lmax, n_p, R, n_b, work, work_bytes, moments, stream);
}

cfd_status cfd_workspace_status(const void *work, cudaStream_t stream) {
    clear_error();
    if (!work) return fail(CFD_ERR_ARG, "work is NULL");
    int st = 0;
    CFD_CUDA(cudaMemcpyAsync(&st, work, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CFD_CUDA(cudaStreamSynchronize(stream));
    if (st == CFD_ERR_TIMEOUT) return fail(CFD_ERR_TIMEOUT, "a bounded device-side wait expired");
    if (st == (CFD_ERR_TIMEOUT | CFD_STATUS_DRAIN_EXPIRED))
        return fail(CFD_ERR_TIMEOUT,
                    "a bounded device-side wait expired and copies of that launch may still have been in flight "
                    "when it returned: the results and the contents of this workspace are invalid");
    if (st == CFD_ERR_BOUNDS)
        return fail(CFD_ERR_BOUNDS, "a Chebyshev moment exceeded mu_0: [lmin, lmax] does not contain the spectrum");
    if (st != 0) return fail(CFD_ERR_INTERNAL, "device status %d", st);
    return CFD_OK;
}

size_t cfd_filter_batched_workspace(int64_t N, int R, int n_s, int n_b, int n_p, int prec_H, int prec_X) {
    if (N < 1 || R < 1 || n_b < 1 || n_p < 2) return 0;
    return batched_workspace(N, R, n_s, n_b, n_p, prec_H & 0xff, prec_X & 0xff);
}

cfd_status cfd_filter_batched(const cfd_matrix *H, const int32_t *chunk_rid, int R, const double *windows, int n_p,
                              cfd_block X, int n_b, void *work, size_t work_bytes, const cfd_filter_opts *opts,
                              cudaStream_t stream) {
    clear_error();
    int vpt = opts ? opts->vpt : 0, pers = opts ? opts->persistent : 0;
    int arith = opts ? opts->arith : 0, graph = opts ? opts->graph : 0;
    return filter_batched_impl(H, chunk_rid, R, windows, n_p, X, n_b, vpt, pers, work, work_bytes, stream, arith,
                               graph);
}

}  // extern "C"
