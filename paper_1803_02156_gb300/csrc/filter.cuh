// Internals of the fused ChebFD step kernels, shared by the filter driver,
// the Lanczos bounds and Rayleigh-Ritz (plain SpMMV = the first step with
// alpha = 1, beta = 0).
#pragma once

#include "common.cuh"

namespace cfd {

constexpr int STEP_WARPS = 8;             // warps per CTA
constexpr int STEP_MAX_CTAS_PER_SM = 8;   // cap on resident CTAs per SM
constexpr int STEP_MAX_GRID = 4096;       // cap on CTAs of one step launch

enum StepKind : int {
    STEP_FIRST = 0,    // w = a (H vin - beta vin)                 (Algorithm 1, line 4)
    STEP_SECOND = 1,   // w = a (H vin - beta vin) - x; x = g0 x + g1 vin + g2 w  (lines 5-6)
    STEP_GENERAL = 2   // w = a (H vin - beta vin) - w; x += g_p w            (lines 9-12)
};

// Arguments of one step launch.  Row i of an operand sits at ptr + i * ld.
// dots receives, per vector j, (<vin_j, vin_j>, Re <w_j, vin_j>).
template <typename T>
struct StepArgs {
    SellView<T> H;
    const cplx_t<T> *vin;   // gathered operand (V_cur; the X block in step 1)
    int64_t ldin;
    cplx_t<T> *w;           // output (read as V_prev in general steps)
    int64_t ldw;
    cplx_t<T> *x;           // accumulator X (steps 2..n_p)
    int64_t ldx;
    double a;               // alpha in step 1, 2 alpha afterwards
    double beta;            // centre of the spectral interval
    const double *gc;       // weights g_k c_k, k = 0..n_p (device)
    int p;                  // step index
    double *partial;        // per-CTA partial dots [grid][nb][2]
    unsigned *ticket;       // CTA completion counter, zero between launches
    double *dots;           // reduced dots of this step [nb][2]
};

template <typename T>
cfd_status launch_step(int kind, int nb, int vpt, const StepArgs<T> &A, int grid_cap,
                       cudaStream_t stream);

struct FilterScratch {
    void *va, *vb, *xn;
    double *gc, *raw, *partial;
    unsigned *ticket;
    int grid_cap;
};

int default_vpt(int prec, int n_b);
size_t filter_workspace(int64_t N, int n_s, int n_b, int n_p, int prec_H, int prec_X);
cfd_status validate_block(const cfd_block &X, int64_t n_rows);
cfd_status launch_filter_coeffs(double alpha, double beta, double lam_l, double lam_r, int n_p,
                                double *gc, cudaStream_t stream);
cfd_status launch_moments(const double *raw, int n_p, int nb, double *mu, int64_t ld_mu,
                          cudaStream_t stream);
cfd_status launch_narrow(const double2 *src, int64_t lds, float2 *dst, int64_t ldd, int64_t n_rows,
                         int nb, cudaStream_t stream);
cfd_status launch_widen(const float2 *src, int64_t lds, double2 *dst, int64_t ldd, int64_t n_rows,
                        int nb, cudaStream_t stream);
// The whole filter with explicit tuning knobs (vpt <= 0: default; grid_cap <= 0: none).
cfd_status filter_impl(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                       int n_p, const cfd_block &X, int n_b, int vpt, int grid_cap, void *work,
                       size_t work_bytes, double *moments, cudaStream_t stream);

}  // namespace cfd
