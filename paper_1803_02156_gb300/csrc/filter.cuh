// Internals of the fused ChebFD step kernels, shared by the filter driver,
// the Lanczos bounds and Rayleigh-Ritz (plain SpMMV = the first step with
// alpha = 1, beta = 0).
#pragma once

#include <functional>

#include "common.cuh"

namespace cfd {

constexpr int STEP_WARPS = 8;             // warps per CTA
constexpr int STEP_MAX_CTAS_PER_SM = 8;   // cap on resident CTAs per SM
constexpr int STEP_MAX_GRID = 4096;       // cap on CTAs of one step launch
constexpr int STEP_GATHER_ALL = 16;       // slots whose gathers a row issues at once (gather option)

enum StepKind : int {
    STEP_FIRST = 0,    // w = a (H vin - beta vin)                 (Algorithm 1, line 4)
    STEP_SECOND = 1,   // w = a (H vin - beta vin) - x; x = g0 x + g1 vin + g2 w  (lines 5-6)
    STEP_GENERAL = 2   // w = a (H vin - beta vin) - w; x += g_p w            (lines 9-12)
};

// Order in which the CTAs of a staged step take the SELL chunks: 0 grid-stride
// (CTA b takes chunks b, b + grid, ...: at any time the GPU works on one
// window of rows); 1 contiguous ranges (CTA b takes ceil(n / grid)
// consecutive chunks, so a row's y-neighbours, a few chunks back, were
// gathered by the same CTA moments before and may still sit in its L1).
#ifndef CFD_STAGED_RASTER
#define CFD_STAGED_RASTER 0
#endif

struct ChunkRange {
    int64_t first, last, stride;
};

__device__ __forceinline__ ChunkRange cta_chunks(int64_t n_chunks) {
    ChunkRange r;
    if (CFD_STAGED_RASTER) {
        const int64_t per = (n_chunks + gridDim.x - 1) / gridDim.x;
        r.first = (int64_t)blockIdx.x * per;
        r.last = r.first + per < n_chunks ? r.first + per : n_chunks;
        r.stride = 1;
    } else {
        r.first = blockIdx.x;
        r.last = n_chunks;
        r.stride = gridDim.x;
    }
    return r;
}

// Arguments of one step launch.  Row i of an operand sits at ptr + i * ld.
// dots receives, per vector j, (<vin_j, vin_j>, Re <w_j, vin_j>).
template <typename T>
struct StepArgs {
    SellView<T> H;
    const cplx_t<T> *vin;   // gathered operand (V_cur; the X block in step 1)
    int64_t ldin;
    cplx_t<T> *w;           // output (read as V_prev in general steps)
    int64_t ldw;
    cplx_t<T> *x;           // accumulator X (steps 2..n_p); nullptr: moments only
    int64_t ldx;
    const cplx_t<T> *x0 = nullptr;   // moments only: the start block (read by step 2)
    int64_t ldx0 = 0;
    double a;               // alpha in step 1, 2 alpha afterwards
    double beta;            // centre of the spectral interval
    const double *gc;       // weights g_k c_k, k = 0..n_p (device)
    int p;                  // step index
    double *partial;        // per-CTA partial dots [grid][nb][2]
    unsigned *ticket;       // CTA completion counter, zero between launches
    double *dots;           // reduced dots of this step [nb][2]
    // batch of realisations (null for a single matrix): chunk -> realisation,
    // per realisation {alpha, beta, g_0 c_0, ..., g_np c_np} with stride rcoef_ld
    const int32_t *chunk_rid = nullptr;
    const double *rcoef = nullptr;
    int64_t rcoef_ld = 0;
    // general steps staged through shared memory by TMA (k_cheb_step_staged);
    // status receives CFD_ERR_TIMEOUT if one of its bounded waits expires
    int staged = 0;
    int *status = nullptr;
    // gathers in flight per row in staged general steps of packed matrices:
    // STEP_GATHER_ALL (all of the first 16 slots at once) or groups of four
    int gather = 0;
    // staged general steps: the matrix values prepared as 2 alpha (H - beta)
    // (launch_prepare_values; same SELL layout and storage as H's values);
    // required by the staged kernel, which then starts each row sum at
    // -V_prev and needs no shift, scale or subtraction
    const void *prep_val = nullptr;
    // staged packed steps of C = 32 matrices: the kernel compiled for that
    // chunk height (>= 0) or the generic one (< 0); results are the same
    int fixed_chunk = 0;
};

template <typename T>
cfd_status launch_step(int kind, int nb, int vpt, const StepArgs<T> &A, int grid_cap,
                       cudaStream_t stream);
// Per (precision, value storage) instantiations, in step_*.cu.
template <typename T, bool PACK>
cfd_status launch_step_p(int kind, int nb, int vpt, const StepArgs<T> &A, int grid_cap, cudaStream_t s);
template <typename T, bool PACK>
cfd_status launch_persistent_p(int nb, int vpt, const StepArgs<T> &A, cplx_t<T> *va, cplx_t<T> *vb, cplx_t<T> *xb,
                               int64_t ldx, int n_p, int grid_cap, cudaStream_t s);

template <typename T>
cfd_status launch_persistent(int nb, int vpt, const StepArgs<T> &A, cplx_t<T> *va, cplx_t<T> *vb, cplx_t<T> *xb,
                             int64_t ldx, int n_p, int grid_cap, cudaStream_t stream);
// General steps 3..n_p of one block in one cooperative launch with the
// TMA-staged chunk loop (packed values prepared in A.prep_val; A.x, A.ldx the
// block; steps 1 and 2 run before it).  Instantiated in step_f*_packed.cu.
template <typename T>
cfd_status launch_persistent_staged(int nb, int vpt, const StepArgs<T> &A, cplx_t<T> *va, cplx_t<T> *vb, int n_p,
                                    int grid_cap, cudaStream_t s);

// Complex-double steps in double-word arithmetic on the fp32 pipe
// (step_dw.cu): step 1, 2 or a general step (last: X written back as complex
// double), the in-place conversion of a block between complex double and
// double-word form, and the double-word prepared values.
cfd_status launch_step_dw(int kind, int nb, int vpt, const StepArgs<double> &A, bool last, int grid_cap,
                          cudaStream_t s);
cfd_status launch_dw_convert(void *p, int64_t ld, int64_t n_rows, int nb, bool to_dw, cudaStream_t stream);
cfd_status launch_prepare_values_dw(const cfd_matrix *H, double alpha, double beta, const int32_t *chunk_rid,
                                    const double *rcoef, int64_t rcoef_ld, void *out, size_t out_bytes,
                                    cudaStream_t stream);

// Per-call footprints of the SELL chunks for the footprint-staged general
// steps (step_fp.cu): the rows of V_cur each chunk reads, as row ranges
// staged by TMA into shared memory, and every slot's column as its row there.
struct FpView {
    const uint16_t *lcol = nullptr;   // per slot (H's SELL layout): the column's row in the staged footprint
    const int2 *desc = nullptr;       // per chunk 32 words: {chunk_len, ranges (-1: not staged)}, {rows, row of
                                      // the first own row}, first slot, 5 unused, 16 ranges {first row, rows}, 8 unused
    int fmax = 0;                     // footprint rows one stage holds (0: footprint steps off)
};
// Workspace bytes of the footprints of an N-row matrix.
size_t footprint_bytes(int64_t N);
// Footprint rows one stage of the footprint step holds for H at n_b / vpt
// (complex float, or complex double in double-word arithmetic); 0 when the
// step does not apply (it needs packed values, C = 32, sigma = 1, n_b = 32)
// or, unless any_size, when H has too few chunks for it to pay.
int footprint_rows_cap(const cfd_matrix *H, int nb, int vpt, bool dw, bool any_size);
// Builds the footprints of H's chunks (at most fmax rows each) in buf; in a
// batch (chunk_rid set) each descriptor also names its chunk's realisation.
cfd_status launch_footprint(const cfd_matrix *H, const int32_t *chunk_rid, int fmax, void *buf, size_t buf_bytes,
                            FpView *out, cudaStream_t stream);
// One general step with the footprints staged (complex float; complex double
// in double-word arithmetic, last: X written back as complex double).
cfd_status launch_step_fp(const StepArgs<float> &A, const FpView &F, int nb, int vpt, int grid_cap, cudaStream_t s);
cfd_status launch_step_fp_dw(const StepArgs<double> &A, const FpView &F, int nb, int vpt, bool last, int grid_cap,
                             cudaStream_t s);

// Runs body(s) captured as a CUDA graph on a library stream and launches the
// graph on `stream`; later calls with the same key bytes (on the same device)
// replay the cached executable without capturing again (graph.cu).
cfd_status run_as_graph(const void *key, size_t key_bytes, cudaStream_t stream,
                        const std::function<cfd_status(cudaStream_t)> &body);

// Arithmetic of the complex-double filter's general steps.
enum FilterArith : int { ARITH_NATIVE = 0, ARITH_DW = 1 };

// How one filter application is run.
struct FilterPlan {
    int n_b = 0, n_p = 0, vpt = 0, grid_cap = 0;
    bool persistent = false;
    int staged = 0;
    int gather = 0;
    int fixed_chunk = 0;
    int arith = ARITH_NATIVE;
    int footprint = 0;                    // footprint steps: 0 where they apply and pay, < 0 never,
                                          // > 0 wherever they apply, at most this many rows a chunk
    double alpha = 0, beta = 0;
    const int32_t *chunk_rid = nullptr;   // batch: chunk -> realisation
    const double *rcoef = nullptr;        // batch: per realisation {alpha, beta, weights}
    int64_t rcoef_ld = 0;
};

// Stored entries per row of the matrices this library builds (Topi: the
// on-site term and two per neighbour): bounds the prepared-values buffer.
constexpr int kMaxRowSlots = 13;

struct FilterScratch {
    int *status;            // device status word (first bytes of the workspace)
    void *va, *vb, *xn;
    void *prep;             // prepared matrix values (2 alpha (H - beta)), prep_bytes long
    size_t prep_bytes;
    void *fp;               // chunk footprints (n_b = 32 only), fp_bytes long
    size_t fp_bytes;
    double *gc, *raw, *partial;
    unsigned *ticket;
    int grid_cap;
};

// Whether the general steps default to the TMA-staged kernel for a matrix precision.
bool default_staged(int prec);
int default_gather(int prec);

int default_vpt(int prec, int n_b);
size_t filter_workspace(int64_t N, int n_s, int n_b, int n_p, int prec_H, int prec_X);
cfd_status validate_block(const cfd_block &X, int64_t n_rows);
// Matrix, block, degree, block width, precision pair and vectors per thread
// of a filter call (CFD_ERR_ARG with a message on the first violation).
cfd_status check_filter_args(const cfd_matrix *H, int n_p, const cfd_block &X, int n_b, int vpt);
// Bit or-ed into CFD_ERR_TIMEOUT in a workspace status word when a CTA also
// gave up waiting for its own bulk copies to land before it returned.
constexpr int CFD_STATUS_DRAIN_EXPIRED = 0x100;
cfd_status launch_filter_coeffs(double alpha, double beta, double lam_l, double lam_r, int n_p,
                                double *gc, cudaStream_t stream);
// Values of 2 alpha (H - beta) in H's SELL layout and storage into out
// (capacity out_bytes): every stored value times 2 alpha, beta subtracted
// first on the diagonal; in a batch (chunk_rid set) each chunk takes its
// realisation's alpha and beta from rcoef (row stride rcoef_ld).
cfd_status launch_prepare_values(const cfd_matrix *H, double alpha, double beta, const int32_t *chunk_rid,
                                 const double *rcoef, int64_t rcoef_ld, void *out, size_t out_bytes,
                                 cudaStream_t stream);
// raw dots -> KPM moments; with status set, also the spectral-bounds guard
// (CFD_ERR_BOUNDS recorded when a moment exceeds mu_0).
cfd_status launch_moments(const double *raw, int n_p, int nb, double *mu, int64_t ld_mu, int *status,
                          cudaStream_t stream);
cfd_status launch_narrow(const double2 *src, int64_t lds, float2 *dst, int64_t ldd, int64_t n_rows,
                         int nb, cudaStream_t stream);
cfd_status launch_widen(const float2 *src, int64_t lds, double2 *dst, int64_t ldd, int64_t n_rows,
                        int nb, cudaStream_t stream);
// The whole filter with all options (persistent: one cooperative launch per block).
cfd_status filter_impl_opts(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r, int n_p,
                            const cfd_block &X, int n_b, int vpt, int grid_cap, int persistent, int staged,
                            void *work, size_t work_bytes, double *moments, cudaStream_t stream, int gather = 0,
                            int fixed_chunk = 0, int arith = ARITH_NATIVE, int graph = 0, int footprint = 0);
size_t batched_workspace(int64_t N, int R, int n_s, int n_b, int n_p, int prec_H, int prec_X);
cfd_status kpm_impl(const cfd_matrix *H, double lmin, double lmax, int n_p, const cfd_block &R, int n_b,
                    void *work, size_t work_bytes, double *moments, cudaStream_t stream);
cfd_status filter_batched_impl(const cfd_matrix *H, const int32_t *chunk_rid, int R, const double *windows, int n_p,
                               const cfd_block &X, int n_b, int vpt, int persistent, void *work, size_t work_bytes,
                               cudaStream_t stream, int arith = ARITH_NATIVE, int graph = 0);
// The whole filter with explicit tuning knobs (vpt <= 0: default; grid_cap <= 0: none).
cfd_status filter_impl(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                       int n_p, const cfd_block &X, int n_b, int vpt, int grid_cap, void *work,
                       size_t work_bytes, double *moments, cudaStream_t stream);

}  // namespace cfd
