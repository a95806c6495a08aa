/*
 * cfd.h -- C ABI of the GB300 ChebFD library (libcfd.so).
 *
 * Chebyshev filter diagonalization (ChebFD) after Kreutzer et al.,
 * "Chebyshev Filter Diagonalization on Modern Manycore Processors and GPGPUs"
 * (arxiv 1803.02156): the block polynomial filter
 *     X <- sum_{k=0}^{n_p} g_k c_k T_k(H~) X,   H~ = alpha (H - beta 1),
 * applied to n_s search vectors in subspace blocks of n_b vectors (Algorithms
 * 1 and 2), on a sparse complex Hermitian matrix H stored in SELL-C-sigma.
 *
 * Conventions shared by every entry point
 *   - Plain C types and pointers only.  "device" pointers are CUDA global
 *     memory on the current device; "host" pointers are ordinary CPU memory.
 *   - The caller allocates all memory.  The library never calls cudaMalloc
 *     or cudaFree; sizes come from the *_size / *_workspace queries.  Buffers
 *     must stay alive until the work queued on the stream has finished.
 *   - All GPU work is queued on the caller's stream.  Entry points that return
 *     host results say so and synchronise that stream only.
 *   - Every call returns a cfd_status.  Nothing aborts or throws across the
 *     ABI.  On failure cfd_last_error() returns a message for the calling
 *     thread.  CUDA errors of earlier asynchronous work may surface at the
 *     next call that checks the stream (reported as CFD_ERR_CUDA).
 *   - Complex scalars are interleaved (re, im): 16 bytes for CFD_C128, 8 bytes
 *     for CFD_C64.  Block vectors are row-major ("interleaved", Sect. 3.1):
 *     element (i, j) of a block sits at ptr + (i * ld + j) * scalar size.
 *   - Device pointers must be 16-byte aligned; ld * scalar size must be a
 *     multiple of 16 bytes.
 */
#ifndef CFD_H
#define CFD_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cfd_status {
    CFD_OK = 0,
    CFD_ERR_ARG = 1,      /* invalid argument (sizes, alignment, window, NULL) */
    CFD_ERR_CUDA = 2,     /* a CUDA runtime call or kernel launch failed */
    CFD_ERR_OOM = 3,      /* the caller's workspace is smaller than required */
    CFD_ERR_BOUNDS = 4,   /* spectrum of H~ left [-1, 1]: moments grew */
    CFD_ERR_TIMEOUT = 5,  /* a bounded device-side wait expired */
    CFD_ERR_NOCONV = 6,   /* the solve hit max_iter without converging */
    CFD_ERR_INTERNAL = 7  /* internal inconsistency */
} cfd_status;

typedef enum cfd_prec {
    CFD_C128 = 0,         /* complex double: fp64 arithmetic */
    CFD_C64 = 1           /* complex float: fp32 arithmetic and accumulation */
} cfd_prec;

/*
 * OR into the `prec` argument of the matrix queries/builds to store every
 * nonzero as one real scalar instead of a complex pair: each row keeps its
 * purely real entries first, then its purely imaginary entries (their
 * imaginary parts), each group in ascending column order.  Valid for
 * matrices whose every entry is purely real or purely imaginary, as all Topi
 * entries are (on-site (m + V) Gamma_1 and hops +-t/2, +-i t/2).  A complex
 * multiply-add with such an entry is two fused multiply-adds instead of four
 * and the value is half the bytes; the row sums add the same products in
 * another order (real group, then imaginary group), so results agree with
 * the complex storage to rounding.
 */
#define CFD_PACK_RI 0x100

/* cfd_matrix.flags bit: values are packed real-or-imaginary scalars. */
#define CFD_MATRIX_PACKED 1
/* cfd_matrix.flags bits 8..15: upper bound on the slots per row of any chunk
 * (0: unknown). */
#define CFD_MATRIX_SLOTS_SHIFT 8

/* Human-readable name of a status code (static string). */
const char *cfd_status_string(int status);

/* Message describing the last failure on the calling thread ("" if none). */
const char *cfd_last_error(void);

/* Library version, e.g. "1.0.0" (static string). */
const char *cfd_version(void);

/* Number of GPU kernels this library has launched in this process (all
 * threads and devices); for accounting in benchmarks. */
unsigned long long cfd_launch_count(void);

/* ------------------------------------------------------------------------ */
/* Matrix: the topological-insulator Hamiltonian in SELL-C-sigma             */
/* ------------------------------------------------------------------------ */

/*
 * Parameters of Topi-Nx-Ny-Nz (Sect. 2.1, "Physical Application and Problem
 * Setting"): a lattice of Nx x Ny x Nz sites with four orbitals each,
 * n = 4 Nx Ny Nz rows, row = 4 site + orbital, site = x + Nx (y + Ny z).
 *   on-site block (m + V_s) Gamma_1, V_s = gamma (u_s - 1/2), u_s uniform in
 *     [0, 1) from counter-based SplitMix64 (seed, stream tag 0, index s);
 *   hop block T_j = -(t/2) Gamma_1 + i (t/2) Gamma_{j+2} at block
 *     (site + e_j, site) and T_j^H at (site, site + e_j);
 *   Gamma_1 = s_z (x) 1, Gamma_{2,3,4} = s_x (x) s_{x,y,z}, index 2a + b;
 *   axis j wraps when periodic_j != 0, else it is open.
 * 13 nonzeros per interior row.  Periodic axes need at least 3 sites.
 */
typedef struct cfd_topi_params {
    int32_t Nx, Ny, Nz;
    int32_t periodic_x, periodic_y, periodic_z;
    double t, m, gamma;
    uint64_t seed;
} cfd_topi_params;

/* Sizes (bytes) of the caller-allocated arrays of a SELL-C-sigma matrix. */
typedef struct cfd_matrix_sizes {
    int64_t n_rows;          /* N */
    int64_t nnz;             /* stored nonzeros of the canonical matrix */
    int64_t n_chunks;        /* ceil(N / C) */
    int64_t n_slots;         /* sum over chunks of C * chunk length (>= nnz) */
    int64_t bytes_val;       /* n_slots complex scalars */
    int64_t bytes_col;       /* n_slots int32 */
    int64_t bytes_chunk_ptr; /* (n_chunks + 1) int64 */
    int64_t bytes_chunk_len; /* n_chunks int32 */
    int64_t bytes_perm;      /* N int32 when sigma > 1, else 0 */
    int64_t bytes_work;      /* build scratch, free again when the build ends */
} cfd_matrix_sizes;

/* Caller-allocated device buffers for cfd_build_matrix (sizes above). */
typedef struct cfd_matrix_buffers {
    void *val, *col, *chunk_ptr, *chunk_len, *perm, *work;
} cfd_matrix_buffers;

/*
 * A SELL-C-sigma matrix (Kreutzer et al. 2014, cited as the GHOST format).
 * Rows are taken in windows of sigma rows, sorted by decreasing length inside
 * each window (stable), and packed into chunks of C consecutive sorted rows.
 * Chunk c holds chunk_len[c] slots per row, stored slot-major: slot k of
 * sorted row r (r = c C + rr) sits at chunk_ptr[c] + k C + rr.  Within a row
 * the slots are in ascending column order; padding slots have col = -1 and
 * value 0.  Sorted row r is canonical row perm[r] (perm == NULL when
 * sigma == 1).  Column indices are canonical.  With CFD_MATRIX_PACKED, val
 * holds one real scalar per slot (double or float); chunk_len[c] holds the
 * chunk's real slot count in its low 16 bits and its imaginary slot count in
 * the high 16 bits, slots [0, n_re) of a row hold real entries and
 * [n_re, n_re + n_im) imaginary ones, each group padded separately (col -1,
 * value 0).  The struct only points into caller memory.
 */
typedef struct cfd_matrix {
    int64_t n_rows, nnz, n_chunks, n_slots;
    int32_t C, sigma, prec, flags;    /* flags: CFD_MATRIX_PACKED, slot bound << CFD_MATRIX_SLOTS_SHIFT */
    void *val;
    int32_t *col;
    int64_t *chunk_ptr;
    int32_t *chunk_len;
    int32_t *perm;
} cfd_matrix;

/*
 * Sizes of the arrays cfd_build_matrix needs for Topi with chunk height C
 * (power of two, 4..128), sorting window sigma (1, or a multiple of C up to
 * 65536) and value precision prec.  Host-only; no GPU work.
 * Errors: CFD_ERR_ARG for invalid lattice, C, sigma or prec.
 */
cfd_status cfd_matrix_query_size(const cfd_topi_params *p, int C, int sigma, int prec,
                                 cfd_matrix_sizes *out);

/*
 * Build Topi (parameters p, see above) in SELL-C-sigma into the caller's
 * device buffers, on `stream`.  Values are computed in fp64 exactly as
 * defined (one rounding each for gamma (u - 1/2) and m + V) and rounded to
 * float for CFD_C64.  Fills *out (host struct) with the metadata and pointers.
 * Asynchronous.  Errors: CFD_ERR_ARG (parameters, NULL or misaligned
 * buffers), CFD_ERR_CUDA (launch failure).
 */
cfd_status cfd_build_matrix(const cfd_topi_params *p, int C, int sigma, int prec,
                            const cfd_matrix_buffers *buf, cfd_matrix *out, cudaStream_t stream);

/* Device scratch bytes cfd_matrix_export_csr needs. */
size_t cfd_export_csr_workspace(const cfd_matrix *H);

/*
 * Export H as canonical CSR (rows in lattice order, columns ascending,
 * padding dropped) into device arrays rowptr[N + 1] (int64), col[nnz]
 * (int32) and val[nnz] (complex of H's precision).  Asynchronous.
 */
cfd_status cfd_matrix_export_csr(const cfd_matrix *H, int64_t *rowptr, int32_t *col, void *val,
                                 void *work, size_t work_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* The ChebFD polynomial filter                                              */
/* ------------------------------------------------------------------------ */

/*
 * Filter weights gc[k] = g_k c_k, k = 0..n_p, written to device memory
 * (n_p + 1 doubles).  H~ = alpha (H - beta), alpha = 2 / (lmax - lmin),
 * beta = (lmax + lmin) / 2 maps [lmin, lmax] onto [-1, 1] (the map
 * alpha H + beta 1 of Algorithm 1 with the paper's beta written as
 * -alpha beta).  c_k are the Chebyshev coefficients of the indicator of the
 * search interval [lam_l, lam_r]: with theta = arccos(alpha (lam - beta)),
 * c_0 = (theta_l - theta_r) / pi, c_k = 2 (sin k theta_l - sin k theta_r) / (k pi);
 * g_k is the Jackson kernel for M = n_p + 1 moments,
 * g_k = [(M - k + 1) cos(pi k / (M + 1)) + sin(pi k / (M + 1)) cot(pi / (M + 1))] / (M + 1).
 * (The paper names c_k, g_k and the window in Sect. 2 and Algorithm 1 and
 * defers their definition to its references.)  Asynchronous.
 * Errors: CFD_ERR_ARG unless lmin <= lam_l < lam_r <= lmax, lmin < lmax, n_p >= 2.
 */
cfd_status cfd_filter_coeffs(double lmin, double lmax, double lam_l, double lam_r, int n_p,
                             double *gc, cudaStream_t stream);

/* A row-major block of n_cols complex vectors of length n_rows. */
typedef struct cfd_block {
    void *ptr;        /* device pointer */
    int64_t n_rows;   /* N */
    int64_t ld;       /* row stride in scalars, >= n_cols */
    int32_t n_cols;   /* n_s */
    int32_t prec;     /* cfd_prec */
} cfd_block;

/*
 * Device scratch bytes cfd_filter needs for an N x n_s block filtered in
 * blocks of n_b vectors with degree n_p, matrix precision prec_H and block
 * precision prec_X.  Flag bits above the low byte (CFD_PACK_RI) are ignored
 * by this and the other workspace queries.  Returns 0 for invalid sizes.
 * Besides the two N x n_b recurrence blocks it holds the matrix values
 * prepared once per call as 2 alpha (H - beta) for the general steps, sized
 * for 13 stored entries per row (the matrices cfd_build_matrix and
 * cfd_build_batch make); a matrix with more is rejected with CFD_ERR_ARG.
 */
size_t cfd_filter_workspace(int64_t N, int n_s, int n_b, int n_p, int prec_H, int prec_X);

/*
 * Apply the ChebFD filter to X in place (Algorithm 1, blocked as Algorithm
 * 2): for each block b of n_b columns [b n_b, (b + 1) n_b),
 *   V1 = H~ X_b;  V2 = 2 H~ V1 - X_b;  X_b <- gc0 X_b + gc1 V1 + gc2 V2;
 *   for p = 3..n_p: swap(V_prev, V_cur); V_prev <- 2 H~ V_cur - V_prev;
 *                   eta_p = Re <V_prev, V_cur>; mu_p = <V_cur, V_cur>;
 *                   X_b <- X_b + gc_p V_prev,
 * each step one fused kernel (the paper's chebfd_op) over the SELL-C-sigma
 * matrix.  H~ and gc as in cfd_filter_coeffs.
 *
 * Precision: X.prec == H->prec runs entirely in that precision.  H->prec ==
 * CFD_C64 with X.prec == CFD_C128 is the mixed mode: each block is rounded to
 * complex float (round to nearest), filtered in fp32 with fp32 accumulation,
 * and widened back.
 *
 * moments (device, nullable): [n_s][2 n_p] doubles, the Chebyshev moments
 * mu_m = <x_j, T_m(H~) x_j>, m = 0..2 n_p - 1, of the input columns, from the
 * per-step dot products (lines 10-11 of Algorithm 1, plus the same dots on
 * the two seed steps) via T_k T_l = (T_{k+l} + T_{|k-l|}) / 2.  The
 * reductions are deterministic (fixed order).
 *
 * Spectral-bounds guard: with moments requested, a moment larger than mu_0
 * by more than 1% (an eigenvalue of H outside [lmin, lmax] makes them grow
 * like cosh(m arccosh |lambda~|)) records CFD_ERR_BOUNDS in the workspace
 * status, reported by cfd_workspace_status; the call itself stays
 * asynchronous.
 *
 * work: device scratch of cfd_filter_workspace(...) bytes.  n_b must divide
 * n_s and be one of 8, 16, 32, 64.  Asynchronous.
 * Errors: CFD_ERR_ARG (sizes, window, precision pair, alignment),
 * CFD_ERR_OOM (work too small), CFD_ERR_CUDA.
 */
cfd_status cfd_filter(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                      int n_p, cfd_block X, int n_b, void *work, size_t work_bytes,
                      double *moments, cudaStream_t stream);

/* Tuning knobs of the fused step kernels (zero = default). */
typedef struct cfd_filter_opts {
    int32_t vpt;          /* vectors per thread: 1 or 2 (threads per row = n_b / vpt); 1 needs n_b <= 32 */
    int32_t grid_cap;     /* upper bound on CTAs per step launch (0: one wave of resident CTAs) */
    int32_t persistent;   /* 1: all n_p steps of a block in one cooperative launch (no moments) */
    int32_t staged;       /* 1: general steps stage matrix chunks in shared memory by TMA bulk copies;
                             -1: never; 0: default (staged);
                             2: test of the bounded waits (no wait can succeed; the filter
                             records CFD_ERR_TIMEOUT, see cfd_workspace_status) */
    int32_t gather;       /* staged general steps of packed matrices: slots of a row whose gathers of
                             V_cur are in flight together; 16 or 8: the first 16 (8) slots at once,
                             the rest in groups of four; 4: groups of four; 0: the library's
                             default.  Results do not depend on it. */
    int32_t fixed_chunk;  /* staged steps of packed matrices with C = 32: 1 uses the kernel compiled
                             for that chunk height (32-bit gather offsets, where they fit); -1 the
                             generic kernel; 0 the default (compiled height for complex float,
                             generic for complex double).  Results do not depend on it. */
    int32_t arith;        /* complex-double filters: 0 native fp64 arithmetic (the FP64 pipe); 1 double-word
                             arithmetic on the fp32 pipe for the general steps (n_p - 2 of n_p): every double
                             carried as hi + lo floats (about 48 significant bits, each operation accurate to
                             a few units of 2^-48 against 2^-53 natively), complex-double storage and memory
                             traffic unchanged; needs packed values (CFD_PACK_RI), not with persistent.
                             Results agree with arith 0 to that rounding, not bit for bit. */
    int32_t graph;        /* 1: the call's launch sequence (weights, prepared values, the n_p steps of every
                             block, moments) is captured once as a CUDA graph on a library stream and launched
                             as one graph on `stream`; later calls with the same arguments (pointers, sizes,
                             bounds, window, options) on the same device replay the cached graph (up to 16
                             are kept).  Results are bit for bit those of graph 0.  The first call of each
                             argument set captures, so make it outside any capture of your own. */
    int32_t footprint;    /* general steps of complex-float filters and double-word complex-double filters
                             (packed values, C = 32, sigma = 1, n_b = 32): 0 (default) stages each chunk's
                             footprint, the rows of V_cur its slots read, by TMA bulk copies into shared
                             memory before the chunk is computed (the row ranges are found once per call),
                             for matrices of at least 16 chunks per SM (smaller ones keep the gathered
                             steps); -1 never (every slot's V_cur row is gathered from global memory); n > 0
                             the footprint steps at any size, with at most n footprint rows per chunk
                             (chunks with more are gathered from global memory).  Results do not depend on
                             it (filtered block bit for bit; moments to the order of their sums). */
} cfd_filter_opts;

/* cfd_filter with explicit kernel options (the autotuner's knobs besides n_b,
 * C and sigma).  The filtered block does not depend on the options; the
 * moments only through the order of their reductions. */
cfd_status cfd_filter_ex(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                         int n_p, cfd_block X, int n_b, void *work, size_t work_bytes,
                         double *moments, const cfd_filter_opts *opts, cudaStream_t stream);

/*
 * The same filter as cfd_filter, computed by a chain of separate standard
 * calls instead of the fused step (the "SpMMV + BLAS1" baseline of Sect. 4,
 * Fig. 2): per recurrence step one SpMMV Y = H U into a third block, three
 * axpby updates (W = 2 alpha Y - W, W -= 2 alpha beta U, X += g_p c_p W) and,
 * when moments is non-NULL, two dot products, each a kernel of its own.
 * It reads and writes 14 block vectors per step where the fused step moves 5;
 * it exists to measure what the fusion saves.  Arguments, layout, precision
 * pairs and errors as cfd_filter; the result agrees with cfd_filter to
 * rounding (the operations are associated differently).  work:
 * cfd_filter_unfused_workspace(...) bytes (cfd_filter's plus one N x n_b
 * block and the dot partials).  Asynchronous.
 */
size_t cfd_filter_unfused_workspace(int64_t N, int n_s, int n_b, int n_p, int prec_H, int prec_X);
cfd_status cfd_filter_unfused(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                              int n_p, cfd_block X, int n_b, void *work, size_t work_bytes,
                              double *moments, cudaStream_t stream);

/*
 * cfd_filter for a search space X held in HOST memory (X.ptr a host pointer,
 * page-locked for copy/compute overlap; pageable memory works but
 * serialises).  Only two n_b-column blocks of X are on the device at a time
 * (Sect. 5: the filter needs fast memory for the active block and the two
 * recurrence blocks only), so n_s N is limited by host memory, not HBM.
 * While block b is filtered on `stream`, an internal copy stream writes block
 * b - 1 back and brings block b + 1 in (pitched 2-D copies of the column
 * window); the filtered X and the moments equal cfd_filter's bit for bit.
 * Asynchronous on `stream`: X must not be touched by the host until the
 * stream has been synchronised.  work: cfd_filter_host_workspace(...) bytes
 * of device memory (the filter workspace for one block plus two N x n_b
 * staging blocks).  moments: device pointer or NULL, as for cfd_filter.
 * Errors as cfd_filter; CFD_ERR_ARG if X.ptr is device or managed memory.
 */
size_t cfd_filter_host_workspace(int64_t N, int n_s, int n_b, int n_p, int prec_H, int prec_X);
cfd_status cfd_filter_host(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                           int n_p, cfd_block X, int n_b, void *work, size_t work_bytes,
                           double *moments, cudaStream_t stream);

/* cfd_filter_host with the arithmetic option of cfd_filter_opts (arith; every
 * other field must be zero): arith = 1 runs the complex-double steps in
 * double-word arithmetic, as cfd_filter_ex does. */
cfd_status cfd_filter_host_ex(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                              int n_p, cfd_block X, int n_b, void *work, size_t work_bytes, double *moments,
                              const cfd_filter_opts *opts, cudaStream_t stream);

/*
 * cfd_filter_host_ex for a search space stored block after block in host
 * memory (block b of n_b columns, N rows of n_b complex values, at
 * X.ptr + b N n_b scalars; X.n_rows = N, X.n_cols = n_s, X.ld = n_b): each
 * block moves over the link as one contiguous copy.  Up to n_p = 40 block
 * b + 1 comes in and b - 1 goes out while b is filtered (gathered steps);
 * above it each block's DMA copies run on `stream` before and after its
 * filter (footprint-staged steps, which starve copies running beside them).
 * Results equal cfd_filter's on the same columns bit for bit.
 */
cfd_status cfd_filter_host_blocked(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                                   int n_p, cfd_block X, int n_b, void *work, size_t work_bytes, double *moments,
                                   const cfd_filter_opts *opts, cudaStream_t stream);

/*
 * Chebyshev moments only (the kernel polynomial method: Algorithm 1 without
 * line 12, Sect. 2): for the columns of R (N x n_s, the matrix's precision,
 * not modified) mu[j][m] = <r_j, T_m(H~) r_j>, m = 0..2 n_p - 1, into
 * moments (device, [n_s][2 n_p]), with the same fused steps as cfd_filter but
 * no accumulation into a filtered block (two fewer block vectors of traffic
 * per step).  work: cfd_filter_workspace(N, n_s, n_b, n_p, prec, prec) bytes.
 * Asynchronous.
 */
cfd_status cfd_kpm_moments(const cfd_matrix *H, double lmin, double lmax, int n_p, cfd_block R, int n_b,
                           void *work, size_t work_bytes, double *moments, cudaStream_t stream);

/*
 * Estimated number of eigenvalues of H in [lam_l, lam_r] from Chebyshev
 * moments (kernel polynomial method; Sect. 2 uses the moments to monitor the
 * number of states in the search interval).  mu: host [n_vec][n_mom] moments
 * <r, T_m(H~) r> of n_vec random vectors (e.g. cfd_filter's output with
 * n_mom = 2 n_p); count = N / n_vec sum_r sum_m g_m c_m mu_m(r) / mu_0(r) with
 * the Jackson kernel g_m for M = n_mom moments and the window coefficients
 * c_m of cfd_filter_coeffs.  Host only.
 */
cfd_status cfd_kpm_count(const double *mu, int n_vec, int n_mom, int64_t N, double lmin, double lmax,
                         double lam_l, double lam_r, double *count);

/*
 * Window [center - d, center + d] whose cfd_kpm_count equals `target`
 * (bisection on d; the Jackson-damped count grows with d).  Host only.
 * Errors: CFD_ERR_ARG if even the widest window holds fewer states.
 */
cfd_status cfd_kpm_window(const double *mu, int n_vec, int n_mom, int64_t N, double lmin, double lmax,
                          double center, double target, double *lam_l, double *lam_r);

/* ------------------------------------------------------------------------ */
/* Batches of independent realisations                                       */
/* ------------------------------------------------------------------------ */

/*
 * Sizes for a batch of R Topi realisations (p[0..R-1]: lattices and disorder
 * seeds may all differ) stored as one block-diagonal SELL-C-sigma matrix.
 * Realisation r owns rows [row_off[r], row_off[r + 1]): its 4 Nx Ny Nz rows
 * followed by empty padding rows up to a multiple of max(C, sigma, 32), so no
 * chunk or sorting window spans two realisations.  row_off (host, nullable)
 * receives R + 1 offsets.  The chunk -> realisation map needs
 * out->n_chunks int32 of device memory.  Host only.
 */
cfd_status cfd_batch_query_size(const cfd_topi_params *p, int R, int C, int sigma, int prec,
                                cfd_matrix_sizes *out, int64_t *row_off);

/*
 * Build the batch into caller buffers (sizes from cfd_batch_query_size) and
 * the chunk -> realisation map chunk_rid (device, n_chunks int32).  Each
 * realisation's rows and values are exactly those of cfd_build_matrix for
 * its parameters, shifted by row_off[r].  Asynchronous.
 */
cfd_status cfd_build_batch(const cfd_topi_params *p, int R, int C, int sigma, int prec,
                           const cfd_matrix_buffers *buf, int32_t *chunk_rid, cfd_matrix *out,
                           cudaStream_t stream);

/* Device scratch bytes of cfd_filter_batched. */
size_t cfd_filter_batched_workspace(int64_t N, int R, int n_s, int n_b, int n_p, int prec_H, int prec_X);

/*
 * The ChebFD filter on every realisation of a batch at once: each row uses
 * the map alpha_r (H - beta_r) and the weights g_k c_k of its realisation r,
 * from windows (device, [R][4] doubles: lmin, lmax, lam_l, lam_r).  X is the
 * N_total x n_s block of all realisations (padding rows must be zero and stay
 * zero).  One launch per step covers all realisations; with
 * opts->persistent each n_b block is instead one cooperative launch running
 * all n_p steps, the grid synchronising between steps (slower on GB300: the
 * three step kinds in one kernel limit occupancy).  Per
 * realisation the result equals cfd_filter on that realisation alone, bit for
 * bit.  No moments.  Same precision rules as cfd_filter.  Asynchronous.
 */
cfd_status cfd_filter_batched(const cfd_matrix *H, const int32_t *chunk_rid, int R, const double *windows,
                              int n_p, cfd_block X, int n_b, void *work, size_t work_bytes,
                              const cfd_filter_opts *opts, cudaStream_t stream);

/*
 * Device-side status of a filter workspace (cfd_filter, cfd_filter_ex,
 * cfd_filter_batched, cfd_kpm_moments, cfd_filter_unfused): the staged
 * kernels bound every wait on their TMA copies and record CFD_ERR_TIMEOUT
 * here if one expires; with moments requested the spectral-bounds guard
 * records CFD_ERR_BOUNDS.  Synchronises `stream`; returns CFD_OK or the
 * recorded status.  A timeout whose CTA also gave up waiting for its own
 * copies in flight is reported as CFD_ERR_TIMEOUT with a message saying so:
 * then the launch's results and the workspace contents are invalid.
 */
cfd_status cfd_workspace_status(const void *work, cudaStream_t stream);

/* Size of the library-owned device scratch used by cfd_filter_noalloc. */
#define CFD_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)

/*
 * cfd_filter without a workspace argument, for callers that are not allowed
 * to allocate device memory: code running under a host application's memory
 * budget or pool, where raw cudaMalloc is forbidden or the pool already holds
 * the memory, and latency-critical loops that cannot pay for cudaMalloc and
 * the device-wide synchronisation it implies.  (The paper has no counterpart;
 * this is a library convenience.)
 *
 * Same arguments, results and errors as cfd_filter, minus work/work_bytes.
 * The scratch is a 64 MiB array inside the library, one copy on every device
 * that loads it, kept until the process exits.  Problems whose
 * cfd_filter_workspace(...) exceeds CFD_NOALLOC_SCRATCH_BYTES are rejected
 * with CFD_ERR_ARG (for complex double roughly N (32 n_b + 208) bytes, plus 34 per row at n_b = 32,
 * <= 64 MiB, e.g. N <= 51000 at n_b = 32).
 * Nothing is allocated: no cudaMalloc/cudaFree and no allocating library call.
 *
 * Argument errors are reported as by cfd_filter before the size check.
 *
 * Every call looks up the scratch array's device address with the current
 * device current (no allocation, no stream work); the first lookup on a
 * device may load the library's device code there, so make the first call on
 * each device before any stream capture.  All calls share the one array and
 * it keeps the last call's contents (what must start at zero is cleared by
 * each call), so calls that can overlap on the GPU -- on different streams,
 * or from different host threads without ordering -- race and corrupt each
 * other; serialise them on one stream.  Device-side errors of the last call
 * (a bounded wait that expired, moments that left [-mu_0, mu_0]) are recorded
 * in the scratch and read by cfd_filter_noalloc_status.
 */
cfd_status cfd_filter_noalloc(const cfd_matrix *H, double lmin, double lmax, double lam_l,
                              double lam_r, int n_p, cfd_block X, int n_b, double *moments,
                              cudaStream_t stream);

/*
 * Device-side status of the last cfd_filter_noalloc call on the current
 * device, as cfd_workspace_status reports it for a caller's workspace:
 * CFD_OK, CFD_ERR_TIMEOUT or CFD_ERR_BOUNDS.  Queue it on the stream of that
 * call; it synchronises `stream`.  (No counterpart in the paper.)
 */
cfd_status cfd_filter_noalloc_status(cudaStream_t stream);


/* ------------------------------------------------------------------------ */
/* Distributed filter: z-slabs with halo exchange (Sect. 6, Algorithms 3, 4) */
/* ------------------------------------------------------------------------ */

/*
 * One rank's share of a Topi lattice distributed over nranks processes
 * (Sect. 6: every process works on a contiguous set of matrix rows and the
 * matching rows of the block vectors; the matrix's stencil structure makes
 * the exchange nearest-neighbour).  Ranks own consecutive z-planes, planes
 * [z0, z1) = rows [row0, row0 + n_local), z0 = rank Nz / nranks.  A rank's
 * local matrix numbers its columns own rows first (0 .. n_local - 1), then
 * the lower halo plane (n_local .. n_local + plane - 1: the plane below z0,
 * owned by lo_rank) and the upper halo plane (the next plane: the one above
 * z1 - 1, owned by hi_rank); a missing neighbour (open z, or one rank) has
 * rank -1 and base -1.  With periodic z the first and last ranks are
 * neighbours.
 */
typedef struct cfd_slab {
    int32_t nranks, rank;
    int32_t z0, z1;
    int64_t row0, n_local, plane;
    int32_t lo_rank, hi_rank;
    int64_t lo_base, hi_base;   /* first canonical row of the lower / upper halo plane */
} cfd_slab;

/* The slab of `rank` among nranks (1 <= nranks <= Nz).  Host only. */
cfd_status cfd_slab_plan(const cfd_topi_params *p, int nranks, int rank, cfd_slab *out);

/* Local column of canonical column col in the slab's numbering (-1 if the
 * slab's rows never reference it).  Host only. */
int64_t cfd_slab_local_col(const cfd_slab *s, int64_t col);

/* Sizes / build of the slab's rows of Topi (as cfd_matrix_query_size and
 * cfd_build_matrix): n_rows = n_local, columns in the slab's numbering.  Each
 * row keeps the entries in the order of the canonical matrix's row, so a
 * slab's row sums are bit for bit those of the whole matrix. */
cfd_status cfd_slab_query_size(const cfd_topi_params *p, const cfd_slab *s, int C, int sigma, int prec,
                               cfd_matrix_sizes *out);
cfd_status cfd_build_matrix_slab(const cfd_topi_params *p, const cfd_slab *s, int C, int sigma, int prec,
                                 const cfd_matrix_buffers *buf, cfd_matrix *out, cudaStream_t stream);

/*
 * Device scratch bytes of one slab's share of the distributed filter (the
 * filter scratch, and the recurrence blocks with their halo rows: one pair,
 * or one pair per subspace block for the pipelined mode).  mode: 0 vector
 * mode (Algorithm 3), 1 pipelined mode (Algorithm 4).
 */
size_t cfd_filter_slab_workspace(const cfd_slab *s, int n_s, int n_b, int n_p, int prec, int mode);

/*
 * The filter (as cfd_filter) distributed over the nranks slabs of one
 * lattice, all held in this process on the current device: slabs[r] is
 * rank r's plan, H[r] its slab matrix, X[r] its n_local x n_s block (same
 * precision as H), work[r] its scratch (work_bytes each).  Before every
 * fused step the boundary planes of the gathered block are copied into the
 * neighbours' halo rows (the exchange of Sect. 6 done by device copies), so
 * each slab's filtered rows are bit for bit those of cfd_filter on the whole
 * matrix.  mode 0 (vector mode, Algorithm 3): block by block, exchange then
 * step; mode 1 (pipelined mode, Algorithm 4): all blocks advance one degree
 * at a time and the exchange of block b + 1 runs on a second stream while
 * block b computes.  moments (device, nullable, [n_s][2 n_p]): the moments of
 * the whole vectors (per-slab dots summed).  opts: vpt, arith and footprint are used.
 * Asynchronous on `stream`.
 */
cfd_status cfd_filter_slabs(int nranks, const cfd_slab *slabs, const cfd_matrix *const *H, double lmin, double lmax,
                            double lam_l, double lam_r, int n_p, const cfd_block *X, int n_b, int mode,
                            void *const *work, size_t work_bytes, double *moments, const cfd_filter_opts *opts,
                            cudaStream_t stream);

/* NCCL communicator for cfd_filter_slab_nccl (libnccl is loaded at first use;
 * CFD_ERR_ARG if it cannot be).  id: 128 bytes, made on one rank by
 * cfd_nccl_unique_id and given to every rank (e.g. through
 * torch.distributed); comm receives the opaque communicator. */
cfd_status cfd_nccl_unique_id(void *id);
cfd_status cfd_nccl_comm_init(const void *id, int nranks, int rank, void **comm);
cfd_status cfd_nccl_comm_destroy(void *comm);

/*
 * One rank's part of the distributed filter, one slab per process and GPU:
 * the halo planes are exchanged with NCCL point-to-point transfers on
 * `stream` (every rank posts: its top plane to hi_rank, its bottom plane to
 * lo_rank, the lower halo from lo_rank, the upper halo from hi_rank) and the
 * moment dots are summed with an NCCL all-reduce, so every rank receives the
 * moments of the whole vectors.  Arguments otherwise as cfd_filter_slabs for
 * one slab.  Every rank must make the call with the same n_s, n_b, n_p, mode
 * and window.
 */
cfd_status cfd_filter_slab_nccl(const cfd_slab *slab, const cfd_matrix *H, double lmin, double lmax, double lam_l,
                                double lam_r, int n_p, cfd_block X, int n_b, int mode, void *work, size_t work_bytes,
                                double *moments, const cfd_filter_opts *opts, void *comm, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Spectral bounds                                                           */
/* ------------------------------------------------------------------------ */

/* Device scratch bytes cfd_spectral_bounds needs. */
size_t cfd_spectral_bounds_workspace(int64_t N, int steps);

/*
 * Interval [lmin, lmax] containing the spectrum of H, for the affine map of
 * the filter (Algorithm 1 maps the spectrum into [-1, 1]; the paper does not
 * say how the bounds are found).  Reading: `steps` Lanczos steps (no
 * reorthogonalisation) from a Gaussian start vector drawn from SplitMix64
 * (seed, stream tag 2); the extreme Ritz values theta_1, theta_m are widened
 * by their residual bounds |beta_m y_{m,i}| plus 1% of theta_m - theta_1 and
 * clipped to the Gershgorin interval.  H must be CFD_C128; steps in 2..256.
 * Host outputs: synchronises `stream`.
 */
cfd_status cfd_spectral_bounds(const cfd_matrix *H, int steps, uint64_t seed, double *lmin, double *lmax,
                               void *work, size_t work_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Dense fp64 kernels: Gram, Hermitian eigensolver                           */
/* ------------------------------------------------------------------------ */

/* Device scratch bytes of cfd_block_gram for N rows, n_x and n_y columns. */
size_t cfd_gram_workspace(int64_t N, int n_x, int n_y);

/*
 * S = X^H Y (n_x x n_y complex double, row-major, ld lds, device) for two
 * CFD_C128 blocks with the same rows, on the FP64 tensor cores, reduced in a
 * fixed order (deterministic).  n_x, n_y <= 256.  Asynchronous.
 */
cfd_status cfd_block_gram(cfd_block X, cfd_block Y, void *S, int64_t lds, void *work, size_t work_bytes,
                          cudaStream_t stream);

/*
 * cfd_block_gram with a choice of arithmetic: arith 0 as cfd_block_gram (fp64
 * on the FP64 tensor cores), 1 double-word arithmetic on the fp32 pipe: every
 * double split once into hi + lo floats, every multiply-add a double-word one
 * (Dekker's product, Knuth's sum, the errors collected in a second float),
 * each split's sums accurate to a few units of 2^-48 of their terms (2^-53
 * natively), the splits folded in fp64 in the same fixed order.  GB300 runs
 * fp64 at 1/64 of the fp32 rate, so the double-word Gram is several times
 * faster.  Same workspace (cfd_gram_workspace); CFD_ERR_ARG for another
 * arith.  Asynchronous.
 */
cfd_status cfd_block_gram_ex(cfd_block X, cfd_block Y, void *S, int64_t lds, void *work, size_t work_bytes,
                             int arith, cudaStream_t stream);

/* Device scratch bytes of cfd_eigh for order n. */
size_t cfd_eigh_workspace(int n);

/*
 * Eigen-decomposition of the Hermitian part of the n x n complex double
 * matrix A (row-major, ld lda, device; n <= 256) by cyclic Jacobi with
 * round-robin parallel ordering: evals (device, n doubles) ascending, Q
 * (device, ld ldq) with the eigenvectors as columns.  Sweeps stop when the
 * off-diagonal Frobenius norm is below n * 2^-52 times the Frobenius norm.
 * Asynchronous.
 */
cfd_status cfd_eigh(const void *A, int64_t lda, int n, double *evals, void *Q, int64_t ldq, void *work,
                    size_t work_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Orthogonalisation and Rayleigh-Ritz (restart step of Sect. 2)             */
/* ------------------------------------------------------------------------ */

/* Device scratch bytes of cfd_orthogonalize for an N x n_s block. */
size_t cfd_orthogonalize_workspace(int64_t N, int n_s);

/*
 * Orthonormalise the columns of X (CFD_C128, n_s <= 256) in place with SVQB
 * (Stathopoulos & Wu 2002, the rank-revealing method Sect. 2 names): S = X^H X,
 * D = diag(S)^{-1/2}, D S D = Q Theta Q^H, X <- X D Q Theta^{-1/2}, where
 * Theta is clamped below at tol * max(Theta) (tol <= 0: 1e-14); applied twice.
 * rank (host, nullable) receives #{theta >= tol max theta} of the first pass
 * and then the call synchronises `stream`; otherwise it is asynchronous.
 */
cfd_status cfd_orthogonalize(cfd_block X, double tol, int *rank, void *work, size_t work_bytes,
                             cudaStream_t stream);

/* cfd_orthogonalize with a choice of arithmetic for its Gram matrices and
 * projections: arith 0 fp64 (as cfd_orthogonalize), 1 double-word arithmetic
 * on the fp32 pipe (as cfd_block_gram_ex).  Same workspace. */
cfd_status cfd_orthogonalize_ex(cfd_block X, double tol, int *rank, void *work, size_t work_bytes, int arith,
                                cudaStream_t stream);

/* Device scratch bytes of cfd_rayleigh_ritz for an N x n_s block. */
size_t cfd_rayleigh_ritz_workspace(int64_t N, int n_s);

/*
 * Rayleigh-Ritz on the orthonormal block X (CFD_C128) with the complex-double
 * matrix H: Z = H X, G = X^H Z, G = Y diag(theta) Y^H (Jacobi), X <- X Y, and
 * resid[j] = ||H x_j - theta_j x_j||_2.  evals (device, n_s, ascending) and
 * resid (device, nullable).  Asynchronous.
 */
cfd_status cfd_rayleigh_ritz(const cfd_matrix *H, cfd_block X, double *evals, double *resid, void *work,
                             size_t work_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* The ChebFD solve                                                          */
/* ------------------------------------------------------------------------ */

typedef enum cfd_policy {
    CFD_POLICY_FP64 = 0,     /* every filter application in fp64 */
    CFD_POLICY_MIXED = 1,    /* fp32 filter until it stalls, then fp64; SVQB and RR always fp64 */
    CFD_POLICY_FP64_DW = 2,  /* as FP64 with double-word arithmetic on the fp32 pipe for the filter's
                                general steps (cfd_filter_opts.arith = 1; H needs packed values) and for the
                                Gram matrices and projections of SVQB and RR (cfd_block_gram_ex arith 1) */
    CFD_POLICY_MIXED_DW = 3  /* as MIXED with the fp64 filter phase, SVQB and RR in double-word arithmetic */
} cfd_policy;

typedef struct cfd_solve_params {
    double lam_l, lam_r;   /* search interval */
    double lmin, lmax;     /* spectral bounds; lmin >= lmax: found by cfd_spectral_bounds */
    double tol;            /* residual tolerance ||H x - theta x||_2, unit vectors (e.g. 1e-10) */
    double switch_tol;     /* mixed: fp32 phase target residual (<= 0: 1e-4) */
    uint64_t seed;         /* start block (stream tag 1) and Lanczos (tag 2) */
    int32_t n_s, n_p, n_b; /* search vectors, filter degree, subspace block */
    int32_t n_t;           /* target eigenpair count (0: unknown) */
    int32_t max_iter;
    int32_t policy;        /* cfd_policy */
    int32_t bounds_steps;  /* Lanczos steps (<= 0: 40) */
    int32_t start;         /* 0: random start block; 1: X holds the start block */
} cfd_solve_params;

typedef struct cfd_solve_result {
    int32_t n_conv;        /* converged Ritz pairs inside the window */
    int32_t iters;         /* restart iterations */
    int32_t iters_low;     /* of which with the fp32 filter */
    int32_t rank_min;      /* smallest SVQB rank seen */
    double lmin, lmax;     /* spectral bounds used */
    double t_filter, t_orth, t_rr, t_total;   /* seconds (device events; t_total wall clock) */
} cfd_solve_result;

/* Device scratch bytes of cfd_solve. */
size_t cfd_solve_workspace(const cfd_matrix *H, const cfd_matrix *H_low, const cfd_solve_params *p);

/*
 * Chebyshev filter diagonalization (Sect. 2): repeat { filter X (Algorithms 1
 * and 2), SVQB-orthogonalise, Rayleigh-Ritz } until done.  The paper gives no
 * stopping rule; reading: a Ritz pair inside [lam_l, lam_r] is converged when
 * its residual <= tol; stop when the converged count reaches n_t (n_t > 0), or
 * when it is >= 1 and unchanged over three consecutive iterations while the
 * smallest residual of the unconverged in-window pairs did not halve in
 * either of the last two (no pair is still converging).
 * Mixed policy: the filter runs on H_low (CFD_C64 copy of H) with fp32
 * arithmetic until the in-window count at switch_tol reaches n_t or stops
 * growing, then on H in fp64, where the solve also stops as soon as at least
 * as many in-window pairs reach tol as the fp32 phase brought to switch_tol;
 * SVQB, Rayleigh-Ritz and residuals stay fp64.
 * H: CFD_C128.  X: N x n_s CFD_C128, in: start block if p->start, out: Ritz
 * vectors.  evals/resid: host arrays of n_s (all Ritz values, ascending, and
 * their residuals).  Synchronises `stream` once per iteration.
 * Errors: CFD_ERR_ARG, CFD_ERR_OOM, CFD_ERR_NOCONV (results still filled).
 */
cfd_status cfd_solve(const cfd_matrix *H, const cfd_matrix *H_low, const cfd_solve_params *p, cfd_block X,
                     double *evals, double *resid, void *work, size_t work_bytes, cfd_solve_result *res,
                     cudaStream_t stream);

/* Device scratch bytes of cfd_solve_batched. */
size_t cfd_solve_batched_workspace(const cfd_matrix *H, int R, const cfd_solve_params *p);

/*
 * The ChebFD solve (see cfd_solve) on every realisation of a batch at once.
 * H (CFD_C128, optionally packed) and H_low (CFD_C64 copy, mixed policy only)
 * come from cfd_build_batch with the chunk -> realisation map chunk_rid.
 * Host arrays: row_off[R + 1] (cfd_batch_query_size), row_end[R] (end of
 * each realisation's real rows, row_off[r] + 4 Nx Ny Nz), windows[R][4]
 * (lmin, lmax, lam_l, lam_r per realisation), n_t[R] (target counts, 0 =
 * unknown).  From p: n_s (<= 64), n_p, n_b, tol, max_iter, policy,
 * switch_tol, seed, start.  X: N_total x n_s complex double with ld = n_s
 * (padding rows are zeroed).  Each iteration is one batched filter (one
 * launch per step for all realisations), a batched SVQB
 * (twice) and a batched Rayleigh-Ritz.  Realisations stop counting once
 * converged; the mixed policy switches to the fp64 filter when every
 * realisation is ready.  Outputs (host): evals[R][n_s], resid[R][n_s],
 * res[R].  Synchronises `stream` once per iteration.
 */
cfd_status cfd_solve_batched(const cfd_matrix *H, const cfd_matrix *H_low, const int32_t *chunk_rid, int R,
                             const int64_t *row_off, const int64_t *row_end, const double *windows,
                             const int32_t *n_t, const cfd_solve_params *p, cfd_block X, double *evals,
                             double *resid, cfd_solve_result *res, void *work, size_t work_bytes,
                             cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Measurement helper                                                        */
/* ------------------------------------------------------------------------ */

/* Device scratch bytes of cfd_probe_fma on the current device. */
size_t cfd_probe_fma_workspace(void);

/*
 * Measured fused multiply-add rate of the current GPU in flop/s (2 flops per
 * FMA): CFD_C128 probes the fp64 pipe, CFD_C64 the fp32 pipe.  Each thread of
 * a full wave of resident CTAs runs 8 independent chains of `iters` FMAs; one
 * short untimed launch precedes the launch timed with CUDA events on
 * `stream`.  It is the denominator of the roofline of an arithmetic-bound
 * step (Sect. 3.4 bounds the filter by min(memory, arithmetic); the paper
 * takes the arithmetic peak from the vendor's figure).  Synchronises
 * `stream`.  work: cfd_probe_fma_workspace() bytes of device memory.
 * Errors: CFD_ERR_ARG (prec, iters < 1, NULL), CFD_ERR_OOM, CFD_ERR_CUDA.
 */
cfd_status cfd_probe_fma(int prec, int iters, double *flops, void *work, size_t work_bytes,
                         cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* CFD_H */
