// Dense fp64 building blocks for orthogonalisation and Rayleigh-Ritz.
#pragma once

#include "common.cuh"

namespace cfd {

constexpr int GRAM_MAX_SPLITS = 256;   // K-splits of a Gram (partials in the workspace)
constexpr int GRAM_TARGET_CTAS = 640;  // CTAs per Gram launch (about 4 per SM)
constexpr int RESID_MAX_CTAS = 1024;
constexpr int DENSE_MAX_COLS = 256;     // widest block for Gram / projection / Jacobi
constexpr int DENSE_BATCH_MAX_N = 64;   // widest block per realisation in batched dense kernels

// S (na x nb complex, ld lds) = X^H Y for N x na and N x nb blocks (unit column
// stride, ld in complex elements).  Deterministic (fixed-order split reduction).
// herm (na == nb, S Hermitian: X^H X, or X^H H X with Y = H X): only the
// output tiles on and above the diagonal are computed (about half the flops
// for n >= 64) and S below them is the conjugate mirror, as LAPACK's
// Hermitian eigensolvers read one triangle.
size_t gram_workspace(int64_t K, int na, int nb);
cfd_status gram(const double2 *X, int64_t ldx, int na, const double2 *Y, int64_t ldy, int nb, int64_t K,
                double2 *S, int64_t lds, double *work, cudaStream_t stream, bool herm = false);

// The same Gram in double-word arithmetic on the fp32 pipe (dense_dw.cu):
// same arguments and workspace; each split's sums accurate to a few units of
// 2^-48 of their terms instead of 2^-53.  gram_dw_split_cap: the most K-splits
// it uses (gram_workspace holds that many partials); launch_gram_fold: the
// fixed-order fold of the partials into S (shared with gram).
cfd_status gram_dw(const double2 *X, int64_t ldx, int na, const double2 *Y, int64_t ldy, int nb, int64_t K,
                   double2 *S, int64_t lds, double *work, cudaStream_t stream, bool herm = false);
int gram_dw_split_cap(int64_t K, int ma, int nb);
void launch_gram_fold(const double *part, int splits, int ma, int nb, double2 *S, int64_t lds, bool herm,
                      cudaStream_t stream);

// X[:, 0:n_out] <- X[:, 0:n_in] M (M n_in x n_out complex, ld ldm), in place, n_out <= n_in.
size_t project_workspace(int n_in, int n_out);
cfd_status project_inplace(double2 *X, int64_t ldx, int64_t n_rows, int n_in, const double2 *M, int64_t ldm,
                           int n_out, double *work, cudaStream_t stream);
// The same projection in double-word arithmetic (dense_dw.cu), same workspace.
cfd_status project_inplace_dw(double2 *X, int64_t ldx, int64_t n_rows, int n_in, const double2 *M, int64_t ldm,
                              int n_out, double *work, cudaStream_t stream);

// Eigen-decomposition of the Hermitian part of A (n x n): eigenvalues ascending
// in evals[n], eigenvectors in the columns of Q (ld ldq).  sweeps (host, nullable)
// receives the Jacobi sweep count after the stream completes.
size_t eigh_workspace(int n);
cfd_status eigh(const double2 *A, int64_t lda, int n, double *evals, double2 *Q, int64_t ldq, void *work,
                size_t work_bytes, cudaStream_t stream, int *sweeps);

// out[j] = || Z_j - theta_j X_j ||_2 (theta, X nullable: column norms of Z).
size_t resid_workspace(int n);
cfd_status resid_norms(const double2 *Z, int64_t ldz, const double2 *X, int64_t ldx, const double *theta, int n,
                       int64_t n_rows, double *out, double *work, cudaStream_t stream);

// Batched forms (realisation r owns rows [row_off[r], row_off[r+1]), device
// row_off; per-realisation outputs are stacked with the given strides).
size_t gram_batched_workspace(int R, int na, int nb);
cfd_status gram_batched(const double2 *X, int64_t ldx, int na, const double2 *Y, int64_t ldy, int nb,
                        const int64_t *row_off_dev, int R, double2 *S, int64_t lds, int64_t s_stride, double *work,
                        cudaStream_t stream, bool herm = false);
size_t project_batched_workspace(int R, int n);
cfd_status project_batched(double2 *X, int64_t ldx, int64_t n_rows, int n, const double2 *M, int64_t ldm,
                           int64_t m_stride, const int64_t *row_off_dev, int R, double *work, cudaStream_t stream);
cfd_status eigh_batched(const double2 *A, int64_t lda, int64_t a_stride, int n, int R, double *evals, double2 *Q,
                        int64_t ldq, int64_t q_stride, cudaStream_t stream);
size_t resid_batched_workspace(int R, int n);
cfd_status resid_norms_batched(const double2 *Z, int64_t ldz, const double2 *X, int64_t ldx, const double *theta,
                               int n, const int64_t *row_off_dev, int R, double *out, double *work,
                               cudaStream_t stream);

}  // namespace cfd
