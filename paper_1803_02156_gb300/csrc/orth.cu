// SVQB orthogonalisation, Rayleigh-Ritz with residual norms, and the dense
// helpers behind them, all in fp64 on the device.
#include <algorithm>

#include "dense.cuh"
#include "filter.cuh"

namespace cfd {

// d_a = 1 / sqrt(Re S_aa) (1 for a zero column); S~ = D S D.
__global__ void k_svqb_scale(double2 *S, int n, double *d) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    int a = e / n, b = e % n;
    double sa = S[(int64_t)a * n + a].x, sb = S[(int64_t)b * n + b].x;
    double da = sa > 0 ? 1.0 / sqrt(sa) : 1.0, db = sb > 0 ? 1.0 / sqrt(sb) : 1.0;
    if (a == b) d[a] = da;
    double2 z = S[e];
    // the scaled copy goes to the second half of the buffer (S stays intact)
    S[(int64_t)n * n + e] = make_double2(z.x * da * db, z.y * da * db);
}

// M_ab = d_a Q_ab / sqrt(max(theta_b, tau theta_max)); rank = #{theta_b >= tau theta_max}.
__global__ void k_svqb_coeff(const double2 *Q, const double *theta, const double *d, int n, double tau,
                             double2 *M, int *rank) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    double tmax = theta[n - 1];
    double floor_ = tau * (tmax > 0 ? tmax : 0.0);
    if (e == 0) {
        int r = 0;
        for (int b = 0; b < n; ++b) r += (theta[b] >= floor_ && theta[b] > 0) ? 1 : 0;
        *rank = r;
    }
    if (e >= n * n) return;
    int a = e / n, b = e % n;
    double th = fmax(theta[b], floor_);
    double s = th > 0 ? d[a] / sqrt(th) : 0.0;
    double2 q = Q[e];
    M[e] = make_double2(q.x * s, q.y * s);
}

size_t svqb_workspace(int64_t N, int n) {
    Carve c(nullptr, 0);
    c.take<double2>((size_t)2 * n * n);    // S, S~
    c.take<double2>((size_t)n * n);        // Q
    c.take<double2>((size_t)n * n);        // M
    c.take<double>((size_t)n);             // theta
    c.take<double>((size_t)n);             // d
    c.take<int>(64);                       // rank
    c.take<char>(gram_workspace(N, n, n));
    c.take<char>(project_workspace(n, n));
    c.take<char>(eigh_workspace(n));
    return round_up(c.off, 256);
}

// The N-row Gram and projection in native fp64 (FP64 tensor cores) or in
// double-word arithmetic on the fp32 pipe (dw).
static cfd_status gram_n(bool dw, const double2 *X, int64_t ldx, int na, const double2 *Y, int64_t ldy, int nb,
                         int64_t K, double2 *S, int64_t lds, double *work, cudaStream_t stream, bool herm) {
    return dw ? gram_dw(X, ldx, na, Y, ldy, nb, K, S, lds, work, stream, herm)
              : gram(X, ldx, na, Y, ldy, nb, K, S, lds, work, stream, herm);
}

static cfd_status project_n(bool dw, double2 *X, int64_t ldx, int64_t n_rows, int n_in, const double2 *M,
                            int64_t ldm, int n_out, double *work, cudaStream_t stream) {
    return dw ? project_inplace_dw(X, ldx, n_rows, n_in, M, ldm, n_out, work, stream)
              : project_inplace(X, ldx, n_rows, n_in, M, ldm, n_out, work, stream);
}

// One SVQB pass (Stathopoulos & Wu 2002): S = X^H X, D = diag(S)^{-1/2},
// D S D = Q Theta Q^H, X <- X D Q Theta^{-1/2} with Theta clamped below at
// tau max(Theta).  dw: the Gram and the projection in double-word arithmetic.
cfd_status svqb_pass(double2 *X, int64_t ldx, int64_t N, int n, double tau, void *work, size_t work_bytes,
                     int *rank_dev, cudaStream_t stream, bool dw) {
    Carve c(work, work_bytes);
    double2 *S = c.take<double2>((size_t)2 * n * n);
    double2 *Q = c.take<double2>((size_t)n * n);
    double2 *M = c.take<double2>((size_t)n * n);
    double *theta = c.take<double>((size_t)n);
    double *d = c.take<double>((size_t)n);
    int *rank = c.take<int>(64);
    double *gw = reinterpret_cast<double *>(c.take<char>(gram_workspace(N, n, n)));
    double *pw = reinterpret_cast<double *>(c.take<char>(project_workspace(n, n)));
    size_t ew_bytes = eigh_workspace(n);
    void *ew = c.take<char>(ew_bytes);
    if (!c.fits()) return fail(CFD_ERR_OOM, "orthogonalisation workspace too small");
    CFD_TRY(gram_n(dw, X, ldx, n, X, ldx, n, N, S, n, gw, stream, true));
    k_svqb_scale<<<(n * n + 255) / 256, 256, 0, stream>>>(S, n, d);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    CFD_TRY(eigh(S + (size_t)n * n, n, n, theta, Q, n, ew, ew_bytes, stream, nullptr));
    k_svqb_coeff<<<(n * n + 255) / 256, 256, 0, stream>>>(Q, theta, d, n, tau, M, rank_dev ? rank_dev : rank);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    CFD_TRY(project_n(dw, X, ldx, N, n, M, n, n, pw, stream));
    return CFD_OK;
}

cfd_status check_c128_block(const cfd_block &X) {
    if (!X.ptr || X.n_rows < 1 || X.n_cols < 1 || X.ld < X.n_cols) return fail(CFD_ERR_ARG, "invalid block");
    if (X.prec != CFD_C128) return fail(CFD_ERR_ARG, "dense fp64 operations need a complex-double block");
    if (!aligned16(X.ptr)) return fail(CFD_ERR_ARG, "block must be 16-byte aligned");
    if (X.n_cols > DENSE_MAX_COLS) return fail(CFD_ERR_ARG, "n_s=%d exceeds %d", X.n_cols, DENSE_MAX_COLS);
    return CFD_OK;
}

size_t orthogonalize_workspace(int64_t N, int n) { return svqb_workspace(N, n); }

cfd_status orthogonalize_impl(const cfd_block &X, double tol, int *rank_host, int *rank_dev, void *work,
                              size_t work_bytes, cudaStream_t stream, bool dw) {
    CFD_TRY(check_c128_block(X));
    if (!work) return fail(CFD_ERR_ARG, "work is NULL");
    if (work_bytes < orthogonalize_workspace(X.n_rows, X.n_cols))
        return fail(CFD_ERR_OOM, "orthogonalisation workspace too small");
    double tau = tol > 0 ? tol : 1e-14;
    double2 *Xp = static_cast<double2 *>(X.ptr);
    Carve c(work, work_bytes);
    int *r1 = c.take<int>(64);
    size_t rest = work_bytes - c.off;
    char *w2 = static_cast<char *>(work) + c.off;
    CFD_TRY(svqb_pass(Xp, X.ld, X.n_rows, X.n_cols, tau, w2, rest, rank_dev ? rank_dev : r1, stream, dw));
    CFD_TRY(svqb_pass(Xp, X.ld, X.n_rows, X.n_cols, tau, w2, rest, nullptr, stream, dw));
    if (rank_host) {
        CFD_CUDA(cudaMemcpyAsync(rank_host, rank_dev ? rank_dev : r1, sizeof(int), cudaMemcpyDeviceToHost, stream));
        CFD_CUDA(cudaStreamSynchronize(stream));
    }
    return CFD_OK;
}

// ---------------------------------------------------------- Rayleigh-Ritz --

int spmmv_width(int n) {
    for (int w : {64, 32, 16, 8})
        if (n % w == 0) return w;
    return 0;
}

// Z = H X, n_b columns at a time, with the plain SpMMV form of the fused step
// (alpha = 1, beta = 0).  partial/ticket/dots: step-kernel scratch.
cfd_status spmmv_block(const cfd_matrix *H, const double2 *X, int64_t ldx, double2 *Z, int64_t ldz, int n,
                       double *partial, unsigned *ticket, double *dots, cudaStream_t stream) {
    int nb = spmmv_width(n);
    if (!nb) return fail(CFD_ERR_ARG, "n_s=%d must be a multiple of 8", n);
    StepArgs<double> A;
    A.H = sell_view<double>(H);
    A.gc = nullptr;
    A.partial = partial;
    A.ticket = ticket;
    A.dots = dots;
    A.a = 1.0;
    A.beta = 0.0;
    A.p = 1;
    A.x = nullptr;
    A.ldx = 0;
    for (int b = 0; b < n / nb; ++b) {
        A.vin = X + (size_t)b * nb;
        A.ldin = ldx;
        A.w = Z + (size_t)b * nb;
        A.ldw = ldz;
        CFD_TRY(launch_step<double>(STEP_FIRST, nb, default_vpt(CFD_C128, nb), A, 0, stream));
    }
    return CFD_OK;
}

size_t rr_workspace(int64_t N, int n) {
    Carve c(nullptr, 0);
    c.take<double2>((size_t)N * n);        // Z
    c.take<double2>((size_t)n * n);        // G
    c.take<double2>((size_t)n * n);        // Y
    c.take<double>((size_t)STEP_MAX_GRID * 2 * 64);
    c.take<unsigned>(64);
    c.take<double>(2 * 64);
    c.take<char>(gram_workspace(N, n, n));
    c.take<char>(project_workspace(n, n));
    c.take<char>(eigh_workspace(n));
    c.take<char>(resid_workspace(n));
    return round_up(c.off, 256);
}

cfd_status rayleigh_ritz_impl(const cfd_matrix *H, const cfd_block &X, double *evals, double *resid, void *work,
                              size_t work_bytes, cudaStream_t stream) {
    CFD_TRY(check_matrix(H));
    CFD_TRY(check_c128_block(X));
    if (H->prec != CFD_C128) return fail(CFD_ERR_ARG, "Rayleigh-Ritz needs the complex-double matrix");
    if (X.n_rows != H->n_rows) return fail(CFD_ERR_ARG, "block rows do not match the matrix");
    if (!evals || !work) return fail(CFD_ERR_ARG, "evals or work is NULL");
    const int64_t N = X.n_rows;
    const int n = X.n_cols;
    if (work_bytes < rr_workspace(N, n)) return fail(CFD_ERR_OOM, "Rayleigh-Ritz workspace too small");
    Carve c(work, work_bytes);
    double2 *Z = c.take<double2>((size_t)N * n);
    double2 *G = c.take<double2>((size_t)n * n);
    double2 *Y = c.take<double2>((size_t)n * n);
    double *partial = c.take<double>((size_t)STEP_MAX_GRID * 2 * 64);
    unsigned *ticket = c.take<unsigned>(64);
    (void)c.take<double>(2 * 64);
    double *gw = reinterpret_cast<double *>(c.take<char>(gram_workspace(N, n, n)));
    double *pw = reinterpret_cast<double *>(c.take<char>(project_workspace(n, n)));
    size_t ewb = eigh_workspace(n);
    void *ew = c.take<char>(ewb);
    double *rw = reinterpret_cast<double *>(c.take<char>(resid_workspace(n)));
    double2 *Xp = static_cast<double2 *>(X.ptr);
    CFD_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), stream));
    CFD_TRY(spmmv_block(H, Xp, X.ld, Z, n, n, partial, ticket, nullptr, stream));   // no moments needed
    CFD_TRY(gram(Xp, X.ld, n, Z, n, n, N, G, n, gw, stream, true));   // X^H H X is Hermitian
    CFD_TRY(eigh(G, n, n, evals, Y, n, ew, ewb, stream, nullptr));
    CFD_TRY(project_inplace(Xp, X.ld, N, n, Y, n, n, pw, stream));
    CFD_TRY(project_inplace(Z, n, N, n, Y, n, n, pw, stream));
    if (resid) CFD_TRY(resid_norms(Z, n, Xp, X.ld, evals, n, N, resid, rw, stream));
    return CFD_OK;
}

// SVQB's second pass folded into Rayleigh-Ritz (the restart step of the
// solve): after the first pass X1 = X0 M1, the second pass would form
// X2 = X1 M2 and Rayleigh-Ritz then Z = H X2, G = X2^H Z.  With Z1 = H X1 and
// G1 = X1^H Z1 instead, H X2 = Z1 M2 and X2^H H X2 = M2^H G1 M2, so
// X <- X1 (M2 Y), Z <- Z1 (M2 Y) give the same Ritz pairs with one N x n x n
// product fewer (three Grams and three projections instead of four).
// Everything else as orthogonalize_impl followed by rayleigh_ritz_impl;
// rank_dev (nullable) receives the first pass's rank, and when e_mid is
// given it is recorded after the first pass.
size_t orth_rr_workspace(int64_t N, int n) {
    Carve c(nullptr, 0);
    c.take<int>(64);
    c.take<char>(svqb_workspace(N, n));
    c.take<double2>((size_t)N * n);        // Z
    c.take<double2>((size_t)2 * n * n);    // S2, S2~
    c.take<double2>((size_t)n * n);        // Q
    c.take<double2>((size_t)n * n);        // M2, then M2 Y
    c.take<double2>((size_t)n * n);        // G1
    c.take<double2>((size_t)n * n);        // T = G1 M2
    c.take<double2>((size_t)n * n);        // G = M2^H T
    c.take<double2>((size_t)n * n);        // Y
    c.take<double>((size_t)n);             // theta
    c.take<double>((size_t)n);             // d
    c.take<double>((size_t)STEP_MAX_GRID * 2 * 64);
    c.take<unsigned>(64);
    c.take<char>(gram_workspace(N, n, n));
    c.take<char>(project_workspace(n, n));
    c.take<char>(eigh_workspace(n));
    c.take<char>(resid_workspace(n));
    return round_up(c.off, 256);
}

cfd_status orth_rr_impl(const cfd_matrix *H, const cfd_block &X, double tol, int *rank_dev, double *evals,
                        double *resid, void *work, size_t work_bytes, cudaEvent_t e_mid, cudaStream_t stream,
                        bool dw) {
    CFD_TRY(check_matrix(H));
    CFD_TRY(check_c128_block(X));
    if (H->prec != CFD_C128) return fail(CFD_ERR_ARG, "Rayleigh-Ritz needs the complex-double matrix");
    if (X.n_rows != H->n_rows) return fail(CFD_ERR_ARG, "block rows do not match the matrix");
    if (!evals || !work) return fail(CFD_ERR_ARG, "evals or work is NULL");
    const int64_t N = X.n_rows;
    const int n = X.n_cols;
    if (work_bytes < orth_rr_workspace(N, n)) return fail(CFD_ERR_OOM, "orthogonalisation workspace too small");
    const double tau = tol > 0 ? tol : 1e-14;
    Carve c(work, work_bytes);
    int *r1 = c.take<int>(64);
    const size_t svqb_bytes = svqb_workspace(N, n);
    char *sw = c.take<char>(svqb_bytes);
    double2 *Z = c.take<double2>((size_t)N * n);
    double2 *S = c.take<double2>((size_t)2 * n * n);
    double2 *Q = c.take<double2>((size_t)n * n);
    double2 *M = c.take<double2>((size_t)n * n);
    double2 *G1 = c.take<double2>((size_t)n * n);
    double2 *T = c.take<double2>((size_t)n * n);
    double2 *G = c.take<double2>((size_t)n * n);
    double2 *Y = c.take<double2>((size_t)n * n);
    double *theta = c.take<double>((size_t)n);
    double *d = c.take<double>((size_t)n);
    double *partial = c.take<double>((size_t)STEP_MAX_GRID * 2 * 64);
    unsigned *ticket = c.take<unsigned>(64);
    double *gw = reinterpret_cast<double *>(c.take<char>(gram_workspace(N, n, n)));
    double *pw = reinterpret_cast<double *>(c.take<char>(project_workspace(n, n)));
    const size_t ewb = eigh_workspace(n);
    void *ew = c.take<char>(ewb);
    double *rw = reinterpret_cast<double *>(c.take<char>(resid_workspace(n)));
    double2 *Xp = static_cast<double2 *>(X.ptr);
    // first pass: X1 = X0 M1
    CFD_TRY(svqb_pass(Xp, X.ld, N, n, tau, sw, svqb_bytes, rank_dev ? rank_dev : r1, stream, dw));
    if (e_mid) CFD_CUDA(cudaEventRecord(e_mid, stream));
    // Z1 = H X1, S2 = X1^H X1, G1 = X1^H Z1
    CFD_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), stream));
    CFD_TRY(spmmv_block(H, Xp, X.ld, Z, n, n, partial, ticket, nullptr, stream));
    CFD_TRY(gram_n(dw, Xp, X.ld, n, Xp, X.ld, n, N, S, n, gw, stream, true));
    CFD_TRY(gram_n(dw, Xp, X.ld, n, Z, n, n, N, G1, n, gw, stream, true));
    // second pass's coefficients M2 = D Q Theta^{-1/2} from S2
    k_svqb_scale<<<(n * n + 255) / 256, 256, 0, stream>>>(S, n, d);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    CFD_TRY(eigh(S + (size_t)n * n, n, n, theta, Q, n, ew, ewb, stream, nullptr));
    k_svqb_coeff<<<(n * n + 255) / 256, 256, 0, stream>>>(Q, theta, d, n, tau, M, r1 + 32);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    // G = M2^H G1 M2 (G1 Hermitian: G1^H M2 = G1 M2), its eigenvectors Y
    CFD_TRY(gram(G1, n, n, M, n, n, n, T, n, gw, stream));
    CFD_TRY(gram(M, n, n, T, n, n, n, G, n, gw, stream));
    CFD_TRY(eigh(G, n, n, evals, Y, n, ew, ewb, stream, nullptr));
    // W = M2 Y; X <- X1 W, Z <- Z1 W; residual norms
    CFD_TRY(project_inplace(M, n, n, n, Y, n, n, pw, stream));
    CFD_TRY(project_n(dw, Xp, X.ld, N, n, M, n, n, pw, stream));
    CFD_TRY(project_n(dw, Z, n, N, n, M, n, n, pw, stream));
    if (resid) CFD_TRY(resid_norms(Z, n, Xp, X.ld, evals, n, N, resid, rw, stream));
    return CFD_OK;
}

}  // namespace cfd

using namespace cfd;

extern "C" {

size_t cfd_gram_workspace(int64_t N, int n_x, int n_y) { return gram_workspace(N, n_x, n_y); }

cfd_status cfd_block_gram(cfd_block X, cfd_block Y, void *S, int64_t lds, void *work, size_t work_bytes,
                          cudaStream_t stream) {
    return cfd_block_gram_ex(X, Y, S, lds, work, work_bytes, 0, stream);
}

cfd_status cfd_block_gram_ex(cfd_block X, cfd_block Y, void *S, int64_t lds, void *work, size_t work_bytes,
                             int arith, cudaStream_t stream) {
    clear_error();
    if (arith != 0 && arith != 1) return fail(CFD_ERR_ARG, "arith=%d not in {0, 1}", arith);
    CFD_TRY(check_c128_block(X));
    CFD_TRY(check_c128_block(Y));
    if (X.n_rows != Y.n_rows) return fail(CFD_ERR_ARG, "blocks differ in rows");
    if (!S || lds < Y.n_cols) return fail(CFD_ERR_ARG, "S is NULL or lds < n_y");
    if (!work || work_bytes < gram_workspace(X.n_rows, X.n_cols, Y.n_cols))
        return fail(CFD_ERR_OOM, "Gram workspace too small");
    return gram_n(arith == 1, static_cast<const double2 *>(X.ptr), X.ld, X.n_cols, static_cast<const double2 *>(Y.ptr), Y.ld,
                Y.n_cols, X.n_rows, static_cast<double2 *>(S), lds, static_cast<double *>(work), stream, false);
}

size_t cfd_eigh_workspace(int n) { return n > 0 ? eigh_workspace(n) : 0; }

cfd_status cfd_eigh(const void *A, int64_t lda, int n, double *evals, void *Q, int64_t ldq, void *work,
                    size_t work_bytes, cudaStream_t stream) {
    clear_error();
    if (!A || !evals || !Q || !work) return fail(CFD_ERR_ARG, "NULL argument");
    if (n < 1 || n > DENSE_MAX_COLS || lda < n || ldq < n) return fail(CFD_ERR_ARG, "bad size n=%d", n);
    return eigh(static_cast<const double2 *>(A), lda, n, evals, static_cast<double2 *>(Q), ldq, work, work_bytes,
                stream, nullptr);
}

size_t cfd_orthogonalize_workspace(int64_t N, int n_s) {
    return (N > 0 && n_s > 0) ? orthogonalize_workspace(N, n_s) + 256 : 0;
}

cfd_status cfd_orthogonalize(cfd_block X, double tol, int *rank, void *work, size_t work_bytes,
                             cudaStream_t stream) {
    clear_error();
    return orthogonalize_impl(X, tol, rank, nullptr, work, work_bytes, stream, false);
}

cfd_status cfd_orthogonalize_ex(cfd_block X, double tol, int *rank, void *work, size_t work_bytes, int arith,
                                cudaStream_t stream) {
    clear_error();
    if (arith != 0 && arith != 1) return fail(CFD_ERR_ARG, "arith=%d not in {0, 1}", arith);
    return orthogonalize_impl(X, tol, rank, nullptr, work, work_bytes, stream, arith == 1);
}

size_t cfd_rayleigh_ritz_workspace(int64_t N, int n_s) { return (N > 0 && n_s > 0) ? rr_workspace(N, n_s) : 0; }

cfd_status cfd_rayleigh_ritz(const cfd_matrix *H, cfd_block X, double *evals, double *resid, void *work,
                             size_t work_bytes, cudaStream_t stream) {
    clear_error();
    return rayleigh_ritz_impl(H, X, evals, resid, work, work_bytes, stream);
}

}  // extern "C"
