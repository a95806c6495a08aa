// The ChebFD restart loop (Sect. 2): filter, SVQB orthogonalisation,
// Rayleigh-Ritz, convergence test; fp64 or mixed-precision filter policy.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "dense.cuh"
#include "filter.cuh"
#include "solve_rules.h"

namespace cfd {

size_t orthogonalize_workspace(int64_t N, int n);
cfd_status orthogonalize_impl(const cfd_block &X, double tol, int *rank_host, int *rank_dev, void *work,
                              size_t work_bytes, cudaStream_t stream, bool dw);
size_t rr_workspace(int64_t N, int n);
size_t orth_rr_workspace(int64_t N, int n);
cfd_status orth_rr_impl(const cfd_matrix *H, const cfd_block &X, double tol, int *rank_dev, double *evals,
                        double *resid, void *work, size_t work_bytes, cudaEvent_t e_mid, cudaStream_t stream,
                        bool dw);
cfd_status rayleigh_ritz_impl(const cfd_matrix *H, const cfd_block &X, double *evals, double *resid, void *work,
                              size_t work_bytes, cudaStream_t stream);
size_t bounds_workspace(int64_t N, int steps);
cfd_status spectral_bounds_dev(const cfd_matrix *H, int steps, uint64_t seed, double *out_dev, void *work,
                               size_t work_bytes, cudaStream_t stream);
cfd_status gaussian_block(double2 *X, int64_t ldx, int64_t N, int n, uint64_t seed, uint64_t tag, int col0,
                          int n_total, cudaStream_t stream);

namespace {

struct SolveWs {
    size_t filt, orth, rr, bnd, total;
};

SolveWs solve_ws(const cfd_matrix *H, const cfd_matrix *Hl, const cfd_solve_params *p) {
    SolveWs w;
    int64_t N = H->n_rows;
    w.filt = filter_workspace(N, p->n_s, p->n_b, p->n_p, CFD_C128, CFD_C128);
    if (Hl) w.filt = std::max(w.filt, filter_workspace(N, p->n_s, p->n_b, p->n_p, CFD_C64, CFD_C128));
    w.orth = orthogonalize_workspace(N, p->n_s) + 256;
    w.rr = std::max(rr_workspace(N, p->n_s), orth_rr_workspace(N, p->n_s));
    w.bnd = bounds_workspace(N, std::max(2, p->bounds_steps > 0 ? p->bounds_steps : 40)) + 256;
    // phases run one after another: the scratch is shared
    w.total = round_up(std::max(std::max(w.filt, w.orth), std::max(w.rr, w.bnd)), 256) + 8192;
    return w;
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

}  // namespace cfd

using namespace cfd;

extern "C" {

size_t cfd_solve_workspace(const cfd_matrix *H, const cfd_matrix *H_low, const cfd_solve_params *p) {
    if (!H || !p || p->n_s < 1 || p->n_b < 1 || p->n_p < 2) return 0;
    return solve_ws(H, H_low, p).total;
}

cfd_status cfd_solve(const cfd_matrix *H, const cfd_matrix *H_low, const cfd_solve_params *p, cfd_block X,
                     double *evals, double *resid, void *work, size_t work_bytes, cfd_solve_result *res,
                     cudaStream_t stream) {
    clear_error();
    CFD_TRY(check_matrix(H));
    if (!p || !evals || !resid || !res || !work) return fail(CFD_ERR_ARG, "NULL argument");
    if (H->prec != CFD_C128) return fail(CFD_ERR_ARG, "cfd_solve needs the complex-double matrix as H");
    if (p->policy < CFD_POLICY_FP64 || p->policy > CFD_POLICY_MIXED_DW)
        return fail(CFD_ERR_ARG, "unknown policy %d", p->policy);
    const bool mixed = p->policy == CFD_POLICY_MIXED || p->policy == CFD_POLICY_MIXED_DW;
    // complex-double filter applications, and the Gram matrices and
    // projections of SVQB and Rayleigh-Ritz, in double-word arithmetic
    const bool dw = p->policy == CFD_POLICY_FP64_DW || p->policy == CFD_POLICY_MIXED_DW;
    if (mixed) {
        if (!H_low) return fail(CFD_ERR_ARG, "mixed policy needs the complex-float matrix H_low");
        CFD_TRY(check_matrix(H_low));
        if (H_low->prec != CFD_C64 || H_low->n_rows != H->n_rows)
            return fail(CFD_ERR_ARG, "H_low must be the complex-float copy of H");
    }
    if (dw && !(H->flags & CFD_MATRIX_PACKED))
        return fail(CFD_ERR_ARG, "double-word policies need H with packed values (CFD_PACK_RI)");
    if (X.prec != CFD_C128 || X.n_cols != p->n_s || X.n_rows != H->n_rows)
        return fail(CFD_ERR_ARG, "X must be the N x n_s complex-double block");
    if (!(p->lam_l < p->lam_r)) return fail(CFD_ERR_ARG, "empty search window");
    if (p->max_iter < 1 || p->tol <= 0) return fail(CFD_ERR_ARG, "max_iter and tol must be positive");
    SolveWs ws = solve_ws(H, mixed ? H_low : nullptr, p);
    if (work_bytes < ws.total) return fail(CFD_ERR_OOM, "solve workspace %zu < %zu bytes", work_bytes, ws.total);

    const double t0 = now_s();
    char *scratch = static_cast<char *>(work) + 8192;      // first 8 KB: small device results
    size_t scratch_bytes = work_bytes - 8192;
    double *small = static_cast<double *>(work);           // [0..3] bounds
    double2 *Xp = static_cast<double2 *>(X.ptr);
    const int n = p->n_s;
    std::memset(res, 0, sizeof(*res));

    if (p->start == 0) CFD_TRY(gaussian_block(Xp, X.ld, X.n_rows, n, p->seed, 1, 0, n, stream));

    double lmin = p->lmin, lmax = p->lmax;
    if (!(lmin < lmax)) {
        int steps = p->bounds_steps > 0 ? p->bounds_steps : 40;
        CFD_TRY(spectral_bounds_dev(H, steps, p->seed, small, scratch, scratch_bytes, stream));
        double h[2];
        CFD_CUDA(cudaMemcpyAsync(h, small, sizeof(h), cudaMemcpyDeviceToHost, stream));
        CFD_CUDA(cudaStreamSynchronize(stream));
        lmin = h[0];
        lmax = h[1];
    }
    res->lmin = lmin;
    res->lmax = lmax;
    if (!(lmin <= p->lam_l && p->lam_r <= lmax))
        return fail(CFD_ERR_ARG, "window [%g, %g] not inside the spectral bounds [%g, %g]", p->lam_l, p->lam_r,
                    lmin, lmax);

    double *ev_dev = reinterpret_cast<double *>(static_cast<char *>(work) + 1024);   // n <= 256 doubles
    double *rs_dev = ev_dev + DENSE_MAX_COLS;
    ConvergenceTracker tr;
    tr.start(p->n_t, mixed);
    const double switch_tol = p->switch_tol > 0 ? p->switch_tol : 1e-4;
    res->rank_min = n;
    PhaseEvents ev;
    CFD_CUDA(ev.create());
    for (int it = 1; it <= p->max_iter; ++it) {
        cudaEvent_t e0 = ev.e[0], e1 = ev.e[1], e2 = ev.e[2], e3 = ev.e[3];
        cudaEventRecord(e0, stream);
        CFD_TRY(filter_impl_opts(tr.low ? H_low : H, lmin, lmax, p->lam_l, p->lam_r, p->n_p, X, p->n_b, 0, 0, 0, 0,
                                 scratch, scratch_bytes, nullptr, stream, 0, 0,
                                 (dw && !tr.low) ? ARITH_DW : ARITH_NATIVE));
        cudaEventRecord(e1, stream);
        int rank = n;
        // SVQB's first pass (t_orth), then its second pass folded into
        // Rayleigh-Ritz (t_rr)
        CFD_TRY(orth_rr_impl(H, X, 1e-14, reinterpret_cast<int *>(small + 8), ev_dev, rs_dev, scratch, scratch_bytes,
                             e2, stream, dw));
        cudaEventRecord(e3, stream);
        CFD_CUDA(cudaMemcpyAsync(evals, ev_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, stream));
        CFD_CUDA(cudaMemcpyAsync(resid, rs_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, stream));
        CFD_CUDA(cudaMemcpyAsync(&rank, small + 8, sizeof(int), cudaMemcpyDeviceToHost, stream));
        int dev_status = 0;          // the filter workspace starts with its status word
        CFD_CUDA(cudaMemcpyAsync(&dev_status, scratch, sizeof(int), cudaMemcpyDeviceToHost, stream));
        CFD_CUDA(cudaStreamSynchronize(stream));
        if ((dev_status & 0xff) == CFD_ERR_TIMEOUT) return fail(CFD_ERR_TIMEOUT, "a bounded device-side wait expired");
        const float a = ev.ms(0, 1), b = ev.ms(1, 2), c = ev.ms(2, 3);
        res->t_filter += a * 1e-3;
        res->t_orth += b * 1e-3;
        res->t_rr += c * 1e-3;
        res->rank_min = std::min(res->rank_min, rank);
        res->iters = it;
        if (tr.low) res->iters_low = it;

        int cnt = 0, cnt_low = 0;
        double mr = kNoPair, mrl = kNoPair;
        for (int j = 0; j < n; ++j) {
            if (!(evals[j] >= p->lam_l && evals[j] <= p->lam_r)) continue;
            if (resid[j] <= p->tol) ++cnt;
            else mr = std::min(mr, resid[j]);
            if (resid[j] <= switch_tol) ++cnt_low;
            else mrl = std::min(mrl, resid[j]);
        }
        res->n_conv = cnt;
        if (tr.update(cnt, cnt_low, mr, mrl)) {
            res->t_total = now_s() - t0;
            return CFD_OK;
        }
        if (tr.low && tr.switch_ready) tr.leave_low();
    }
    res->t_total = now_s() - t0;
    return fail(CFD_ERR_NOCONV, "no convergence in %d iterations (%d converged)", p->max_iter, res->n_conv);
}

}  // extern "C"
