// ChebFD restart loop on a batch of independent realisations (block-diagonal
// batch matrix from cfd_build_batch): every iteration runs the batched filter
// (one launch per step for all realisations), a batched SVQB and a batched
// Rayleigh-Ritz, each a handful of launches for the whole batch.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "dense.cuh"
#include "filter.cuh"
#include "solve_rules.h"

namespace cfd {

cfd_status spmmv_block(const cfd_matrix *H, const double2 *X, int64_t ldx, double2 *Z, int64_t ldz, int n,
                       double *partial, unsigned *ticket, double *dots, cudaStream_t stream);
cfd_status gaussian_block(double2 *X, int64_t ldx, int64_t N, int n, uint64_t seed, uint64_t tag, int col0,
                          int n_total, cudaStream_t stream);

namespace {

// Per realisation: d = diag(S)^{-1/2}, S~ = D S D (into S + n^2 of each slot).
__global__ void k_bsvqb_scale(double2 *S, int n, double *d) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    S += (int64_t)blockIdx.y * 2 * n * n;
    d += (int64_t)blockIdx.y * n;
    int a = e / n, b = e % n;
    double sa = S[a * n + a].x, sb = S[b * n + b].x;
    double da = sa > 0 ? 1.0 / sqrt(sa) : 1.0, db = sb > 0 ? 1.0 / sqrt(sb) : 1.0;
    if (a == b) d[a] = da;
    double2 z = S[e];
    S[n * n + e] = make_double2(z.x * da * db, z.y * da * db);
}

// Per realisation: M_ab = d_a Q_ab / sqrt(max(theta_b, tau theta_max)).
__global__ void k_bsvqb_coeff(const double2 *Q, const double *theta, const double *d, int n, double tau,
                              double2 *M, int *rank) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    Q += (int64_t)blockIdx.y * n * n;
    M += (int64_t)blockIdx.y * n * n;
    theta += (int64_t)blockIdx.y * n;
    d += (int64_t)blockIdx.y * n;
    double tmax = theta[n - 1];
    double floor_ = tau * (tmax > 0 ? tmax : 0.0);
    if (e == 0 && rank) {
        int r = 0;
        for (int b = 0; b < n; ++b) r += (theta[b] >= floor_ && theta[b] > 0) ? 1 : 0;
        rank[blockIdx.y] = r;
    }
    if (e >= n * n) return;
    int a = e / n, b = e % n;
    double th = fmax(theta[b], floor_);
    double s = th > 0 ? d[a] / sqrt(th) : 0.0;
    double2 q = Q[e];
    M[e] = make_double2(q.x * s, q.y * s);
}

// Zero the padding rows [row_end[r], row_off[r+1]) of every realisation.
__global__ void k_zero_padding(double2 *X, int64_t ldx, int n, const int64_t *row_off, const int64_t *row_end,
                               int R) {
    int r = blockIdx.y;
    int64_t a = row_end[r], e = row_off[r + 1];
    for (int64_t i = a + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < e; i += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < n; ++j) X[i * ldx + j] = make_double2(0.0, 0.0);
}

struct BWs {
    size_t small, dense, big, total;
};

BWs bws(const cfd_matrix *H, int R, const cfd_solve_params *p) {
    BWs w;
    const int n = p->n_s;
    const int64_t N = H->n_rows;
    Carve s(nullptr, 0);
    s.take<int64_t>((size_t)R + 1);                  // row_off
    s.take<int64_t>((size_t)R);                      // row_end
    s.take<double>((size_t)4 * R);                   // windows
    s.take<double>((size_t)R * n);                   // theta / evals
    s.take<double>((size_t)R * n);                   // resid
    s.take<double>((size_t)R * n);                   // d
    s.take<int>((size_t)R + 64);                     // rank
    w.small = round_up(s.off, 256);
    Carve d(nullptr, 0);
    d.take<double2>((size_t)R * 2 * n * n);          // S, S~
    d.take<double2>((size_t)R * n * n);              // Q
    d.take<double2>((size_t)R * n * n);              // M
    w.dense = round_up(d.off, 256);
    size_t filt = batched_workspace(N, R, n, p->n_b, p->n_p, CFD_C128, CFD_C128);
    filt = std::max(filt, batched_workspace(N, R, n, p->n_b, p->n_p, CFD_C64, CFD_C128));
    Carve r(nullptr, 0);
    r.take<double2>((size_t)N * n);                  // Z
    r.take<double>((size_t)STEP_MAX_GRID * 2 * 64);  // step partials
    r.take<unsigned>(64);
    r.take<char>(gram_batched_workspace(R, n, n));
    r.take<char>(project_batched_workspace(R, n));
    r.take<char>(resid_batched_workspace(R, n));
    w.big = round_up(std::max(filt, r.off), 256);
    w.total = w.small + w.dense + w.big;
    return w;
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" {

size_t cfd_solve_batched_workspace(const cfd_matrix *H, int R, const cfd_solve_params *p) {
    if (!H || !p || R < 1 || p->n_s < 1 || p->n_b < 1 || p->n_p < 2) return 0;
    return bws(H, R, p).total;
}

cfd_status cfd_solve_batched(const cfd_matrix *H, const cfd_matrix *H_low, const int32_t *chunk_rid, int R,
                             const int64_t *row_off, const int64_t *row_end, const double *windows,
                             const int32_t *n_t, const cfd_solve_params *p, cfd_block X, double *evals,
                             double *resid, cfd_solve_result *res, void *work, size_t work_bytes,
                             cudaStream_t stream) {
    clear_error();
    CFD_TRY(check_matrix(H));
    if (!p || !chunk_rid || !row_off || !row_end || !windows || !n_t || !evals || !resid || !res || !work || R < 1)
        return fail(CFD_ERR_ARG, "NULL argument");
    if (H->prec != CFD_C128) return fail(CFD_ERR_ARG, "H must be the complex-double batch");
    if (p->policy != CFD_POLICY_FP64 && p->policy != CFD_POLICY_MIXED)
        return fail(CFD_ERR_ARG, "the batched solve supports the FP64 and MIXED policies (got %d)", p->policy);
    const bool mixed = p->policy == CFD_POLICY_MIXED;
    if (mixed) {
        if (!H_low) return fail(CFD_ERR_ARG, "mixed policy needs the complex-float batch H_low");
        CFD_TRY(check_matrix(H_low));
        if (H_low->prec != CFD_C64 || H_low->n_rows != H->n_rows) return fail(CFD_ERR_ARG, "H_low mismatch");
    }
    const int n = p->n_s;
    if (n > DENSE_BATCH_MAX_N) return fail(CFD_ERR_ARG, "batched solve supports n_s <= %d", DENSE_BATCH_MAX_N);
    if (X.prec != CFD_C128 || X.n_cols != n || X.n_rows != H->n_rows || X.ld != n)
        return fail(CFD_ERR_ARG, "X must be the contiguous N_total x n_s complex-double block");
    if (p->max_iter < 1 || p->tol <= 0) return fail(CFD_ERR_ARG, "max_iter and tol must be positive");
    if (row_off[0] != 0 || row_off[R] != H->n_rows) return fail(CFD_ERR_ARG, "row offsets do not span the batch");
    for (int r = 0; r < R; ++r) {
        if (row_off[r] % 32 || row_end[r] < row_off[r] || row_end[r] > row_off[r + 1])
            return fail(CFD_ERR_ARG, "bad rows of realisation %d", r);
        const double *w = windows + 4 * r;
        if (!(w[0] < w[1] && w[0] <= w[2] && w[2] < w[3] && w[3] <= w[1]))
            return fail(CFD_ERR_ARG, "bad window of realisation %d", r);
    }
    BWs ws = bws(H, R, p);
    if (work_bytes < ws.total) return fail(CFD_ERR_OOM, "batched solve workspace %zu < %zu", work_bytes, ws.total);

    const double t0 = now_s();
    Carve sm(work, ws.small);
    int64_t *d_off = sm.take<int64_t>((size_t)R + 1);
    int64_t *d_end = sm.take<int64_t>((size_t)R);
    double *d_win = sm.take<double>((size_t)4 * R);
    double *theta = sm.take<double>((size_t)R * n);
    double *rs = sm.take<double>((size_t)R * n);
    double *dsc = sm.take<double>((size_t)R * n);
    int *rank = sm.take<int>((size_t)R + 64);
    Carve dn(static_cast<char *>(work) + ws.small, ws.dense);
    double2 *S = dn.take<double2>((size_t)R * 2 * n * n);
    double2 *Q = dn.take<double2>((size_t)R * n * n);
    double2 *M = dn.take<double2>((size_t)R * n * n);
    char *big = static_cast<char *>(work) + ws.small + ws.dense;
    Carve bg(big, ws.big);
    double2 *Z = bg.take<double2>((size_t)H->n_rows * n);
    double *spart = bg.take<double>((size_t)STEP_MAX_GRID * 2 * 64);
    unsigned *ticket = bg.take<unsigned>(64);
    double *gw = reinterpret_cast<double *>(bg.take<char>(gram_batched_workspace(R, n, n)));
    double *pw = reinterpret_cast<double *>(bg.take<char>(project_batched_workspace(R, n)));
    double *rw = reinterpret_cast<double *>(bg.take<char>(resid_batched_workspace(R, n)));

    CFD_CUDA(cudaMemcpyAsync(d_off, row_off, sizeof(int64_t) * (R + 1), cudaMemcpyHostToDevice, stream));
    CFD_CUDA(cudaMemcpyAsync(d_end, row_end, sizeof(int64_t) * R, cudaMemcpyHostToDevice, stream));
    CFD_CUDA(cudaMemcpyAsync(d_win, windows, sizeof(double) * 4 * R, cudaMemcpyHostToDevice, stream));
    double2 *Xp = static_cast<double2 *>(X.ptr);
    if (p->start == 0) CFD_TRY(gaussian_block(Xp, n, H->n_rows, n, p->seed, 1, 0, n, stream));
    k_zero_padding<<<dim3(4, R), 256, 0, stream>>>(Xp, n, n, d_off, d_end, R);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    CFD_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), stream));

    std::memset(res, 0, sizeof(cfd_solve_result) * R);
    std::vector<ConvergenceTracker> trk(R);
    for (int r = 0; r < R; ++r) trk[r].start(n_t[r], mixed);
    std::vector<char> done(R, 0);
    bool low = mixed;
    const double switch_tol = p->switch_tol > 0 ? p->switch_tol : 1e-4;
    const int nn = n * n;
    double tf = 0, to = 0, tr = 0;
    for (int r = 0; r < R; ++r) res[r].rank_min = n;
    PhaseEvents ev;
    CFD_CUDA(ev.create());
    cudaEvent_t *e = ev.e;
    for (int it = 1; it <= p->max_iter; ++it) {
        cudaEventRecord(e[0], stream);
        CFD_TRY(filter_batched_impl(low ? H_low : H, chunk_rid, R, d_win, p->n_p, X, p->n_b, 0, 0, big, ws.big,
                                    stream));
        cudaEventRecord(e[1], stream);
        // SVQB twice (Stathopoulos & Wu), batched over realisations
        for (int pass = 0; pass < 2; ++pass) {
            CFD_TRY(gram_batched(Xp, n, n, Xp, n, n, d_off, R, S, n, 2 * nn, gw, stream, true));
            k_bsvqb_scale<<<dim3((nn + 255) / 256, R), 256, 0, stream>>>(S, n, dsc);
            CFD_COUNT_LAUNCH();
            CFD_LAUNCH_CHECK();
            CFD_TRY(eigh_batched(S + nn, n, 2 * nn, n, R, theta, Q, n, nn, stream));
            k_bsvqb_coeff<<<dim3((nn + 255) / 256, R), 256, 0, stream>>>(Q, theta, dsc, n, 1e-14, M,
                                                                         pass == 0 ? rank : nullptr);
            CFD_COUNT_LAUNCH();
            CFD_LAUNCH_CHECK();
            CFD_TRY(project_batched(Xp, n, H->n_rows, n, M, n, nn, d_off, R, pw, stream));
        }
        cudaEventRecord(e[2], stream);
        // Rayleigh-Ritz: Z = H X (block diagonal), G_r = X_r^H Z_r, G_r = Y_r Theta_r Y_r^H
        CFD_TRY(spmmv_block(H, Xp, n, Z, n, n, spart, ticket, nullptr, stream));
        CFD_TRY(gram_batched(Xp, n, n, Z, n, n, d_off, R, S, n, 2 * nn, gw, stream, true));
        CFD_TRY(eigh_batched(S, n, 2 * nn, n, R, theta, Q, n, nn, stream));
        CFD_TRY(project_batched(Xp, n, H->n_rows, n, Q, n, nn, d_off, R, pw, stream));
        CFD_TRY(project_batched(Z, n, H->n_rows, n, Q, n, nn, d_off, R, pw, stream));
        CFD_TRY(resid_norms_batched(Z, n, Xp, n, theta, n, d_off, R, rs, rw, stream));
        cudaEventRecord(e[3], stream);
        std::vector<int> rk(R);
        CFD_CUDA(cudaMemcpyAsync(evals, theta, sizeof(double) * R * n, cudaMemcpyDeviceToHost, stream));
        CFD_CUDA(cudaMemcpyAsync(resid, rs, sizeof(double) * R * n, cudaMemcpyDeviceToHost, stream));
        CFD_CUDA(cudaMemcpyAsync(rk.data(), rank, sizeof(int) * R, cudaMemcpyDeviceToHost, stream));
        int dev_status = 0;          // the filter workspace starts with its status word
        CFD_CUDA(cudaMemcpyAsync(&dev_status, big, sizeof(int), cudaMemcpyDeviceToHost, stream));
        CFD_CUDA(cudaStreamSynchronize(stream));
        if ((dev_status & 0xff) == CFD_ERR_TIMEOUT) return fail(CFD_ERR_TIMEOUT, "a bounded device-side wait expired");
        const float a = ev.ms(0, 1), b = ev.ms(1, 2), c = ev.ms(2, 3);
        tf += a * 1e-3;
        to += b * 1e-3;
        tr += c * 1e-3;
        bool all_done = true, all_ready = true;
        for (int r = 0; r < R; ++r) {
            const double *w = windows + 4 * r;
            int cnt = 0, cnt_low = 0;
            double mr = kNoPair, mrl = kNoPair;
            for (int j = 0; j < n; ++j) {
                double th = evals[(int64_t)r * n + j], rr = resid[(int64_t)r * n + j];
                if (!(th >= w[2] && th <= w[3])) continue;
                if (rr <= p->tol) ++cnt;
                else mr = std::min(mr, rr);
                if (rr <= switch_tol) ++cnt_low;
                else mrl = std::min(mrl, rr);
            }
            res[r].n_conv = cnt;
            res[r].rank_min = std::min(res[r].rank_min, rk[r]);
            if (done[r]) continue;
            res[r].iters = it;
            if (low) {
                res[r].iters_low = it;
                if (!trk[r].switch_ready) trk[r].update(cnt, cnt_low, mr, mrl);
                all_ready = all_ready && trk[r].switch_ready;
                all_done = false;
            } else {
                if (trk[r].update(cnt, cnt_low, mr, mrl)) done[r] = 1;
                all_done = all_done && done[r];
            }
        }
        if (low && all_ready) {          // every realisation ready: continue in fp64
            low = false;
            for (auto &t : trk) t.leave_low();
        }
        if (!low && all_done) {
            double tt = now_s() - t0;
            for (int r = 0; r < R; ++r) {
                res[r].t_filter = tf;
                res[r].t_orth = to;
                res[r].t_rr = tr;
                res[r].t_total = tt;
            }
            return CFD_OK;
        }
    }
    double tt = now_s() - t0;
    for (int r = 0; r < R; ++r) {
        res[r].t_filter = tf;
        res[r].t_orth = to;
        res[r].t_rr = tr;
        res[r].t_total = tt;
    }
    return fail(CFD_ERR_NOCONV, "batched solve: not every realisation converged in %d iterations", p->max_iter);
}

}  // extern "C"
