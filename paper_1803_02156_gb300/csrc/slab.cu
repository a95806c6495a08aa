// The ChebFD filter distributed over z-slabs (Sect. 6): every rank holds the
// rows of its slab (cfd_build_matrix_slab), and before each fused step the
// boundary planes of the gathered block are exchanged with the neighbouring
// ranks into halo rows at the end of the recurrence blocks, so the unchanged
// step kernels gather local and halo rows alike.  Two schedules:
//   vector mode (Algorithm 3): block after block, exchange then step;
//   pipelined mode (Algorithm 4): all blocks advance one degree at a time,
//     the exchange for block b + 1 running on a second stream while block b
//     computes.
// Two exchangers share the driver: every slab in one process on the current
// device (halo planes moved by device copies: the distributed filter on one
// GPU, bit for bit the single-matrix filter), and one slab per process with
// NCCL point-to-point transfers (libnccl loaded at first use).  The partial
// moment dots of the slabs are summed (a kernel, or an NCCL all-reduce)
// before the moments are formed.
#include <dlfcn.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "filter.cuh"

namespace cfd {

namespace {

// ------------------------------------------------------------- NCCL API --

// The handful of NCCL entry points used, resolved from libnccl at run time
// (no link-time dependency: the library loads without NCCL).
struct NcclUniqueId {
    char internal[128];
};
enum { kNcclUint8 = 1, kNcclFloat64 = 8, kNcclSum = 0 };

struct NcclApi {
    bool ok = false;
    int (*get_unique_id)(NcclUniqueId *) = nullptr;
    int (*comm_init_rank)(void **, int, NcclUniqueId, int) = nullptr;
    int (*comm_destroy)(void *) = nullptr;
    int (*send)(const void *, size_t, int, int, void *, cudaStream_t) = nullptr;
    int (*recv)(void *, size_t, int, int, void *, cudaStream_t) = nullptr;
    int (*group_start)() = nullptr;
    int (*group_end)() = nullptr;
    int (*all_reduce)(const void *, void *, size_t, int, int, void *, cudaStream_t) = nullptr;
    const char *(*error_string)(int) = nullptr;
};

std::mutex g_nccl_mu;

const NcclApi *nccl() {
    static NcclApi api;
    static bool tried = false;
    std::lock_guard<std::mutex> lock(g_nccl_mu);
    if (tried) return api.ok ? &api : nullptr;
    tried = true;
    void *h = dlopen("libnccl.so.2", RTLD_NOW | RTLD_GLOBAL);
    if (!h) h = dlopen("libnccl.so", RTLD_NOW | RTLD_GLOBAL);
    if (!h) return nullptr;
    auto sym = [&](const char *n) { return dlsym(h, n); };
    api.get_unique_id = reinterpret_cast<int (*)(NcclUniqueId *)>(sym("ncclGetUniqueId"));
    api.comm_init_rank = reinterpret_cast<int (*)(void **, int, NcclUniqueId, int)>(sym("ncclCommInitRank"));
    api.comm_destroy = reinterpret_cast<int (*)(void *)>(sym("ncclCommDestroy"));
    api.send = reinterpret_cast<int (*)(const void *, size_t, int, int, void *, cudaStream_t)>(sym("ncclSend"));
    api.recv = reinterpret_cast<int (*)(void *, size_t, int, int, void *, cudaStream_t)>(sym("ncclRecv"));
    api.group_start = reinterpret_cast<int (*)()>(sym("ncclGroupStart"));
    api.group_end = reinterpret_cast<int (*)()>(sym("ncclGroupEnd"));
    api.all_reduce =
        reinterpret_cast<int (*)(const void *, void *, size_t, int, int, void *, cudaStream_t)>(sym("ncclAllReduce"));
    api.error_string = reinterpret_cast<const char *(*)(int)>(sym("ncclGetErrorString"));
    api.ok = api.get_unique_id && api.comm_init_rank && api.comm_destroy && api.send && api.recv &&
             api.group_start && api.group_end && api.all_reduce && api.error_string;
    return api.ok ? &api : nullptr;
}

#define CFD_NCCL(call)                                                                            \
    do {                                                                                          \
        int r_ = (call);                                                                          \
        if (r_ != 0) return ::cfd::fail(CFD_ERR_CUDA, "%s failed: %s", #call, api->error_string(r_)); \
    } while (0)

// ----------------------------------------------------------- slab state --

// One slab's buffers, carved from its workspace: the filter scratch (status,
// prepared values, weights, CTA partials, ticket), the per-block raw dots and
// the recurrence blocks, each n_local + 2 plane rows of n_b (halo rows last).
struct SlabState {
    const cfd_slab *slab = nullptr;
    const cfd_matrix *H = nullptr;
    cfd_block X{};
    int64_t rows_ext = 0;
    FilterScratch ws{};
    double *raw = nullptr;               // [n_raw_blocks][n_p][n_b][2]
    std::vector<char *> va, vb;          // per block (pipelined) or one pair
};

struct SlabLayout {
    size_t prep, raw, vbuf, fp, total;
    int n_vpairs;
};

SlabLayout slab_layout(const cfd_slab &s, int n_s, int n_b, int n_p, int prec, int mode) {
    const size_t sH = prec == CFD_C128 ? 16 : 8;
    const int n_blocks = n_s / n_b;
    SlabLayout L;
    L.n_vpairs = mode == 1 ? n_blocks : 1;
    L.prep = (size_t)kMaxRowSlots * (size_t)(s.n_local + 127) * sH;
    L.raw = (size_t)(mode == 1 ? n_blocks : 1) * n_p * n_b * 2;
    L.vbuf = (size_t)(s.n_local + 2 * s.plane) * n_b * sH;
    L.fp = n_b == 32 ? footprint_bytes(s.n_local) : 0;      // chunk footprints of the slab's rows
    Carve c(nullptr, 0);
    c.take<int>(64);
    c.take<char>(L.prep);
    c.take<double>((size_t)n_p + 1);
    c.take<double>((size_t)STEP_MAX_GRID * 2 * n_b);
    c.take<unsigned>(64);
    c.take<double>(L.raw);
    for (int k = 0; k < 2 * L.n_vpairs; ++k) c.take<char>(L.vbuf);
    if (L.fp) c.take<char>(L.fp);
    L.total = round_up(c.off, 256);
    return L;
}

// ------------------------------------------------------------ exchangers --

struct Exchanger {
    virtual ~Exchanger() = default;
    // fill the halo rows of recurrence buffer (which = 0: va, 1: vb) of
    // block pair k on every local slab, on stream s
    virtual cfd_status halo(std::vector<SlabState> &S, int which, int k, int n_b, size_t elem, cudaStream_t s) = 0;
    // raw dots of block pair k: every slab's array replaced by the sum over
    // all ranks (count doubles)
    virtual cfd_status sum_dots(std::vector<SlabState> &S, size_t off, size_t count, cudaStream_t s) = 0;
};

inline char *buf_of(SlabState &st, int which, int k) { return which ? st.vb[k] : st.va[k]; }

__global__ void k_add_into(double *dst, const double *src, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) dst[e] += src[e];
}

// Every slab in this process: planes moved by device copies.
struct LocalExchanger : Exchanger {
    cfd_status halo(std::vector<SlabState> &S, int which, int k, int n_b, size_t elem, cudaStream_t s) override {
        for (auto &st : S) {
            const cfd_slab &sl = *st.slab;
            const size_t pb = (size_t)sl.plane * n_b * elem;
            char *dst = buf_of(st, which, k);
            if (sl.lo_rank >= 0) {
                SlabState &lo = S[sl.lo_rank];
                const char *src = buf_of(lo, which, k) + (size_t)(lo.slab->n_local - lo.slab->plane) * n_b * elem;
                CFD_CUDA(cudaMemcpyAsync(dst + (size_t)sl.n_local * n_b * elem, src, pb, cudaMemcpyDeviceToDevice, s));
            }
            if (sl.hi_rank >= 0) {
                SlabState &hi = S[sl.hi_rank];
                CFD_CUDA(cudaMemcpyAsync(dst + (size_t)(sl.n_local + sl.plane) * n_b * elem, buf_of(hi, which, k), pb,
                                         cudaMemcpyDeviceToDevice, s));
            }
        }
        return CFD_OK;
    }
    cfd_status sum_dots(std::vector<SlabState> &S, size_t off, size_t count, cudaStream_t s) override {
        for (size_t r = 1; r < S.size(); ++r) {
            k_add_into<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(S[0].raw + off, S[r].raw + off, (int64_t)count);
            CFD_COUNT_LAUNCH();
            CFD_LAUNCH_CHECK();
        }
        for (size_t r = 1; r < S.size(); ++r)
            CFD_CUDA(cudaMemcpyAsync(S[r].raw + off, S[0].raw + off, count * sizeof(double), cudaMemcpyDeviceToDevice,
                                     s));
        return CFD_OK;
    }
};

// One slab per process over NCCL.  Per exchange every rank posts, in this
// order, the send of its top plane to hi_rank, the send of its bottom plane
// to lo_rank, the receive of the lower halo from lo_rank and the receive of
// the upper halo from hi_rank; a pair of ranks that are each other's lower
// and upper neighbour (two ranks, periodic z) then matches the top plane with
// the lower halo and the bottom plane with the upper halo.
struct NcclExchanger : Exchanger {
    const NcclApi *api;
    void *comm;
    NcclExchanger(const NcclApi *a, void *c) : api(a), comm(c) {}
    cfd_status halo(std::vector<SlabState> &S, int which, int k, int n_b, size_t elem, cudaStream_t s) override {
        SlabState &st = S[0];
        const cfd_slab &sl = *st.slab;
        const size_t pb = (size_t)sl.plane * n_b * elem;
        char *b = buf_of(st, which, k);
        CFD_NCCL(api->group_start());
        if (sl.hi_rank >= 0)
            CFD_NCCL(api->send(b + (size_t)(sl.n_local - sl.plane) * n_b * elem, pb, kNcclUint8, sl.hi_rank, comm, s));
        if (sl.lo_rank >= 0) CFD_NCCL(api->send(b, pb, kNcclUint8, sl.lo_rank, comm, s));
        if (sl.lo_rank >= 0)
            CFD_NCCL(api->recv(b + (size_t)sl.n_local * n_b * elem, pb, kNcclUint8, sl.lo_rank, comm, s));
        if (sl.hi_rank >= 0)
            CFD_NCCL(api->recv(b + (size_t)(sl.n_local + sl.plane) * n_b * elem, pb, kNcclUint8, sl.hi_rank, comm, s));
        CFD_NCCL(api->group_end());
        return CFD_OK;
    }
    cfd_status sum_dots(std::vector<SlabState> &S, size_t off, size_t count, cudaStream_t s) override {
        CFD_NCCL(api->all_reduce(S[0].raw + off, S[0].raw + off, count, kNcclFloat64, kNcclSum, comm, s));
        return CFD_OK;
    }
};

// ----------------------------------------------------------------- driver --

// Copy the n_b-column window X_b (ld ldx, n rows) into a contiguous buffer
// (ld n_b): the input of step 1, whose halo rows the exchange then fills.
cfd_status copy_window(const void *src, int64_t ldx, void *dst, int64_t n_rows, int n_b, size_t elem, cudaStream_t s) {
    CFD_CUDA(cudaMemcpy2DAsync(dst, (size_t)n_b * elem, src, (size_t)ldx * elem, (size_t)n_b * elem, (size_t)n_rows,
                               cudaMemcpyDeviceToDevice, s));
    return CFD_OK;
}

struct DistArgs {
    double lmin, lmax, lam_l, lam_r;
    int n_p, n_b, mode, arith, vpt;
    double *moments;
    int footprint;       // as cfd_filter_opts.footprint
};

template <typename T>
cfd_status run_dist(std::vector<SlabState> &S, Exchanger &ex, const DistArgs &D, cudaStream_t stream) {
    using C = cplx_t<T>;
    const int n_b = D.n_b, n_p = D.n_p;
    const int n_blocks = S[0].X.n_cols / n_b;
    const size_t elem = sizeof(C);
    const double alpha = 2.0 / (D.lmax - D.lmin), beta = 0.5 * (D.lmax + D.lmin);
    const bool dw = std::is_same<T, double>::value && D.arith == ARITH_DW && n_p >= 3;
    const int vpt = D.vpt > 0 ? D.vpt : default_vpt(S[0].H->prec, n_b);
    std::vector<StepArgs<T>> A(S.size());
    std::vector<FpView> F(S.size());     // the general steps' footprints, per slab (fmax 0: gathered steps)
    for (size_t r = 0; r < S.size(); ++r) {
        SlabState &st = S[r];
        CFD_CUDA(cudaMemsetAsync(st.ws.ticket, 0, sizeof(unsigned), stream));
        CFD_CUDA(cudaMemsetAsync(st.ws.status, 0, sizeof(int), stream));
        CFD_TRY(launch_filter_coeffs(alpha, beta, D.lam_l, D.lam_r, n_p, st.ws.gc, stream));
        if (dw)
            CFD_TRY(launch_prepare_values_dw(st.H, alpha, beta, nullptr, nullptr, 0, st.ws.prep, st.ws.prep_bytes,
                                             stream));
        else
            CFD_TRY(launch_prepare_values(st.H, alpha, beta, nullptr, nullptr, 0, st.ws.prep, st.ws.prep_bytes,
                                          stream));
        StepArgs<T> &a = A[r];
        a.H = sell_view<T>(st.H);
        a.gc = st.ws.gc;
        a.partial = st.ws.partial;
        a.ticket = st.ws.ticket;
        a.beta = beta;
        a.staged = (int)default_staged(st.H->prec);
        a.gather = default_gather(st.H->prec);
        a.status = st.ws.status;
        a.prep_val = st.ws.prep;
        // the footprint-staged general steps: a slab row's halo columns are
        // rows of the recurrence buffers past n_local, so footprints reach them
        if (D.footprint >= 0 && st.ws.fp && (dw || std::is_same<T, float>::value)) {
            int fmax = footprint_rows_cap(st.H, n_b, vpt, dw, D.footprint > 0);
            if (D.footprint > 0) fmax = std::min(fmax, D.footprint);
            if (fmax > 0) CFD_TRY(launch_footprint(st.H, nullptr, fmax, st.ws.fp, st.ws.fp_bytes, &F[r], stream));
        }
    }
    auto step = [&](size_t r, int kind, int p, bool last, cudaStream_t s) -> cfd_status {
        (void)p;
        if constexpr (std::is_same<T, double>::value) {
            if (dw && kind == STEP_GENERAL && F[r].fmax > 0)
                return launch_step_fp_dw(A[r], F[r], n_b, vpt, last, STEP_MAX_GRID, s);
            if (dw) return launch_step_dw(kind, n_b, vpt, A[r], last, STEP_MAX_GRID, s);
        } else {
            if (kind == STEP_GENERAL && F[r].fmax > 0) return launch_step_fp(A[r], F[r], n_b, vpt, STEP_MAX_GRID, s);
        }
        return launch_step<T>(kind, n_b, vpt, A[r], STEP_MAX_GRID, s);
    };
    // raw dots of block b: in pair k's region (vector mode: k = 0 for all)
    auto raw_of = [&](size_t r, int k, int p) { return S[r].raw + ((size_t)k * n_p + (p - 1)) * n_b * 2; };
    // steps 1 and 2 of block b with pair k
    auto seed_steps = [&](int b, int k) -> cfd_status {
        for (size_t r = 0; r < S.size(); ++r) {
            SlabState &st = S[r];
            C *xb = static_cast<C *>(st.X.ptr) + (size_t)b * n_b;
            if (dw) CFD_TRY(launch_dw_convert(xb, st.X.ld, st.X.n_rows, n_b, true, stream));
            CFD_TRY(copy_window(xb, st.X.ld, st.vb[k], st.X.n_rows, n_b, elem, stream));
        }
        CFD_TRY(ex.halo(S, 1, k, n_b, elem, stream));
        for (size_t r = 0; r < S.size(); ++r) {
            StepArgs<T> &a = A[r];
            a.vin = reinterpret_cast<C *>(S[r].vb[k]); a.ldin = n_b;
            a.w = reinterpret_cast<C *>(S[r].va[k]); a.ldw = n_b; a.x = nullptr; a.ldx = 0;
            a.a = alpha; a.p = 1; a.dots = D.moments ? raw_of(r, k, 1) : nullptr;
            CFD_TRY(step(r, STEP_FIRST, 1, false, stream));
        }
        CFD_TRY(ex.halo(S, 0, k, n_b, elem, stream));
        for (size_t r = 0; r < S.size(); ++r) {
            StepArgs<T> &a = A[r];
            a.vin = reinterpret_cast<C *>(S[r].va[k]); a.ldin = n_b;
            a.w = reinterpret_cast<C *>(S[r].vb[k]); a.ldw = n_b;
            a.x = static_cast<C *>(S[r].X.ptr) + (size_t)b * n_b; a.ldx = S[r].X.ld;
            a.a = 2.0 * alpha; a.p = 2; a.dots = D.moments ? raw_of(r, k, 2) : nullptr;
            CFD_TRY(step(r, STEP_SECOND, 2, false, stream));
        }
        return CFD_OK;
    };
    auto general = [&](int b, int k, int p, cudaStream_t s) -> cfd_status {
        for (size_t r = 0; r < S.size(); ++r) {
            StepArgs<T> &a = A[r];
            a.vin = reinterpret_cast<C *>((p & 1) ? S[r].vb[k] : S[r].va[k]); a.ldin = n_b;
            a.w = reinterpret_cast<C *>((p & 1) ? S[r].va[k] : S[r].vb[k]); a.ldw = n_b;
            a.x = static_cast<C *>(S[r].X.ptr) + (size_t)b * n_b; a.ldx = S[r].X.ld;
            a.p = p; a.dots = D.moments ? raw_of(r, k, p) : nullptr;
            CFD_TRY(step(r, STEP_GENERAL, p, p == n_p, s));
        }
        return CFD_OK;
    };
    auto finish_moments = [&](int b, int k) -> cfd_status {
        if (!D.moments) return CFD_OK;
        const size_t off = (size_t)k * n_p * n_b * 2;
        CFD_TRY(ex.sum_dots(S, off, (size_t)n_p * n_b * 2, stream));
        return launch_moments(S[0].raw + off, n_p, n_b, D.moments + (int64_t)b * n_b * 2 * n_p, 2 * n_p,
                              S[0].ws.status, stream);
    };

    if (D.mode == 0) {
        // vector mode (Algorithm 3): per block, exchange before every step
        for (int b = 0; b < n_blocks; ++b) {
            CFD_TRY(seed_steps(b, 0));
            for (int p = 3; p <= n_p; ++p) {
                CFD_TRY(ex.halo(S, (p & 1) ? 1 : 0, 0, n_b, elem, stream));
                CFD_TRY(general(b, 0, p, stream));
            }
            CFD_TRY(finish_moments(b, 0));
        }
        return CFD_OK;
    }
    // pipelined mode (Algorithm 4): the degree outside, the blocks inside; the
    // exchange for block b + 1 runs on a second stream while block b computes
    for (int b = 0; b < n_blocks; ++b) CFD_TRY(seed_steps(b, b));
    cudaStream_t xs = nullptr;
    CFD_CUDA(cudaStreamCreateWithFlags(&xs, cudaStreamNonBlocking));
    std::vector<cudaEvent_t> ev_done(n_blocks, nullptr), ev_halo(n_blocks, nullptr);
    struct Release {
        cudaStream_t &s;
        std::vector<cudaEvent_t> &a, &b;
        ~Release() {
            for (auto e : a) if (e) cudaEventDestroy(e);
            for (auto e : b) if (e) cudaEventDestroy(e);
            if (s) cudaStreamDestroy(s);
        }
    } rel{xs, ev_done, ev_halo};
    for (int b = 0; b < n_blocks; ++b) {
        CFD_CUDA(cudaEventCreateWithFlags(&ev_done[b], cudaEventDisableTiming));
        CFD_CUDA(cudaEventCreateWithFlags(&ev_halo[b], cudaEventDisableTiming));
        CFD_CUDA(cudaEventRecord(ev_done[b], stream));             // seed steps of every block done
    }
    for (int p = 3; p <= n_p; ++p) {
        const int which = (p & 1) ? 1 : 0;                           // buffer gathered at degree p
        CFD_CUDA(cudaStreamWaitEvent(xs, ev_done[0], 0));
        CFD_TRY(ex.halo(S, which, 0, n_b, elem, xs));
        CFD_CUDA(cudaEventRecord(ev_halo[0], xs));
        for (int b = 0; b < n_blocks; ++b) {
            if (b + 1 < n_blocks) {
                CFD_CUDA(cudaStreamWaitEvent(xs, ev_done[b + 1], 0));
                CFD_TRY(ex.halo(S, which, b + 1, n_b, elem, xs));
                CFD_CUDA(cudaEventRecord(ev_halo[b + 1], xs));
            }
            CFD_CUDA(cudaStreamWaitEvent(stream, ev_halo[b], 0));
            CFD_TRY(general(b, b, p, stream));
            CFD_CUDA(cudaEventRecord(ev_done[b], stream));
        }
    }
    for (int b = 0; b < n_blocks; ++b) CFD_TRY(finish_moments(b, b));
    return CFD_OK;
}

cfd_status check_dist(int n, const cfd_slab *slabs, const cfd_matrix *const *H, const cfd_block *X, int n_p, int n_b,
                      int mode, double lmin, double lmax, double lam_l, double lam_r) {
    if (!slabs || !H || !X) return fail(CFD_ERR_ARG, "NULL argument");
    if (mode != 0 && mode != 1) return fail(CFD_ERR_ARG, "mode=%d not in {0, 1}", mode);
    if (!(lmin < lmax) || !(lmin <= lam_l && lam_l < lam_r && lam_r <= lmax))
        return fail(CFD_ERR_ARG, "need lmin <= lam_l < lam_r <= lmax");
    for (int r = 0; r < n; ++r) {
        CFD_TRY(check_filter_args(H[r], n_p, X[r], n_b, 0));
        if (X[r].prec != H[r]->prec) return fail(CFD_ERR_ARG, "the distributed filter needs X in H's precision");
        if (H[r]->n_rows != slabs[r].n_local) return fail(CFD_ERR_ARG, "matrix %d is not its slab's", r);
        if (X[r].n_cols != X[0].n_cols || H[r]->prec != H[0]->prec)
            return fail(CFD_ERR_ARG, "slabs differ in block width or precision");
        // the step kernels' 32-bit gather offsets are chosen from the matrix's
        // own rows; a slab's halo rows must stay inside that range too
        if ((uint64_t)(slabs[r].n_local + 2 * slabs[r].plane) * (uint64_t)n_b >= (1ULL << 32))
            return fail(CFD_ERR_ARG, "slab %d too large: (n_local + 2 plane) n_b must stay below 2^32", r);
    }
    return CFD_OK;
}

cfd_status setup_states(std::vector<SlabState> &S, int n, const cfd_slab *slabs, const cfd_matrix *const *H,
                        const cfd_block *X, int n_p, int n_b, int mode, void *const *work, size_t work_bytes) {
    S.resize(n);
    for (int r = 0; r < n; ++r) {
        const SlabLayout L = slab_layout(slabs[r], X[r].n_cols, n_b, n_p, H[r]->prec, mode);
        if (!work[r] || work_bytes < L.total)
            return fail(CFD_ERR_OOM, "slab workspace %zu < %zu bytes", work_bytes, L.total);
        if (!aligned16(work[r])) return fail(CFD_ERR_ARG, "work must be 16-byte aligned");
        SlabState &st = S[r];
        st.slab = slabs + r;
        st.H = H[r];
        st.X = X[r];
        st.rows_ext = slabs[r].n_local + 2 * slabs[r].plane;
        Carve c(work[r], work_bytes);
        st.ws.status = c.take<int>(64);
        st.ws.prep_bytes = L.prep;
        st.ws.prep = c.take<char>(L.prep);
        st.ws.gc = c.take<double>((size_t)n_p + 1);
        st.ws.partial = c.take<double>((size_t)STEP_MAX_GRID * 2 * n_b);
        st.ws.ticket = c.take<unsigned>(64);
        st.raw = c.take<double>(L.raw);
        st.va.resize(L.n_vpairs);
        st.vb.resize(L.n_vpairs);
        for (int k = 0; k < L.n_vpairs; ++k) {
            st.va[k] = c.take<char>(L.vbuf);
            st.vb[k] = c.take<char>(L.vbuf);
        }
        st.ws.fp_bytes = L.fp;
        st.ws.fp = L.fp ? c.take<char>(L.fp) : nullptr;
        st.ws.grid_cap = STEP_MAX_GRID;
    }
    return CFD_OK;
}

cfd_status dist_filter(std::vector<SlabState> &S, Exchanger &ex, const DistArgs &D, cudaStream_t stream) {
    if (S[0].H->prec == CFD_C128) return run_dist<double>(S, ex, D, stream);
    return run_dist<float>(S, ex, D, stream);
}

}  // namespace

}  // namespace cfd

using namespace cfd;

extern "C" {

size_t cfd_filter_slab_workspace(const cfd_slab *s, int n_s, int n_b, int n_p, int prec, int mode) {
    if (!s || n_s < 1 || n_b < 1 || n_s % n_b || n_p < 2) return 0;
    return slab_layout(*s, n_s, n_b, n_p, prec & 0xff, mode).total;
}

cfd_status cfd_filter_slabs(int nranks, const cfd_slab *slabs, const cfd_matrix *const *H, double lmin, double lmax,
                            double lam_l, double lam_r, int n_p, const cfd_block *X, int n_b, int mode,
                            void *const *work, size_t work_bytes, double *moments, const cfd_filter_opts *opts,
                            cudaStream_t stream) {
    clear_error();
    if (nranks < 1 || !slabs) return fail(CFD_ERR_ARG, "nranks < 1 or slabs NULL");
    for (int r = 0; r < nranks; ++r)
        if (slabs[r].nranks != nranks || slabs[r].rank != r) return fail(CFD_ERR_ARG, "slab %d is not rank %d of %d", r, r, nranks);
    CFD_TRY(check_dist(nranks, slabs, H, X, n_p, n_b, mode, lmin, lmax, lam_l, lam_r));
    const int arith = opts ? opts->arith : 0;
    if (arith == ARITH_DW && (H[0]->prec != CFD_C128 || !(H[0]->flags & CFD_MATRIX_PACKED)))
        return fail(CFD_ERR_ARG, "double-word arithmetic needs packed complex-double slabs");
    std::vector<SlabState> S;
    CFD_TRY(setup_states(S, nranks, slabs, H, X, n_p, n_b, mode, work, work_bytes));
    LocalExchanger ex;
    if (opts && opts->footprint < -1) return fail(CFD_ERR_ARG, "footprint=%d < -1", opts->footprint);
    DistArgs D{lmin, lmax, lam_l, lam_r, n_p, n_b, mode, arith, opts ? opts->vpt : 0, moments,
               opts ? opts->footprint : 0};
    return dist_filter(S, ex, D, stream);
}

cfd_status cfd_nccl_unique_id(void *id) {
    clear_error();
    if (!id) return fail(CFD_ERR_ARG, "id is NULL");
    const NcclApi *api = nccl();
    if (!api) return fail(CFD_ERR_ARG, "libnccl could not be loaded");
    CFD_NCCL(api->get_unique_id(static_cast<NcclUniqueId *>(id)));
    return CFD_OK;
}

cfd_status cfd_nccl_comm_init(const void *id, int nranks, int rank, void **comm) {
    clear_error();
    if (!id || !comm) return fail(CFD_ERR_ARG, "id or comm is NULL");
    const NcclApi *api = nccl();
    if (!api) return fail(CFD_ERR_ARG, "libnccl could not be loaded");
    NcclUniqueId u;
    std::memcpy(&u, id, sizeof(u));
    CFD_NCCL(api->comm_init_rank(comm, nranks, u, rank));
    return CFD_OK;
}

cfd_status cfd_nccl_comm_destroy(void *comm) {
    clear_error();
    const NcclApi *api = nccl();
    if (!api) return fail(CFD_ERR_ARG, "libnccl could not be loaded");
    if (comm) CFD_NCCL(api->comm_destroy(comm));
    return CFD_OK;
}

cfd_status cfd_filter_slab_nccl(const cfd_slab *slab, const cfd_matrix *H, double lmin, double lmax, double lam_l,
                                double lam_r, int n_p, cfd_block X, int n_b, int mode, void *work, size_t work_bytes,
                                double *moments, const cfd_filter_opts *opts, void *comm, cudaStream_t stream) {
    clear_error();
    if (!slab || !comm) return fail(CFD_ERR_ARG, "slab or comm is NULL");
    CFD_TRY(check_dist(1, slab, &H, &X, n_p, n_b, mode, lmin, lmax, lam_l, lam_r));
    const int arith = opts ? opts->arith : 0;
    if (arith == ARITH_DW && (H->prec != CFD_C128 || !(H->flags & CFD_MATRIX_PACKED)))
        return fail(CFD_ERR_ARG, "double-word arithmetic needs a packed complex-double slab");
    const NcclApi *api = nccl();
    if (!api) return fail(CFD_ERR_ARG, "libnccl could not be loaded");
    std::vector<SlabState> S;
    void *w[1] = {work};
    CFD_TRY(setup_states(S, 1, slab, &H, &X, n_p, n_b, mode, w, work_bytes));
    NcclExchanger ex(api, comm);
    if (opts && opts->footprint < -1) return fail(CFD_ERR_ARG, "footprint=%d < -1", opts->footprint);
    DistArgs D{lmin, lmax, lam_l, lam_r, n_p, n_b, mode, arith, opts ? opts->vpt : 0, moments,
               opts ? opts->footprint : 0};
    return dist_filter(S, ex, D, stream);
}

}  // extern "C"
