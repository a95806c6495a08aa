// Footprint-staged general steps (Algorithm 1, lines 9-12) for complex-float
// data and for complex double in double-word arithmetic.
//
// The gathered general steps read each row's V_cur entries with a dependent
// global load per slot, and their time goes to waiting for those loads.  Here
// the rows of V_cur one SELL chunk reads (its footprint) are copied into
// shared memory by TMA bulk copies before the chunk is computed, so the
// sparse product itself reads shared memory only.  The footprint of a chunk
// of a nearest-neighbour Hamiltonian is a handful of contiguous row ranges
// (for a Topi chunk of 32 rows = 8 sites: the chunk and its x-neighbours,
// and one range each for the y- and z-neighbour sites, about 168 rows), so a
// few bulk copies move it.  Per call, k_footprint finds each chunk's ranges
// and replaces every slot's column by its row in the staged footprint (16
// bits).  A CTA keeps S chunks in flight: while it computes chunk k from
// stage k mod S, the copies of the next S - 1 chunks (matrix slots, prepared
// values, V_prev rows, the X rows and the V_cur footprint) are landing.
// Chunks whose footprint does not fit a stage (more than FP_RMAX ranges or
// more rows than the stage holds) keep their slots' columns and are computed
// from global memory in the same launch.
//
// Every row's arithmetic is that of the gathered staged steps, operation for
// operation (k_cheb_step_staged with packed prepared values; k_cheb_step_dw),
// so the new vector and X are bit for bit theirs; the moments differ only by
// the order of their cross-row sums.
#include "dw_arith.cuh"
#include "step_kernels.cuh"

namespace cfd {

namespace {

constexpr int FP_RMAX = 16;     // row ranges of a staged footprint
constexpr int FP_GAP = 4;       // rows two ranges may be apart and still be merged
constexpr int FP_KEYS = 512;    // slots + own rows of a chunk the builder sorts
constexpr int FP_C = 32;        // chunk height the footprint steps are built for
// Slots of a chunk whose rows all have six neighbours (Topi, packed values):
// the on-site entry and 8 real hop entries, 4 imaginary ones.  Chunks of this
// shape take a fully unrolled row sum (compile-time slot indices, every
// shared-memory load of the row issued before its multiply-adds).
constexpr int FP_FULL_RE = 9, FP_FULL_IM = 4;
// Whether a thread loads its X row of its next chunk while it computes this
// one (where each thread has one row per chunk and X is not staged).
#ifndef CFD_FP_XPRE
#define CFD_FP_XPRE 1
#endif

// fn(K0), fn(K0 + 1), ..., fn(K1 - 1) with compile-time indices.
template <int K0, int K1, typename Fn>
__device__ __forceinline__ void unrolled(Fn &&fn) {
    if constexpr (K0 < K1) {
        fn(K0);
        unrolled<K0 + 1, K1>(fn);
    }
}

}  // namespace

// One arrival on a shared-memory mbarrier (release semantics).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Offsets of one stage's parts in dynamic shared memory (bytes), the same on
// host and device: slot rows (uint16), prepared values, the chunk's V_prev
// rows, its X rows (when staged), then the footprint rows.
struct FpLayout {
    uint32_t lcol, val, prev, xs, rows, stage;
};

__host__ __device__ inline uint32_t fp_round(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline FpLayout fp_layout(int slots_cap, int val_bytes, int row_bytes, int fmax, bool xst) {
    FpLayout L;
    L.lcol = 0;
    L.val = fp_round((uint32_t)slots_cap * 2u, 16);
    L.prev = L.val + fp_round((uint32_t)slots_cap * (uint32_t)val_bytes, 16);
    L.xs = L.prev + (uint32_t)FP_C * (uint32_t)row_bytes;
    L.rows = L.xs + (xst ? (uint32_t)FP_C * (uint32_t)row_bytes : 0u);
    L.stage = fp_round(L.rows + (uint32_t)fmax * (uint32_t)row_bytes, 128);
    return L;
}

// ------------------------------------------------------- footprint build --

// One CTA per chunk (grid-stride): the chunk's slot columns and own rows are
// sorted (bitonic, FP_KEYS keys, padding slots and unused keys INT_MAX),
// runs of keys no more than FP_GAP apart become ranges, and each slot's
// column is replaced by its row in the concatenated ranges.  The chunk's
// descriptor desc[c 32 + l] (32 int2, one coalesced 256-byte load for a
// warp) holds in word 0 {chunk_len, ranges (-1: not staged)}, word 1
// {footprint rows, row of the chunk's first own row}, word 2 the chunk's
// first slot (low, high 32 bits), word 3 {the chunk's realisation in a batch,
// 0}, words 8 + r {first row, rows} of range r.
__global__ void __launch_bounds__(256) k_footprint(const int32_t *col, const int64_t *chunk_ptr,
                                                   const int32_t *chunk_len, int64_t n_rows, int64_t n_chunks,
                                                   const int32_t *chunk_rid, int fmax, uint16_t *lcol, int2 *desc) {
    __shared__ int key[FP_KEYS];
    __shared__ int rs[FP_RMAX], re[FP_RMAX], ro[FP_RMAX];
    __shared__ int s_nr, s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const int cl = chunk_len[c];
        const int nslot = ((cl & 0xffff) + (cl >> 16)) * FP_C;
        const int64_t base = chunk_ptr[c];
        const int64_t r0 = c * FP_C;
        const int own = (int)(n_rows - r0 < FP_C ? n_rows - r0 : FP_C);
        const bool fits = nslot + own <= FP_KEYS;
        if (fits) {
            for (int t = tid; t < FP_KEYS; t += blockDim.x) {
                int k = INT_MAX;
                if (t < nslot) {
                    const int cc = col[base + t];
                    if (cc >= 0) k = cc;
                } else if (t < nslot + own) {
                    k = (int)(r0 + (t - nslot));
                }
                key[t] = k;
            }
            __syncthreads();
            for (int k = 2; k <= FP_KEYS; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int p = tid; p < FP_KEYS / 2; p += blockDim.x) {
                        const int i = 2 * p - (p & (j - 1));
                        const int a = key[i], b = key[i + j];
                        if ((a > b) == ((i & k) == 0)) {
                            key[i] = b;
                            key[i + j] = a;
                        }
                    }
                    __syncthreads();
                }
            }
        }
        if (warp == 0) {
            int nr = 0;
            if (fits) {
                for (int it = 0; it < FP_KEYS / 32; ++it) {
                    const int e = it * 32 + lane;
                    const int k = key[e];
                    const bool valid = k != INT_MAX;
                    const int kp = e > 0 ? key[e - 1] : INT_MAX;
                    const int kn = e + 1 < FP_KEYS ? key[e + 1] : INT_MAX;
                    const bool start = valid && (e == 0 || (int64_t)k - kp > FP_GAP);
                    const bool end = valid && (kn == INT_MAX || (int64_t)kn - k > FP_GAP);
                    const unsigned ms = __ballot_sync(0xffffffffu, start);
                    const int rid = nr + __popc(ms & (0xffffffffu >> (31 - lane))) - 1;
                    if (start && rid < FP_RMAX) rs[rid] = k;
                    if (end && rid >= 0 && rid < FP_RMAX) re[rid] = k + 1;
                    nr += __popc(ms);
                }
            }
            if (lane == 0) {
                bool ok = fits && nr <= FP_RMAX;
                int total = 0;
                if (ok)
                    for (int r = 0; r < nr; ++r) {
                        ro[r] = total;
                        total += re[r] - rs[r];
                    }
                ok = ok && total <= fmax;
                s_nr = ok ? nr : -1;
                s_total = ok ? total : 0;
            }
        }
        __syncthreads();
        const int nr = s_nr;
        auto local = [&](int cc) {     // row of column cc in the footprint (cc in one of the ranges)
            int lo = 0, hi = nr - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (rs[mid] <= cc) lo = mid;
                else hi = mid - 1;
            }
            return ro[lo] + (cc - rs[lo]);
        };
        if (tid < 32) {
            int2 d = make_int2(0, 0);
            if (tid == 0) d = make_int2(cl, nr);
            else if (tid == 1) d = make_int2(s_total, nr >= 0 ? local((int)r0) : 0);
            else if (tid == 2) d = make_int2((int)(uint32_t)base, (int)(uint32_t)((uint64_t)base >> 32));
            else if (tid == 3) d = make_int2(chunk_rid ? chunk_rid[c] : 0, 0);
            else if (tid >= 8 && tid - 8 < nr) d = make_int2(rs[tid - 8], re[tid - 8] - rs[tid - 8]);
            desc[c * 32 + tid] = d;
        }
        for (int t = tid; t < nslot; t += blockDim.x) {
            const int cc = col[base + t];
            lcol[base + t] = (uint16_t)((nr >= 0 && cc >= 0) ? local(cc) : 0);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- the step --

namespace {

enum FpMode : int { FPM_C64 = 0, FPM_DW = 1 };

// Scalar of the step arguments, one complex element of a block (complex float,
// or a double-word {re_hi, im_hi, re_lo, im_lo}), one packed slot value.
template <int MODE> struct FpTypes;
template <> struct FpTypes<FPM_C64> {
    using T = float;
    using E = float2;
    using V = float;
};
template <> struct FpTypes<FPM_DW> {
    using T = double;
    using E = float4;
    using V = float2;
};

// VPT consecutive elements (complex float pairs as one 16-byte access).
template <typename E, int VPT>
__device__ __forceinline__ void ld_elems(const E *p, E (&v)[VPT]) {
    if constexpr (std::is_same<E, float2>::value && VPT == 2) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        v[0] = make_float2(a.x, a.y);
        v[1] = make_float2(a.z, a.w);
    } else {
#pragma unroll
        for (int q = 0; q < VPT; ++q) v[q] = p[q];
    }
}

template <typename E, int VPT>
__device__ __forceinline__ void ldg_elems(const E *p, E (&v)[VPT]) {
    if constexpr (std::is_same<E, float2>::value && VPT == 2) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = make_float2(a.x, a.y);
        v[1] = make_float2(a.z, a.w);
    } else {
#pragma unroll
        for (int q = 0; q < VPT; ++q) v[q] = __ldg(p + q);
    }
}

template <typename E, int VPT>
__device__ __forceinline__ void st_elems(E *p, const E (&v)[VPT]) {
    if constexpr (std::is_same<E, float2>::value && VPT == 2) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    } else {
#pragma unroll
        for (int q = 0; q < VPT; ++q) p[q] = v[q];
    }
}

}  // namespace

// One general step W = P V_cur - V_prev, X += g_p W (P = 2 alpha (H - beta),
// prepared values), with the moments' dots <V_cur, V_cur>, Re <W, V_cur>.
// MODE FPM_C64: complex float; FPM_DW: complex double in double-word
// arithmetic (LAST: X written back as complex double).  Needs a C = 32 matrix
// with sigma = 1, packed values, V_cur and V_prev with row stride NB.
//
// One CTA per SM, chunks grid-stride, warp-specialised: warp W (the
// producer) stages chunk after chunk into a ring of S stages (TMA bulk
// copies completing on the stage's `full` mbarrier) and warps 0..W-1 (the
// consumers) compute each chunk's rows from shared memory, each warp
// releasing the stage through the stage's `empty` mbarrier when it is done
// with it; the producer refills a stage once all W consumer warps released
// it.  No CTA-wide barrier per chunk.  XST: the chunk's X rows are staged
// too (else each row's X is loaded when the row starts).  In the
// double-word step a thread's vectors are lane % TPR + q TPR, so the 16-byte
// shared-memory loads of a half-warp are contiguous (no bank conflicts).
// Bounded waits as in the other staged steps: a wait that expires stops the
// CTA (every warp leaves its loop; a shared flag tells the others), the
// producer waits for every copy it issued to land (also bounded) and records
// CFD_ERR_TIMEOUT in *A.status (with CFD_STATUS_DRAIN_EXPIRED if that wait
// expired too), and the CTA returns without its moments.  A.staged == 2 is
// the test of that path (every stage expects 16 bytes more than are copied).
template <int MODE, int NB, int VPT, bool MOM, bool LAST, int S, bool XST, int W, int CGT>
__global__ void __launch_bounds__((W + 1) * 32, 1)
k_cheb_step_fp(const StepArgs<typename FpTypes<MODE>::T> A, const FpView F, int slots_cap) {
    using E = typename FpTypes<MODE>::E;
    using V = typename FpTypes<MODE>::V;
    constexpr bool DW = MODE == FPM_DW;
    // a thread's vectors in units of G consecutive ones (16 bytes): unit u of
    // the row's NB vectors starts at u TPR G + (lane % TPR) G, so the 16-byte
    // shared-memory loads of the threads of a row are contiguous
    constexpr int G = 16 / (int)sizeof(E);
    static_assert(VPT % G == 0, "vectors per thread in whole 16-byte units");
    constexpr int TPR = NB / VPT;
    constexpr int RPW = 32 / TPR;
    constexpr int ROWS_PASS = W * RPW;
    // consumer groups: the warps split into CG groups of WG warps and group g
    // computes the CTA's chunks j = g (mod CG), each chunk's rows GROUP_PASS
    // at a time (CGT = 0: as many groups as the warps' rows fill chunks)
    constexpr int CG = CGT > 0 ? CGT : (ROWS_PASS > FP_C ? ROWS_PASS / FP_C : 1);
    constexpr int WG = W / CG;
    constexpr int GROUP_PASS = WG * RPW;
    static_assert(W % CG == 0 && S % CG == 0 && GROUP_PASS <= FP_C && FP_C % GROUP_PASS == 0,
                  "bad consumer groups");
    constexpr int RB = NB * (int)sizeof(E);
    static_assert(TPR >= 1 && TPR <= 32 && (32 % TPR) == 0, "bad thread split");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t empty[S];
    __shared__ int4 s_info[S];
    __shared__ float4 s_w[S];     // the chunk's weight g_p c_p: {as a float, double-word hi, lo, 0}
    __shared__ int s_abort;
    const FpLayout L = fp_layout(slots_cap, (int)sizeof(V), RB, F.fmax, XST);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = lane / TPR;
    const int jt = lane % TPR;
    auto jq = [&](int q) { return (q / G) * TPR * G + jt * G + q % G; };
    const int64_t n_rows = A.H.n_rows;
    const int64_t n_chunks = (n_rows + FP_C - 1) / FP_C;
    const E *vin = reinterpret_cast<const E *>(A.vin);
    E *wout = reinterpret_cast<E *>(A.w);
    E *xio = reinterpret_cast<E *>(A.x);
    const int64_t ldx = A.ldx;
    const V *gval = reinterpret_cast<const V *>(A.prep_val);
    const uint32_t tx_extra = A.staged == 2 ? 16u : 0u;
    const long long limit = A.staged == 2 ? (1LL << 24) : (1LL << 32);
    volatile int *abort_flag = &s_abort;

    MomentAcc<float> uu[VPT], wu[VPT];                       // complex float
    float2 uu_s2[VPT], uu_e2[VPT], wu_s2[VPT], wu_e2[VPT];   // double-word, per lane (re, im)
#pragma unroll
    for (int q = 0; q < VPT; ++q) uu_s2[q] = uu_e2[q] = wu_s2[q] = wu_e2[q] = make_float2(0.f, 0.f);

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], WG);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int64_t first = blockIdx.x, stride = gridDim.x;
    int issued = 0;              // producer: chunks issued
    bool drained_done = false;   // producer: stopped, its copies waited for and the status recorded
    // producer lane 0, after the CTA stopped: wait for the copies of the last
    // S issues (all issued ones, if fewer) and record the timeout
    auto drain = [&]() {
        const int j0 = issued > S ? issued - S : 0;
        if (tx_extra)
            for (int j = j0; j < issued; ++j) mbar_complete_tx(&full[j % S], tx_extra);
        bool drained = true;
        for (int j = j0; j < issued; ++j)
            drained = mbar_wait_bounded(&full[j % S], (uint32_t)((j / S) & 1), 1LL << 32) && drained;
        atomicOr(A.status, drained ? (int)CFD_ERR_TIMEOUT : (int)CFD_ERR_TIMEOUT | CFD_STATUS_DRAIN_EXPIRED);
    };

    if (warp == W) {
        // ------------------------------------------------------ producer --
        // a weight as a float and as a double-word {hi, lo}
        auto weight = [](double gd) {
            const float gh = __double2float_rn(gd);
            return make_float4(gh, gh, __double2float_rn(gd - (double)gh), 0.f);
        };
        const float4 w_step = A.chunk_rid ? make_float4(0.f, 0.f, 0.f, 0.f) : weight(A.gc[A.p]);
        // chunk c into stage s from its descriptor (lane l holds word l)
        auto issue = [&](int64_t c, int s, int2 d, double wd) {
            unsigned char *st = smem_raw + (size_t)s * L.stage;
            const int cl = __shfl_sync(0xffffffffu, d.x, 0);
            const int nr = __shfl_sync(0xffffffffu, d.y, 0);
            const int tot = __shfl_sync(0xffffffffu, d.x, 1);
            const int own_off = __shfl_sync(0xffffffffu, d.y, 1);
            const long long base = (long long)(((uint64_t)(uint32_t)__shfl_sync(0xffffffffu, d.y, 2) << 32) |
                                               (uint32_t)__shfl_sync(0xffffffffu, d.x, 2));
            const uint32_t nslot = (uint32_t)((cl & 0xffff) + (cl >> 16)) * FP_C;
            const int own = (int)(n_rows - c * FP_C < FP_C ? n_rows - c * FP_C : FP_C);
            int2 g;
            g.x = __shfl_sync(0xffffffffu, d.x, 8 + (lane & (FP_RMAX - 1)));
            g.y = __shfl_sync(0xffffffffu, d.y, 8 + (lane & (FP_RMAX - 1)));
            if (lane >= nr) g = make_int2(0, 0);
            // each range's first row in the stage: exclusive prefix of the rows
            int off = g.y;
#pragma unroll
            for (int d = 1; d < FP_RMAX; d <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, off, d);
                if (lane >= d) off += t;
            }
            off -= g.y;
            const uint32_t bytes = nslot * (uint32_t)sizeof(V) + (uint32_t)own * RB * (XST ? 2u : 1u) +
                                   (nr >= 0 ? nslot * 2u + (uint32_t)tot * RB : 0u) + tx_extra;
            if (lane == 0) {
                s_info[s] = make_int4(cl, nr, own_off, own);
                // the step's weight g_p c_p (in a batch, that of the chunk's realisation)
                s_w[s] = A.chunk_rid ? weight(wd) : w_step;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (lane == 0) mbar_expect_tx(&full[s], bytes);
            __syncwarp();
            if (lane == 0 && nr >= 0 && nslot) tma_load_1d(st + L.lcol, F.lcol + base, nslot * 2u, &full[s]);
            if (lane == 1 && nslot) tma_load_1d(st + L.val, gval + base, nslot * (uint32_t)sizeof(V), &full[s]);
            if (lane == 2) tma_load_1d(st + L.prev, wout + c * FP_C * NB, (uint32_t)own * RB, &full[s]);
            if (XST && lane < own) tma_load_1d(st + L.xs + lane * RB, xio + (c * FP_C + lane) * ldx, RB, &full[s]);
            if (lane < nr)
                tma_load_1d(st + L.rows + (uint32_t)off * RB, vin + (int64_t)g.x * NB, (uint32_t)g.y * RB, &full[s]);
        };
        bool failed = false;
        // descriptors two chunks ahead and (in a batch) each chunk's weight
        // one chunk ahead, so no load latency sits on the issue path
        auto ld_desc = [&](int64_t c) { return c < n_chunks ? __ldg(F.desc + c * 32 + lane) : make_int2(0, 0); };
        auto ld_weight = [&](int64_t c, int2 d) {
            if (!A.chunk_rid || c >= n_chunks) return 0.0;
            const int rid = __shfl_sync(0xffffffffu, d.x, 3);
            return __ldg(A.rcoef + (int64_t)rid * A.rcoef_ld + 2 + A.p);
        };
        int2 d1 = ld_desc(first), d2 = ld_desc(first + stride);
        double w1 = ld_weight(first, d1);
        for (int64_t c = first; c < n_chunks; c += stride, ++issued) {
            const int2 d = d1;
            const double wd = w1;
            d1 = d2;
            d2 = ld_desc(c + 2 * stride);
            w1 = ld_weight(c + stride, d1);
            const int s = issued % S;
            if (issued >= S) {
                const bool ok = mbar_wait_bounded(&empty[s], (uint32_t)((issued / S - 1) & 1), limit);
                if (__any_sync(0xffffffffu, !ok || *abort_flag)) {
                    failed = true;
                    break;
                }
            }
            issue(c, s, d, wd);
        }
        if (failed && lane == 0) {
            *abort_flag = 1;
            drain();
            drained_done = true;
        }
    } else {
        // ----------------------------------------------------- consumers --
        auto lds_row = [&](const E *rowp, E (&v)[VPT]) {     // shared memory, or plain global loads
#pragma unroll
            for (int u = 0; u < VPT / G; ++u) {
                E w[G];
                ld_elems<E, G>(rowp + u * TPR * G + jt * G, w);
#pragma unroll
                for (int t = 0; t < G; ++t) v[u * G + t] = w[t];
            }
        };
        auto ldg_row = [&](const E *rowp, E (&v)[VPT]) {     // read-only global loads
#pragma unroll
            for (int u = 0; u < VPT / G; ++u) {
                E w[G];
                ldg_elems<E, G>(rowp + u * TPR * G + jt * G, w);
#pragma unroll
                for (int t = 0; t < G; ++t) v[u * G + t] = w[t];
            }
        };
        auto st_row = [&](E *rowp, const E (&v)[VPT]) {
#pragma unroll
            for (int u = 0; u < VPT / G; ++u) {
                E w[G];
#pragma unroll
                for (int t = 0; t < G; ++t) w[t] = v[u * G + t];
                st_elems<E, G>(rowp + u * TPR * G + jt * G, w);
            }
        };
        // this warp's rows of one chunk from stage s; SM: V_cur rows from the
        // staged footprint (else, for an unstaged chunk, from global memory)
        // one row per thread and chunk, X not staged: each thread loads its X
        // row of the next chunk while it computes this one
        constexpr bool XPRE = CFD_FP_XPRE && !XST && GROUP_PASS == FP_C;
        const int grp = warp / WG;
        const int my_rr = (warp % WG) * RPW + sub;
        auto x_row_exists = [&](int64_t c) { return c < n_chunks && c * FP_C + my_rr < n_rows; };
        E xpre[VPT];
        auto rows = [&](auto sm_tag, int64_t c, int s, const E (&xin)[VPT]) {
            constexpr bool SM = decltype(sm_tag)::value;
            const int4 inf = s_info[s];
            const int cl = inf.x, own_off = inf.z, own = inf.w;
            const float4 wv = s_w[s];
            const float g0 = wv.x, gh = wv.y, gl = wv.z;
            (void)g0, (void)gh, (void)gl;
            const int nre = cl & 0xffff, len = nre + (cl >> 16);
            const unsigned char *st = smem_raw + (size_t)s * L.stage;
            const uint16_t *lc_s = reinterpret_cast<const uint16_t *>(st + L.lcol);
            const V *val_s = reinterpret_cast<const V *>(st + L.val);
            const E *prev_s = reinterpret_cast<const E *>(st + L.prev);
            const E *x_s = reinterpret_cast<const E *>(st + L.xs);
            (void)x_s;
            const E *rows_s = reinterpret_cast<const E *>(st + L.rows);
            const int64_t gbase = SM ? 0 : __ldg(A.H.chunk_ptr + c);
            for (int rr = my_rr; rr < own; rr += GROUP_PASS) {
                const int64_t i = c * FP_C + rr;
                auto vrow = [&](int kk, E (&v)[VPT]) {
                    if constexpr (SM) {
                        lds_row(rows_s + (int)lc_s[kk * FP_C + rr] * NB, v);
                    } else {
                        const int cc = max(__ldg(A.H.col + gbase + kk * FP_C + rr), 0);   // padding: col -1, value 0
                        ldg_row(vin + (int64_t)cc * NB, v);
                    }
                };
                E wo[VPT], xo[VPT], u[VPT];
                lds_row(prev_s + rr * NB, wo);
                if constexpr (XST) {
                    lds_row(x_s + rr * NB, xo);
                } else if constexpr (XPRE) {
#pragma unroll
                    for (int q = 0; q < VPT; ++q) xo[q] = xin[q];
                } else {
                    lds_row(xio + i * ldx, xo);
                }
                if constexpr (!DW) {
                    // complex float: the row sum starts at -V_prev; real slots
                    // add h v, imaginary slots i h v
                    E acc[VPT];
#pragma unroll
                    for (int q = 0; q < VPT; ++q) {
                        acc[q].x = -wo[q].x;
                        acc[q].y = -wo[q].y;
                    }
                    auto madd_re = [&](int kk) {
                        E v[VPT];
                        vrow(kk, v);
                        const float h = val_s[kk * FP_C + rr];
#pragma unroll
                        for (int q = 0; q < VPT; ++q) {
                            acc[q].x = fmaf(h, v[q].x, acc[q].x);
                            acc[q].y = fmaf(h, v[q].y, acc[q].y);
                        }
                    };
                    auto madd_im = [&](int kk) {
                        E v[VPT];
                        vrow(kk, v);
                        const float h = val_s[kk * FP_C + rr];
#pragma unroll
                        for (int q = 0; q < VPT; ++q) {
                            acc[q].x = fmaf(-h, v[q].y, acc[q].x);
                            acc[q].y = fmaf(h, v[q].x, acc[q].y);
                        }
                    };
                    if (nre == FP_FULL_RE && len == FP_FULL_RE + FP_FULL_IM) {
                        unrolled<0, FP_FULL_RE>(madd_re);
                        unrolled<FP_FULL_RE, FP_FULL_RE + FP_FULL_IM>(madd_im);
                    } else {
#pragma unroll 4
                        for (int kk = 0; kk < nre; ++kk) madd_re(kk);
#pragma unroll 4
                        for (int kk = nre; kk < len; ++kk) madd_im(kk);
                    }
                    E xn[VPT];
#pragma unroll
                    for (int q = 0; q < VPT; ++q) {
                        xn[q].x = fmaf(g0, acc[q].x, xo[q].x);
                        xn[q].y = fmaf(g0, acc[q].y, xo[q].y);
                    }
                    st_row(wout + i * NB, acc);
                    st_row(xio + i * ldx, xn);
                    if (MOM) {
                        if constexpr (SM) lds_row(rows_s + (own_off + rr) * NB, u);
                        else ldg_row(vin + i * NB, u);
#pragma unroll
                        for (int q = 0; q < VPT; ++q) {
                            uu[q].add2(u[q].x, u[q].x, u[q].y, u[q].y);
                            wu[q].add2(acc[q].x, u[q].x, acc[q].y, u[q].y);
                        }
                    }
                } else {
                    // double-word: (s, e) per lane (re, im), started at -V_prev;
                    // the imaginary group runs with the accumulator lanes swapped
                    float2 s2[VPT], e2[VPT];
#pragma unroll
                    for (int q = 0; q < VPT; ++q) {
                        s2[q] = make_float2(-wo[q].x, -wo[q].y);
                        e2[q] = make_float2(-wo[q].z, -wo[q].w);
                    }
                    auto madd_re = [&](int kk) {
                        E v[VPT];
                        vrow(kk, v);
                        const float2 h = val_s[kk * FP_C + rr];
                        const float2 hh = make_float2(h.x, h.x);
                        const float2 nhh = neg2(hh);
                        const float2 nhl = make_float2(-h.y, -h.y);
#pragma unroll
                        for (int q = 0; q < VPT; ++q)
                            dw_mac2(s2[q], e2[q], hh, nhh, nhl, make_float2(v[q].x, v[q].y),
                                    make_float2(v[q].z, v[q].w));
                    };
                    auto madd_im = [&](int kk) {
                        E v[VPT];
                        vrow(kk, v);
                        const float2 h = val_s[kk * FP_C + rr];
                        const float2 hh = make_float2(h.x, -h.x);
                        const float2 nhh = neg2(hh);
                        const float2 nhl = make_float2(-h.y, h.y);
#pragma unroll
                        for (int q = 0; q < VPT; ++q)
                            dw_mac2(s2[q], e2[q], hh, nhh, nhl, make_float2(v[q].x, v[q].y),
                                    make_float2(v[q].z, v[q].w));
                    };
                    auto swap_acc = [&]() {
#pragma unroll
                        for (int q = 0; q < VPT; ++q) {
                            s2[q] = swap2(s2[q]);
                            e2[q] = swap2(e2[q]);
                        }
                    };
                    if (nre == FP_FULL_RE && len == FP_FULL_RE + FP_FULL_IM) {
                        unrolled<0, FP_FULL_RE>(madd_re);
                        swap_acc();
                        unrolled<FP_FULL_RE, FP_FULL_RE + FP_FULL_IM>(madd_im);
                        swap_acc();
                    } else {
#pragma unroll 2
                        for (int kk = 0; kk < nre; ++kk) madd_re(kk);
                        swap_acc();
#pragma unroll 2
                        for (int kk = nre; kk < len; ++kk) madd_im(kk);
                        swap_acc();
                    }
                    if (MOM) {
                        if constexpr (SM) lds_row(rows_s + (own_off + rr) * NB, u);
                        else ldg_row(vin + i * NB, u);
                    }
                    E wn[VPT];
#pragma unroll
                    for (int q = 0; q < VPT; ++q) {
                        float2 nh, nl;
                        two_sum2(s2[q], e2[q], nh, nl);
                        wn[q] = make_float4(nh.x, nh.y, nl.x, nl.y);
                    }
                    st_row(wout + i * NB, wn);
#pragma unroll
                    for (int q = 0; q < VPT; ++q) {
                        const float2 wh = make_float2(wn[q].x, wn[q].y), wl = make_float2(wn[q].z, wn[q].w);
                        float2 xh = make_float2(xo[q].x, xo[q].y), xl = make_float2(xo[q].z, xo[q].w);
                        dw_axpy2(xh, xl, bcast2(gh), bcast2(-gh), bcast2(-gl), wh, wl);
                        if (LAST) {
                            double2 *xd = reinterpret_cast<double2 *>(xio + i * ldx + jq(q));
                            *xd = make_double2((double)xh.x + (double)xl.x, (double)xh.y + (double)xl.y);
                        } else {
                            xio[i * ldx + jq(q)] = make_float4(xh.x, xh.y, xl.x, xl.y);
                        }
                        if (MOM) {
                            const float2 uh = make_float2(u[q].x, u[q].y), ul = make_float2(u[q].z, u[q].w);
                            dw_mac2(uu_s2[q], uu_e2[q], uh, neg2(uh), neg2(ul), uh, ul);
                            dw_mac2(wu_s2[q], wu_e2[q], wh, neg2(wh), neg2(wl), uh, ul);
                        }
                    }
                }
            }
        };
        const int64_t gfirst = first + grp * stride;
        if (XPRE && x_row_exists(gfirst)) lds_row(xio + (gfirst * FP_C + my_rr) * ldx, xpre);
        int k = grp;
        for (int64_t c = gfirst; c < n_chunks; c += CG * stride, k += CG) {
            if (__any_sync(0xffffffffu, *abort_flag)) break;
            const int s = k % S;
            E xcur[VPT];
#pragma unroll
            for (int q = 0; q < VPT; ++q) xcur[q] = xpre[q];
            if (XPRE && x_row_exists(c + CG * stride)) lds_row(xio + ((c + CG * stride) * FP_C + my_rr) * ldx, xpre);
            const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((k / S) & 1), limit);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) *abort_flag = 1;
                break;
            }
            if (s_info[s].y >= 0) rows(std::integral_constant<bool, true>{}, c, s, xcur);
            else rows(std::integral_constant<bool, false>{}, c, s, xcur);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    __syncthreads();
    if (*abort_flag) {
        if (warp == W && lane == 0 && !drained_done) drain();
        return;
    }
    if (MOM) {
        if constexpr (DW) {
            // (s.x + e.x) + (s.y + e.y) as a Kahan-form accumulator (value s - c)
            auto lanes = [](float2 s2, float2 e2, MomentAcc<float> &m) {
                float t, err;
                two_sum(s2.x, s2.y, t, err);
                m.s = t;
                m.c = -__fadd_rn(__fadd_rn(e2.x, e2.y), err);
            };
#pragma unroll
            for (int q = 0; q < VPT; ++q) {
                lanes(uu_s2[q], uu_e2[q], uu[q]);
                lanes(wu_s2[q], wu_e2[q], wu[q]);
            }
        }
        reduce_moments<float, NB, VPT, W + 1, G>(A.partial, A.ticket, A.dots, uu, wu);
    }
}

// ---------------------------------------------------------------- launch --

// Stages in flight and whether X rows are staged, per mode: the tuned
// values, fixed at compile time.
#ifndef CFD_FP_C64_STAGES
#define CFD_FP_C64_STAGES 4
#endif
#ifndef CFD_FP_C64_XST
#define CFD_FP_C64_XST 0
#endif
#ifndef CFD_FP_DW_STAGES
#define CFD_FP_DW_STAGES 2
#endif
// Chunks per SM below which the filter keeps the gathered steps (unless the
// caller asks for the footprint steps explicitly).
#ifndef CFD_FP_MIN_CHUNKS_PER_SM
#define CFD_FP_MIN_CHUNKS_PER_SM 16
#endif
// Vectors per thread, and consumer warps of the CTA (one CTA per SM, plus
// the producer warp; 0: one row per thread and chunk, n_b / vpt warps).
// Complex float: 4 vectors per thread in 16 warps, two groups of 8 warps
// taking alternate chunks (fewer shared-memory loads of slot columns and
// values per row than 2 vectors per thread, and as many warps).
#ifndef CFD_FP_C64_VPT
#define CFD_FP_C64_VPT 4
#endif
#ifndef CFD_FP_DW_VPT
#define CFD_FP_DW_VPT 2
#endif
#ifndef CFD_FP_C64_WARPS
#define CFD_FP_C64_WARPS 16
#endif
#ifndef CFD_FP_DW_WARPS
#define CFD_FP_DW_WARPS 0
#endif
// Consumer groups (0: as many as the warps' rows fill chunks).
#ifndef CFD_FP_C64_GROUPS
#define CFD_FP_C64_GROUPS 0
#endif

namespace {

constexpr int FP_NB = 32;

template <int MODE> struct FpConf;
template <> struct FpConf<FPM_C64> {
    static constexpr int S = CFD_FP_C64_STAGES;
    static constexpr bool XST = CFD_FP_C64_XST != 0;
    static constexpr int VPT = CFD_FP_C64_VPT;
    static constexpr int W = CFD_FP_C64_WARPS ? CFD_FP_C64_WARPS : FP_NB / VPT;
    static constexpr int CG = CFD_FP_C64_GROUPS;
};
template <> struct FpConf<FPM_DW> {
    static constexpr int S = CFD_FP_DW_STAGES;
    static constexpr bool XST = false;
    static constexpr int VPT = CFD_FP_DW_VPT;
    static constexpr int W = CFD_FP_DW_WARPS ? CFD_FP_DW_WARPS : FP_NB / VPT;
    static constexpr int CG = 0;
};

// Dynamic shared memory a CTA may take next to the kernel's static shared
// memory (per device, cached).
template <int MODE>
cfd_status fp_smem_budget(size_t *out) {
    using Ty = FpTypes<MODE>;
    constexpr int S = FpConf<MODE>::S;
    constexpr bool XST = FpConf<MODE>::XST;
    static std::mutex mu;
    static size_t cache[64];
    int dev = 0;
    CFD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CFD_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!cache[dev]) {
        int optin = 0;
        CFD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        // the moments variant carries the reduction's static arrays
        cudaFuncAttributes fa{};
        constexpr int W = FpConf<MODE>::W;
        CFD_CUDA(cudaFuncGetAttributes(&fa, k_cheb_step_fp<MODE, FP_NB, FpConf<MODE>::VPT, true, false, S, XST, W, FpConf<MODE>::CG>));
        cudaFuncAttributes fb{};
        CFD_CUDA(cudaFuncGetAttributes(&fb, k_cheb_step_fp<MODE, FP_NB, FpConf<MODE>::VPT, true, true, S, XST, W, FpConf<MODE>::CG>));
        const size_t stat = std::max(fa.sharedSizeBytes, fb.sharedSizeBytes);
        cache[dev] = (size_t)optin > stat + 1024 ? (size_t)optin - stat - 1024 : 1;
    }
    *out = cache[dev];
    (void)sizeof(typename Ty::E);
    return CFD_OK;
}

template <int MODE>
int fp_rows_cap_t(int slots_cap) {
    using Ty = FpTypes<MODE>;
    constexpr int S = FpConf<MODE>::S;
    constexpr int RB = FP_NB * (int)sizeof(typename Ty::E);
    size_t budget = 0;
    if (fp_smem_budget<MODE>(&budget) != CFD_OK) {
        clear_error();
        return 0;
    }
    const FpLayout L0 = fp_layout(slots_cap, (int)sizeof(typename Ty::V), RB, 0, FpConf<MODE>::XST);
    const size_t per = budget / S / 128 * 128;
    if (per <= L0.rows) return 0;
    return (int)std::min<size_t>((per - L0.rows) / RB, 4096);
}

template <int MODE, bool MOM, bool LAST>
cfd_status launch_fp_t(const StepArgs<typename FpTypes<MODE>::T> &A, const FpView &F, int grid_cap,
                       cudaStream_t stream) {
    using Ty = FpTypes<MODE>;
    constexpr int S = FpConf<MODE>::S;
    constexpr bool XST = FpConf<MODE>::XST;
    constexpr int RB = FP_NB * (int)sizeof(typename Ty::E);
    const int slots_cap = A.H.slots_bound * FP_C;
    const FpLayout L = fp_layout(slots_cap, (int)sizeof(typename Ty::V), RB, F.fmax, XST);
    const size_t smem = (size_t)S * L.stage;
    size_t budget = 0;
    CFD_TRY(fp_smem_budget<MODE>(&budget));
    if (smem > budget) return fail(CFD_ERR_ARG, "footprint stages of %d rows need %zu bytes of shared memory", F.fmax, smem);
    constexpr int W = FpConf<MODE>::W;
    auto kern = k_cheb_step_fp<MODE, FP_NB, FpConf<MODE>::VPT, MOM, LAST, S, XST, W, FpConf<MODE>::CG>;
    struct Cache {
        std::mutex mu;
        int occ[64];
        size_t occ_smem[64];
        size_t attr_smem[64];
    };
    static Cache cache{};
    int dev = 0;
    CFD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CFD_ERR_ARG, "device ordinal %d out of range", dev);
    int resident = 0;
    {
        std::lock_guard<std::mutex> lock(cache.mu);
        if (smem > cache.attr_smem[dev]) {
            CFD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            cache.attr_smem[dev] = smem;
        }
        if (cache.occ[dev] == 0 || cache.occ_smem[dev] != smem) {
            int o = 0;
            CFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, (W + 1) * 32, smem));
            cache.occ[dev] = std::max(1, std::min(o, STEP_MAX_CTAS_PER_SM));
            cache.occ_smem[dev] = smem;
        }
        resident = cache.occ[dev];
    }
    const int64_t n_chunks = (A.H.n_rows + FP_C - 1) / FP_C;
    int64_t grid = std::min<int64_t>((int64_t)resident * sm_count(), n_chunks);
    if (grid_cap > 0) grid = std::min<int64_t>(grid, grid_cap);
    grid = std::max<int64_t>(grid, 1);
    kern<<<(unsigned)grid, (W + 1) * 32, smem, stream>>>(A, F, slots_cap);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

template <typename T>
cfd_status fp_check(const StepArgs<T> &A, const FpView &F, int nb, int vpt) {
    (void)vpt;    // the footprint step's own thread split; results do not depend on it
    if (nb != FP_NB) return fail(CFD_ERR_INTERNAL, "footprint step built for n_b = %d", FP_NB);
    if (!A.H.packed || A.H.log2C != 5 || A.H.perm || (A.chunk_rid && !A.rcoef))
        return fail(CFD_ERR_INTERNAL, "footprint step needs a packed C = 32, sigma = 1 matrix");
    if (A.ldin != FP_NB || A.ldw != FP_NB || !A.x || !A.status || !A.prep_val || F.fmax <= 0 || !F.lcol)
        return fail(CFD_ERR_INTERNAL, "footprint step arguments incomplete");
    return CFD_OK;
}

}  // namespace

size_t footprint_bytes(int64_t N) {
    const int64_t n_chunks = (N + FP_C - 1) / FP_C;
    return round_up((size_t)kMaxRowSlots * (size_t)(N + 127) * 2, 256) + round_up((size_t)n_chunks * 256, 256);
}

int footprint_rows_cap(const cfd_matrix *H, int nb, int vpt, bool dw, bool any_size) {
    const int slots_bound = (H->flags >> CFD_MATRIX_SLOTS_SHIFT) & 0xff;
    (void)vpt;
    if (nb != FP_NB || H->C != FP_C || H->perm || !(H->flags & CFD_MATRIX_PACKED)) return 0;
    if (slots_bound < 1 || slots_bound * FP_C + FP_C > FP_KEYS) return 0;
    if (H->n_rows >= (int64_t)INT_MAX) return 0;
    // one CTA per SM ramps its pipeline up per launch: below a few chunks per
    // SM the gathered steps (several CTAs per SM) are faster
    if (!any_size && H->n_chunks < (int64_t)CFD_FP_MIN_CHUNKS_PER_SM * sm_count()) return 0;
    if (dw ? H->prec != CFD_C128 : H->prec != CFD_C64) return 0;
    const int cap = dw ? fp_rows_cap_t<FPM_DW>(slots_bound * FP_C) : fp_rows_cap_t<FPM_C64>(slots_bound * FP_C);
    return std::min(cap, 65535);
}

cfd_status launch_footprint(const cfd_matrix *H, const int32_t *chunk_rid, int fmax, void *buf, size_t buf_bytes,
                            FpView *out, cudaStream_t stream) {
    const int64_t n_chunks = (H->n_rows + FP_C - 1) / FP_C;
    if (H->C != FP_C || H->n_chunks != n_chunks) return fail(CFD_ERR_INTERNAL, "footprint needs C = 32");
    if (H->n_slots > (int64_t)kMaxRowSlots * (H->n_rows + 127) || footprint_bytes(H->n_rows) > buf_bytes)
        return fail(CFD_ERR_INTERNAL, "footprint buffer too small");
    Carve c(buf, buf_bytes);
    uint16_t *lcol = c.take<uint16_t>((size_t)kMaxRowSlots * (size_t)(H->n_rows + 127));
    int2 *desc = c.take<int2>((size_t)n_chunks * 32);
    const int grid = (int)std::min<int64_t>(n_chunks, (int64_t)sm_count() * 8);
    k_footprint<<<grid, 256, 0, stream>>>(H->col, H->chunk_ptr, H->chunk_len, H->n_rows, n_chunks, chunk_rid, fmax,
                                          lcol, desc);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    out->lcol = lcol;
    out->desc = desc;
    out->fmax = fmax;
    return CFD_OK;
}

cfd_status launch_step_fp(const StepArgs<float> &A, const FpView &F, int nb, int vpt, int grid_cap,
                          cudaStream_t s) {
    CFD_TRY(fp_check(A, F, nb, vpt));
    return A.dots ? launch_fp_t<FPM_C64, true, false>(A, F, grid_cap, s)
                  : launch_fp_t<FPM_C64, false, false>(A, F, grid_cap, s);
}

cfd_status launch_step_fp_dw(const StepArgs<double> &A, const FpView &F, int nb, int vpt, bool last, int grid_cap,
                             cudaStream_t s) {
    CFD_TRY(fp_check(A, F, nb, vpt));
    if (A.dots)
        return last ? launch_fp_t<FPM_DW, true, true>(A, F, grid_cap, s)
                    : launch_fp_t<FPM_DW, true, false>(A, F, grid_cap, s);
    return last ? launch_fp_t<FPM_DW, false, true>(A, F, grid_cap, s)
                : launch_fp_t<FPM_DW, false, false>(A, F, grid_cap, s);
}

}  // namespace cfd
