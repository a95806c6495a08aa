// Fused ChebFD step kernels (templates).  Included by the four step_*.cu
// translation units, each instantiating one (precision, value storage) pair.
#pragma once

#include <algorithm>
#include <atomic>
#include <cooperative_groups.h>
#include <mutex>
#include <type_traits>

#include "filter.cuh"

// Gathers of a row in flight together in the grouped loops, and the CTAs
// per SM the complex-float staged step's registers are capped for (0: no
// cap): the tuned values, fixed at compile time.
#ifndef CFD_STAGED_UNR
#define CFD_STAGED_UNR 4
#endif
#ifndef CFD_STAGED_MINB_F32
#define CFD_STAGED_MINB_F32 0
#endif

namespace cfd {

namespace cg = cooperative_groups;

__device__ __forceinline__ size_t round_up_dev(size_t x, size_t a) { return (x + a - 1) / a * a; }

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ------------------------------------------------------ step kernel --

namespace {

template <typename T> struct MomentAcc;

// fp64 path: plain fp64 sums per thread.
template <> struct MomentAcc<double> {
    double s = 0.0;
    // s += a b + c d as two fused multiply-adds (fp64 is the scarce pipe)
    __device__ void add2(double a, double b, double c, double d) { s = fma(c, d, fma(a, b, s)); }
    __device__ double value() const { return s; }
};

// fp32 path: compensated (Kahan) fp32 sums per thread, widened once at the end.
template <> struct MomentAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ void add2(float a, float b, float c2, float d) {
        float y = fma(a, b, c2 * d) - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ double value() const { return (double)s - (double)c; }
};

template <typename C, int VPT> struct Pack { C v[VPT]; };


template <typename C, int VPT>
__device__ __forceinline__ Pack<C, VPT> ld_nc(const C *p) {
    Pack<C, VPT> r;
#pragma unroll
    for (int q = 0; q < VPT; ++q) r.v[q] = __ldg(p + q);
    return r;
}

template <>
__device__ __forceinline__ Pack<float2, 2> ld_nc<float2, 2>(const float2 *p) {
    float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    Pack<float2, 2> r;
    r.v[0] = make_float2(a.x, a.y);
    r.v[1] = make_float2(a.z, a.w);
    return r;
}

template <typename C, int VPT>
__device__ __forceinline__ Pack<C, VPT> ld_rw(const C *p) {
    Pack<C, VPT> r;
#pragma unroll
    for (int q = 0; q < VPT; ++q) r.v[q] = p[q];
    return r;
}

template <>
__device__ __forceinline__ Pack<float2, 2> ld_rw<float2, 2>(const float2 *p) {
    float4 a = *reinterpret_cast<const float4 *>(p);
    Pack<float2, 2> r;
    r.v[0] = make_float2(a.x, a.y);
    r.v[1] = make_float2(a.z, a.w);
    return r;
}

template <typename C, int VPT>
__device__ __forceinline__ void st(C *p, const Pack<C, VPT> &r) {
#pragma unroll
    for (int q = 0; q < VPT; ++q) p[q] = r.v[q];
}

template <>
__device__ __forceinline__ void st<float2, 2>(float2 *p, const Pack<float2, 2> &r) {
    *reinterpret_cast<float4 *>(p) = make_float4(r.v[0].x, r.v[0].y, r.v[1].x, r.v[1].y);
}

}  // namespace


// Load of one slot word: shared memory (staged chunks) or the read-only path.
template <bool SMEM, typename V>
__device__ __forceinline__ V ld_slot(const V *p) {
    if constexpr (SMEM) return *p;
    else return __ldg(p);
}

// Packed slots [k0, k1) of one row (slot k at colp[k << log2C]): each holds
// one real scalar h; the group is real (h v added to acc) or imaginary
// (i h v added: (-h vy, h vx)).  Padding slots (col -1, h 0) gather row 0 and
// add zero.  U loads in flight.
template <typename T, int VPT, bool IMAG, int U, bool SMEM>
__device__ __forceinline__ void packed_group(const StepArgs<T> &A, const int32_t *colp, const T *valp, int log2C,
                                             int k0, int k1, int j0, cplx_t<T> (&acc)[VPT]) {
    using C = cplx_t<T>;
    int k = k0;
    for (; k + U <= k1; k += U) {
        int cc[U];
        T hv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cc[u] = max(ld_slot<SMEM>(colp + ((int64_t)(k + u) << log2C)), 0);
            hv[u] = ld_slot<SMEM>(valp + ((int64_t)(k + u) << log2C));
        }
        Pack<C, VPT> vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) vv[u] = ld_nc<C, VPT>(A.vin + (int64_t)cc[u] * A.ldin + j0);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < VPT; ++q) {
                if (IMAG) {
                    acc[q].x = fma(-hv[u], vv[u].v[q].y, acc[q].x);
                    acc[q].y = fma(hv[u], vv[u].v[q].x, acc[q].y);
                } else {
                    acc[q].x = fma(hv[u], vv[u].v[q].x, acc[q].x);
                    acc[q].y = fma(hv[u], vv[u].v[q].y, acc[q].y);
                }
            }
    }
    for (; k < k1; ++k) {
        const int c = max(ld_slot<SMEM>(colp + ((int64_t)k << log2C)), 0);
        const T h = ld_slot<SMEM>(valp + ((int64_t)k << log2C));
        Pack<C, VPT> v = ld_nc<C, VPT>(A.vin + (int64_t)c * A.ldin + j0);
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            if (IMAG) {
                acc[q].x = fma(-h, v.v[q].y, acc[q].x);
                acc[q].y = fma(h, v.v[q].x, acc[q].y);
            } else {
                acc[q].x = fma(h, v.v[q].x, acc[q].x);
                acc[q].y = fma(h, v.v[q].y, acc[q].y);
            }
        }
    }
}

// Packed slots [0, len) of one row with every gather of the first KMAX
// slots in flight at once: indices and values are read (from shared memory
// when staged), all gathers issued, then the multiply-adds run in slot order
// (real group, then imaginary group: the order of packed_group, so the sums
// are bitwise the same).  Slots beyond KMAX go through packed_group.  The
// slot counts are uniform over a chunk, so the guards do not diverge.
template <typename T, int VPT, int KMAX, bool SMEM>
__device__ __forceinline__ void packed_all(const StepArgs<T> &A, const int32_t *colp, const T *valp, int log2C,
                                           int nre, int len, int j0, cplx_t<T> (&acc)[VPT]) {
    using C = cplx_t<T>;
    const int kk = min(len, KMAX);
    Pack<C, VPT> vv[KMAX];
    // staged: the values are read again from shared memory after the
    // gathers (no registers held across them); else kept from the first read
    T hv[SMEM ? 1 : KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < kk) {
            const int c = max(ld_slot<SMEM>(colp + ((int64_t)k << log2C)), 0);
            if constexpr (!SMEM) hv[k] = ld_slot<SMEM>(valp + ((int64_t)k << log2C));
            vv[k] = ld_nc<C, VPT>(A.vin + (int64_t)c * A.ldin + j0);
        }
    }
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < kk) {
            const T h = SMEM ? ld_slot<SMEM>(valp + ((int64_t)k << log2C)) : hv[SMEM ? 0 : k];
#pragma unroll
            for (int q = 0; q < VPT; ++q) {
                if (k < nre) {
                    acc[q].x = fma(h, vv[k].v[q].x, acc[q].x);
                    acc[q].y = fma(h, vv[k].v[q].y, acc[q].y);
                } else {
                    acc[q].x = fma(-h, vv[k].v[q].y, acc[q].x);
                    acc[q].y = fma(h, vv[k].v[q].x, acc[q].y);
                }
            }
        }
    }
    if (len > KMAX) {
        const int r1 = max(nre, KMAX);
        packed_group<T, VPT, false, 4, SMEM>(A, colp, valp, log2C, KMAX, r1, j0, acc);
        packed_group<T, VPT, true, 4, SMEM>(A, colp, valp, log2C, r1, len, j0, acc);
    }
}

// Packed slots [0, len) of one staged row with the chunk height CH fixed at
// compile time: slot k of the row sits at shared offset k * CH (immediate
// offsets), and row c of V_cur at byte offset (c * ld16) * 16 from the
// thread's base vbase (ld16 = the row stride in 16-byte units; the host
// checks that n_rows * ld16 fits in 32 bits), so a gather costs one 32-bit
// multiply and one wide multiply-add instead of 64-bit index arithmetic.
// Same products in the same order as packed_group / packed_all: KMAX > 0
// issues the first KMAX slots' gathers together, else groups of U.
template <typename T, int VPT, int U, int KMAX, int CH>
__device__ __forceinline__ void packed_row_fixed(const char *vbase, uint32_t ld16, const int32_t *colp,
                                                 const T *valp, int nre, int len, cplx_t<T> (&acc)[VPT]) {
    using C = cplx_t<T>;
    auto gather = [&](int k) {
        const uint32_t c = (uint32_t)max(colp[k * CH], 0);
        return ld_nc<C, VPT>(reinterpret_cast<const C *>(vbase + (uint64_t)(c * ld16) * 16u));
    };
    auto madd = [&](int k, bool imag, const Pack<C, VPT> &v) {
        const T h = valp[k * CH];
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            if (imag) {
                acc[q].x = fma(-h, v.v[q].y, acc[q].x);
                acc[q].y = fma(h, v.v[q].x, acc[q].y);
            } else {
                acc[q].x = fma(h, v.v[q].x, acc[q].x);
                acc[q].y = fma(h, v.v[q].y, acc[q].y);
            }
        }
    };
    int k0 = 0;
    if constexpr (KMAX > 0) {
        const int kk = min(len, KMAX);
        Pack<C, VPT> vv[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < kk) vv[k] = gather(k);
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < kk) madd(k, k >= nre, vv[k]);
        k0 = kk;
    }
    // the rest (all of the row when KMAX == 0): real group, then imaginary
    for (int g = 0; g < 2; ++g) {
        const bool imag = g == 1;
        int k = imag ? max(k0, nre) : k0;
        const int k1 = imag ? len : nre;
        for (; k + U <= k1; k += U) {
            Pack<C, VPT> vv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) vv[u] = gather(k + u);
#pragma unroll
            for (int u = 0; u < U; ++u) madd(k + u, imag, vv[u]);
        }
        for (; k < k1; ++k) madd(k, imag, gather(k));
    }
}

// Complex slots [0, len) of one row.
template <typename T, int VPT, int U, bool SMEM>
__device__ __forceinline__ void complex_slots(const StepArgs<T> &A, const int32_t *colp, const cplx_t<T> *valp,
                                              int log2C, int len, int j0, cplx_t<T> (&acc)[VPT]) {
    using C = cplx_t<T>;
    int k = 0;
    for (; k + U <= len; k += U) {
        int cc[U];
        C hh[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cc[u] = max(ld_slot<SMEM>(colp + ((int64_t)(k + u) << log2C)), 0);      // padding: col -1, value 0
            hh[u] = ld_slot<SMEM>(valp + ((int64_t)(k + u) << log2C));
        }
        Pack<C, VPT> vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) vv[u] = ld_nc<C, VPT>(A.vin + (int64_t)cc[u] * A.ldin + j0);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < VPT; ++q) cfma(acc[q], hh[u], vv[u].v[q]);
    }
    for (; k < len; ++k) {
        const int c = max(ld_slot<SMEM>(colp + ((int64_t)k << log2C)), 0);
        const C h = ld_slot<SMEM>(valp + ((int64_t)k << log2C));
        Pack<C, VPT> v = ld_nc<C, VPT>(A.vin + (int64_t)c * A.ldin + j0);
#pragma unroll
        for (int q = 0; q < VPT; ++q) cfma(acc[q], h, v.v[q]);
    }
}

// Map and weights of one step for a row: the step's own, or in a batch
// (A.chunk_rid set) those of the chunk's realisation.
template <typename T, int KIND>
struct StepCoef {
    T a, beta, g0, g1, g2;
    __device__ __forceinline__ void init(const StepArgs<T> &A) {
        a = (T)A.a;
        beta = (T)A.beta;
        g0 = g1 = g2 = 0;
        if (!A.chunk_rid) {
            if (KIND == STEP_SECOND) {
                g0 = (T)A.gc[0];
                g1 = (T)A.gc[1];
                g2 = (T)A.gc[2];
            } else if (KIND == STEP_GENERAL) {
                g0 = (T)A.gc[A.p];
            }
        }
    }
    __device__ __forceinline__ void for_chunk(const StepArgs<T> &A, int64_t ch) {
        if (!A.chunk_rid) return;
        const double *rc = A.rcoef + (int64_t)__ldg(A.chunk_rid + ch) * A.rcoef_ld;
        a = (T)((KIND == STEP_FIRST ? 1.0 : 2.0) * __ldg(rc));
        beta = (T)__ldg(rc + 1);
        if (KIND == STEP_SECOND) {
            g0 = (T)__ldg(rc + 2);
            g1 = (T)__ldg(rc + 3);
            g2 = (T)__ldg(rc + 4);
        } else if (KIND == STEP_GENERAL) {
            g0 = (T)__ldg(rc + 2 + A.p);
        }
    }
};

// One row i of a fused step: the row's slots (colp/valp, slot k at
// k << log2C; nre real slots first when packed) gathered against V_cur, then
// shift, scale, three-term recurrence, accumulation into X, moment dots.
// KMAX > 0 (packed values): the first KMAX slots' gathers all in flight at
// once (packed_all); 0: groups of four.  CH > 0 (staged packed rows): chunk
// height fixed at compile time, 32-bit gather offsets (packed_row_fixed).
// PREP (general steps): the row's values are those of 2 alpha (H - beta)
// (launch_prepare_values), so the row sum started at -V_prev is the new
// vector itself: W = 2 alpha (H - beta) V_cur - V_prev costs the sum alone,
// and V_cur's own row is read only for the moments.
template <typename T, int NB, int VPT, int KIND, bool MOM, bool PACK, bool SMEM, int KMAX = 0, int CH = 0,
          bool PREP = false>
__device__ __forceinline__ void process_row(const StepArgs<T> &A, int64_t i, const int32_t *colp, const void *valp,
                                            int log2C, int nre, int len, int j0, const StepCoef<T, KIND> &cf,
                                            MomentAcc<T> (&uu)[VPT], MomentAcc<T> (&wu)[VPT]) {
    using C = cplx_t<T>;
    constexpr int UNR = CFD_STAGED_UNR;
    static_assert(!PREP || KIND == STEP_GENERAL, "prepared values only in general steps");
    // operands of the epilogue do not depend on the gathers: issue their
    // (streaming) loads first so their latency overlaps the SpMMV
    Pack<C, VPT> u;
    if (!PREP || MOM) u = ld_nc<C, VPT>(A.vin + i * A.ldin + j0);
    // A.x == nullptr: moments only (Algorithm 1 without line 12), X untouched;
    // step 2 then needs the start block's row i, which is V_prev's role here
    Pack<C, VPT> wo, xo;
    if (KIND == STEP_GENERAL) wo = ld_rw<C, VPT>(A.w + i * A.ldw + j0);
    if (KIND == STEP_SECOND) xo = ld_rw<C, VPT>(A.x ? A.x + i * A.ldx + j0 : A.x0 + i * A.ldx0 + j0);
    if (KIND == STEP_GENERAL && A.x) xo = ld_rw<C, VPT>(A.x + i * A.ldx + j0);

    C acc[VPT];
#pragma unroll
    for (int q = 0; q < VPT; ++q) acc[q] = PREP ? cmake<T>(-wo.v[q].x, -wo.v[q].y) : cmake<T>(0, 0);
    if constexpr (PACK && CH > 0) {
        const uint32_t ld16 = (uint32_t)((A.ldin * (int64_t)sizeof(C)) >> 4);
        packed_row_fixed<T, VPT, UNR, KMAX, CH>(reinterpret_cast<const char *>(A.vin + j0), ld16, colp,
                                                static_cast<const T *>(valp), nre, len, acc);
    } else if constexpr (PACK && KMAX > 0) {
        packed_all<T, VPT, KMAX, SMEM>(A, colp, static_cast<const T *>(valp), log2C, nre, len, j0, acc);
    } else if constexpr (PACK) {
        packed_group<T, VPT, false, UNR, SMEM>(A, colp, static_cast<const T *>(valp), log2C, 0, nre, j0, acc);
        packed_group<T, VPT, true, UNR, SMEM>(A, colp, static_cast<const T *>(valp), log2C, nre, len, j0, acc);
    } else {
        complex_slots<T, VPT, UNR, SMEM>(A, colp, static_cast<const C *>(valp), log2C, len, j0, acc);
    }

    const T a = cf.a, beta = cf.beta, g0 = cf.g0, g1 = cf.g1, g2 = cf.g2;
    Pack<C, VPT> wn;
    if (KIND == STEP_FIRST) {
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            wn.v[q].x = a * fma(-beta, u.v[q].x, acc[q].x);
            wn.v[q].y = a * fma(-beta, u.v[q].y, acc[q].y);
        }
        st<C, VPT>(A.w + i * A.ldw + j0, wn);
    } else if (KIND == STEP_SECOND) {
        C *xp = A.x + i * A.ldx + j0;
        Pack<C, VPT> xn;
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            wn.v[q].x = fma(a, fma(-beta, u.v[q].x, acc[q].x), -xo.v[q].x);
            wn.v[q].y = fma(a, fma(-beta, u.v[q].y, acc[q].y), -xo.v[q].y);
            xn.v[q].x = fma(g2, wn.v[q].x, fma(g1, u.v[q].x, g0 * xo.v[q].x));
            xn.v[q].y = fma(g2, wn.v[q].y, fma(g1, u.v[q].y, g0 * xo.v[q].y));
        }
        st<C, VPT>(A.w + i * A.ldw + j0, wn);
        if (A.x) st<C, VPT>(xp, xn);
    } else {
        C *wp = A.w + i * A.ldw + j0;
        C *xp = A.x + i * A.ldx + j0;
        Pack<C, VPT> xn;
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            if (PREP) {
                wn.v[q] = acc[q];
            } else {
                wn.v[q].x = fma(a, fma(-beta, u.v[q].x, acc[q].x), -wo.v[q].x);
                wn.v[q].y = fma(a, fma(-beta, u.v[q].y, acc[q].y), -wo.v[q].y);
            }
            xn.v[q].x = fma(g0, wn.v[q].x, xo.v[q].x);
            xn.v[q].y = fma(g0, wn.v[q].y, xo.v[q].y);
        }
        st<C, VPT>(wp, wn);
        if (A.x) st<C, VPT>(xp, xn);
    }
    if (MOM) {
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            uu[q].add2(u.v[q].x, u.v[q].x, u.v[q].y, u.v[q].y);
            wu[q].add2(wn.v[q].x, u.v[q].x, wn.v[q].y, u.v[q].y);
        }
    }
}

// Rows of one fused ChebFD step for a block of NB vectors, accumulating the
// thread's moment dot products.  Thread layout: a warp covers RPW = 32 / TPR
// rows at a time, TPR = NB / VPT threads per row, each thread VPT
// consecutive vectors of its row.  Each CTA sweeps whole SELL chunks (its
// warps cover the chunk's C rows, RPW rows per warp at a time), so a chunk's
// matrix lines are read by one SM; CTAs take chunks grid-stride, so at any
// time the GPU works on a contiguous window of rows and the gathered rows of
// V_cur stay in L2.
template <typename T, int NB, int VPT, int KIND, bool MOM, bool PACK>
__device__ __forceinline__ void step_rows(const StepArgs<T> &A, MomentAcc<T> (&uu)[VPT],
                                          MomentAcc<T> (&wu)[VPT]) {
    constexpr int TPR = NB / VPT;
    constexpr int RPW = 32 / TPR;
    static_assert(TPR >= 1 && TPR <= 32 && (32 % TPR) == 0, "bad thread split");
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int sub = lane / TPR;
    const int j0 = (lane % TPR) * VPT;
    const int log2C = A.H.log2C;
    StepCoef<T, KIND> cf;
    cf.init(A);

    const int64_t n_rows = A.H.n_rows;
    const int chunk_h = 1 << log2C;
    const int64_t n_chunks = (n_rows + chunk_h - 1) >> log2C;
    const int rows_per_pass = STEP_WARPS * RPW;
    const int passes = (chunk_h + rows_per_pass - 1) / rows_per_pass;
    const int64_t n_items = n_chunks * passes;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int64_t ch = item / passes;
        const int rr = (int)(item % passes) * rows_per_pass + warp * RPW + sub;
        if (rr >= chunk_h) continue;
        const int64_t r = (ch << log2C) + rr;
        if (r >= n_rows) continue;
        const int64_t base = __ldg(A.H.chunk_ptr + ch) + rr;
        const int cl = __ldg(A.H.chunk_len + ch);
        // packed: cl holds the real (low 16 bits) and imaginary (high) slot counts
        const int nre = PACK ? (cl & 0xffff) : cl;
        const int len = PACK ? nre + (cl >> 16) : cl;
        const int64_t i = A.H.perm ? (int64_t)__ldg(A.H.perm + r) : r;
        cf.for_chunk(A, ch);
        const void *valp = PACK ? (const void *)(A.H.pval + base) : (const void *)(A.H.val + base);
        process_row<T, NB, VPT, KIND, MOM, PACK, false>(A, i, A.H.col + base, valp, log2C, nre, len, j0, cf, uu, wu);
    }
}

// Arithmetic of the moment reductions.  fp64 steps add in fp64.  fp32 steps
// add double-float pairs (hi + lo, Knuth's TwoSum, about 44 significant
// bits) on the fp32 pipe: GB300 runs fp64 at 1/64 of the fp32 rate, and the
// fp64 reductions after the rows formed a tail of several microseconds per
// complex64 step.  A cross-CTA partial is one 8-byte word either way (a
// double, or the pair as float2); the reduced dot is widened to fp64 once.
template <typename T> struct MomentRed;

template <> struct MomentRed<double> {
    using R = double;
    static __device__ __forceinline__ R from(const MomentAcc<double> &m) { return m.value(); }
    static __device__ __forceinline__ R zero() { return 0.0; }
    static __device__ __forceinline__ R add(R a, R b) { return a + b; }
    static __device__ __forceinline__ R shfl_xor(R a, int off) { return __shfl_xor_sync(0xffffffffu, a, off); }
    static __device__ __forceinline__ void store(double *p, R a) { *p = a; }
    static __device__ __forceinline__ R load(const double *p) { return __ldcg(p); }
    static __device__ __forceinline__ double widen(R a) { return a; }
};

template <> struct MomentRed<float> {
    struct R { float hi, lo; };
    // (hi, lo) with |lo| <= ulp(hi) / 2 from an unnormalised pair
    static __device__ __forceinline__ R fast_two_sum(float a, float b) {
        const float h = a + b;
        return R{h, b - (h - a)};
    }
    // Kahan's running sum s with compensation c stands for s - c
    static __device__ __forceinline__ R from(const MomentAcc<float> &m) { return fast_two_sum(m.s, -m.c); }
    static __device__ __forceinline__ R zero() { return R{0.f, 0.f}; }
    static __device__ __forceinline__ R add(R a, R b) {
        const float s = a.hi + b.hi;                     // TwoSum of the high parts
        const float bv = s - a.hi;
        const float e = ((a.hi - (s - bv)) + (b.hi - bv)) + (a.lo + b.lo);
        return fast_two_sum(s, e);
    }
    static __device__ __forceinline__ R shfl_xor(R a, int off) {
        return R{__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off)};
    }
    static __device__ __forceinline__ void store(double *p, R a) {
        *reinterpret_cast<float2 *>(p) = make_float2(a.hi, a.lo);
    }
    static __device__ __forceinline__ R load(const double *p) {
        const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
        return R{v.x, v.y};
    }
    static __device__ __forceinline__ double widen(R a) { return (double)a.hi + (double)a.lo; }
};

// Deterministic reduction of the threads' moment sums: warps (shuffles), the
// CTA (shared memory, fixed order), then across CTAs by the last CTA to finish
// (ticket counter), each in a fixed order.  WARPS: the CTA's warps.  A
// thread's vectors q < VPT come in units of G consecutive vectors: vector q
// is (q / G) TPR G + (lane % TPR) G + q % G (G = VPT: VPT consecutive
// vectors; G = 1: vectors lane % TPR + q TPR).
template <typename T, int NB, int VPT, int WARPS = STEP_WARPS, int G = VPT>
__device__ __forceinline__ void reduce_moments(double *partial, unsigned *ticket, double *dots,
                                               MomentAcc<T> (&uu)[VPT], MomentAcc<T> (&wu)[VPT]) {
    using Op = MomentRed<T>;
    using R = typename Op::R;
    constexpr int TPR = NB / VPT;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int sub = lane / TPR;
    const int jt = lane % TPR;
    auto jq = [&](int q) { return (q / G) * TPR * G + jt * G + q % G; };
    __shared__ R red[WARPS][NB][2];
    __shared__ bool last_cta;
    R s_uu[VPT], s_wu[VPT];
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
        s_uu[q] = Op::from(uu[q]);
        s_wu[q] = Op::from(wu[q]);
#pragma unroll
        for (int off = TPR; off < 32; off <<= 1) {
            s_uu[q] = Op::add(s_uu[q], Op::shfl_xor(s_uu[q], off));
            s_wu[q] = Op::add(s_wu[q], Op::shfl_xor(s_wu[q], off));
        }
    }
    if (sub == 0) {
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            red[warp][jq(q)][0] = s_uu[q];
            red[warp][jq(q)][1] = s_wu[q];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * NB; e += blockDim.x) {
        R s = Op::zero();
#pragma unroll
        for (int w = 0; w < WARPS; ++w) s = Op::add(s, red[w][e >> 1][e & 1]);
        Op::store(partial + (int64_t)blockIdx.x * 2 * NB + e, s);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last_cta = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last_cta) {
        __threadfence();
        for (int e = warp; e < 2 * NB; e += WARPS) {
            R s = Op::zero();
            for (int b = lane; b < (int)gridDim.x; b += 32) s = Op::add(s, Op::load(partial + (int64_t)b * 2 * NB + e));
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s = Op::add(s, Op::shfl_xor(s, off));
            if (lane == 0) dots[e] = Op::widen(s);
        }
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

// One fused ChebFD step (the paper's chebfd_op) over all rows, with the
// moments reduced deterministically when MOM.
template <typename T, int NB, int VPT, int KIND, bool MOM, bool PACK>
__global__ void __launch_bounds__(STEP_WARPS * 32)
k_cheb_step(const StepArgs<T> A) {
    MomentAcc<T> uu[VPT], wu[VPT];
    step_rows<T, NB, VPT, KIND, MOM, PACK>(A, uu, wu);
    if (MOM) reduce_moments<T, NB, VPT>(A.partial, A.ticket, A.dots, uu, wu);
}

// ------------------------------------------------- TMA-staged general step --


__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of a barrier, giving up after `limit` cycles:
// returns false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Count `bytes` of a barrier's expected transaction bytes as arrived without a
// copy (used only to cancel the surplus the wait test expects).
__device__ __forceinline__ void mbar_complete_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared memory (TMA), completing on `bar`.
// Addresses 16-byte aligned, size a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// General step with the matrix staged through shared memory: each CTA takes
// whole chunks grid-stride; one thread copies the next chunk's column indices
// and values with two TMA bulk copies into the other half of a double buffer
// while the CTA computes the current chunk from shared memory, so a row's
// critical path holds only its V_cur gathers.  The values are those of
// 2 alpha (H - beta) (A.prep_val), so each row sum starts at -V_prev and is
// the new vector when it ends.  Slot counts of a chunk are
// multiples of C >= 4, so every copy is 16-byte aligned and sized.  A wait
// that expires (after ~2^32 cycles, about two seconds) records
// CFD_ERR_TIMEOUT in *A.status and the CTA returns once its own copies in
// flight (the current chunk's and the prefetched one's) have landed; if that
// drain wait expires too (bounded the same way), the status also carries
// CFD_STATUS_DRAIN_EXPIRED and the launch's results and workspace are
// invalid.  A.staged == 2 is the test of that path: every barrier expects
// 16 bytes more than are copied, so no chunk wait can succeed and waits give
// up after 2^24 cycles; the drain then cancels the surplus
// (mbarrier.complete_tx) and waits for the real copies only.
// KMAX > 0: every gather of a row's first KMAX slots in flight at once
// (packed values; registers capped so that two CTAs fit on an SM, three for
// KMAX <= 8).  CH > 0:
// the matrix's chunk height, fixed at compile time (packed values; the
// host launches it only for C == CH and 32-bit gather offsets).
template <typename T, int NB, int VPT, bool MOM, bool PACK, int KMAX = 0, int CH = 0>
__global__ void __launch_bounds__(STEP_WARPS * 32,
                                  KMAX > 8 ? 2 : (KMAX > 0 ? 3 : (sizeof(T) == 4 ? CFD_STAGED_MINB_F32 : 0)))
k_cheb_step_staged(const StepArgs<T> A, int slots_cap) {
    using C = cplx_t<T>;
    using V = typename std::conditional<PACK, T, C>::type;
    constexpr int TPR = NB / VPT;
    constexpr int RPW = 32 / TPR;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_len[2];
    const int col_bytes = (int)round_up_dev((size_t)slots_cap * 4, 16);
    // buffer b: indices at smem_raw + b col_bytes, values after both index buffers
    auto col_s = [&](int b) { return reinterpret_cast<int32_t *>(smem_raw + b * col_bytes); };
    auto val_s = [&](int b) {
        return reinterpret_cast<V *>(smem_raw + 2 * col_bytes + (size_t)b * slots_cap * sizeof(V));
    };
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int sub = lane / TPR;
    const int j0 = (lane % TPR) * VPT;
    const int log2C = CH > 0 ? __ffs(CH) - 1 : A.H.log2C;
    const int chunk_h = CH > 0 ? CH : 1 << log2C;
    const int64_t n_rows = A.H.n_rows;
    const int64_t n_chunks = (n_rows + chunk_h - 1) >> log2C;
    // the values of 2 alpha (H - beta), prepared once per filter call
    const V *gval = reinterpret_cast<const V *>(A.prep_val);
    const uint32_t tx_extra = A.staged == 2 ? 16u : 0u;
    const long long limit = A.staged == 2 ? (1LL << 24) : (1LL << 32);
    StepCoef<T, STEP_GENERAL> cf;
    cf.init(A);
    MomentAcc<T> uu[VPT], wu[VPT];

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int64_t c, int b) {     // thread 0: stage chunk c into buffer b
        const int cl = __ldg(A.H.chunk_len + c);
        const int len = PACK ? (cl & 0xffff) + (cl >> 16) : cl;
        const int64_t base = __ldg(A.H.chunk_ptr + c);
        const uint32_t nslot = (uint32_t)len << log2C;
        s_len[b] = cl;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[b], nslot * (uint32_t)(4 + sizeof(V)) + tx_extra);
        if (nslot) {
            tma_load_1d(col_s(b), A.H.col + base, nslot * 4u, &bar[b]);
            tma_load_1d(val_s(b), gval + base, nslot * (uint32_t)sizeof(V), &bar[b]);
        }
    };

    int k = 0;
    bool ok = true;
    bool prefetched = false;      // thread 0: the next chunk's copies were issued this iteration
    const ChunkRange cr = cta_chunks(n_chunks);
    if (tid == 0 && cr.first < cr.last) issue(cr.first, 0);
    __syncthreads();              // s_len[0] written by thread 0
    for (int64_t c = cr.first; c < cr.last; c += cr.stride, ++k) {
        const int b = k & 1;
        prefetched = c + cr.stride < cr.last;
        if (tid == 0 && prefetched) issue(c + cr.stride, b ^ 1);
        // every thread waits for the chunk's copies itself; a thread whose
        // wait expired skips the chunk, and the barrier below then stops all
        const bool landed = mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1), limit);
        if (landed) {
            const int cl = s_len[b];
            const int nre = PACK ? (cl & 0xffff) : cl;
            const int len = PACK ? nre + (cl >> 16) : cl;
            cf.for_chunk(A, c);
            for (int rr = warp * RPW + sub; rr < chunk_h; rr += STEP_WARPS * RPW) {
                const int64_t r = (c << log2C) + rr;
                if (r >= n_rows) continue;
                const int64_t i = A.H.perm ? (int64_t)__ldg(A.H.perm + r) : r;
                process_row<T, NB, VPT, STEP_GENERAL, MOM, PACK, true, KMAX, CH, true>(
                A, i, col_s(b) + rr, val_s(b) + rr, log2C, nre, len, j0, cf, uu, wu);
            }
        }
        // one barrier per chunk: buffer b is refilled only after every thread
        // read it, and an expired wait anywhere ends the sweep
        if (!__syncthreads_and(landed)) {
            ok = false;
            break;
        }
    }
    if (!ok) {
        if (tid == 0) {
            // drain this CTA's copies still in flight (bounded): the current
            // chunk's and, if issued, the prefetched one; in the wait test
            // first cancel the surplus each armed barrier expects
            const int b = k & 1;
            if (tx_extra) {
                mbar_complete_tx(&bar[b], tx_extra);
                if (prefetched) mbar_complete_tx(&bar[b ^ 1], tx_extra);
            }
            const long long drain_limit = 1LL << 32;
            bool drained = mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1), drain_limit);
            if (prefetched) drained = mbar_wait_bounded(&bar[b ^ 1], (uint32_t)(((k + 1) >> 1) & 1), drain_limit) && drained;
            atomicOr(A.status, drained ? (int)CFD_ERR_TIMEOUT : (int)CFD_ERR_TIMEOUT | CFD_STATUS_DRAIN_EXPIRED);
        }
        return;
    }
    if (MOM) reduce_moments<T, NB, VPT>(A.partial, A.ticket, A.dots, uu, wu);
}

// All n_p steps of Algorithm 1 for one block in a single cooperative launch:
// the grid synchronises between steps (every step reads V_cur rows that
// other CTAs wrote in the previous step).  No moments.  The CTA count must
// not exceed the co-resident capacity (cooperative launch checks it).
template <typename T, int NB, int VPT, bool PACK>
__global__ void __launch_bounds__(STEP_WARPS * 32, 3)
k_cheb_persistent(const StepArgs<T> A0, cplx_t<T> *va, cplx_t<T> *vb, cplx_t<T> *xb, int64_t ldx, int n_p) {
    cg::grid_group grid = cg::this_grid();
    MomentAcc<T> uu[VPT], wu[VPT];
    StepArgs<T> A = A0;
    const double alpha = A0.a;
    // step 1: V1 = H~ X_b
    A.vin = xb; A.ldin = ldx; A.w = va; A.ldw = NB; A.x = nullptr; A.ldx = 0; A.a = alpha; A.p = 1;
    step_rows<T, NB, VPT, STEP_FIRST, false, PACK>(A, uu, wu);
    grid.sync();
    // step 2: V2 = 2 H~ V1 - X_b, X_b = gc0 X_b + gc1 V1 + gc2 V2
    A.vin = va; A.ldin = NB; A.w = vb; A.ldw = NB; A.x = xb; A.ldx = ldx; A.a = 2.0 * alpha; A.p = 2;
    step_rows<T, NB, VPT, STEP_SECOND, false, PACK>(A, uu, wu);
    for (int p = 3; p <= n_p; ++p) {
        grid.sync();
        A.vin = (p & 1) ? vb : va;
        A.w = (p & 1) ? va : vb;
        A.p = p;
        step_rows<T, NB, VPT, STEP_GENERAL, false, PACK>(A, uu, wu);
    }
}

// General steps 3..n_p of one block in a single cooperative launch, each step
// the TMA-staged chunk loop of k_cheb_step_staged (packed values prepared as
// 2 alpha (H - beta), A.prep_val), the grid synchronising between steps
// (every step gathers V_cur rows other CTAs wrote in the previous one).
// Steps 1 and 2 are launched before it, so the kernel holds only the general
// step's registers.  A CTA keeps the same chunks in every step, and the copy
// of its first chunk of step p + 1 is issued while it computes its last chunk
// of step p.  No moments.  A bounded wait that expires records
// CFD_ERR_TIMEOUT in *A.status; the CTA drains its copies and still meets
// every grid barrier, and after the barrier all CTAs see the status and
// return together (no CTA waits at a barrier another has left).
template <typename T, int NB, int VPT, int CH>
__global__ void __launch_bounds__(STEP_WARPS * 32, sizeof(T) == 4 ? 5 : 3)
k_cheb_persistent_staged(const StepArgs<T> A0, cplx_t<T> *va, cplx_t<T> *vb, int n_p, int slots_cap) {
    cg::grid_group grid = cg::this_grid();
    constexpr int TPR = NB / VPT;
    constexpr int RPW = 32 / TPR;
    using V = T;                                  // packed values
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_len[2];
    const int col_bytes = (int)round_up_dev((size_t)slots_cap * 4, 16);
    auto col_s = [&](int b) { return reinterpret_cast<int32_t *>(smem_raw + b * col_bytes); };
    auto val_s = [&](int b) {
        return reinterpret_cast<V *>(smem_raw + 2 * col_bytes + (size_t)b * slots_cap * sizeof(V));
    };
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int sub = lane / TPR;
    const int j0 = (lane % TPR) * VPT;
    const int log2C = CH > 0 ? __ffs(CH) - 1 : A0.H.log2C;
    const int chunk_h = CH > 0 ? CH : 1 << log2C;
    const int64_t n_rows = A0.H.n_rows;
    const int64_t n_chunks = (n_rows + chunk_h - 1) >> log2C;
    const V *gval = reinterpret_cast<const V *>(A0.prep_val);
    const uint32_t tx_extra = A0.staged == 2 ? 16u : 0u;
    const long long limit = A0.staged == 2 ? (1LL << 24) : (1LL << 32);
    MomentAcc<T> uu[VPT], wu[VPT];                // unused (no moments)
    volatile int *status = A0.status;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int64_t c, int b) {
        const int cl = __ldg(A0.H.chunk_len + c);
        const int len = (cl & 0xffff) + (cl >> 16);
        const int64_t base = __ldg(A0.H.chunk_ptr + c);
        const uint32_t nslot = (uint32_t)len << log2C;
        s_len[b] = cl;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[b], nslot * (uint32_t)(4 + sizeof(V)) + tx_extra);
        if (nslot) {
            tma_load_1d(col_s(b), A0.H.col + base, nslot * 4u, &bar[b]);
            tma_load_1d(val_s(b), gval + base, nslot * (uint32_t)sizeof(V), &bar[b]);
        }
    };
    const bool has_work = (int64_t)blockIdx.x < n_chunks;
    int k = 0;                     // chunk iterations over all steps (buffer k & 1, phase (k >> 1) & 1)
    bool in_flight = false;        // a copy for iteration k was issued and not yet waited for
    if (tid == 0 && has_work) issue(blockIdx.x, 0);
    in_flight = has_work;
    __syncthreads();
    StepArgs<T> A = A0;
    for (int p = 3; p <= n_p; ++p) {
        A.vin = (p & 1) ? vb : va;
        A.ldin = NB;
        A.w = (p & 1) ? va : vb;
        A.ldw = NB;
        A.p = p;
        StepCoef<T, STEP_GENERAL> cf;
        cf.init(A);
        bool ok = true;
        bool issued_next = false;  // the copy for iteration k + 1 was issued
        for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x, ++k) {
            const int b = k & 1;
            // the next chunk: of this step, else this CTA's first of the next step
            int64_t cn = c + gridDim.x;
            issued_next = true;
            if (cn >= n_chunks) {
                cn = blockIdx.x;
                issued_next = p < n_p;
            }
            if (tid == 0 && issued_next) issue(cn, b ^ 1);
            const bool landed = mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1), limit);
            if (landed) {
                const int cl = s_len[b];
                const int nre = cl & 0xffff;
                const int len = nre + (cl >> 16);
                cf.for_chunk(A, c);
                for (int rr = warp * RPW + sub; rr < chunk_h; rr += STEP_WARPS * RPW) {
                    const int64_t r = (c << log2C) + rr;
                    if (r >= n_rows) continue;
                    const int64_t i = A.H.perm ? (int64_t)__ldg(A.H.perm + r) : r;
                    process_row<T, NB, VPT, STEP_GENERAL, false, true, true, 0, CH, true>(
                        A, i, col_s(b) + rr, val_s(b) + rr, log2C, nre, len, j0, cf, uu, wu);
                }
            }
            if (!__syncthreads_and(landed)) {
                ok = false;
                break;
            }
            in_flight = issued_next;
        }
        if (!ok) {
            in_flight = false;
            if (tid == 0) {
                // drain: the copy of iteration k (not landed) and, if issued, of k + 1
                const int b = k & 1;
                if (tx_extra) {
                    mbar_complete_tx(&bar[b], tx_extra);
                    if (issued_next) mbar_complete_tx(&bar[b ^ 1], tx_extra);
                }
                const long long drain_limit = 1LL << 32;
                bool drained = mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1), drain_limit);
                if (issued_next)
                    drained = mbar_wait_bounded(&bar[b ^ 1], (uint32_t)(((k + 1) >> 1) & 1), drain_limit) && drained;
                atomicOr(A0.status, drained ? (int)CFD_ERR_TIMEOUT : (int)CFD_ERR_TIMEOUT | CFD_STATUS_DRAIN_EXPIRED);
            }
        }
        grid.sync();
        if (*status != 0) {
            // every CTA leaves here, after the same barrier; one that did not
            // fail may still have the copy of its next chunk in flight
            if (tid == 0 && in_flight) {
                const int b = k & 1;
                if (tx_extra) mbar_complete_tx(&bar[b], tx_extra);
                if (!mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1), 1LL << 32))
                    atomicOr(A0.status, (int)CFD_ERR_TIMEOUT | CFD_STATUS_DRAIN_EXPIRED);
            }
            return;
        }
    }
}

// --------------------------------------------------------- launching --

namespace {

template <typename T, int NB, int VPT, int KIND, bool MOM, bool PACK>
cfd_status launch_one(const StepArgs<T> &A, int grid_cap, cudaStream_t stream) {
    constexpr bool STAGEABLE = (KIND == STEP_GENERAL);
    const bool staged = STAGEABLE && A.staged;
    using V = typename std::conditional<PACK, T, cplx_t<T>>::type;
    int slots_cap = 0;
    size_t smem = 0;
    if (staged) {
        if (!A.status) return fail(CFD_ERR_INTERNAL, "staged step without a status word");
        if (!A.prep_val) return fail(CFD_ERR_INTERNAL, "staged step without prepared matrix values");
        slots_cap = A.H.slots_bound << A.H.log2C;
        if (slots_cap <= 0) return fail(CFD_ERR_ARG, "matrix has no slot bound; cannot stage");
        smem = 2 * round_up((size_t)slots_cap * 4, 16) + round_up(2 * (size_t)slots_cap * sizeof(V), 16);
        if (smem > 200 * 1024) return fail(CFD_ERR_ARG, "chunk too large to stage (%zu bytes)", smem);
    }
    auto kern = k_cheb_step<T, NB, VPT, KIND, MOM, PACK>;
    // staged general steps of packed matrices: the first 16 (or 8) slots'
    // gathers of a row in flight at once, else groups of four
    const int kmax = (staged && PACK) ? (A.gather >= STEP_GATHER_ALL ? STEP_GATHER_ALL : (A.gather >= 8 ? 8 : 0)) : 0;
    // chunk height 32 compiled in, with 32-bit gather offsets (fits when
    // every gathered row's offset in 16-byte units stays below 2^32); by
    // default for fp32 only: the fp64 variant needs more registers, which
    // costs a resident CTA on the FP64-bound step
    const bool want_fixed = A.fixed_chunk > 0 || (A.fixed_chunk == 0 && sizeof(T) == 4);
    const bool fixed = staged && PACK && want_fixed && A.H.log2C == 5 &&
                       (uint64_t)A.H.n_rows * (uint64_t)((A.ldin * (int64_t)sizeof(cplx_t<T>)) >> 4) < (1ULL << 32);
    auto skern = k_cheb_step_staged<T, NB, VPT, MOM, PACK>;
    if constexpr (PACK && STAGEABLE) {
        if (kmax == STEP_GATHER_ALL)
            skern = fixed ? k_cheb_step_staged<T, NB, VPT, MOM, PACK, STEP_GATHER_ALL, 32>
                          : k_cheb_step_staged<T, NB, VPT, MOM, PACK, STEP_GATHER_ALL>;
        else if (kmax == 8)
            skern = fixed ? k_cheb_step_staged<T, NB, VPT, MOM, PACK, 8, 32> : k_cheb_step_staged<T, NB, VPT, MOM, PACK, 8>;
        else if (fixed)
            skern = k_cheb_step_staged<T, NB, VPT, MOM, PACK, 0, 32>;
    }
    // Occupancy per device and kernel variant (0 plain; staged generic 1
    // (groups of four), 2 (8 at once), 3 (16 at once); staged fixed 4, 5, 6),
    // and the shared-memory limit set on the kernel, which only ever grows so
    // that a concurrent launch with a larger chunk never finds it lowered.
    // One mutex per instantiation guards the cache and the attribute.
    struct Cache {
        std::mutex mu;
        int occ[64][7];
        size_t occ_smem[64][7];
        size_t attr_smem[64][7];
    };
    static Cache cache{};
    int dev = 0;
    CFD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CFD_ERR_ARG, "device ordinal %d out of range", dev);
    int which = 0;
    if (staged) which = (kmax == STEP_GATHER_ALL ? 3 : (kmax == 8 ? 2 : 1)) + (fixed ? 3 : 0);
    int resident = 0;
    {
        std::lock_guard<std::mutex> lock(cache.mu);
        if (staged && smem > cache.attr_smem[dev][which]) {
            CFD_CUDA(cudaFuncSetAttribute(skern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            cache.attr_smem[dev][which] = smem;
        }
        if (cache.occ[dev][which] == 0 || (staged && cache.occ_smem[dev][which] != smem)) {
            int o = 0;
            if (staged) {
                CFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, skern, STEP_WARPS * 32, smem));
                cache.occ_smem[dev][which] = smem;
            } else {
                CFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, STEP_WARPS * 32, 0));
            }
            cache.occ[dev][which] = std::max(1, std::min(o, STEP_MAX_CTAS_PER_SM));
        }
        resident = cache.occ[dev][which];
    }
    constexpr int RPW = 32 / (NB / VPT);
    const int64_t C = 1LL << A.H.log2C;
    const int64_t passes = (C + STEP_WARPS * RPW - 1) / (STEP_WARPS * RPW);
    const int64_t n_chunks = (A.H.n_rows + C - 1) / C;
    int64_t need = staged ? n_chunks : n_chunks * passes;     // work items
    int64_t grid = std::min<int64_t>((int64_t)resident * sm_count(), need);
    if (grid_cap > 0) grid = std::min<int64_t>(grid, grid_cap);
    grid = std::max<int64_t>(grid, 1);
    if (staged) {
        if constexpr (STAGEABLE) skern<<<(unsigned)grid, STEP_WARPS * 32, smem, stream>>>(A, slots_cap);
    } else {
        kern<<<(unsigned)grid, STEP_WARPS * 32, 0, stream>>>(A);
    }
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

template <typename T, int NB, int VPT, bool MOM, bool PACK>
cfd_status launch_kind_mp(int kind, const StepArgs<T> &A, int grid_cap, cudaStream_t s) {
    switch (kind) {
    case STEP_FIRST: return launch_one<T, NB, VPT, STEP_FIRST, MOM, PACK>(A, grid_cap, s);
    case STEP_SECOND: return launch_one<T, NB, VPT, STEP_SECOND, MOM, PACK>(A, grid_cap, s);
    default: return launch_one<T, NB, VPT, STEP_GENERAL, MOM, PACK>(A, grid_cap, s);
    }
}

// Moments are reduced only when the caller asks for the dot products.
template <typename T, int NB, int VPT, bool PACK>
cfd_status launch_kind(int kind, const StepArgs<T> &A, int grid_cap, cudaStream_t s) {
    if (A.dots) return launch_kind_mp<T, NB, VPT, true, PACK>(kind, A, grid_cap, s);
    return launch_kind_mp<T, NB, VPT, false, PACK>(kind, A, grid_cap, s);
}

}  // namespace

template <typename T, bool PACK>
cfd_status launch_step_p(int kind, int nb, int vpt, const StepArgs<T> &A, int grid_cap, cudaStream_t s) {
#define CFD_CASE(NB_, VPT_) \
    if (nb == NB_ && vpt == VPT_) return launch_kind<T, NB_, VPT_, PACK>(kind, A, grid_cap, s);
    CFD_CASE(1, 1)
    CFD_CASE(8, 1)
    CFD_CASE(8, 2)
    CFD_CASE(16, 1)
    CFD_CASE(16, 2)
    CFD_CASE(32, 1)
    CFD_CASE(32, 2)
    CFD_CASE(64, 2)
#undef CFD_CASE
    return fail(CFD_ERR_ARG, "unsupported block width n_b=%d with %d vectors per thread", nb, vpt);
}


namespace {

template <typename T, int NB, int VPT, bool PACK>
cfd_status launch_persistent_nbp(const StepArgs<T> &A, cplx_t<T> *va, cplx_t<T> *vb, cplx_t<T> *xb, int64_t ldx,
                                 int n_p, int grid_cap, cudaStream_t stream) {
    auto kern = k_cheb_persistent<T, NB, VPT, PACK>;
    static std::atomic<int> occ[64] = {};      // resident CTAs per SM, per device (0: not yet known)
    int dev = 0;
    CFD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CFD_ERR_ARG, "device ordinal %d out of range", dev);
    if (occ[dev].load() == 0) {
        int o = 0;
        CFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, STEP_WARPS * 32, 0));
        occ[dev].store(std::max(1, std::min(o, STEP_MAX_CTAS_PER_SM)));
    }
    constexpr int RPW = 32 / (NB / VPT);
    const int64_t C = 1LL << A.H.log2C;
    const int64_t passes = (C + STEP_WARPS * RPW - 1) / (STEP_WARPS * RPW);
    int64_t need = (A.H.n_rows + C - 1) / C * passes;       // work items (chunk passes)
    int64_t grid = std::min<int64_t>((int64_t)occ[dev].load() * sm_count(), need);
    if (grid_cap > 0) grid = std::min<int64_t>(grid, grid_cap);
    grid = std::max<int64_t>(grid, 1);
    StepArgs<T> a = A;
    void *args[] = {&a, &va, &vb, &xb, &ldx, &n_p};
    CFD_CUDA(cudaLaunchCooperativeKernel((void *)kern, dim3((unsigned)grid), dim3(STEP_WARPS * 32), args, 0, stream));
    CFD_COUNT_LAUNCH();
    return CFD_OK;
}

}  // namespace

namespace {

template <typename T, int NB, int VPT, int CH>
cfd_status launch_persistent_staged_nb(const StepArgs<T> &A, cplx_t<T> *va, cplx_t<T> *vb, int n_p, int grid_cap,
                                       cudaStream_t stream) {
    const int slots_cap = A.H.slots_bound << A.H.log2C;
    if (slots_cap <= 0) return fail(CFD_ERR_ARG, "matrix has no slot bound; cannot stage");
    const size_t smem = 2 * round_up((size_t)slots_cap * 4, 16) + round_up(2 * (size_t)slots_cap * sizeof(T), 16);
    if (smem > 200 * 1024) return fail(CFD_ERR_ARG, "chunk too large to stage (%zu bytes)", smem);
    auto kern = k_cheb_persistent_staged<T, NB, VPT, CH>;
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
            CFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, STEP_WARPS * 32, smem));
            if (o < 1) return fail(CFD_ERR_ARG, "persistent staged step does not fit on an SM");
            cache.occ[dev] = std::min(o, STEP_MAX_CTAS_PER_SM);
            cache.occ_smem[dev] = smem;
        }
        resident = cache.occ[dev];
    }
    const int64_t n_chunks = (A.H.n_rows + (1LL << A.H.log2C) - 1) >> A.H.log2C;
    // every CTA co-resident (cooperative launch), at most one per chunk
    int64_t grid = std::min<int64_t>((int64_t)resident * sm_count(), n_chunks);
    if (grid_cap > 0) grid = std::min<int64_t>(grid, grid_cap);
    grid = std::max<int64_t>(grid, 1);
    StepArgs<T> a = A;
    int np = n_p, sc = slots_cap;
    void *args[] = {&a, &va, &vb, &np, &sc};
    CFD_CUDA(cudaLaunchCooperativeKernel((void *)kern, dim3((unsigned)grid), dim3(STEP_WARPS * 32), args, smem, stream));
    CFD_COUNT_LAUNCH();
    return CFD_OK;
}

template <typename T, int NB, int VPT>
cfd_status launch_persistent_staged_ch(const StepArgs<T> &A, cplx_t<T> *va, cplx_t<T> *vb, int n_p, int grid_cap,
                                       cudaStream_t s) {
    const bool fixed = A.H.log2C == 5 &&
                       (uint64_t)A.H.n_rows * (uint64_t)((NB * (int64_t)sizeof(cplx_t<T>)) >> 4) < (1ULL << 32);
    if (fixed) return launch_persistent_staged_nb<T, NB, VPT, 32>(A, va, vb, n_p, grid_cap, s);
    return launch_persistent_staged_nb<T, NB, VPT, 0>(A, va, vb, n_p, grid_cap, s);
}

}  // namespace

// General steps 3..n_p in one cooperative launch (packed values prepared in
// A.prep_val; steps 1 and 2 already run).
template <typename T>
cfd_status launch_persistent_staged(int nb, int vpt, const StepArgs<T> &A, cplx_t<T> *va, cplx_t<T> *vb, int n_p,
                                    int grid_cap, cudaStream_t s) {
    if (!A.H.packed) return fail(CFD_ERR_ARG, "the staged persistent filter needs packed matrix values");
    if (!A.status || !A.prep_val) return fail(CFD_ERR_INTERNAL, "staged persistent steps without status or values");
#define CFD_PSCASE(NB_, VPT_) \
    if (nb == NB_ && vpt == VPT_) return launch_persistent_staged_ch<T, NB_, VPT_>(A, va, vb, n_p, grid_cap, s);
    CFD_PSCASE(8, 1)
    CFD_PSCASE(8, 2)
    CFD_PSCASE(16, 1)
    CFD_PSCASE(16, 2)
    CFD_PSCASE(32, 1)
    CFD_PSCASE(32, 2)
    CFD_PSCASE(64, 2)
#undef CFD_PSCASE
    return fail(CFD_ERR_ARG, "unsupported block width n_b=%d with %d vectors per thread", nb, vpt);
}

template <typename T, bool PACK>
cfd_status launch_persistent_p(int nb, int vpt, const StepArgs<T> &A, cplx_t<T> *va, cplx_t<T> *vb, cplx_t<T> *xb,
                               int64_t ldx, int n_p, int grid_cap, cudaStream_t s) {
#define CFD_PCASE(NB_, VPT_) \
    if (nb == NB_ && vpt == VPT_) return launch_persistent_nbp<T, NB_, VPT_, PACK>(A, va, vb, xb, ldx, n_p, grid_cap, s);
    CFD_PCASE(8, 1)
    CFD_PCASE(8, 2)
    CFD_PCASE(16, 1)
    CFD_PCASE(16, 2)
    CFD_PCASE(32, 1)
    CFD_PCASE(32, 2)
    CFD_PCASE(64, 2)
#undef CFD_PCASE
    return fail(CFD_ERR_ARG, "unsupported block width n_b=%d with %d vectors per thread", nb, vpt);
}


}  // namespace cfd
