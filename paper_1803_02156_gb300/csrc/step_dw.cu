// Fused ChebFD steps (Algorithm 1) for complex double data in double-word
// arithmetic on the fp32 pipe.
//
// GB300 executes fp64 fused multiply-adds at 1/64 of the fp32 rate, so the
// native complex128 step is bound by the FP64 pipe at about a fifth of the
// HBM bandwidth.  Here every double is carried as an unevaluated sum of two
// floats hi + lo (|lo| <= ulp(hi) / 2, about 48 significant bits; Dekker
// 1971, "A floating-point technique for extending the available precision")
// and every operation of the step runs on the fp32 pipe:
//   * products exactly as hi*hi plus its rounding error from one FMA
//     (Dekker's TwoProduct via FMA) plus the two cross terms hi*lo, lo*hi;
//   * sums with Knuth's TwoSum (exact error of a rounded addition), the
//     error terms of a row sum collected in a second float and added once
//     at the end (the accumulation of Ogita, Rump and Oishi 2005, "Accurate
//     sum and dot product", Dot2);
//   * the result renormalised with TwoSum.
// Each operation is accurate to a few units of 2^-48 relative to the sum of
// the magnitudes of its terms (lo*lo products, below 2^-48 |hi*hi|, are
// dropped), against 2^-53 for native fp64.  The real and imaginary parts of
// an element go through the same sequence together, in Blackwell's packed
// fp32x2 instructions (two lanes per issue slot).
//
// Storage stays 16 bytes per complex element: the recurrence blocks V_a, V_b
// and, during one filter application, the caller's X block hold the
// double-word form {re_hi, im_hi, re_lo, im_lo}; the driver converts X to it
// before step 1 and the last step writes it back as complex double.  The matrix
// values are prepared once per application as the double-word form of
// 2 alpha (H - beta) (8 bytes per packed slot, the bytes of a packed double),
// so the minimum traffic per step equals the native step's.
#include "dw_arith.cuh"
#include "step_kernels.cuh"

namespace cfd {

// Gathers of a row in flight together (group size) and the CTAs per SM the
// registers are capped for: the tuned values; both fixed at compile time.
#ifndef CFD_DW_GROUP
#define CFD_DW_GROUP 2
#endif
#ifndef CFD_DW_MIN_CTAS
#define CFD_DW_MIN_CTAS 4
#endif

// x h for a double-word x and a float h that is a power of two (exact).
__device__ __forceinline__ float4 dw_scale(float4 v, float h) {
    return make_float4(v.x * h, v.y * h, v.z * h, v.w * h);
}

// One fused step (KIND: STEP_FIRST, STEP_SECOND or STEP_GENERAL, Algorithm 1
// lines 4-6 and 9-12) with the prepared values P = 2 alpha (H - beta):
//   first:   V1 = (1/2) P X                       (X: vin)
//   second:  V2 = P V1 - X;  X <- g0 X + g1 V1 + g2 V2
//   general: V_new = P V_cur - V_prev;  X <- X + g_p V_new
// with the moments' dots <vin, vin>, Re <w, vin>.  Arguments: those of the
// native steps (StepArgs<double>); the block pointers hold double-words,
// prep_val the double-word prepared values (float2 {hi, lo} per slot).
// LAST: X is written back as complex double.  A row's X and own vin entries
// are loaded after its row sum (loading them before holds their registers
// across the gathers and costs a resident CTA: measured slower).
template <int NB, int VPT, int KIND, bool MOM, int CH, bool LAST>
__global__ void __launch_bounds__(STEP_WARPS * 32, CFD_DW_MIN_CTAS)
k_cheb_step_dw(const StepArgs<double> A, int slots_cap) {
    constexpr int TPR = NB / VPT;
    constexpr int RPW = 32 / TPR;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_len[2];
    const int col_bytes = (int)round_up_dev((size_t)slots_cap * 4, 16);
    auto col_s = [&](int b) { return reinterpret_cast<int32_t *>(smem_raw + b * col_bytes); };
    auto val_s = [&](int b) {
        return reinterpret_cast<float2 *>(smem_raw + 2 * col_bytes + (size_t)b * slots_cap * sizeof(float2));
    };
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int sub = lane / TPR;
    const int j0 = (lane % TPR) * VPT;
    const int log2C = CH > 0 ? __ffs(CH) - 1 : A.H.log2C;
    const int chunk_h = CH > 0 ? CH : 1 << log2C;
    const int64_t n_rows = A.H.n_rows;
    const int64_t n_chunks = (n_rows + chunk_h - 1) >> log2C;
    const float2 *gval = reinterpret_cast<const float2 *>(A.prep_val);
    const float4 *vin = reinterpret_cast<const float4 *>(A.vin);
    float4 *wout = reinterpret_cast<float4 *>(A.w);
    float4 *xdw = reinterpret_cast<float4 *>(A.x);
    const uint32_t tx_extra = A.staged == 2 ? 16u : 0u;
    const long long limit = A.staged == 2 ? (1LL << 24) : (1LL << 32);
    // the step's weights as double-words: g_p c_p (general), g_0 c_0,
    // g_1 c_1, g_2 c_2 (second); in a batch per chunk, those of its realisation
    float gh[3] = {0.f, 0.f, 0.f}, gl[3] = {0.f, 0.f, 0.f};
    constexpr int NW = KIND == STEP_SECOND ? 3 : (KIND == STEP_GENERAL ? 1 : 0);
    auto set_weights = [&](const double *g) {
#pragma unroll
        for (int t = 0; t < NW; ++t) {
            const double gd = g[t];
            gh[t] = __double2float_rn(gd);
            gl[t] = __double2float_rn(gd - (double)gh[t]);
        }
    };
    const int w0 = KIND == STEP_GENERAL ? A.p : 0;
    if (!A.chunk_rid && NW) set_weights(A.gc + w0);
    // 32-bit gather offsets (16-byte units) when the chunk height is compiled in
    const uint32_t ld16 = (uint32_t)A.ldin;
    float2 uu_s2[VPT], uu_e2[VPT], wu_s2[VPT], wu_e2[VPT];     // per lane (real part, imaginary part)
#pragma unroll
    for (int q = 0; q < VPT; ++q) uu_s2[q] = uu_e2[q] = wu_s2[q] = wu_e2[q] = make_float2(0.f, 0.f);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int64_t c, int b) {     // thread 0: stage chunk c into buffer b
        const int cl = __ldg(A.H.chunk_len + c);
        const int len = (cl & 0xffff) + (cl >> 16);
        const int64_t base = __ldg(A.H.chunk_ptr + c);
        const uint32_t nslot = (uint32_t)len << log2C;
        s_len[b] = cl;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[b], nslot * (uint32_t)(4 + sizeof(float2)) + tx_extra);
        if (nslot) {
            tma_load_1d(col_s(b), A.H.col + base, nslot * 4u, &bar[b]);
            tma_load_1d(val_s(b), gval + base, nslot * (uint32_t)sizeof(float2), &bar[b]);
        }
    };

    int k = 0;
    bool ok = true;
    bool prefetched = false;
    const ChunkRange cr = cta_chunks(n_chunks);
    if (tid == 0 && cr.first < cr.last) issue(cr.first, 0);
    __syncthreads();
    for (int64_t c = cr.first; c < cr.last; c += cr.stride, ++k) {
        const int b = k & 1;
        prefetched = c + cr.stride < cr.last;
        if (tid == 0 && prefetched) issue(c + cr.stride, b ^ 1);
        const bool landed = mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1), limit);
        if (landed) {
            const int cl = s_len[b];
            const int nre = cl & 0xffff;
            const int len = nre + (cl >> 16);
            if (A.chunk_rid && NW) set_weights(A.rcoef + (int64_t)__ldg(A.chunk_rid + c) * A.rcoef_ld + 2 + w0);
            for (int rr = warp * RPW + sub; rr < chunk_h; rr += STEP_WARPS * RPW) {
                const int64_t r = (c << log2C) + rr;
                if (r >= n_rows) continue;
                const int64_t i = A.H.perm ? (int64_t)__ldg(A.H.perm + r) : r;
                const int32_t *colp = col_s(b) + rr;
                const float2 *valp = val_s(b) + rr;
                // the row sum starts at -V_prev (general), -X (second) or 0:
                // (s, e), lane 0 the real part, lane 1 the imaginary part
                float4 u[VPT], xo[VPT];
                float2 s2[VPT], e2[VPT];
#pragma unroll
                for (int q = 0; q < VPT; ++q) {
                    float4 w0v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (KIND == STEP_GENERAL) w0v = wout[i * A.ldw + j0 + q];
                    if (KIND == STEP_SECOND) w0v = xdw[i * A.ldx + j0 + q];
                    s2[q] = make_float2(-w0v.x, -w0v.y);
                    e2[q] = make_float2(-w0v.z, -w0v.w);
                }
                auto gather = [&](int kk, float4 (&v)[VPT]) {
                    const int cc = max(colp[kk << log2C], 0);          // padding: col -1, value 0
                    if constexpr (CH > 0) {
                        const float4 *row = vin + (uint64_t)((uint32_t)cc * ld16) + j0;
#pragma unroll
                        for (int q = 0; q < VPT; ++q) v[q] = ld_nc4(row + q);
                    } else {
#pragma unroll
                        for (int q = 0; q < VPT; ++q) v[q] = ld_nc4(vin + (int64_t)cc * A.ldin + j0 + q);
                    }
                };
                // real slot: (re, im) += h (v_re, v_im); imaginary slot, with
                // the accumulator lanes swapped to (im, re) for the whole
                // group: (im, re) += (h, -h) (v_re, v_im), i.e. i h v
                auto madd = [&](int kk, bool imag, const float4 (&v)[VPT]) {
                    const float2 h = valp[kk << log2C];
                    const float2 hh = make_float2(h.x, imag ? -h.x : h.x);
                    const float2 nhh = neg2(hh);
                    const float2 nhl = make_float2(-h.y, imag ? h.y : -h.y);
#pragma unroll
                    for (int q = 0; q < VPT; ++q)
                        dw_mac2(s2[q], e2[q], hh, nhh, nhl, make_float2(v[q].x, v[q].y), make_float2(v[q].z, v[q].w));
                };
                constexpr int U = CFD_DW_GROUP;
                for (int g = 0; g < 2; ++g) {             // real group, then imaginary group
                    const bool imag = g == 1;
                    int kk = imag ? nre : 0;
                    const int k1 = imag ? len : nre;
                    if (imag) {
#pragma unroll
                        for (int q = 0; q < VPT; ++q) { s2[q] = swap2(s2[q]); e2[q] = swap2(e2[q]); }
                    }
                    for (; kk + U <= k1; kk += U) {
                        float4 vv[U][VPT];
#pragma unroll
                        for (int uo = 0; uo < U; ++uo) gather(kk + uo, vv[uo]);
#pragma unroll
                        for (int uo = 0; uo < U; ++uo) madd(kk + uo, imag, vv[uo]);
                    }
                    for (; kk < k1; ++kk) {
                        float4 v[VPT];
                        gather(kk, v);
                        madd(kk, imag, v);
                    }
                    if (imag) {
#pragma unroll
                        for (int q = 0; q < VPT; ++q) { s2[q] = swap2(s2[q]); e2[q] = swap2(e2[q]); }
                    }
                }
                // the own row of vin (moments; V1 in the second step's X
                // update) and X
#pragma unroll
                for (int q = 0; q < VPT; ++q) {
                    if (MOM || KIND == STEP_SECOND) u[q] = ld_nc4(vin + i * A.ldin + j0 + q);
                    if (KIND != STEP_FIRST) xo[q] = xdw[i * A.ldx + j0 + q];
                }
                // the new vector = the renormalised sum; X update; moments
#pragma unroll
                for (int q = 0; q < VPT; ++q) {
                    float2 nh, nl;
                    two_sum2(s2[q], e2[q], nh, nl);
                    float4 wn = make_float4(nh.x, nh.y, nl.x, nl.y);
                    if (KIND == STEP_FIRST) wn = dw_scale(wn, 0.5f);
                    wout[i * A.ldw + j0 + q] = wn;
                    const float2 wh = make_float2(wn.x, wn.y), wl = make_float2(wn.z, wn.w);
                    const float2 uh = make_float2(u[q].x, u[q].y), ul = make_float2(u[q].z, u[q].w);
                    if (KIND != STEP_FIRST) {
                        float2 xh = make_float2(xo[q].x, xo[q].y), xl = make_float2(xo[q].z, xo[q].w);
                        if (KIND == STEP_SECOND) {
                            // g0 X + g1 V1 + g2 V2 as (0 + g0 X) + g1 V1 + g2 V2
                            float2 ah = make_float2(0.f, 0.f), al = make_float2(0.f, 0.f);
                            dw_axpy2(ah, al, bcast2(gh[0]), bcast2(-gh[0]), bcast2(-gl[0]), xh, xl);
                            dw_axpy2(ah, al, bcast2(gh[1]), bcast2(-gh[1]), bcast2(-gl[1]), uh, ul);
                            xh = ah;
                            xl = al;
                        }
                        dw_axpy2(xh, xl, bcast2(gh[NW - 1]), bcast2(-gh[NW - 1]), bcast2(-gl[NW - 1]), wh, wl);
                        if (LAST) {
                            double2 *xd = reinterpret_cast<double2 *>(xdw + i * A.ldx + j0 + q);
                            *xd = make_double2((double)xh.x + (double)xl.x, (double)xh.y + (double)xl.y);
                        } else {
                            xdw[i * A.ldx + j0 + q] = make_float4(xh.x, xh.y, xl.x, xl.y);
                        }
                    }
                    if (MOM) {
                        // lanewise: (re^2, im^2) and (wn_re u_re, wn_im u_im)
                        dw_mac2(uu_s2[q], uu_e2[q], uh, neg2(uh), neg2(ul), uh, ul);
                        dw_mac2(wu_s2[q], wu_e2[q], wh, neg2(wh), neg2(wl), uh, ul);
                    }
                }
            }
        }
        if (!__syncthreads_and(landed)) {
            ok = false;
            break;
        }
    }
    if (!ok) {
        if (tid == 0) {
            const int b = k & 1;
            if (tx_extra) {
                mbar_complete_tx(&bar[b], tx_extra);
                if (prefetched) mbar_complete_tx(&bar[b ^ 1], tx_extra);
            }
            const long long drain_limit = 1LL << 32;
            bool drained = mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1), drain_limit);
            if (prefetched)
                drained = mbar_wait_bounded(&bar[b ^ 1], (uint32_t)(((k + 1) >> 1) & 1), drain_limit) && drained;
            atomicOr(A.status, drained ? (int)CFD_ERR_TIMEOUT : (int)CFD_ERR_TIMEOUT | CFD_STATUS_DRAIN_EXPIRED);
        }
        return;
    }
    if (MOM) {
        // the threads' double-word sums (s + e) as Kahan-form accumulators
        // (value s - c) for the shared deterministic reduction
        // after adding the two lanes: (s.x + e.x) + (s.y + e.y) = t + lo
        MomentAcc<float> uu[VPT], wu[VPT];
        auto lanes = [](float2 s, float2 e, MomentAcc<float> &m) {
            float t, err;
            two_sum(s.x, s.y, t, err);
            m.s = t;
            m.c = -__fadd_rn(__fadd_rn(e.x, e.y), err);
        };
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            lanes(uu_s2[q], uu_e2[q], uu[q]);
            lanes(wu_s2[q], wu_e2[q], wu[q]);
        }
        reduce_moments<float, NB, VPT>(A.partial, A.ticket, A.dots, uu, wu);
    }
}

// ------------------------------------------------------------ conversions --

// In place, N x nb complex elements of a block with row stride ld (elements):
// complex double -> double-word {re_hi, im_hi, re_lo, im_lo} (TO_DW) or back.
// hi = fl32(x), lo = fl32(x - hi): x - hi is exact in fp64, so hi + lo is x
// rounded to 48 bits; back: hi + lo evaluated in fp64 (exact).
template <bool TO_DW>
__global__ void k_dw_convert(double2 *p, int64_t ld, int64_t n_rows, int nb) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_rows * nb) return;
    const int64_t i = e / nb;
    const int j = (int)(e % nb);
    double2 *a = p + i * ld + j;
    if (TO_DW) {
        const double2 z = *a;
        const float rh = __double2float_rn(z.x), ih = __double2float_rn(z.y);
        const float rl = __double2float_rn(z.x - (double)rh), il = __double2float_rn(z.y - (double)ih);
        *reinterpret_cast<float4 *>(a) = make_float4(rh, ih, rl, il);
    } else {
        const float4 d = *reinterpret_cast<const float4 *>(a);
        *a = make_double2((double)d.x + (double)d.z, (double)d.y + (double)d.w);
    }
}

// Prepared values 2 alpha (H - beta) as double-words {hi, lo}, one per packed
// slot, in H's SELL layout (the double-word form of k_prepare_values' output).
__global__ void k_prepare_values_dw(SellView<double> H, int64_t n_pos, double alpha, double beta,
                                    const int32_t *chunk_rid, const double *rcoef, int64_t rcoef_ld, float2 *out) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_pos) return;
    const int64_t ch = r >> H.log2C;
    const int64_t base = H.chunk_ptr[ch] + (r & ((1 << H.log2C) - 1));
    const int cl = H.chunk_len[ch];
    const int len = (cl & 0xffff) + (cl >> 16);
    const int64_t i = r < H.n_rows ? (H.perm ? (int64_t)H.perm[r] : r) : -2;
    if (chunk_rid) {
        const double *rc = rcoef + (int64_t)chunk_rid[ch] * rcoef_ld;
        alpha = rc[0];
        beta = rc[1];
    }
    const double a2 = 2.0 * alpha;
    for (int k = 0; k < len; ++k) {
        const int64_t s = base + ((int64_t)k << H.log2C);
        const double h = H.pval[s];
        const double v = H.col[s] == i ? a2 * (h - beta) : a2 * h;
        const float hi = __double2float_rn(v);
        out[s] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

// ---------------------------------------------------------------- launch --

namespace {

template <int NB, int VPT, int KIND, bool MOM, int CH, bool LAST>
cfd_status launch_dw_t(const StepArgs<double> &A, int grid_cap, cudaStream_t stream) {
    const int slots_cap = A.H.slots_bound << A.H.log2C;
    if (slots_cap <= 0) return fail(CFD_ERR_ARG, "matrix has no slot bound; cannot stage");
    const size_t smem = 2 * round_up((size_t)slots_cap * 4, 16) + round_up(2 * (size_t)slots_cap * sizeof(float2), 16);
    if (smem > 200 * 1024) return fail(CFD_ERR_ARG, "chunk too large to stage (%zu bytes)", smem);
    auto kern = k_cheb_step_dw<NB, VPT, KIND, MOM, CH, LAST>;
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
            cache.occ[dev] = std::max(1, std::min(o, STEP_MAX_CTAS_PER_SM));
            cache.occ_smem[dev] = smem;
        }
        resident = cache.occ[dev];
    }
    const int64_t n_chunks = (A.H.n_rows + (1LL << A.H.log2C) - 1) >> A.H.log2C;
    int64_t grid = std::min<int64_t>((int64_t)resident * sm_count(), n_chunks);
    if (grid_cap > 0) grid = std::min<int64_t>(grid, grid_cap);
    grid = std::max<int64_t>(grid, 1);
    kern<<<(unsigned)grid, STEP_WARPS * 32, smem, stream>>>(A, slots_cap);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

template <int NB, int VPT, bool MOM>
cfd_status launch_dw_m(int kind, const StepArgs<double> &A, bool last, int grid_cap, cudaStream_t s) {
    // chunk height 32 compiled in when the gathers' 16-byte offsets fit in 32 bits
    const bool fixed = A.H.log2C == 5 && (uint64_t)A.H.n_rows * (uint64_t)A.ldin < (1ULL << 32);
#define CFD_DW_K(CH_)                                                                                  \
    if (kind == STEP_FIRST) return launch_dw_t<NB, VPT, STEP_FIRST, MOM, CH_, false>(A, grid_cap, s);  \
    if (kind == STEP_SECOND) return launch_dw_t<NB, VPT, STEP_SECOND, MOM, CH_, false>(A, grid_cap, s); \
    return last ? launch_dw_t<NB, VPT, STEP_GENERAL, MOM, CH_, true>(A, grid_cap, s)                   \
                : launch_dw_t<NB, VPT, STEP_GENERAL, MOM, CH_, false>(A, grid_cap, s);
    if (fixed) {
        CFD_DW_K(32)
    }
    CFD_DW_K(0)
#undef CFD_DW_K
}

}  // namespace

// vpt: vectors per thread, as for the native step (default 1 at n_b = 8,
// else 2; 1 also at n_b = 16 and 32).  last (general steps): X written back
// as complex double.
cfd_status launch_step_dw(int kind, int nb, int vpt, const StepArgs<double> &A, bool last, int grid_cap,
                          cudaStream_t s) {
    if (!A.H.packed) return fail(CFD_ERR_ARG, "double-word arithmetic needs packed matrix values (CFD_PACK_RI)");
    if (!A.status || !A.prep_val) return fail(CFD_ERR_INTERNAL, "double-word step without status or prepared values");
    const bool mom = A.dots != nullptr;
#define CFD_DW_CASE(NB_, VPT_)                                                                   \
    if (nb == NB_ && vpt == VPT_)                                                                \
        return mom ? launch_dw_m<NB_, VPT_, true>(kind, A, last, grid_cap, s)                    \
                   : launch_dw_m<NB_, VPT_, false>(kind, A, last, grid_cap, s);
    CFD_DW_CASE(8, 1)
    CFD_DW_CASE(16, 1)
    CFD_DW_CASE(16, 2)
    CFD_DW_CASE(32, 1)
    CFD_DW_CASE(32, 2)
    CFD_DW_CASE(64, 2)
#undef CFD_DW_CASE
    return fail(CFD_ERR_ARG, "double-word step: n_b=%d with %d vectors per thread is not built", nb, vpt);
}

cfd_status launch_dw_convert(void *p, int64_t ld, int64_t n_rows, int nb, bool to_dw, cudaStream_t stream) {
    const int64_t n = n_rows * nb;
    if (n == 0) return CFD_OK;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (to_dw) k_dw_convert<true><<<grid, 256, 0, stream>>>(static_cast<double2 *>(p), ld, n_rows, nb);
    else k_dw_convert<false><<<grid, 256, 0, stream>>>(static_cast<double2 *>(p), ld, n_rows, nb);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

cfd_status launch_prepare_values_dw(const cfd_matrix *H, double alpha, double beta, const int32_t *chunk_rid,
                                    const double *rcoef, int64_t rcoef_ld, void *out, size_t out_bytes,
                                    cudaStream_t stream) {
    const SellView<double> v = sell_view<double>(H);
    if (!v.packed) return fail(CFD_ERR_ARG, "double-word arithmetic needs packed matrix values (CFD_PACK_RI)");
    if ((size_t)H->n_slots * sizeof(float2) > out_bytes)
        return fail(CFD_ERR_ARG, "matrix stores %lld slots, more than the filter workspace prepares (%d per row)",
                    (long long)H->n_slots, kMaxRowSlots);
    const int64_t n_pos = H->n_chunks << v.log2C;
    if (n_pos == 0) return CFD_OK;
    k_prepare_values_dw<<<(unsigned)((n_pos + 255) / 256), 256, 0, stream>>>(v, n_pos, alpha, beta, chunk_rid, rcoef,
                                                                            rcoef_ld, static_cast<float2 *>(out));
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

}  // namespace cfd
