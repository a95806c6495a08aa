// The ChebFD polynomial filter (Algorithm 1, blocked as Algorithm 2): one
// fused SELL-C-sigma SpMMV kernel per recurrence step (the paper's
// chebfd_op), weights table, moment finalisation, precision conversion.
#include <algorithm>

#include "filter.cuh"

namespace cfd {

// ------------------------------------------------------------ weights --

// gc[k] = g_k c_k (window coefficients times Jackson kernel), k = 0..n_p.
__global__ void k_filter_coeffs(double alpha, double beta, double lam_l, double lam_r, int n_p,
                                double *gc) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n_p) return;
    const double pi = 3.141592653589793238462643383279502884;
    double xl = fmin(fmax(alpha * (lam_l - beta), -1.0), 1.0);
    double xr = fmin(fmax(alpha * (lam_r - beta), -1.0), 1.0);
    double tl = acos(xl), tr = acos(xr);
    double c = (k == 0) ? (tl - tr) / pi : 2.0 * (sin(k * tl) - sin(k * tr)) / (k * pi);
    double M = n_p + 1.0;
    double q = pi / (M + 1.0);
    double g = ((M - k + 1.0) * cos(q * k) + sin(q * k) / tan(q)) / (M + 1.0);
    gc[k] = g * c;
}

cfd_status launch_filter_coeffs(double alpha, double beta, double lam_l, double lam_r, int n_p,
                                double *gc, cudaStream_t stream) {
    k_filter_coeffs<<<(n_p + 1 + 127) / 128, 128, 0, stream>>>(alpha, beta, lam_l, lam_r, n_p, gc);
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

// ------------------------------------------------------ step kernel --

namespace {

template <typename T> struct MomentAcc;

// fp64 path: plain fp64 sums per thread.
template <> struct MomentAcc<double> {
    double s = 0.0;
    __device__ void add(double v) { s += v; }
    __device__ double value() const { return s; }
};

// fp32 path: compensated (Kahan) fp32 sums per thread, widened once at the end.
template <> struct MomentAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ void add(float v) {
        float y = v - c;
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

// One fused ChebFD step over all rows of H for a block of NB vectors.
// Thread layout: a warp covers RPW = 32 / TPR rows at a time, TPR = NB / VPT
// threads per row, each thread VPT consecutive vectors of its row.  Warps
// sweep the (sorted) rows grid-stride, so at any time the whole GPU works on
// a contiguous window of rows and the gathered neighbour rows of V_cur are
// shared through L2.  Each thread reduces its moment dot products over its
// rows; warps, then CTAs, then the last CTA to finish (ticket counter) reduce
// in a fixed order, so the moments are deterministic.
template <typename T, int NB, int VPT, int KIND>
__global__ void __launch_bounds__(STEP_WARPS * 32)
k_cheb_step(const StepArgs<T> A) {
    using C = cplx_t<T>;
    constexpr int TPR = NB / VPT;
    constexpr int RPW = 32 / TPR;
    constexpr int UNR = 4;
    static_assert(TPR >= 1 && TPR <= 32 && (32 % TPR) == 0, "bad thread split");
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int sub = lane / TPR;
    const int j0 = (lane % TPR) * VPT;
    const int log2C = A.H.log2C;
    const T a = (T)A.a;
    const T beta = (T)A.beta;
    T g0 = 0, g1 = 0, g2 = 0;
    if (KIND == STEP_SECOND) {
        g0 = (T)A.gc[0];
        g1 = (T)A.gc[1];
        g2 = (T)A.gc[2];
    } else if (KIND == STEP_GENERAL) {
        g0 = (T)A.gc[A.p];
    }
    MomentAcc<T> uu[VPT], wu[VPT];

    const int64_t n_rows = A.H.n_rows;
    const int64_t n_groups = (n_rows + RPW - 1) / RPW;
    for (int64_t grp = (int64_t)blockIdx.x * STEP_WARPS + warp; grp < n_groups;
         grp += (int64_t)gridDim.x * STEP_WARPS) {
        const int64_t r = grp * RPW + sub;
        if (r >= n_rows) continue;
        const int64_t ch = r >> log2C;
        const int64_t base = __ldg(A.H.chunk_ptr + ch) + (r & ((1 << log2C) - 1));
        const int len = __ldg(A.H.chunk_len + ch);
        const int64_t i = A.H.perm ? (int64_t)__ldg(A.H.perm + r) : r;

        C acc[VPT];
#pragma unroll
        for (int q = 0; q < VPT; ++q) acc[q] = cmake<T>(0, 0);

        int k = 0;
        for (; k + UNR <= len; k += UNR) {
            int cc[UNR];
            C hh[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const int64_t at = base + ((int64_t)(k + u) << log2C);
                cc[u] = max(__ldg(A.H.col + at), 0);      // padding: col -1, value 0
                hh[u] = __ldg(A.H.val + at);
            }
            Pack<C, VPT> vv[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) vv[u] = ld_nc<C, VPT>(A.vin + (int64_t)cc[u] * A.ldin + j0);
#pragma unroll
            for (int u = 0; u < UNR; ++u)
#pragma unroll
                for (int q = 0; q < VPT; ++q) cfma(acc[q], hh[u], vv[u].v[q]);
        }
        for (; k < len; ++k) {
            const int64_t at = base + ((int64_t)k << log2C);
            const int c = max(__ldg(A.H.col + at), 0);
            const C h = __ldg(A.H.val + at);
            Pack<C, VPT> v = ld_nc<C, VPT>(A.vin + (int64_t)c * A.ldin + j0);
#pragma unroll
            for (int q = 0; q < VPT; ++q) cfma(acc[q], h, v.v[q]);
        }

        // epilogue: shift, scale, recurrence, accumulation, moment dots
        const Pack<C, VPT> u = ld_nc<C, VPT>(A.vin + i * A.ldin + j0);
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
            Pack<C, VPT> xo = ld_rw<C, VPT>(xp), xn;
#pragma unroll
            for (int q = 0; q < VPT; ++q) {
                wn.v[q].x = fma(a, fma(-beta, u.v[q].x, acc[q].x), -xo.v[q].x);
                wn.v[q].y = fma(a, fma(-beta, u.v[q].y, acc[q].y), -xo.v[q].y);
                xn.v[q].x = fma(g2, wn.v[q].x, fma(g1, u.v[q].x, g0 * xo.v[q].x));
                xn.v[q].y = fma(g2, wn.v[q].y, fma(g1, u.v[q].y, g0 * xo.v[q].y));
            }
            st<C, VPT>(A.w + i * A.ldw + j0, wn);
            st<C, VPT>(xp, xn);
        } else {
            C *wp = A.w + i * A.ldw + j0;
            C *xp = A.x + i * A.ldx + j0;
            Pack<C, VPT> wo = ld_rw<C, VPT>(wp);
            Pack<C, VPT> xo = ld_rw<C, VPT>(xp), xn;
#pragma unroll
            for (int q = 0; q < VPT; ++q) {
                wn.v[q].x = fma(a, fma(-beta, u.v[q].x, acc[q].x), -wo.v[q].x);
                wn.v[q].y = fma(a, fma(-beta, u.v[q].y, acc[q].y), -wo.v[q].y);
                xn.v[q].x = fma(g0, wn.v[q].x, xo.v[q].x);
                xn.v[q].y = fma(g0, wn.v[q].y, xo.v[q].y);
            }
            st<C, VPT>(wp, wn);
            st<C, VPT>(xp, xn);
        }
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            uu[q].add(fma(u.v[q].x, u.v[q].x, u.v[q].y * u.v[q].y));
            wu[q].add(fma(wn.v[q].x, u.v[q].x, wn.v[q].y * u.v[q].y));
        }
    }

    // ---- deterministic moment reduction ----
    __shared__ double red[STEP_WARPS][NB][2];
    __shared__ bool last_cta;
    double s_uu[VPT], s_wu[VPT];
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
        s_uu[q] = uu[q].value();
        s_wu[q] = wu[q].value();
#pragma unroll
        for (int off = TPR; off < 32; off <<= 1) {
            s_uu[q] += __shfl_xor_sync(0xffffffffu, s_uu[q], off);
            s_wu[q] += __shfl_xor_sync(0xffffffffu, s_wu[q], off);
        }
    }
    if (sub == 0) {
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            red[warp][j0 + q][0] = s_uu[q];
            red[warp][j0 + q][1] = s_wu[q];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * NB; e += blockDim.x) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < STEP_WARPS; ++w) s += red[w][e >> 1][e & 1];
        A.partial[(int64_t)blockIdx.x * 2 * NB + e] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last_cta = (atomicAdd(A.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last_cta) {
        __threadfence();
        for (int e = warp; e < 2 * NB; e += STEP_WARPS) {
            double s = 0.0;
            for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(A.partial + (int64_t)b * 2 * NB + e);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) A.dots[e] = s;
        }
        if (threadIdx.x == 0) *A.ticket = 0u;
    }
}

// --------------------------------------------------------- launching --

namespace {

template <typename T, int NB, int VPT, int KIND>
cfd_status launch_one(const StepArgs<T> &A, int grid_cap, cudaStream_t stream) {
    auto kern = k_cheb_step<T, NB, VPT, KIND>;
    static int occ[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (occ[dev] == 0) {
        int o = 0;
        CFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, STEP_WARPS * 32, 0));
        occ[dev] = std::max(1, std::min(o, STEP_MAX_CTAS_PER_SM));
    }
    constexpr int RPW = 32 / (NB / VPT);
    int64_t groups = (A.H.n_rows + RPW - 1) / RPW;
    int64_t need = (groups + STEP_WARPS - 1) / STEP_WARPS;
    int64_t grid = std::min<int64_t>((int64_t)occ[dev] * sm_count(), need);
    if (grid_cap > 0) grid = std::min<int64_t>(grid, grid_cap);
    grid = std::max<int64_t>(grid, 1);
    kern<<<(unsigned)grid, STEP_WARPS * 32, 0, stream>>>(A);
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

template <typename T, int NB, int VPT>
cfd_status launch_kind(int kind, const StepArgs<T> &A, int grid_cap, cudaStream_t s) {
    switch (kind) {
    case STEP_FIRST: return launch_one<T, NB, VPT, STEP_FIRST>(A, grid_cap, s);
    case STEP_SECOND: return launch_one<T, NB, VPT, STEP_SECOND>(A, grid_cap, s);
    default: return launch_one<T, NB, VPT, STEP_GENERAL>(A, grid_cap, s);
    }
}

}  // namespace

template <typename T>
cfd_status launch_step(int kind, int nb, int vpt, const StepArgs<T> &A, int grid_cap,
                       cudaStream_t s) {
#define CFD_CASE(NB_, VPT_) \
    if (nb == NB_ && vpt == VPT_) return launch_kind<T, NB_, VPT_>(kind, A, grid_cap, s);
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

template cfd_status launch_step<double>(int, int, int, const StepArgs<double> &, int, cudaStream_t);
template cfd_status launch_step<float>(int, int, int, const StepArgs<float> &, int, cudaStream_t);

// ------------------------------------------------- moments, conversion --

// raw[p-1][j][0] = <T_{p-1}x_j, T_{p-1}x_j>, raw[p-1][j][1] = Re <T_p x_j, T_{p-1}x_j>
// -> mu[j][m] = <x_j, T_m x_j>, m = 0..2 n_p - 1 (T_k T_l = (T_{k+l} + T_{|k-l|}) / 2).
__global__ void k_moments(const double *raw, int n_p, int nb, double *mu, int64_t ld_mu) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)nb * 2 * n_p) return;
    int j = (int)(e / (2 * n_p));
    int m = (int)(e % (2 * n_p));
    double mu0 = raw[2 * j + 0], mu1 = raw[2 * j + 1];
    double v;
    if (m == 0) v = mu0;
    else if (m == 1) v = mu1;
    else {
        int p = m / 2 + 1;
        const double *d = raw + (int64_t)(p - 1) * 2 * nb + 2 * j;
        v = (m & 1) ? 2.0 * d[1] - mu1 : 2.0 * d[0] - mu0;
    }
    mu[(int64_t)j * ld_mu + m] = v;
}

cfd_status launch_moments(const double *raw, int n_p, int nb, double *mu, int64_t ld_mu,
                          cudaStream_t stream) {
    int64_t n = (int64_t)nb * 2 * n_p;
    k_moments<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(raw, n_p, nb, mu, ld_mu);
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

// Round a strided complex-double block to a contiguous complex-float block
// (round to nearest) or widen it back.
__global__ void k_narrow(const double2 *src, int64_t lds, float2 *dst, int64_t ldd, int64_t n_rows,
                         int nb) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_rows * nb) return;
    int64_t i = e / nb;
    int j = (int)(e % nb);
    double2 z = src[i * lds + j];
    dst[i * ldd + j] = make_float2(__double2float_rn(z.x), __double2float_rn(z.y));
}

__global__ void k_widen(const float2 *src, int64_t lds, double2 *dst, int64_t ldd, int64_t n_rows,
                        int nb) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_rows * nb) return;
    int64_t i = e / nb;
    int j = (int)(e % nb);
    float2 z = src[i * lds + j];
    dst[i * ldd + j] = make_double2((double)z.x, (double)z.y);
}

cfd_status launch_narrow(const double2 *src, int64_t lds, float2 *dst, int64_t ldd, int64_t n_rows,
                         int nb, cudaStream_t stream) {
    int64_t n = n_rows * nb;
    k_narrow<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(src, lds, dst, ldd, n_rows, nb);
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

cfd_status launch_widen(const float2 *src, int64_t lds, double2 *dst, int64_t ldd, int64_t n_rows,
                        int nb, cudaStream_t stream) {
    int64_t n = n_rows * nb;
    k_widen<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(src, lds, dst, ldd, n_rows, nb);
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

// ------------------------------------------------------------- driver --

int default_vpt(int prec, int n_b) {
    if (prec == CFD_C64) return 2;          // float4 = two complex floats per 16-byte access
    return n_b > 32 ? 2 : 1;                // one complex double per 16-byte access
}

size_t filter_workspace(int64_t N, int n_s, int n_b, int n_p, int prec_H, int prec_X) {
    (void)n_s;
    size_t sH = prec_H == CFD_C128 ? 16 : 8;
    Carve c(nullptr, 0);
    c.take<char>((size_t)N * n_b * sH);                      // V_a
    c.take<char>((size_t)N * n_b * sH);                      // V_b
    if (prec_H != prec_X) c.take<char>((size_t)N * n_b * 8); // narrowed X block
    c.take<double>((size_t)n_p + 1);                          // weights
    c.take<double>((size_t)n_p * n_b * 2);                    // raw dots
    c.take<double>((size_t)STEP_MAX_GRID * 2 * n_b);       // CTA partials
    c.take<unsigned>(64);                                     // ticket
    return round_up(c.off, 256);
}

cfd_status validate_block(const cfd_block &X, int64_t n_rows) {
    if (!X.ptr) return fail(CFD_ERR_ARG, "block pointer is NULL");
    if (X.n_rows != n_rows) return fail(CFD_ERR_ARG, "block has %lld rows, matrix %lld",
                                        (long long)X.n_rows, (long long)n_rows);
    if (X.n_cols < 1 || X.ld < X.n_cols) return fail(CFD_ERR_ARG, "block ld/n_cols invalid");
    if (X.prec != CFD_C128 && X.prec != CFD_C64) return fail(CFD_ERR_ARG, "block precision invalid");
    size_t s = X.prec == CFD_C128 ? 16 : 8;
    if (!aligned16(X.ptr) || ((size_t)X.ld * s) % 16) return fail(CFD_ERR_ARG, "block must be 16-byte aligned with ld * scalar a multiple of 16 bytes");
    return CFD_OK;
}

template <typename T>
static cfd_status run_filter(const cfd_matrix *H, double alpha, double beta, int n_p, const cfd_block &X,
                             int n_b, int vpt, const FilterScratch &ws, double *moments,
                             cudaStream_t stream) {
    using C = cplx_t<T>;
    const bool mixed = (X.prec != H->prec);
    StepArgs<T> A;
    A.H = sell_view<T>(H);
    A.gc = ws.gc;
    A.partial = ws.partial;
    A.ticket = ws.ticket;
    C *va = static_cast<C *>(ws.va), *vb = static_cast<C *>(ws.vb);
    const int n_blocks = X.n_cols / n_b;
    const size_t sX = X.prec == CFD_C128 ? 16 : 8;
    for (int b = 0; b < n_blocks; ++b) {
        C *xb;
        int64_t ldx;
        char *xsrc = static_cast<char *>(X.ptr) + (size_t)b * n_b * sX;
        if (mixed) {
            CFD_TRY(launch_narrow(reinterpret_cast<const double2 *>(xsrc), X.ld, static_cast<float2 *>(ws.xn),
                                  n_b, X.n_rows, n_b, stream));
            xb = static_cast<C *>(ws.xn);
            ldx = n_b;
        } else {
            xb = reinterpret_cast<C *>(xsrc);
            ldx = X.ld;
        }
        // step 1: V1 = H~ X_b
        A.vin = xb; A.ldin = ldx; A.w = va; A.ldw = n_b; A.x = nullptr; A.ldx = 0;
        A.a = alpha; A.beta = beta; A.p = 1; A.dots = ws.raw;
        CFD_TRY(launch_step<T>(STEP_FIRST, n_b, vpt, A, ws.grid_cap, stream));
        // step 2: V2 = 2 H~ V1 - X_b, X_b = gc0 X_b + gc1 V1 + gc2 V2
        A.vin = va; A.ldin = n_b; A.w = vb; A.ldw = n_b; A.x = xb; A.ldx = ldx;
        A.a = 2.0 * alpha; A.p = 2; A.dots = ws.raw + 2 * n_b;
        CFD_TRY(launch_step<T>(STEP_SECOND, n_b, vpt, A, ws.grid_cap, stream));
        // steps 3..n_p: swap(V_prev, V_cur); V_prev = 2 H~ V_cur - V_prev; X_b += gc_p V_prev
        for (int p = 3; p <= n_p; ++p) {
            C *cur = (p & 1) ? vb : va;
            C *prev = (p & 1) ? va : vb;
            A.vin = cur; A.ldin = n_b; A.w = prev; A.ldw = n_b; A.p = p;
            A.dots = ws.raw + (int64_t)(p - 1) * 2 * n_b;
            CFD_TRY(launch_step<T>(STEP_GENERAL, n_b, vpt, A, ws.grid_cap, stream));
        }
        if (moments) CFD_TRY(launch_moments(ws.raw, n_p, n_b, moments + (int64_t)b * n_b * 2 * n_p, 2 * n_p, stream));
        if (mixed)
            CFD_TRY(launch_widen(static_cast<const float2 *>(ws.xn), n_b, reinterpret_cast<double2 *>(xsrc),
                                 X.ld, X.n_rows, n_b, stream));
    }
    return CFD_OK;
}

cfd_status filter_impl(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r,
                       int n_p, const cfd_block &X, int n_b, int vpt, int grid_cap, void *work,
                       size_t work_bytes, double *moments, cudaStream_t stream) {
    CFD_TRY(check_matrix(H));
    CFD_TRY(validate_block(X, H->n_rows));
    if (!(lmin < lmax) || !(lmin <= lam_l && lam_l < lam_r && lam_r <= lmax))
        return fail(CFD_ERR_ARG, "need lmin <= lam_l < lam_r <= lmax (got %g %g %g %g)", lmin, lam_l, lam_r, lmax);
    if (n_p < 2) return fail(CFD_ERR_ARG, "n_p=%d < 2", n_p);
    if (n_b != 8 && n_b != 16 && n_b != 32 && n_b != 64) return fail(CFD_ERR_ARG, "n_b=%d not in {8,16,32,64}", n_b);
    if (X.n_cols % n_b) return fail(CFD_ERR_ARG, "n_b=%d does not divide n_s=%d", n_b, X.n_cols);
    if (!(X.prec == H->prec || (H->prec == CFD_C64 && X.prec == CFD_C128)))
        return fail(CFD_ERR_ARG, "unsupported precision pair (matrix %d, block %d)", H->prec, X.prec);
    if (vpt <= 0) vpt = default_vpt(H->prec, n_b);
    if (!work) return fail(CFD_ERR_ARG, "work is NULL");
    size_t need = filter_workspace(H->n_rows, X.n_cols, n_b, n_p, H->prec, X.prec);
    if (work_bytes < need) return fail(CFD_ERR_OOM, "filter workspace %zu < %zu bytes", work_bytes, need);
    if (!aligned16(work)) return fail(CFD_ERR_ARG, "work must be 16-byte aligned");

    size_t sH = H->prec == CFD_C128 ? 16 : 8;
    Carve c(work, work_bytes);
    FilterScratch ws;
    ws.va = c.take<char>((size_t)H->n_rows * n_b * sH);
    ws.vb = c.take<char>((size_t)H->n_rows * n_b * sH);
    ws.xn = (H->prec != X.prec) ? c.take<char>((size_t)H->n_rows * n_b * 8) : nullptr;
    ws.gc = c.take<double>((size_t)n_p + 1);
    ws.raw = c.take<double>((size_t)n_p * n_b * 2);
    ws.partial = c.take<double>((size_t)STEP_MAX_GRID * 2 * n_b);
    ws.ticket = c.take<unsigned>(64);
    ws.grid_cap = std::min(grid_cap > 0 ? grid_cap : STEP_MAX_GRID, STEP_MAX_GRID);
    CFD_CUDA(cudaMemsetAsync(ws.ticket, 0, sizeof(unsigned), stream));

    const double alpha = 2.0 / (lmax - lmin);
    const double beta = 0.5 * (lmax + lmin);
    CFD_TRY(launch_filter_coeffs(alpha, beta, lam_l, lam_r, n_p, ws.gc, stream));
    if (H->prec == CFD_C128) return run_filter<double>(H, alpha, beta, n_p, X, n_b, vpt, ws, moments, stream);
    return run_filter<float>(H, alpha, beta, n_p, X, n_b, vpt, ws, moments, stream);
}

}  // namespace cfd

using namespace cfd;

extern "C" {

cfd_status cfd_filter_coeffs(double lmin, double lmax, double lam_l, double lam_r, int n_p, double *gc,
                             cudaStream_t stream) {
    clear_error();
    if (!gc) return fail(CFD_ERR_ARG, "gc is NULL");
    if (!(lmin < lmax) || !(lmin <= lam_l && lam_l < lam_r && lam_r <= lmax))
        return fail(CFD_ERR_ARG, "need lmin <= lam_l < lam_r <= lmax");
    if (n_p < 2) return fail(CFD_ERR_ARG, "n_p < 2");
    return launch_filter_coeffs(2.0 / (lmax - lmin), 0.5 * (lmax + lmin), lam_l, lam_r, n_p, gc, stream);
}

size_t cfd_filter_workspace(int64_t N, int n_s, int n_b, int n_p, int prec_H, int prec_X) {
    if (N < 1 || n_b < 1 || n_p < 2) return 0;
    return filter_workspace(N, n_s, n_b, n_p, prec_H, prec_X);
}

cfd_status cfd_filter(const cfd_matrix *H, double lmin, double lmax, double lam_l, double lam_r, int n_p,
                      cfd_block X, int n_b, void *work, size_t work_bytes, double *moments,
                      cudaStream_t stream) {
    clear_error();
    return filter_impl(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, 0, 0, work, work_bytes, moments, stream);
}

}  // extern "C"
