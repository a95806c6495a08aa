// Spectral bounds for the affine map of the filter: Lanczos on the device,
// widened by the Ritz residual bounds and clipped to the Gershgorin interval.
// (The paper needs [lmin, lmax] for alpha H + beta 1 in Algorithm 1 but does
// not say how they are found.)
#include <algorithm>

#include "dense.cuh"
#include "filter.cuh"

namespace cfd {
namespace {

constexpr int LZ_THREADS = 256;

__device__ inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ inline double sm64_uniform(uint64_t seed, uint64_t tag, uint64_t i) {
    const uint64_t G = 0x9E3779B97F4A7C15ULL;
    uint64_t key = sm64_mix(seed + G * (2 * tag + 1));
    return (double)(sm64_mix(key + (i + 1) * G) >> 11) * (1.0 / 9007199254740992.0);
}

// Complex Gaussian entries (Box-Muller on SplitMix64 uniforms), row-major N x n.
__global__ void k_gaussian(double2 *X, int64_t ldx, int64_t N, int n, uint64_t seed, uint64_t tag, int col0,
                           int n_total) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * n) return;
    int64_t i = e / n;
    int j = (int)(e % n);
    uint64_t k = (uint64_t)(i * n_total + col0 + j);
    double u1 = sm64_uniform(seed, tag, 2 * k), u2 = sm64_uniform(seed, tag, 2 * k + 1);
    double r = sqrt(-2.0 * log1p(-u1)) * 0.70710678118654752440;
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    X[i * ldx + j] = make_double2(r * c, r * s);
}

// Per-CTA [min(center - radius), max(center + radius)] over SELL rows.
template <typename C>
__global__ void __launch_bounds__(LZ_THREADS) k_gersh_part(SellView<double> H0, const C *val, double *part) {
    double lo = 1e308, hi = -1e308;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < H0.n_rows; r += stride) {
        int64_t ch = r >> H0.log2C;
        int64_t base = H0.chunk_ptr[ch] + (r & ((1 << H0.log2C) - 1));
        int64_t i = H0.perm ? H0.perm[r] : r;
        double cen = 0.0, rad = 0.0;
        const int cl = H0.chunk_len[ch];
        const int nre = H0.packed ? (cl & 0xffff) : cl;       // packed: real group, then imaginary group
        const int len = H0.packed ? nre + (cl >> 16) : cl;
        for (int k = 0; k < len; ++k) {
            int64_t at = base + ((int64_t)k << H0.log2C);
            int c = H0.col[at];
            if (c < 0) continue;
            double re, im;
            if (H0.packed) {
                re = k < nre ? H0.pval[at] : 0.0;
                im = k < nre ? 0.0 : H0.pval[at];
            } else {
                C v = val[at];
                re = v.x;
                im = v.y;
            }
            if (c == i) cen += re;
            else rad += sqrt(re * re + im * im);
        }
        lo = fmin(lo, cen - rad);
        hi = fmax(hi, cen + rad);
    }
    __shared__ double slo[LZ_THREADS], shi[LZ_THREADS];
    slo[threadIdx.x] = lo;
    shi[threadIdx.x] = hi;
    __syncthreads();
    for (int o = LZ_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + o]);
            shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = slo[0];
        part[2 * blockIdx.x + 1] = shi[0];
    }
}

// Sum of squares of a complex vector (or of w after w -= a v + b vprev).
// mode 0: norm only; mode 1: w <- w - alpha[k] v - beta[k-1] vprev first.
__global__ void __launch_bounds__(LZ_THREADS)
k_lz_update(double2 *w, const double2 *v, const double2 *vprev, const double *dots, const double *beta, int k,
            int64_t N, double *part) {
    const double a = dots[2 * k + 1];
    const double bp = k > 0 ? beta[k - 1] : 0.0;
    double s = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
        double2 x = w[i], y = v[i];
        double2 z = k > 0 ? vprev[i] : make_double2(0.0, 0.0);
        x.x = x.x - a * y.x - bp * z.x;
        x.y = x.y - a * y.y - bp * z.y;
        w[i] = x;
        s += x.x * x.x + x.y * x.y;
    }
    __shared__ double sh[LZ_THREADS];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = LZ_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_lz_fold(const double *part, int nparts, double *beta, int k) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[b];
        beta[k] = sqrt(s);
    }
}

__global__ void k_scale(double2 *w, int64_t N, const double *beta, int k) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double b = beta[k];
    double s = b > 0 ? 1.0 / b : 0.0;
    double2 x = w[i];
    w[i] = make_double2(x.x * s, x.y * s);
}

// Tridiagonal T (m x m, complex storage) from alpha = dots[2k + 1], beta.
__global__ void k_lz_tridiag(const double *dots, const double *beta, int m, double2 *T) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    int i = e / m, j = e % m;
    double v = 0.0;
    if (i == j) v = dots[2 * i + 1];
    else if (j == i + 1) v = beta[i];
    else if (i == j + 1) v = beta[j];
    T[e] = make_double2(v, 0.0);
}

// Bounds: extreme Ritz values widened by |beta_m y_{m,i}| and 1% of their
// spread, clipped to the Gershgorin interval (part folded here).
__global__ void k_lz_bounds(const double *theta, const double2 *Y, int m, const double *beta, const double *gpart,
                            int ngp, double *out) {
    if (blockIdx.x || threadIdx.x) return;
    double glo = 1e308, ghi = -1e308;
    for (int b = 0; b < ngp; ++b) {
        glo = fmin(glo, gpart[2 * b]);
        ghi = fmax(ghi, gpart[2 * b + 1]);
    }
    double bm = beta[m - 1];
    double2 y0 = Y[(int64_t)(m - 1) * m + 0], y1 = Y[(int64_t)(m - 1) * m + (m - 1)];
    double r0 = fabs(bm) * sqrt(y0.x * y0.x + y0.y * y0.y);
    double r1 = fabs(bm) * sqrt(y1.x * y1.x + y1.y * y1.y);
    double spread = theta[m - 1] - theta[0];
    double lo = theta[0] - r0 - 0.01 * spread;
    double hi = theta[m - 1] + r1 + 0.01 * spread;
    out[0] = fmax(lo, glo);
    out[1] = fmin(hi, ghi);
    out[2] = glo;
    out[3] = ghi;
}

int lz_ctas(int64_t N) { return (int)std::min<int64_t>(std::max<int64_t>(1, (N + LZ_THREADS - 1) / LZ_THREADS), 2 * sm_count()); }

}  // namespace

size_t bounds_workspace(int64_t N, int steps) {
    Carve c(nullptr, 0);
    for (int q = 0; q < 3; ++q) c.take<double2>((size_t)N);
    c.take<double>(4096);                      // partials
    c.take<double>((size_t)2 * steps + 2);     // dots (alpha)
    c.take<double>((size_t)steps + 2);         // beta
    c.take<double2>((size_t)steps * steps);    // T
    c.take<double2>((size_t)steps * steps);    // Y
    c.take<double>((size_t)steps);             // theta
    c.take<double>(8);                         // out
    c.take<double>((size_t)STEP_MAX_GRID * 2); // step partials
    c.take<unsigned>(64);
    c.take<char>(eigh_workspace(steps));
    return round_up(c.off, 256);
}

cfd_status gaussian_block(double2 *X, int64_t ldx, int64_t N, int n, uint64_t seed, uint64_t tag, int col0,
                          int n_total, cudaStream_t stream) {
    int64_t e = N * n;
    k_gaussian<<<(unsigned)((e + 255) / 256), 256, 0, stream>>>(X, ldx, N, n, seed, tag, col0, n_total);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

// Device-only: bounds land in out_dev[0..1] (lmin, lmax), Gershgorin in [2..3].
cfd_status spectral_bounds_dev(const cfd_matrix *H, int steps, uint64_t seed, double *out_dev, void *work,
                               size_t work_bytes, cudaStream_t stream) {
    CFD_TRY(check_matrix(H));
    if (steps < 2 || steps > 256) return fail(CFD_ERR_ARG, "Lanczos steps %d not in 2..256", steps);
    if (H->prec != CFD_C128) return fail(CFD_ERR_ARG, "spectral bounds need the complex-double matrix");
    if (!work || work_bytes < bounds_workspace(H->n_rows, steps)) return fail(CFD_ERR_OOM, "bounds workspace too small");
    const int64_t N = H->n_rows;
    Carve c(work, work_bytes);
    double2 *B[3];
    for (int q = 0; q < 3; ++q) B[q] = c.take<double2>((size_t)N);
    double *part = c.take<double>(4096);
    double *dots = c.take<double>((size_t)2 * steps + 2);
    double *beta = c.take<double>((size_t)steps + 2);
    double2 *T = c.take<double2>((size_t)steps * steps);
    double2 *Y = c.take<double2>((size_t)steps * steps);
    double *theta = c.take<double>((size_t)steps);
    double *outw = c.take<double>(8);
    double *spart = c.take<double>((size_t)STEP_MAX_GRID * 2);
    unsigned *ticket = c.take<unsigned>(64);
    size_t ewb = eigh_workspace(steps);
    void *ew = c.take<char>(ewb);
    (void)outw;
    const int ctas = lz_ctas(N);
    SellView<double> H0 = sell_view<double>(H);
    k_gersh_part<double2><<<ctas, LZ_THREADS, 0, stream>>>(H0, static_cast<const double2 *>(H->val), part + 2048);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    CFD_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), stream));
    // v_0: normalised Gaussian vector
    double2 *vprev = B[0], *v = B[1], *w = B[2];
    CFD_TRY(gaussian_block(v, 1, N, 1, seed, 2, 0, 1, stream));
    CFD_CUDA(cudaMemsetAsync(dots, 0, sizeof(double) * 2, stream));
    k_lz_update<<<ctas, LZ_THREADS, 0, stream>>>(v, v, v, dots, beta, 0, N, part);   // alpha = 0: norm only
    k_lz_fold<<<1, 1, 0, stream>>>(part, ctas, beta, steps + 1);
    CFD_COUNT_LAUNCH();
    k_scale<<<(unsigned)((N + 255) / 256), 256, 0, stream>>>(v, N, beta, steps + 1);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    StepArgs<double> A;
    A.H = H0;
    A.gc = nullptr;
    A.partial = spart;
    A.ticket = ticket;
    A.a = 1.0;
    A.beta = 0.0;
    A.p = 1;
    A.x = nullptr;
    A.ldx = 0;
    for (int k = 0; k < steps; ++k) {
        A.vin = v;
        A.ldin = 1;
        A.w = w;
        A.ldw = 1;
        A.dots = dots + 2 * k;                 // (<v, v>, alpha_k = Re <H v, v>)
        CFD_TRY(launch_step<double>(STEP_FIRST, 1, 1, A, 0, stream));
        k_lz_update<<<ctas, LZ_THREADS, 0, stream>>>(w, v, vprev, dots, beta, k, N, part);
        CFD_COUNT_LAUNCH();
        k_lz_fold<<<1, 1, 0, stream>>>(part, ctas, beta, k);
        CFD_COUNT_LAUNCH();
        k_scale<<<(unsigned)((N + 255) / 256), 256, 0, stream>>>(w, N, beta, k);
        CFD_COUNT_LAUNCH();
        CFD_LAUNCH_CHECK();
        double2 *t = vprev;
        vprev = v;
        v = w;
        w = t;
    }
    k_lz_tridiag<<<(steps * steps + 255) / 256, 256, 0, stream>>>(dots, beta, steps, T);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    CFD_TRY(eigh(T, steps, steps, theta, Y, steps, ew, ewb, stream, nullptr));
    k_lz_bounds<<<1, 1, 0, stream>>>(theta, Y, steps, beta, part + 2048, ctas, out_dev);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

}  // namespace cfd

using namespace cfd;

extern "C" {

size_t cfd_spectral_bounds_workspace(int64_t N, int steps) {
    return (N > 0 && steps > 1) ? bounds_workspace(N, steps) + 256 : 0;
}

cfd_status cfd_spectral_bounds(const cfd_matrix *H, int steps, uint64_t seed, double *lmin, double *lmax,
                               void *work, size_t work_bytes, cudaStream_t stream) {
    clear_error();
    if (!lmin || !lmax || !work || work_bytes < 256) return fail(CFD_ERR_ARG, "NULL argument");
    double *out = static_cast<double *>(work);
    CFD_TRY(spectral_bounds_dev(H, steps, seed, out, static_cast<char *>(work) + 256, work_bytes - 256, stream));
    double h[4];
    CFD_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, stream));
    CFD_CUDA(cudaStreamSynchronize(stream));
    *lmin = h[0];
    *lmax = h[1];
    if (!(h[0] < h[1])) return fail(CFD_ERR_INTERNAL, "Lanczos bounds degenerate (%g, %g)", h[0], h[1]);
    return CFD_OK;
}

}  // extern "C"
