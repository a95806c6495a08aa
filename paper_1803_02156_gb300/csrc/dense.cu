// Dense fp64 kernels for orthogonalisation and Rayleigh-Ritz on tall-skinny
// complex blocks: Gram matrices and in-place projections on the FP64 tensor
// cores (mma.sync m8n8k4 f64; tcgen05 has no f64 kind), the cyclic Jacobi
// eigensolver for small complex Hermitian matrices, and column residual norms.
//
// A complex N x n block with unit column stride is viewed as a real N x 2n
// matrix (interleaved re, im).  The complex Gram S = X^H Y follows from the
// real Gram G = Xr^T Yr:  S_ab = (G_2a,2b + G_2a+1,2b+1) + i (G_2a,2b+1 - G_2a+1,2b),
// and X M equals Xr Mr with the real representation Mr of M
// (Mr_2a,2b = Mr_2a+1,2b+1 = Re M_ab, Mr_2a,2b+1 = Im M_ab, Mr_2a+1,2b = -Im M_ab).
#include <algorithm>
#include <atomic>
#include <cooperative_groups.h>

#include "dense.cuh"

namespace cg = cooperative_groups;

namespace cfd {

// D += A B for one 8x8x4 fp64 tile; a: A[lane>>2][lane&3], b: B[lane&3][lane>>2],
// d: D[lane>>2][2 (lane&3) + {0, 1}].
__device__ __forceinline__ void dmma(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

// ------------------------------------------------------------------ Gram --

constexpr int GR_TILE = 64;      // output tile (real) 64 x 64
constexpr int GR_KS = 32;        // rows per slab
constexpr int GR_LDS = GR_TILE + 4;  // smem row stride (doubles), conflict-free fragments
constexpr int GR_THREADS = 256;

// Partial real Gram of a K-range: part[split][m][n] = sum_k A[k][m0 + m] B[k][n0 + n]
// over rows k of this split.  grid = (tiles, splits[, R]): all tiles_m x
// tiles_n output tiles, or with herm (a Hermitian result, ma == nb) only the
// tiles on and above the diagonal, the fold mirroring the rest.  With
// row_off (batch), grid.z indexes the realisation whose rows
// [row_off[z], row_off[z+1]) are split evenly.
__global__ void __launch_bounds__(GR_THREADS)
k_gram(const double *__restrict__ A, int64_t lda, int ma, const double *__restrict__ B, int64_t ldb,
       int nb, int64_t K, int64_t rows_per_split, double *part, const int64_t *row_off, int herm) {
    __shared__ __align__(16) double As[GR_KS][GR_LDS];
    __shared__ __align__(16) double Bs[GR_KS][GR_LDS];
    const int tiles_n = (nb + GR_TILE - 1) / GR_TILE;
    int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
    if (herm) {                      // blockIdx.x enumerates the upper tiles row by row
        int t = blockIdx.x;
        tm = 0;
        while (t >= tiles_n - tm) {
            t -= tiles_n - tm;
            ++tm;
        }
        tn = tm + t;
    }
    const int m0 = tm * GR_TILE;
    const int n0 = tn * GR_TILE;
    int64_t k_begin, k_end;
    double *out;
    if (row_off) {
        const int64_t r0 = row_off[blockIdx.z], r1 = row_off[blockIdx.z + 1];
        const int64_t rps = ((r1 - r0 + gridDim.y - 1) / gridDim.y + GR_KS - 1) / GR_KS * GR_KS;
        k_begin = r0 + (int64_t)blockIdx.y * rps;
        k_end = min(r1, k_begin + rps);
        out = part + ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * ma * nb;
    } else {
        k_begin = (int64_t)blockIdx.y * rows_per_split;
        k_end = min(K, k_begin + rows_per_split);
        out = part + (int64_t)blockIdx.y * ma * nb;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = (warp >> 2) * 32;   // warp tile: 32 rows (4 m-tiles) x 16 cols (2 n-tiles)
    const int wn = (warp & 3) * 16;
    double acc[4][2][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    for (int64_t k0 = k_begin; k0 < k_end; k0 += GR_KS) {
        // stage 32 x 64 of A and of B (zero-filled past the edges)
        for (int e = threadIdx.x; e < GR_KS * GR_TILE; e += GR_THREADS) {
            int r = e / GR_TILE, c = e % GR_TILE;
            int64_t k = k0 + r;
            As[r][c] = (k < k_end && m0 + c < ma) ? A[k * lda + m0 + c] : 0.0;
            Bs[r][c] = (k < k_end && n0 + c < nb) ? B[k * ldb + n0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GR_KS; kk += 4) {
            const int kr = kk + (lane & 3);
            double a[4], b[2];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kr][wm + 8 * i + (lane >> 2)];
#pragma unroll
            for (int j = 0; j < 2; ++j) b[j] = Bs[kr][wn + 8 * j + (lane >> 2)];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) dmma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int m = m0 + wm + 8 * i + (lane >> 2);
                int n = n0 + wn + 8 * j + 2 * (lane & 3) + h;
                if (m < ma && n < nb) out[(int64_t)m * nb + n] = acc[i][j][h];
            }
}

// S[a][b] (complex, ld lds) = sum over splits (fixed order) of the real Gram,
// folded; grid.y = realisation in a batch (S advanced by s_stride, part by
// splits * ma * nb).  herm: an entry whose real tile lies below the diagonal
// is the conjugate of its mirror, S[a][b] = conj(S[b][a]).
__global__ void k_gram_fold(const double *part, int splits, int ma, int nb, double2 *S, int64_t lds,
                            int64_t s_stride, int herm) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int na = ma / 2, nbc = nb / 2;
    if (e >= na * nbc) return;
    part += (int64_t)blockIdx.y * splits * ma * nb;
    S += (int64_t)blockIdx.y * s_stride;
    const int a = e / nbc, b = e % nbc;
    const bool mirror = herm && (2 * a) / GR_TILE > (2 * b) / GR_TILE;
    const int r = mirror ? b : a, c = mirror ? a : b;     // the computed entry
    double g00 = 0, g11 = 0, g01 = 0, g10 = 0;
    for (int s = 0; s < splits; ++s) {
        const double *P = part + (int64_t)s * ma * nb;
        g00 += P[(int64_t)(2 * r) * nb + 2 * c];
        g11 += P[(int64_t)(2 * r + 1) * nb + 2 * c + 1];
        g01 += P[(int64_t)(2 * r) * nb + 2 * c + 1];
        g10 += P[(int64_t)(2 * r + 1) * nb + 2 * c];
    }
    const double im = g01 - g10;
    S[(int64_t)a * lds + b] = make_double2(g00 + g11, mirror ? -im : im);
}

// Output tiles a Gram launch computes: all of them, or the upper triangle.
static int gram_tiles(int ma, int nb, bool herm) {
    const int tm = (ma + GR_TILE - 1) / GR_TILE, tn = (nb + GR_TILE - 1) / GR_TILE;
    return herm ? tn * (tn + 1) / 2 : tm * tn;
}

// K-splits of a Gram: about GRAM_TARGET_CTAS CTAs in total, at least 4 slabs of
// rows per split.  Independent of the device, so the partial layout (and the
// fixed reduction order) is the same everywhere.
int gram_splits(int64_t K, int ma, int nb) {
    int tiles = ((ma + GR_TILE - 1) / GR_TILE) * ((nb + GR_TILE - 1) / GR_TILE);
    int64_t want = std::max<int64_t>(1, GRAM_TARGET_CTAS / tiles);
    int64_t max_by_rows = std::max<int64_t>(1, (K + 4 * GR_KS - 1) / (4 * GR_KS));
    return (int)std::min<int64_t>(std::min<int64_t>(want, max_by_rows), GRAM_MAX_SPLITS);
}

size_t gram_workspace(int64_t K, int na, int nbc) {
    int ma = 2 * na, nb = 2 * nbc;
    const int splits = std::max(gram_splits(K, ma, nb), gram_dw_split_cap(K, ma, nb));
    return round_up((size_t)splits * ma * nb * sizeof(double), 256);
}

void launch_gram_fold(const double *part, int splits, int ma, int nb, double2 *S, int64_t lds, bool herm,
                      cudaStream_t stream) {
    const int n = (ma / 2) * (nb / 2);
    k_gram_fold<<<(n + 255) / 256, 256, 0, stream>>>(part, std::max(splits, 1), ma, nb, S, lds, 0, herm ? 1 : 0);
}

cfd_status gram(const double2 *X, int64_t ldx, int na, const double2 *Y, int64_t ldy, int nbc, int64_t K,
                double2 *S, int64_t lds, double *work, cudaStream_t stream, bool herm) {
    int ma = 2 * na, nb = 2 * nbc;
    if (herm && ma != nb) return fail(CFD_ERR_INTERNAL, "Hermitian Gram of non-square shape");
    int splits = gram_splits(K, ma, nb);     // the workspace holds this many partials
    int64_t rps = ((K + splits - 1) / splits + GR_KS - 1) / GR_KS * GR_KS;
    splits = (int)((K + rps - 1) / rps);
    dim3 grid(gram_tiles(ma, nb, herm), std::max(splits, 1));
    k_gram<<<grid, GR_THREADS, 0, stream>>>(reinterpret_cast<const double *>(X), 2 * ldx, ma,
                                           reinterpret_cast<const double *>(Y), 2 * ldy, nb, K, rps, work, nullptr,
                                           herm ? 1 : 0);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    int n = na * nbc;
    k_gram_fold<<<(n + 255) / 256, 256, 0, stream>>>(work, std::max(splits, 1), ma, nb, S, lds, 0, herm ? 1 : 0);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

// ----------------------------------------------------------- batched Gram --

int gram_batched_splits(int R, int ma, int nb) {
    int tiles = ((ma + GR_TILE - 1) / GR_TILE) * ((nb + GR_TILE - 1) / GR_TILE);
    return std::max(1, std::min(GRAM_MAX_SPLITS, GRAM_TARGET_CTAS / (tiles * R)));
}

size_t gram_batched_workspace(int R, int na, int nbc) {
    int ma = 2 * na, nb = 2 * nbc;
    return round_up((size_t)R * gram_batched_splits(R, ma, nb) * ma * nb * sizeof(double), 256);
}

cfd_status gram_batched(const double2 *X, int64_t ldx, int na, const double2 *Y, int64_t ldy, int nbc,
                        const int64_t *row_off_dev, int R, double2 *S, int64_t lds, int64_t s_stride, double *work,
                        cudaStream_t stream, bool herm) {
    int ma = 2 * na, nb = 2 * nbc;
    if (herm && ma != nb) return fail(CFD_ERR_INTERNAL, "Hermitian Gram of non-square shape");
    int splits = gram_batched_splits(R, ma, nb);
    dim3 grid(gram_tiles(ma, nb, herm), splits, R);
    k_gram<<<grid, GR_THREADS, 0, stream>>>(reinterpret_cast<const double *>(X), 2 * ldx, ma,
                                           reinterpret_cast<const double *>(Y), 2 * ldy, nb, 0, 0, work,
                                           row_off_dev, herm ? 1 : 0);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    int n = na * nbc;
    k_gram_fold<<<dim3((n + 255) / 256, R), 256, 0, stream>>>(work, splits, ma, nb, S, lds, s_stride, herm ? 1 : 0);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

// --------------------------------------------------- in-place projection --

constexpr int PJ_ROWS = 32;      // rows of X per CTA (whole rows staged in smem)
constexpr int PJ_NT = 64;        // output columns (real) per pass
constexpr int PJ_KS = 32;        // k-slab of M
constexpr int PJ_THREADS = 256;

// Real representation of a complex n_in x n_out matrix M (ld ldm): Mr is
// 2 n_in x 2 n_out, row-major.
__global__ void k_real_rep(const double2 *M, int64_t ldm, int n_in, int n_out, double *Mr) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_in * n_out) return;
    M += (int64_t)blockIdx.y * n_in * ldm;                     // batch: one matrix per realisation
    Mr += (int64_t)blockIdx.y * (2 * n_in) * (2 * n_out);
    int a = e / n_out, b = e % n_out;
    double2 z = M[(int64_t)a * ldm + b];
    int64_t W = 2 * n_out;
    Mr[(int64_t)(2 * a) * W + 2 * b] = z.x;
    Mr[(int64_t)(2 * a) * W + 2 * b + 1] = z.y;
    Mr[(int64_t)(2 * a + 1) * W + 2 * b] = -z.y;
    Mr[(int64_t)(2 * a + 1) * W + 2 * b + 1] = z.x;
}

// X[rows, 0:2 n_out] <- X[rows, 0:2 n_in] Mr, in place: each CTA stages its
// PJ_ROWS whole rows in shared memory before writing any of them back, and
// no other CTA touches those rows.  Dynamic smem: PJ_ROWS * (2 n_in + 4) doubles
// for the rows plus a PJ_KS x (PJ_NT + 4) slab of Mr.
__global__ void __launch_bounds__(PJ_THREADS)
k_project(double *X, int64_t ldx, int kin, int nout, const double *__restrict__ Mr, int64_t n_rows,
          const int64_t *row_off, int R) {
    extern __shared__ __align__(16) double sm[];
    if (row_off) {        // batch: this panel's realisation (panels never straddle two)
        const int64_t r0 = (int64_t)blockIdx.x * PJ_ROWS;
        int lo = 0, hi = R - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) / 2;
            if (row_off[mid] <= r0) lo = mid;
            else hi = mid - 1;
        }
        Mr += (int64_t)lo * kin * nout;
    }
    const int lda = kin + 4;
    double *Xs = sm;                              // [PJ_ROWS][lda]
    double *Ms = sm + (size_t)PJ_ROWS * lda;      // [PJ_KS][PJ_NT + 4]
    const int ldm = PJ_NT + 4;
    const int64_t r0 = (int64_t)blockIdx.x * PJ_ROWS;
    for (int e = threadIdx.x; e < PJ_ROWS * kin; e += PJ_THREADS) {
        int r = e / kin, c = e % kin;
        Xs[r * lda + c] = (r0 + r < n_rows) ? X[(r0 + r) * ldx + c] : 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = (warp >> 2) * 16;     // warp tile 16 rows (2 m-tiles) x 16 cols (2 n-tiles)
    const int wn = (warp & 3) * 16;
    for (int n0 = 0; n0 < nout; n0 += PJ_NT) {
        double acc[2][2][2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
        for (int k0 = 0; k0 < kin; k0 += PJ_KS) {
            for (int e = threadIdx.x; e < PJ_KS * PJ_NT; e += PJ_THREADS) {
                int r = e / PJ_NT, c = e % PJ_NT;
                Ms[r * ldm + c] = (k0 + r < kin && n0 + c < nout) ? Mr[(int64_t)(k0 + r) * nout + n0 + c] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < PJ_KS; kk += 4) {
                const int kc = k0 + kk + (lane & 3);
                double a[2], b[2];
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    a[i] = (kc < kin) ? Xs[(wm + 8 * i + (lane >> 2)) * lda + kc] : 0.0;
#pragma unroll
                for (int j = 0; j < 2; ++j) b[j] = Ms[(kk + (lane & 3)) * ldm + wn + 8 * j + (lane >> 2)];
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) dmma(acc[i][j], a[i], b[j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    int64_t r = r0 + wm + 8 * i + (lane >> 2);
                    int c = n0 + wn + 8 * j + 2 * (lane & 3) + h;
                    if (r < n_rows && c < nout) X[r * ldx + c] = acc[i][j][h];
                }
    }
}

size_t project_workspace(int n_in, int n_out) {
    return round_up((size_t)(2 * n_in) * (2 * n_out) * sizeof(double), 256);
}

cfd_status project_inplace(double2 *X, int64_t ldx, int64_t n_rows, int n_in, const double2 *M, int64_t ldm,
                           int n_out, double *work, cudaStream_t stream) {
    if (n_out > n_in) return fail(CFD_ERR_ARG, "in-place projection cannot widen (%d -> %d)", n_in, n_out);
    int n = n_in * n_out;
    k_real_rep<<<(n + 255) / 256, 256, 0, stream>>>(M, ldm, n_in, n_out, work);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    int kin = 2 * n_in, nout = 2 * n_out;
    size_t smem = ((size_t)PJ_ROWS * (kin + 4) + (size_t)PJ_KS * (PJ_NT + 4)) * sizeof(double);
    // the limit is always the same 227 KB, so concurrent first calls may both set it
    static std::atomic<int> configured[64] = {};
    int dev = 0;
    CFD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !configured[dev].load()) {
        CFD_CUDA(cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        if (dev >= 0 && dev < 64) configured[dev].store(1);
    }
    if (smem > 227 * 1024) return fail(CFD_ERR_ARG, "block too wide for in-place projection (n=%d)", n_in);
    unsigned grid = (unsigned)((n_rows + PJ_ROWS - 1) / PJ_ROWS);
    k_project<<<grid, PJ_THREADS, smem, stream>>>(reinterpret_cast<double *>(X), 2 * ldx, kin, nout, work,
                                                  n_rows, nullptr, 0);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

// X_r <- X_r M_r for every realisation r of a batch (M: R matrices n x n,
// stride m_stride), in place.  Panel rows must not straddle realisations
// (row offsets are multiples of 32).
cfd_status project_batched(double2 *X, int64_t ldx, int64_t n_rows, int n, const double2 *M, int64_t ldm,
                           int64_t m_stride, const int64_t *row_off_dev, int R, double *work, cudaStream_t stream) {
    if (m_stride != (int64_t)n * ldm) return fail(CFD_ERR_ARG, "batched projection needs packed matrices");
    int nn = n * n;
    k_real_rep<<<dim3((nn + 255) / 256, R), 256, 0, stream>>>(M, ldm, n, n, work);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    int kin = 2 * n;
    size_t smem = ((size_t)PJ_ROWS * (kin + 4) + (size_t)PJ_KS * (PJ_NT + 4)) * sizeof(double);
    if (smem > 227 * 1024) return fail(CFD_ERR_ARG, "block too wide for in-place projection (n=%d)", n);
    CFD_CUDA(cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    unsigned grid = (unsigned)((n_rows + PJ_ROWS - 1) / PJ_ROWS);
    k_project<<<grid, PJ_THREADS, smem, stream>>>(reinterpret_cast<double *>(X), 2 * ldx, kin, kin, work, n_rows,
                                                  row_off_dev, R);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

size_t project_batched_workspace(int R, int n) { return round_up((size_t)R * (2 * n) * (2 * n) * sizeof(double), 256); }

// ------------------------------------------------------ Jacobi eigensolver --

__device__ __forceinline__ double4 ld_rot(const double4 *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldcg(q), b = __ldcg(q + 1);
    return make_double4(a.x, a.y, b.x, b.y);
}

// Round-robin (circle method) pairing: with m = n rounded up to even, round r
// pairs position i with position m - 1 - i; position 0 is fixed, the others
// rotate.  Index n (odd n) is a dummy.
__device__ __forceinline__ int rr_player(int pos, int r, int m) {
    return pos == 0 ? 0 : ((pos - 1 + r) % (m - 1)) + 1;
}

// Cyclic Jacobi for a complex Hermitian n x n matrix W (row-major, ld n,
// overwritten), eigenvectors accumulated in V (columns), one cooperative
// launch.  Each round applies n/2 disjoint rotations: the rotation for (p, q)
// with a_pq = |a_pq| e^{i phi}, tau = (a_qq - a_pp) / (2 |a_pq|),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c is
// J = [[c, s e^{i phi}], [-s e^{-i phi}, c]] on columns p, q, and A <- J^H A J
// zeroes a_pq (Golub & Van Loan's symmetric Schur rotation after a diagonal
// phase change).  Sweeps end when the off-diagonal Frobenius norm is below
// tol times the Frobenius norm, or after max_sweeps.
__global__ void k_jacobi(double2 *W, double2 *V, int n, double tol, int max_sweeps, double4 *rot,
                         double *part, int *sweeps_out) {
    cg::grid_group grid = cg::this_grid();
    const int m = n + (n & 1);
    const int npairs = m / 2;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    __shared__ double red[1024 / 32];

    for (int64_t e = tid; e < (int64_t)n * n; e += nthr) {
        int i = (int)(e / n), j = (int)(e % n);
        V[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    grid.sync();

    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        // convergence test: off^2 <= tol^2 total^2 (fixed-order reductions)
        double off = 0.0, tot = 0.0;
        for (int64_t e = tid; e < (int64_t)n * n; e += nthr) {
            double2 z = __ldcg(W + e);
            double q = z.x * z.x + z.y * z.y;
            tot += q;
            if (e / n != e % n) off += q;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        if (lane == 0) red[wid] = off;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int w = 0; w < nw; ++w) s += red[w];
            part[2 * blockIdx.x] = s;
        }
        __syncthreads();
        if (lane == 0) red[wid] = tot;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int w = 0; w < nw; ++w) s += red[w];
            part[2 * blockIdx.x + 1] = s;
        }
        grid.sync();
        double so = 0, st = 0;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            so += __ldcg(part + 2 * b);
            st += __ldcg(part + 2 * b + 1);
        }
        grid.sync();   // everyone has read part before it is rewritten
        if (so <= tol * tol * st || so == 0.0) break;

        for (int r = 0; r < m - 1; ++r) {
            // rotation parameters (c, Re s e^{i phi}, Im s e^{i phi}, t |a_pq|)
            for (int64_t k = tid; k < npairs; k += nthr) {
                int p = rr_player((int)k, r, m), q = rr_player(m - 1 - (int)k, r, m);
                if (p > q) { int tmp = p; p = q; q = tmp; }
                double4 R = make_double4(1.0, 0.0, 0.0, 0.0);
                if (q < n) {
                    double2 apq = __ldcg(W + (int64_t)p * n + q);
                    double g = sqrt(apq.x * apq.x + apq.y * apq.y);
                    double app = __ldcg(W + (int64_t)p * n + p).x, aqq = __ldcg(W + (int64_t)q * n + q).x;
                    if (g > 1e-300 * (fabs(app) + fabs(aqq)) && g > 0.0) {
                        double tau = (aqq - app) / (2.0 * g);
                        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                        R = make_double4(c, s * apq.x / g, s * apq.y / g, t * g);
                    }
                }
                rot[k] = R;
            }
            grid.sync();
            // rows p, q: a_pk <- c a_pk - s e^{i phi} a_qk, a_qk <- s e^{-i phi} a_pk + c a_qk
            for (int64_t e = tid; e < (int64_t)npairs * n; e += nthr) {
                int k = (int)(e / n), col = (int)(e % n);
                int p = rr_player(k, r, m), q = rr_player(m - 1 - k, r, m);
                if (p > q) { int tmp = p; p = q; q = tmp; }
                if (q >= n) continue;
                double4 R = ld_rot(rot + k);
                if (R.y == 0.0 && R.z == 0.0) continue;
                double2 ap = __ldcg(W + (int64_t)p * n + col), aq = __ldcg(W + (int64_t)q * n + col);
                double2 np_, nq;
                np_.x = R.x * ap.x - (R.y * aq.x - R.z * aq.y);
                np_.y = R.x * ap.y - (R.y * aq.y + R.z * aq.x);
                nq.x = (R.y * ap.x + R.z * ap.y) + R.x * aq.x;
                nq.y = (R.y * ap.y - R.z * ap.x) + R.x * aq.y;
                __stcg(W + (int64_t)p * n + col, np_);
                __stcg(W + (int64_t)q * n + col, nq);
            }
            grid.sync();
            // columns p, q of W and V: a_kp <- c a_kp - s e^{-i phi} a_kq, a_kq <- s e^{i phi} a_kp + c a_kq
            for (int64_t e = tid; e < (int64_t)npairs * n * 2; e += nthr) {
                int which = (int)(e / ((int64_t)npairs * n));
                int64_t f = e % ((int64_t)npairs * n);
                int k = (int)(f / n), row = (int)(f % n);
                int p = rr_player(k, r, m), q = rr_player(m - 1 - k, r, m);
                if (p > q) { int tmp = p; p = q; q = tmp; }
                if (q >= n) continue;
                double4 R = ld_rot(rot + k);
                if (R.y == 0.0 && R.z == 0.0) continue;
                double2 *M = which ? V : W;
                double2 ap = __ldcg(M + (int64_t)row * n + p), aq = __ldcg(M + (int64_t)row * n + q);
                double2 np_, nq;
                np_.x = R.x * ap.x - (R.y * aq.x + R.z * aq.y);
                np_.y = R.x * ap.y - (R.y * aq.y - R.z * aq.x);
                nq.x = (R.y * ap.x - R.z * ap.y) + R.x * aq.x;
                nq.y = (R.y * ap.y + R.z * ap.x) + R.x * aq.y;
                __stcg(M + (int64_t)row * n + p, np_);
                __stcg(M + (int64_t)row * n + q, nq);
            }
            grid.sync();
            // set the rotated 2x2 blocks exactly: diag a_pp - t|a_pq|, a_qq + t|a_pq|, off-diagonal 0
            for (int64_t k = tid; k < npairs; k += nthr) {
                int p = rr_player((int)k, r, m), q = rr_player(m - 1 - (int)k, r, m);
                if (p > q) { int tmp = p; p = q; q = tmp; }
                if (q >= n) continue;
                double4 R = ld_rot(rot + k);
                if (R.y == 0.0 && R.z == 0.0) continue;
                __stcg(W + (int64_t)p * n + q, make_double2(0.0, 0.0));
                __stcg(W + (int64_t)q * n + p, make_double2(0.0, 0.0));
                double2 dp = __ldcg(W + (int64_t)p * n + p), dq = __ldcg(W + (int64_t)q * n + q);
                __stcg(W + (int64_t)p * n + p, make_double2(dp.x, 0.0));
                __stcg(W + (int64_t)q * n + q, make_double2(dq.x, 0.0));
            }
            grid.sync();
        }
    }
    if (tid == 0) *sweeps_out = sweep;
}

// Eigenvalues ascending (stable by index) and the matching eigenvector columns.
__global__ void k_eig_sort(const double2 *W, const double2 *V, int n, double *evals, double2 *Q, int64_t ldq) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double li = W[(int64_t)i * n + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
        double lj = W[(int64_t)j * n + j].x;
        if (lj < li || (lj == li && j < i)) ++rank;
    }
    evals[rank] = li;
    for (int k = 0; k < n; ++k) Q[(int64_t)k * ldq + rank] = V[(int64_t)k * n + i];
}

__global__ void k_copy_sym(const double2 *A, int64_t lda, int n, double2 *W) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    int i = (int)(e / n), j = (int)(e % n);
    // Hermitian part (A + A^H) / 2
    double2 a = A[(int64_t)i * lda + j], b = A[(int64_t)j * lda + i];
    W[e] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
}

size_t eigh_workspace(int n) {
    Carve c(nullptr, 0);
    c.take<double2>((size_t)n * n);
    c.take<double2>((size_t)n * n);
    c.take<double4>((size_t)n / 2 + 1);
    c.take<double>(2 * 4096);
    c.take<int>(64);
    return round_up(c.off, 256);
}

cfd_status eigh(const double2 *A, int64_t lda, int n, double *evals, double2 *Q, int64_t ldq, void *work,
                size_t work_bytes, cudaStream_t stream, int *sweeps) {
    if (n < 1) return fail(CFD_ERR_ARG, "eigh: n < 1");
    if (work_bytes < eigh_workspace(n)) return fail(CFD_ERR_OOM, "eigh workspace too small");
    Carve c(work, work_bytes);
    double2 *W = c.take<double2>((size_t)n * n);
    double2 *V = c.take<double2>((size_t)n * n);
    double4 *rot = c.take<double4>((size_t)n / 2 + 1);
    double *part = c.take<double>(2 * 4096);
    int *sw = c.take<int>(64);
    int64_t nn = (int64_t)n * n;
    k_copy_sym<<<(unsigned)((nn + 255) / 256), 256, 0, stream>>>(A, lda, n, W);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    // grid: one CTA for small problems, more for large (all co-resident)
    const int threads = 512;
    int per_sm = 0;
    CFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, threads, 0));
    int want = n <= 64 ? 1 : std::min<int>(sm_count(), (int)((nn / 2 + threads - 1) / threads));
    int blocks = std::max(1, std::min(want, per_sm * sm_count()));
    blocks = std::min(blocks, 4096);
    double tol = 2.220446049250313e-16 * std::max(n, 4);   // off-diagonal Frobenius <= n eps |A|_F
    int max_sweeps = 40;
    void *args[] = {&W, &V, &n, &tol, &max_sweeps, &rot, &part, &sw};
    CFD_CUDA(cudaLaunchCooperativeKernel((void *)k_jacobi, dim3(blocks), dim3(threads), args, 0, stream));
    CFD_COUNT_LAUNCH();
    k_eig_sort<<<(n + 127) / 128, 128, 0, stream>>>(W, V, n, evals, Q, ldq);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    if (sweeps) CFD_CUDA(cudaMemcpyAsync(sweeps, sw, sizeof(int), cudaMemcpyDeviceToHost, stream));
    return CFD_OK;
}

// ------------------------------------------------- batched small Jacobi --

// One CTA per problem: cyclic Jacobi (same rotations as k_jacobi) on a
// complex Hermitian n x n matrix (n <= 64) held with its eigenvectors in
// shared memory.  Problem b reads the Hermitian part of A + b a_stride and
// writes ascending eigenvalues to evals + b n and eigenvectors (columns) to
// Q + b q_stride.
__global__ void __launch_bounds__(256)
k_jacobi_blocks(const double2 *A, int64_t lda, int64_t a_stride, int n, double tol, int max_sweeps,
                double *evals, double2 *Q, int64_t ldq, int64_t q_stride, int *sweeps_out) {
    extern __shared__ __align__(16) double2 shj[];
    double2 *W = shj, *V = shj + n * n;
    __shared__ double4 rot[DENSE_BATCH_MAX_N / 2 + 1];
    __shared__ double red[2][256 / 32];
    __shared__ int done;
    const int m = n + (n & 1), npairs = m / 2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    A += (int64_t)blockIdx.x * a_stride;
    for (int e = tid; e < n * n; e += nthr) {
        int i = e / n, j = e % n;
        double2 a = A[(int64_t)i * lda + j], b = A[(int64_t)j * lda + i];
        W[e] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        V[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < n * n; e += nthr) {
            double q = W[e].x * W[e].x + W[e].y * W[e].y;
            tot += q;
            if (e / n != e % n) off += q;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = off;
            red[1][tid >> 5] = tot;
        }
        __syncthreads();
        if (tid == 0) {
            double so = 0, st = 0;
            for (int w = 0; w < (nthr >> 5); ++w) {
                so += red[0][w];
                st += red[1][w];
            }
            done = (so <= tol * tol * st || so == 0.0);
        }
        __syncthreads();
        if (done) break;
        for (int r = 0; r < m - 1; ++r) {
            for (int k = tid; k < npairs; k += nthr) {
                int p = rr_player(k, r, m), q = rr_player(m - 1 - k, r, m);
                if (p > q) { int t2 = p; p = q; q = t2; }
                double4 R = make_double4(1.0, 0.0, 0.0, 0.0);
                if (q < n) {
                    double2 apq = W[p * n + q];
                    double g = sqrt(apq.x * apq.x + apq.y * apq.y);
                    double app = W[p * n + p].x, aqq = W[q * n + q].x;
                    if (g > 0.0) {
                        double tau = (aqq - app) / (2.0 * g);
                        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                        R = make_double4(c, sn * apq.x / g, sn * apq.y / g, t * g);
                    }
                }
                rot[k] = R;
            }
            __syncthreads();
            for (int e = tid; e < npairs * n; e += nthr) {          // rows p, q
                int k = e / n, col = e % n;
                int p = rr_player(k, r, m), q = rr_player(m - 1 - k, r, m);
                if (p > q) { int t2 = p; p = q; q = t2; }
                if (q >= n) continue;
                double4 R = rot[k];
                if (R.y == 0.0 && R.z == 0.0) continue;
                double2 ap = W[p * n + col], aq = W[q * n + col];
                W[p * n + col] = make_double2(R.x * ap.x - (R.y * aq.x - R.z * aq.y),
                                              R.x * ap.y - (R.y * aq.y + R.z * aq.x));
                W[q * n + col] = make_double2((R.y * ap.x + R.z * ap.y) + R.x * aq.x,
                                              (R.y * ap.y - R.z * ap.x) + R.x * aq.y);
            }
            __syncthreads();
            for (int e = tid; e < 2 * npairs * n; e += nthr) {      // columns p, q of W and V
                int which = e / (npairs * n), f = e % (npairs * n);
                int k = f / n, row = f % n;
                int p = rr_player(k, r, m), q = rr_player(m - 1 - k, r, m);
                if (p > q) { int t2 = p; p = q; q = t2; }
                if (q >= n) continue;
                double4 R = rot[k];
                if (R.y == 0.0 && R.z == 0.0) continue;
                double2 *M = which ? V : W;
                double2 ap = M[row * n + p], aq = M[row * n + q];
                M[row * n + p] = make_double2(R.x * ap.x - (R.y * aq.x + R.z * aq.y),
                                              R.x * ap.y - (R.y * aq.y - R.z * aq.x));
                M[row * n + q] = make_double2((R.y * ap.x - R.z * ap.y) + R.x * aq.x,
                                              (R.y * ap.y + R.z * ap.x) + R.x * aq.y);
            }
            __syncthreads();
            for (int k = tid; k < npairs; k += nthr) {               // exact 2x2 blocks
                int p = rr_player(k, r, m), q = rr_player(m - 1 - k, r, m);
                if (p > q) { int t2 = p; p = q; q = t2; }
                if (q >= n) continue;
                double4 R = rot[k];
                if (R.y == 0.0 && R.z == 0.0) continue;
                W[p * n + q] = make_double2(0.0, 0.0);
                W[q * n + p] = make_double2(0.0, 0.0);
                W[p * n + p].y = 0.0;
                W[q * n + q].y = 0.0;
            }
            __syncthreads();
        }
    }
    // ascending eigenvalues (stable by index) and their eigenvectors
    evals += (int64_t)blockIdx.x * n;
    Q += (int64_t)blockIdx.x * q_stride;
    for (int i = tid; i < n; i += nthr) {
        double li = W[i * n + i].x;
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            double lj = W[j * n + j].x;
            if (lj < li || (lj == li && j < i)) ++rank;
        }
        evals[rank] = li;
        for (int k = 0; k < n; ++k) Q[(int64_t)k * ldq + rank] = V[k * n + i];
    }
    if (tid == 0 && sweeps_out) sweeps_out[blockIdx.x] = sweep;
}

cfd_status eigh_batched(const double2 *A, int64_t lda, int64_t a_stride, int n, int R, double *evals, double2 *Q,
                        int64_t ldq, int64_t q_stride, cudaStream_t stream) {
    if (n < 1 || n > DENSE_BATCH_MAX_N) return fail(CFD_ERR_ARG, "batched eigensolver needs 1 <= n <= %d", DENSE_BATCH_MAX_N);
    size_t smem = (size_t)2 * n * n * sizeof(double2);
    CFD_CUDA(cudaFuncSetAttribute(k_jacobi_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    double tol = 2.220446049250313e-16 * std::max(n, 4);
    k_jacobi_blocks<<<R, 256, smem, stream>>>(A, lda, a_stride, n, tol, 40, evals, Q, ldq, q_stride, nullptr);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

// ----------------------------------------------------------- residuals --

constexpr int RS_THREADS = 256;

// part[cta][j] = sum over this CTA's rows of |Z_ij - theta_j X_ij|^2 (theta
// nullable: plain column norms of Z).
__global__ void __launch_bounds__(RS_THREADS)
k_resid_part(const double2 *Z, int64_t ldz, const double2 *X, int64_t ldx, const double *theta, int n,
             int64_t n_rows, int64_t rows_per_cta, double *part, const int64_t *row_off) {
    int64_t r0, r1;
    if (row_off) {        // batch: grid.y = realisation, its rows split over grid.x CTAs
        const int64_t a = row_off[blockIdx.y], e = row_off[blockIdx.y + 1];
        const int64_t rpc = (e - a + gridDim.x - 1) / gridDim.x;
        r0 = a + (int64_t)blockIdx.x * rpc;
        r1 = min(e, r0 + rpc);
        theta += (int64_t)blockIdx.y * n;
        part += (int64_t)blockIdx.y * gridDim.x * n;
    } else {
        r0 = (int64_t)blockIdx.x * rows_per_cta;
        r1 = min(n_rows, r0 + rows_per_cta);
    }
    __shared__ double red[RS_THREADS];
    for (int j0 = 0; j0 < n; j0 += 32) {
        const int j = j0 + (threadIdx.x & 31);
        const int rl = threadIdx.x >> 5;          // 8 row lanes
        double s = 0.0;
        if (j < n) {
            double th = theta ? theta[j] : 0.0;
            for (int64_t r = r0 + rl; r < r1; r += RS_THREADS / 32) {
                double2 z = Z[r * ldz + j];
                double2 x = X ? X[r * ldx + j] : make_double2(0.0, 0.0);
                double dx = z.x - th * x.x, dy = z.y - th * x.y;
                s += dx * dx + dy * dy;
            }
        }
        red[threadIdx.x] = s;
        __syncthreads();
        if (threadIdx.x < 32 && j < n) {
            double t = 0.0;
            for (int q = 0; q < RS_THREADS / 32; ++q) t += red[q * 32 + threadIdx.x];
            part[(int64_t)blockIdx.x * n + j] = t;
        }
        __syncthreads();
    }
}

__global__ void k_resid_fold(const double *part, int ctas, int n, double *out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    part += (int64_t)blockIdx.y * ctas * n;                  // batch: one fold per realisation
    out += (int64_t)blockIdx.y * n;
    double s = 0.0;
    for (int b = 0; b < ctas; ++b) s += part[(int64_t)b * n + j];
    out[j] = sqrt(s);
}

size_t resid_workspace(int n) { return round_up((size_t)RESID_MAX_CTAS * n * sizeof(double), 256); }

cfd_status resid_norms(const double2 *Z, int64_t ldz, const double2 *X, int64_t ldx, const double *theta, int n,
                       int64_t n_rows, double *out, double *work, cudaStream_t stream) {
    int64_t ctas = std::min<int64_t>(RESID_MAX_CTAS, std::max<int64_t>(1, (n_rows + 255) / 256));
    ctas = std::min<int64_t>(ctas, 4LL * sm_count());
    int64_t rpc = (n_rows + ctas - 1) / ctas;
    ctas = (n_rows + rpc - 1) / rpc;
    k_resid_part<<<(unsigned)ctas, RS_THREADS, 0, stream>>>(Z, ldz, X, ldx, theta, n, n_rows, rpc, work, nullptr);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    k_resid_fold<<<(n + 127) / 128, 128, 0, stream>>>(work, (int)ctas, n, out);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

cfd_status resid_norms_batched(const double2 *Z, int64_t ldz, const double2 *X, int64_t ldx, const double *theta,
                               int n, const int64_t *row_off_dev, int R, double *out, double *work,
                               cudaStream_t stream) {
    const int per = 8;     // CTAs per realisation
    k_resid_part<<<dim3(per, R), RS_THREADS, 0, stream>>>(Z, ldz, X, ldx, theta, n, 0, 0, work, row_off_dev);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    k_resid_fold<<<dim3((n + 127) / 128, R), 128, 0, stream>>>(work, per, n, out);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

size_t resid_batched_workspace(int R, int n) { return round_up((size_t)R * 8 * n * sizeof(double), 256); }

}  // namespace cfd
