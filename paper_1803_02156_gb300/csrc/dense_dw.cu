// Gram matrices and in-place projections of tall complex-double blocks in
// double-word arithmetic on the fp32 pipe.
//
// GB300 runs fp64 at 1/64 of the fp32 rate: its FP64 tensor cores (the DMMA
// kernels of dense.cu) reach about 1.1 TFLOP/s, which makes the Gram
// matrices and projections of orthogonalisation and Rayleigh-Ritz the
// larger part of a mixed-precision solve.  Here the same real-embedded
// products (dense.cu's header) run with every double split once into
// hi + lo floats and every multiply-add as a double-word multiply-add
// (dw_arith.cuh: Dekker's TwoProduct by FMA plus the cross terms, Knuth's
// TwoSum, the errors collected in a second float and folded back into the
// sum after every slab of rows), two output columns per packed fp32x2
// instruction.  A real multiply-add costs 12 fp32 operations,
// so the fp32 pipe gives about 3 TFLOP/s of fp64-equivalent work; each
// product and sum is accurate to a few units of 2^-48 of its terms (2^-53
// natively).  The Gram's partials and the fold are those of dense.cu (the
// same layout, split order and fp64 fold), so only the arithmetic inside a
// split differs.
#include <algorithm>
#include <atomic>

#include "dense.cuh"
#include "dw_arith.cuh"

namespace cfd {

namespace {

constexpr int GD_TM = 64;           // output tile (real) 64 rows x 128 columns
constexpr int GD_TN = 128;
constexpr int GD_KS = 16;           // rows per slab
constexpr int GD_THREADS = 256;
constexpr int GD_TARGET_CTAS = 304; // two waves of one CTA per SM on a 152-SM GB300

constexpr int PD_ROWS = 32;         // rows per CTA of the projection
constexpr int PD_NT = 128;          // output columns per pass
constexpr int PD_KS = 32;           // k-slab of M
constexpr int PD_THREADS = 256;

// x = hi + lo: hi = fl32(x), lo = fl32(x - hi) (x - hi is exact in fp64).
__device__ __forceinline__ void split_dw(double x, float &hi, float &lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
}

}  // namespace

// Partial real Gram of a K-range in double-word arithmetic: part[split][m][n]
// = sum_k A[k][m0 + m] B[k][n0 + n] over the split's rows, rounded to fp64
// once.  grid = (tiles, splits) over all 64 x 128 output tiles; with herm a
// tile wholly below the diagonal returns at once (the fold mirrors those
// entries).  A thread owns rows ty 4 + i (i < 4) and the column pairs
// {tx 4, tx 4 + 2, 64 + tx 4, 64 + tx 4 + 2} of the tile, so a warp's
// 16-byte shared loads are contiguous or broadcast.
__global__ void __launch_bounds__(GD_THREADS, 1)
k_gram_dw(const double *__restrict__ A, int64_t lda, int ma, const double *__restrict__ B, int64_t ldb, int nb,
          int64_t K, int64_t rows_per_split, double *part, int herm) {
    __shared__ __align__(16) float Ah[GD_KS][GD_TM + 4], Al[GD_KS][GD_TM + 4];
    __shared__ __align__(16) float Bh[GD_KS][GD_TN + 4], Bl[GD_KS][GD_TN + 4];
    const int tiles_n = (nb + GD_TN - 1) / GD_TN;
    const int m0 = (blockIdx.x / tiles_n) * GD_TM, n0 = (blockIdx.x % tiles_n) * GD_TN;
    if (herm && m0 >= n0 + GD_TN) return;
    const int64_t k_begin = (int64_t)blockIdx.y * rows_per_split;
    const int64_t k_end = min(K, k_begin + rows_per_split);
    double *out = part + (int64_t)blockIdx.y * ma * nb;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    float2 s2[4][4], e2[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) s2[i][j] = e2[i][j] = make_float2(0.f, 0.f);

    // the next slab's values are loaded into registers while the current
    // slab is computed, then split into shared memory
    constexpr int PA = GD_KS * GD_TM / GD_THREADS, PB = GD_KS * GD_TN / GD_THREADS;
    double pa[PA], pb[PB];
    auto load = [&](int64_t k0) {
#pragma unroll
        for (int t = 0; t < PA; ++t) {
            const int e = threadIdx.x + t * GD_THREADS, r = e / GD_TM, c = e % GD_TM;
            const int64_t k = k0 + r;
            pa[t] = (k < k_end && m0 + c < ma) ? A[k * lda + m0 + c] : 0.0;
        }
#pragma unroll
        for (int t = 0; t < PB; ++t) {
            const int e = threadIdx.x + t * GD_THREADS, r = e / GD_TN, c = e % GD_TN;
            const int64_t k = k0 + r;
            pb[t] = (k < k_end && n0 + c < nb) ? B[k * ldb + n0 + c] : 0.0;
        }
    };
    if (k_begin < k_end) load(k_begin);
    for (int64_t k0 = k_begin; k0 < k_end; k0 += GD_KS) {
#pragma unroll
        for (int t = 0; t < PA; ++t) {
            const int e = threadIdx.x + t * GD_THREADS;
            split_dw(pa[t], Ah[e / GD_TM][e % GD_TM], Al[e / GD_TM][e % GD_TM]);
        }
#pragma unroll
        for (int t = 0; t < PB; ++t) {
            const int e = threadIdx.x + t * GD_THREADS;
            split_dw(pb[t], Bh[e / GD_TN][e % GD_TN], Bl[e / GD_TN][e % GD_TN]);
        }
        __syncthreads();
        if (k0 + GD_KS < k_end) load(k0 + GD_KS);
#pragma unroll 2
        for (int kk = 0; kk < GD_KS; ++kk) {
            const float4 x = *reinterpret_cast<const float4 *>(&Ah[kk][4 * ty]);
            const float4 y = *reinterpret_cast<const float4 *>(&Al[kk][4 * ty]);
            const float ah[4] = {x.x, x.y, x.z, x.w};
            const float al[4] = {y.x, y.y, y.z, y.w};
            float2 bh[4], bl[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 u = *reinterpret_cast<const float4 *>(&Bh[kk][64 * h + 4 * tx]);
                const float4 v = *reinterpret_cast<const float4 *>(&Bl[kk][64 * h + 4 * tx]);
                bh[2 * h + 0] = make_float2(u.x, u.y);
                bh[2 * h + 1] = make_float2(u.z, u.w);
                bl[2 * h + 0] = make_float2(v.x, v.y);
                bl[2 * h + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 hh = bcast2(ah[i]), nhh = bcast2(-ah[i]), nhl = bcast2(-al[i]);
#pragma unroll
                for (int j = 0; j < 4; ++j) dw_mac2(s2[i][j], e2[i][j], hh, nhh, nhl, bh[j], bl[j]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) renorm2(s2[i][j], e2[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + 4 * ty + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + 64 * (j / 2) + 4 * tx + 2 * (j % 2);
            if (m < ma && n < nb) out[(int64_t)m * nb + n] = (double)s2[i][j].x + (double)e2[i][j].x;
            if (m < ma && n + 1 < nb) out[(int64_t)m * nb + n + 1] = (double)s2[i][j].y + (double)e2[i][j].y;
        }
    }
}

// Real representation Mr (2 n_in x 2 n_out, row-major, see dense.cu) of a
// complex matrix M, split into hi and lo float arrays.
__global__ void k_real_rep_dw(const double2 *M, int64_t ldm, int n_in, int n_out, float *Mh, float *Ml) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_in * n_out) return;
    const int a = e / n_out, b = e % n_out;
    const double2 z = M[(int64_t)a * ldm + b];
    const int64_t W = 2 * n_out;
    float rh, rl, ih, il;
    split_dw(z.x, rh, rl);
    split_dw(z.y, ih, il);
    Mh[(int64_t)(2 * a) * W + 2 * b] = rh;
    Ml[(int64_t)(2 * a) * W + 2 * b] = rl;
    Mh[(int64_t)(2 * a) * W + 2 * b + 1] = ih;
    Ml[(int64_t)(2 * a) * W + 2 * b + 1] = il;
    Mh[(int64_t)(2 * a + 1) * W + 2 * b] = -ih;
    Ml[(int64_t)(2 * a + 1) * W + 2 * b] = -il;
    Mh[(int64_t)(2 * a + 1) * W + 2 * b + 1] = rh;
    Ml[(int64_t)(2 * a + 1) * W + 2 * b + 1] = rl;
}

// X[rows, 0:nout] <- X[rows, 0:kin] Mr in double-word arithmetic, in place:
// each CTA splits its PD_ROWS whole rows into shared memory (transposed,
// hi and lo) before writing any of them back, and no other CTA touches
// those rows.  A thread owns rows ty 4 + i (i < 4) and the column pairs
// {2 tx, 64 + 2 tx} of each PD_NT-wide pass.  Dynamic smem: the rows,
// 2 kin x (PD_ROWS + 4) floats, plus a 2 x PD_KS x (PD_NT + 4) slab of Mr.
__global__ void __launch_bounds__(PD_THREADS, 1)
k_project_dw(double *X, int64_t ldx, int kin, int nout, const float *__restrict__ Mh, const float *__restrict__ Ml,
             int64_t n_rows) {
    extern __shared__ __align__(16) float smd[];
    constexpr int LR = PD_ROWS + 4;
    constexpr int LM = PD_NT + 4;
    float *XhT = smd;                              // [kin][LR]
    float *XlT = smd + (size_t)kin * LR;
    float *Msh = smd + 2 * (size_t)kin * LR;       // [PD_KS][LM]
    float *Msl = Msh + PD_KS * LM;
    const int64_t r0 = (int64_t)blockIdx.x * PD_ROWS;
    for (int e = threadIdx.x; e < PD_ROWS * kin; e += PD_THREADS) {
        const int r = e / kin, c = e % kin;
        const double x = (r0 + r < n_rows) ? X[(r0 + r) * ldx + c] : 0.0;
        split_dw(x, XhT[c * LR + r], XlT[c * LR + r]);
    }
    __syncthreads();
    const int ty = threadIdx.x / 32, tx = threadIdx.x % 32;
    for (int n0 = 0; n0 < nout; n0 += PD_NT) {
        float2 s2[4][2], e2[4][2];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) s2[i][j] = e2[i][j] = make_float2(0.f, 0.f);
        for (int k0 = 0; k0 < kin; k0 += PD_KS) {
            for (int e = threadIdx.x; e < PD_KS * PD_NT; e += PD_THREADS) {
                const int r = e / PD_NT, c = e % PD_NT;
                const bool in = k0 + r < kin && n0 + c < nout;
                Msh[r * LM + c] = in ? Mh[(int64_t)(k0 + r) * nout + n0 + c] : 0.f;
                Msl[r * LM + c] = in ? Ml[(int64_t)(k0 + r) * nout + n0 + c] : 0.f;
            }
            __syncthreads();
            const int kmax = min(PD_KS, kin - k0);
#pragma unroll 4
            for (int kk = 0; kk < kmax; ++kk) {
                const int k = k0 + kk;
                const float4 xh = *reinterpret_cast<const float4 *>(&XhT[k * LR + 4 * ty]);
                const float4 xl = *reinterpret_cast<const float4 *>(&XlT[k * LR + 4 * ty]);
                const float ah[4] = {xh.x, xh.y, xh.z, xh.w};
                const float al[4] = {xl.x, xl.y, xl.z, xl.w};
                float2 bh[2], bl[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    bh[j] = *reinterpret_cast<const float2 *>(&Msh[kk * LM + 64 * j + 2 * tx]);
                    bl[j] = *reinterpret_cast<const float2 *>(&Msl[kk * LM + 64 * j + 2 * tx]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 hh = bcast2(ah[i]), nhh = bcast2(-ah[i]), nhl = bcast2(-al[i]);
#pragma unroll
                    for (int j = 0; j < 2; ++j) dw_mac2(s2[i][j], e2[i][j], hh, nhh, nhl, bh[j], bl[j]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) renorm2(s2[i][j], e2[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t r = r0 + 4 * ty + i;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int c = n0 + 64 * j + 2 * tx;
                if (r < n_rows && c < nout) X[r * ldx + c] = (double)s2[i][j].x + (double)e2[i][j].x;
                if (r < n_rows && c + 1 < nout) X[r * ldx + c + 1] = (double)s2[i][j].y + (double)e2[i][j].y;
            }
        }
    }
}

// ---------------------------------------------------------------- launch --

// Output tiles of a launch, and those that compute (herm: not wholly below
// the diagonal).
static int gram_dw_tiles(int ma, int nb) {
    return ((ma + GD_TM - 1) / GD_TM) * ((nb + GD_TN - 1) / GD_TN);
}

static int gram_dw_busy_tiles(int ma, int nb, bool herm) {
    int t = 0;
    for (int m0 = 0; m0 < ma; m0 += GD_TM)
        for (int n0 = 0; n0 < nb; n0 += GD_TN) t += (!herm || m0 < n0 + GD_TN) ? 1 : 0;
    return std::max(t, 1);
}

int gram_dw_split_cap(int64_t K, int ma, int nb) {
    const int64_t max_by_rows = std::max<int64_t>(1, (K + 4 * GD_KS - 1) / (4 * GD_KS));
    const int64_t most = std::max(1, GD_TARGET_CTAS / gram_dw_busy_tiles(ma, nb, ma == nb));
    return (int)std::min<int64_t>(most, max_by_rows);
}

// K-splits of a double-word Gram: about one wave of CTAs, at least 4 slabs
// of rows per split, never more partials than the Gram workspace holds.
// Independent of the device, so the split order is the same everywhere.
static int gram_dw_splits(int64_t K, int ma, int nb, bool herm) {
    const int64_t want = std::max(1, GD_TARGET_CTAS / gram_dw_busy_tiles(ma, nb, herm));
    const int64_t max_by_rows = std::max<int64_t>(1, (K + 4 * GD_KS - 1) / (4 * GD_KS));
    return (int)std::min<int64_t>({want, max_by_rows, (int64_t)gram_dw_split_cap(K, ma, nb)});
}

cfd_status gram_dw(const double2 *X, int64_t ldx, int na, const double2 *Y, int64_t ldy, int nbc, int64_t K,
                   double2 *S, int64_t lds, double *work, cudaStream_t stream, bool herm) {
    const int ma = 2 * na, nb = 2 * nbc;
    if (herm && ma != nb) return fail(CFD_ERR_INTERNAL, "Hermitian Gram of non-square shape");
    int splits = gram_dw_splits(K, ma, nb, herm);
    const int64_t rps = ((K + splits - 1) / splits + GD_KS - 1) / GD_KS * GD_KS;
    splits = (int)std::max<int64_t>(1, (K + rps - 1) / rps);
    dim3 grid(gram_dw_tiles(ma, nb), splits);
    k_gram_dw<<<grid, GD_THREADS, 0, stream>>>(reinterpret_cast<const double *>(X), 2 * ldx, ma,
                                              reinterpret_cast<const double *>(Y), 2 * ldy, nb, K, rps, work,
                                              herm ? 1 : 0);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    launch_gram_fold(work, splits, ma, nb, S, lds, herm, stream);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

cfd_status project_inplace_dw(double2 *X, int64_t ldx, int64_t n_rows, int n_in, const double2 *M, int64_t ldm,
                              int n_out, double *work, cudaStream_t stream) {
    if (n_out > n_in) return fail(CFD_ERR_ARG, "in-place projection cannot widen (%d -> %d)", n_in, n_out);
    const int kin = 2 * n_in, nout = 2 * n_out;
    float *Mh = reinterpret_cast<float *>(work);
    float *Ml = Mh + (size_t)kin * nout;
    const int n = n_in * n_out;
    k_real_rep_dw<<<(n + 255) / 256, 256, 0, stream>>>(M, ldm, n_in, n_out, Mh, Ml);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    const size_t smem = (2 * (size_t)kin * (PD_ROWS + 4) + 2 * (size_t)PD_KS * (PD_NT + 4)) * sizeof(float);
    if (smem > 227 * 1024) return fail(CFD_ERR_ARG, "block too wide for in-place projection (n=%d)", n_in);
    static std::atomic<int> configured[64] = {};
    int dev = 0;
    CFD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !configured[dev].load()) {
        CFD_CUDA(cudaFuncSetAttribute(k_project_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        if (dev >= 0 && dev < 64) configured[dev].store(1);
    }
    const unsigned grid = (unsigned)((n_rows + PD_ROWS - 1) / PD_ROWS);
    k_project_dw<<<grid, PD_THREADS, smem, stream>>>(reinterpret_cast<double *>(X), 2 * ldx, kin, nout, Mh, Ml,
                                                     n_rows);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

}  // namespace cfd
