/*
 * ChebFD oracle, plain C part.  TEST INFRASTRUCTURE ONLY: nothing in the
 * library path may call it; tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm are its only users.
 *
 * Plain, slow, obviously correct CPU code in fp64.  It shares no code with the
 * CUDA library.  Built with -O2 -ffp-contract=off so every product and sum is
 * rounded exactly as written.
 *
 * Contents
 *   - counter-based SplitMix64 (Steele, Lea, Flood, "Fast splittable
 *     pseudorandom number generators", OOPSLA 2014) for the on-site disorder;
 *   - the topological-insulator Hamiltonian of Sect. 2.1 ("Topi-Nx-Ny-Nz",
 *     n = 4 Nx Ny Nz, 13 nonzeros per interior row) as canonical CSR;
 *   - CSR SpMMV on row-major block vectors (Sect. 3.1);
 *   - the ChebFD polynomial filter of Algorithm 1, applied block by block as
 *     in Algorithm 2, with the Chebyshev moment dot products of Algorithm 1.
 *
 * Complex numbers are stored as interleaved (re, im) doubles.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ RNG -- */

/* SplitMix64 output function (mix64 variant 13 of Stafford, as published with
 * SplitMix64). */
static uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

/* Draw number i (0-based) of the SplitMix64 stream whose initial state is
 * key(seed, tag) = mix(seed + GAMMA * (2 tag + 1)).  SplitMix64 advances its
 * state by GAMMA before each output, so draw i is mix(key + (i + 1) GAMMA). */
uint64_t orc_splitmix64(uint64_t seed, uint64_t tag, uint64_t i)
{
    uint64_t key = sm64_mix(seed + SM64_GAMMA * (2 * tag + 1));
    return sm64_mix(key + (i + 1) * SM64_GAMMA);
}

/* Uniform double in [0, 1) from the top 53 bits. */
double orc_uniform(uint64_t seed, uint64_t tag, uint64_t i)
{
    return (double)(orc_splitmix64(seed, tag, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------- Topi matrix ----- */

/* Site index of lattice point (x, y, z): x fastest. */
static int64_t site_of(int64_t x, int64_t y, int64_t z, int64_t Nx, int64_t Ny)
{
    return x + Nx * (y + Ny * z);
}

/* Number of stored nonzeros of Topi-Nx-Ny-Nz. */
int64_t orc_topi_nnz(int Nx, int Ny, int Nz, const int *periodic)
{
    int64_t n = 0;
    int L[3] = {Nx, Ny, Nz};
    for (int64_t z = 0; z < Nz; ++z)
        for (int64_t y = 0; y < Ny; ++y)
            for (int64_t x = 0; x < Nx; ++x) {
                int64_t c[3] = {x, y, z};
                int64_t per_orb = 1; /* on-site */
                for (int j = 0; j < 3; ++j) {
                    int has_back = periodic[j] || c[j] > 0;
                    int has_fwd = periodic[j] || c[j] < L[j] - 1;
                    per_orb += 2 * has_back + 2 * has_fwd;
                }
                n += 4 * per_orb;
            }
    return n;
}

/*
 * Gamma matrices of the model: Gamma_1 = sz (x) 1, Gamma_{2,3,4} = sx (x)
 * sx, sy, sz, with the 4x4 index of s_a (x) s_b entry [(a1,b1),(a2,b2)] equal
 * to 2 a1 + b1 (row) and 2 a2 + b2 (column).
 * pauli(k, r, c) gives entry (r, c) of s_k, k = 0 (identity), 1 (x), 2 (y),
 * 3 (z), as a complex number.
 */
static void pauli(int k, int r, int c, double *re, double *im)
{
    *re = 0.0;
    *im = 0.0;
    if (k == 0) {
        if (r == c) *re = 1.0;
    } else if (k == 1) {
        if (r != c) *re = 1.0;
    } else if (k == 2) {
        if (r == 0 && c == 1) *im = -1.0;
        if (r == 1 && c == 0) *im = 1.0;
    } else {
        if (r == c) *re = (r == 0) ? 1.0 : -1.0;
    }
}

/* Entry (r, c) of s_a (x) s_b. */
static void kron_entry(int a, int b, int r, int c, double *re, double *im)
{
    double ar, ai, br, bi;
    pauli(a, r / 2, c / 2, &ar, &ai);
    pauli(b, r % 2, c % 2, &br, &bi);
    *re = ar * br - ai * bi;
    *im = ar * bi + ai * br;
}

/* Hop block T_j = -(t/2) Gamma_1 + i (t/2) Gamma_{j+2}, entry (r, c);
 * axis j = 0 (x), 1 (y), 2 (z).  Gamma_{j+2} = s_x (x) s_{j+1}. */
static void hop_entry(int j, double t, int r, int c, double *re, double *im)
{
    double g1r, g1i, gjr, gji;
    kron_entry(3, 0, r, c, &g1r, &g1i);
    kron_entry(1, j + 1, r, c, &gjr, &gji);
    double h = t / 2.0;
    /* -(h) g1 + i h gj  ;  i (gjr + i gji) = -gji + i gjr */
    *re = -h * g1r + h * (-gji);
    *im = -h * g1i + h * gjr;
}

typedef struct {
    int64_t col;
    double re, im;
} entry_t;

/* Stored values carry no negative zeros: -0.0 becomes +0.0. */
static double no_neg_zero(double v)
{
    return v == 0.0 ? 0.0 : v;
}

static int cmp_entry(const void *a, const void *b)
{
    int64_t x = ((const entry_t *)a)->col, y = ((const entry_t *)b)->col;
    return (x > y) - (x < y);
}

/*
 * Build Topi-Nx-Ny-Nz as CSR: rows 4 site + orbital, columns ascending.
 *   on-site block (m + V_s) Gamma_1, V_s = gamma (u_s - 1/2), u_s uniform from
 *     SplitMix64(seed, tag 0, s);
 *   block (site + e_j, site) = T_j and block (site, site + e_j) = T_j^H.
 * rowptr has N + 1 entries; col and val (interleaved re, im) nnz entries.
 * Returns 0, or -1 when a periodic axis is shorter than 3 sites (its two
 * neighbours would coincide) or an axis is empty.
 */
int orc_topi_csr(int Nx, int Ny, int Nz, const int *periodic, double t, double m,
                 double gamma, uint64_t seed, int64_t *rowptr, int32_t *col, double *val)
{
    int L[3] = {Nx, Ny, Nz};
    for (int j = 0; j < 3; ++j) {
        if (L[j] < 1) return -1;
        if (periodic[j] && L[j] < 3) return -1;
    }
    int64_t pos = 0;
    rowptr[0] = 0;
    for (int64_t z = 0; z < Nz; ++z)
        for (int64_t y = 0; y < Ny; ++y)
            for (int64_t x = 0; x < Nx; ++x) {
                int64_t s = site_of(x, y, z, Nx, Ny);
                int64_t c[3] = {x, y, z};
                double u = orc_uniform(seed, 0, (uint64_t)s);
                double V = gamma * (u - 0.5);
                double onsite = m + V;
                for (int o = 0; o < 4; ++o) {
                    entry_t e[13];
                    int ne = 0;
                    double g1r, g1i;
                    kron_entry(3, 0, o, o, &g1r, &g1i);
                    e[ne].col = 4 * s + o;
                    e[ne].re = no_neg_zero(onsite * g1r);
                    e[ne].im = 0.0;
                    ++ne;
                    for (int j = 0; j < 3; ++j) {
                        /* backward neighbour s - e_j: row s is "site + e_j" of
                         * that site, so the block is T_j. */
                        if (periodic[j] || c[j] > 0) {
                            int64_t cb[3] = {c[0], c[1], c[2]};
                            cb[j] = (c[j] - 1 + L[j]) % L[j];
                            int64_t sb = site_of(cb[0], cb[1], cb[2], Nx, Ny);
                            for (int o2 = 0; o2 < 4; ++o2) {
                                double hr, hi;
                                hop_entry(j, t, o, o2, &hr, &hi);
                                if (hr != 0.0 || hi != 0.0) {
                                    e[ne].col = 4 * sb + o2;
                                    e[ne].re = no_neg_zero(hr);
                                    e[ne].im = no_neg_zero(hi);
                                    ++ne;
                                }
                            }
                        }
                        /* forward neighbour s + e_j: block T_j^H, whose entry
                         * (o, o2) is conj(T_j(o2, o)). */
                        if (periodic[j] || c[j] < L[j] - 1) {
                            int64_t cf[3] = {c[0], c[1], c[2]};
                            cf[j] = (c[j] + 1) % L[j];
                            int64_t sf = site_of(cf[0], cf[1], cf[2], Nx, Ny);
                            for (int o2 = 0; o2 < 4; ++o2) {
                                double hr, hi;
                                hop_entry(j, t, o2, o, &hr, &hi);
                                if (hr != 0.0 || hi != 0.0) {
                                    e[ne].col = 4 * sf + o2;
                                    e[ne].re = no_neg_zero(hr);
                                    e[ne].im = no_neg_zero(-hi);
                                    ++ne;
                                }
                            }
                        }
                    }
                    qsort(e, (size_t)ne, sizeof(entry_t), cmp_entry);
                    for (int k = 0; k < ne; ++k) {
                        col[pos] = (int32_t)e[k].col;
                        val[2 * pos] = e[k].re;
                        val[2 * pos + 1] = e[k].im;
                        ++pos;
                    }
                    rowptr[4 * s + o + 1] = pos;
                }
            }
    return 0;
}

/* ------------------------------------------------------------ SpMMV ----- */

/* y = H x for row-major blocks of nb complex vectors: x(i, j) at
 * x[2 (i ldx + j)], y(i, j) at y[2 (i ldy + j)].  Rows are independent, so the
 * OpenMP split over rows does not change any result. */
void orc_csr_spmmv(int64_t N, const int64_t *rowptr, const int32_t *col, const double *val,
                   const double *x, int64_t ldx, double *y, int64_t ldy, int nb)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int j = 0; j < nb; ++j) {
            double sr = 0.0, si = 0.0;
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                double hr = val[2 * k], hi = val[2 * k + 1];
                const double *xv = x + 2 * ((int64_t)col[k] * ldx + j);
                sr = sr + (hr * xv[0] - hi * xv[1]);
                si = si + (hr * xv[1] + hi * xv[0]);
            }
            y[2 * (i * ldy + j)] = sr;
            y[2 * (i * ldy + j) + 1] = si;
        }
    }
}

/* ------------------------------------------------------ ChebFD filter ---- */

/* Column-wise dot products over a block of N rows and nb vectors (ld = nb):
 * uu[j] = <u_j, u_j>, wu[j] = Re <w_j, u_j>, with <a, b> = sum conj(a) b.
 * Plain serial sums in row order. */
static void block_dots(int64_t N, int nb, const double *w, const double *u, double *wu,
                       double *uu)
{
    for (int j = 0; j < nb; ++j) {
        wu[j] = 0.0;
        uu[j] = 0.0;
    }
    for (int64_t i = 0; i < N; ++i)
        for (int j = 0; j < nb; ++j) {
            const double *a = w + 2 * (i * nb + j), *b = u + 2 * (i * nb + j);
            wu[j] = wu[j] + (a[0] * b[0] + a[1] * b[1]);
            uu[j] = uu[j] + (b[0] * b[0] + b[1] * b[1]);
        }
}

/* out = 2 (a h + b u) - prev, elementwise over N x nb (paper's affine map
 * a H + b 1 applied to u, with h = H u already computed).  out may alias prev. */
static void cheb_combine(int64_t N, int nb, double a, double b, const double *h,
                         const double *u, const double *prev, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N * nb; ++i) {
        for (int c = 0; c < 2; ++c) {
            double s = a * h[2 * i + c] + b * u[2 * i + c];
            out[2 * i + c] = 2.0 * s - prev[2 * i + c];
        }
    }
}

/*
 * Apply the ChebFD filter p(a H + b 1) = sum_{k=0}^{n_p} gc[k] T_k(a H + b 1)
 * to the n_s columns of X (row-major, row stride ldX) in place, n_b columns
 * at a time (Algorithm 2; n_b divides n_s), each block by Algorithm 1:
 *   U = (aH + b) X;  W = 2 (aH + b) U - X;  X = gc0 X + gc1 U + gc2 W;
 *   for p = 3..n_p: swap(W, U); W = 2 (aH + b) U - W;
 *                   eta_p = <W, U>; mu_p = <U, U>; X = X + gc_p W.
 * dots (nullable) receives, for column j and step p = 1..n_p,
 *   dots[(j n_p + p - 1) 2 + 0] = <T_{p-1} x_j, T_{p-1} x_j>   (mu_p)
 *   dots[(j n_p + p - 1) 2 + 1] = Re <T_p x_j, T_{p-1} x_j>    (eta_p)
 * Steps 1 and 2 are the same dot products taken on the seed vectors (the
 * paper's loop records p >= 3 only); they give the first Chebyshev moments.
 * Returns 0, or -1 on bad sizes / allocation failure.
 */
int orc_chebfd_filter(int64_t N, const int64_t *rowptr, const int32_t *col, const double *val,
                      double a, double b, int n_p, const double *gc, double *X, int64_t ldX,
                      int n_s, int n_b, double *dots)
{
    if (n_p < 2 || n_b < 1 || n_s % n_b != 0) return -1;
    size_t bytes = (size_t)N * (size_t)n_b * 2 * sizeof(double);
    double *x = malloc(bytes), *U = malloc(bytes), *W = malloc(bytes), *h = malloc(bytes);
    double *wu = malloc((size_t)n_b * sizeof(double)), *uu = malloc((size_t)n_b * sizeof(double));
    if (!x || !U || !W || !h || !wu || !uu) {
        free(x); free(U); free(W); free(h); free(wu); free(uu);
        return -1;
    }
    for (int blk = 0; blk < n_s / n_b; ++blk) {
        /* X_b: columns blk n_b .. (blk + 1) n_b - 1 (half-open). */
        for (int64_t i = 0; i < N; ++i)
            memcpy(x + 2 * i * n_b, X + 2 * (i * ldX + (int64_t)blk * n_b), 2 * n_b * sizeof(double));

        /* U = (aH + b) X */
        orc_csr_spmmv(N, rowptr, col, val, x, n_b, h, n_b, n_b);
        for (int64_t i = 0; i < N * n_b; ++i)
            for (int c = 0; c < 2; ++c) U[2 * i + c] = a * h[2 * i + c] + b * x[2 * i + c];
        block_dots(N, n_b, U, x, wu, uu);
        if (dots)
            for (int j = 0; j < n_b; ++j) {
                double *d = dots + 2 * ((int64_t)(blk * n_b + j) * n_p + 0);
                d[0] = uu[j];
                d[1] = wu[j];
            }

        /* W = 2 (aH + b) U - X */
        orc_csr_spmmv(N, rowptr, col, val, U, n_b, h, n_b, n_b);
        cheb_combine(N, n_b, a, b, h, U, x, W);
        block_dots(N, n_b, W, U, wu, uu);
        if (dots)
            for (int j = 0; j < n_b; ++j) {
                double *d = dots + 2 * ((int64_t)(blk * n_b + j) * n_p + 1);
                d[0] = uu[j];
                d[1] = wu[j];
            }

        /* X = g0 c0 X + g1 c1 U + g2 c2 W */
        for (int64_t i = 0; i < 2 * N * n_b; ++i)
            x[i] = gc[0] * x[i] + gc[1] * U[i] + gc[2] * W[i];

        for (int p = 3; p <= n_p; ++p) {
            double *tmp = W; /* swap(W, U) */
            W = U;
            U = tmp;
            orc_csr_spmmv(N, rowptr, col, val, U, n_b, h, n_b, n_b);
            cheb_combine(N, n_b, a, b, h, U, W, W);
            block_dots(N, n_b, W, U, wu, uu);
            if (dots)
                for (int j = 0; j < n_b; ++j) {
                    double *d = dots + 2 * ((int64_t)(blk * n_b + j) * n_p + (p - 1));
                    d[0] = uu[j];
                    d[1] = wu[j];
                }
            for (int64_t i = 0; i < 2 * N * n_b; ++i) x[i] = x[i] + gc[p] * W[i];
        }
        for (int64_t i = 0; i < N; ++i)
            memcpy(X + 2 * (i * ldX + (int64_t)blk * n_b), x + 2 * i * n_b, 2 * n_b * sizeof(double));
    }
    free(x); free(U); free(W); free(h); free(wu); free(uu);
    return 0;
}

/* Number of OpenMP threads the parallel loops above use (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
