// Topological-insulator Hamiltonian (Sect. 2.1) built on the device directly
// into SELL-C-sigma, and canonical CSR export.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace cfd {
namespace {

constexpr int TOPI_MAX_ROW = 13;

// The lattice, and the rows built: all of them, or the rows [row0, row0 +
// n_rows) of one z-slab, whose columns are then renumbered locally (own rows
// first, then the lower and the upper halo plane; cfd_slab_local_col).
struct Lattice {
    int32_t L[3];
    int32_t per[3];
    int64_t n_rows;              // rows built
    int64_t row0 = 0;            // canonical index of built row 0
    int32_t slab = 0;            // 1: renumber columns as a slab
    int64_t plane = 0, lo_base = -1, hi_base = -1;
};

Lattice lattice_of(const cfd_topi_params *p) {
    Lattice g;
    g.L[0] = p->Nx;
    g.L[1] = p->Ny;
    g.L[2] = p->Nz;
    g.per[0] = p->periodic_x != 0;
    g.per[1] = p->periodic_y != 0;
    g.per[2] = p->periodic_z != 0;
    g.n_rows = 4LL * p->Nx * p->Ny * p->Nz;
    return g;
}

Lattice lattice_of_slab(const cfd_topi_params *p, const cfd_slab *s) {
    Lattice g = lattice_of(p);
    g.n_rows = s->n_local;
    g.row0 = s->row0;
    g.slab = 1;
    g.plane = s->plane;
    g.lo_base = s->lo_base;
    g.hi_base = s->hi_base;
    return g;
}

// Column of canonical index c in the built rows' numbering.
__host__ __device__ inline int64_t local_col(int64_t c, const Lattice &g) {
    if (!g.slab) return c;
    if (c >= g.row0 && c < g.row0 + g.n_rows) return c - g.row0;
    if (g.lo_base >= 0 && c >= g.lo_base && c < g.lo_base + g.plane) return g.n_rows + (c - g.lo_base);
    if (g.hi_base >= 0 && c >= g.hi_base && c < g.hi_base + g.plane) return g.n_rows + g.plane + (c - g.hi_base);
    return -1;
}

// Stored entries of canonical row i: one on-site entry and two per existing
// neighbour (periodic axes always have both neighbours).
__host__ __device__ inline int topi_row_len(int64_t i, const Lattice &g) {
    int64_t s = i >> 2;
    int64_t c[3];
    c[0] = s % g.L[0];
    c[1] = (s / g.L[0]) % g.L[1];
    c[2] = s / ((int64_t)g.L[0] * g.L[1]);
    int len = 1;
    for (int j = 0; j < 3; ++j) {
        if (g.per[j] || c[j] > 0) len += 2;
        if (g.per[j] || c[j] < g.L[j] - 1) len += 2;
    }
    return len;
}

// Real and imaginary entries of canonical row i: on-site real; per existing
// neighbour along x a real diagonal-orbital entry and an imaginary partner,
// along y two real entries, along z a real and an imaginary entry.
__host__ __device__ inline void topi_row_counts(int64_t i, const Lattice &g, int *n_re, int *n_im) {
    int64_t s = i >> 2;
    int64_t c[3];
    c[0] = s % g.L[0];
    c[1] = (s / g.L[0]) % g.L[1];
    c[2] = s / ((int64_t)g.L[0] * g.L[1]);
    int nb[3];
    for (int j = 0; j < 3; ++j) nb[j] = (g.per[j] || c[j] > 0) + (g.per[j] || c[j] < g.L[j] - 1);
    *n_re = 1 + nb[0] + 2 * nb[1] + nb[2];
    *n_im = nb[0] + nb[2];
}

// SplitMix64 (Steele, Lea, Flood 2014): output function and counter-based
// draw i of stream (seed, tag), key = mix(seed + GAMMA (2 tag + 1)).
__device__ inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ inline uint64_t sm64_draw(uint64_t seed, uint64_t tag, uint64_t i) {
    const uint64_t G = 0x9E3779B97F4A7C15ULL;
    uint64_t key = sm64_mix(seed + G * (2 * tag + 1));
    return sm64_mix(key + (i + 1) * G);
}

struct TopiValues {
    double t, m, gamma;
    uint64_t seed;
};

// Entries of canonical row i = 4 s + o, in ascending column order.
// Hop block T_j = -(t/2) Gamma_1 + i (t/2) Gamma_{j+2}:
//   diagonal (o, o):          -(t/2) g1(o), g1 = +1 for o < 2, -1 otherwise;
//   partner (o, q_j(o)):      q = 3 - o for j = x, y and q = o ^ 2 for j = z,
//     x: +i t/2;  y: +t/2 (o even) / -t/2 (o odd);  z: +i t/2 (o even) / -i t/2 (o odd).
// Row s meets T_j towards s - e_j and T_j^H towards s + e_j; the partner entry
// of T_j^H in row o is conj(T_j(q, o)).
__device__ int topi_row(int64_t i, const Lattice &g, const TopiValues &v, int32_t *col,
                        double2 *val) {
    const int64_t s = i >> 2;
    const int o = (int)(i & 3);
    int64_t c[3];
    c[0] = s % g.L[0];
    c[1] = (s / g.L[0]) % g.L[1];
    c[2] = s / ((int64_t)g.L[0] * g.L[1]);
    const int64_t stride[3] = {1, (int64_t)g.L[0], (int64_t)g.L[0] * g.L[1]};
    const double h = 0.5 * v.t;
    const double g1 = (o < 2) ? 1.0 : -1.0;
    int n = 0;

    // on-site (m + V_s) Gamma_1, V_s = gamma (u_s - 1/2)
    double u = (double)(sm64_draw(v.seed, 0, (uint64_t)s) >> 11) * (1.0 / 9007199254740992.0);
    double onsite = __dadd_rn(v.m, __dmul_rn(v.gamma, u - 0.5));
    double d = onsite * g1;
    col[n] = (int32_t)i;
    val[n] = make_double2(d == 0.0 ? 0.0 : d, 0.0);
    ++n;

    for (int j = 0; j < 3; ++j) {
        const int q = (j < 2) ? 3 - o : (o ^ 2);
        // backward neighbour: block T_j, row o
        if (g.per[j] || c[j] > 0) {
            int64_t sb = s + ((c[j] > 0) ? -stride[j] : (int64_t)(g.L[j] - 1) * stride[j]);
            col[n] = (int32_t)(4 * sb + o);
            val[n] = make_double2(-h * g1, 0.0);
            ++n;
            col[n] = (int32_t)(4 * sb + q);
            if (j == 0) val[n] = make_double2(0.0, h);
            else if (j == 1) val[n] = make_double2((o & 1) ? -h : h, 0.0);
            else val[n] = make_double2(0.0, (o & 1) ? -h : h);
            ++n;
        }
        // forward neighbour: block T_j^H, row o
        if (g.per[j] || c[j] < g.L[j] - 1) {
            int64_t sf = s + ((c[j] < g.L[j] - 1) ? stride[j] : -(int64_t)(g.L[j] - 1) * stride[j]);
            col[n] = (int32_t)(4 * sf + o);
            val[n] = make_double2(-h * g1, 0.0);
            ++n;
            col[n] = (int32_t)(4 * sf + q);
            if (j == 0) val[n] = make_double2(0.0, -h);                      // conj(+i t/2)
            else if (j == 1) val[n] = make_double2((q & 1) ? -h : h, 0.0);    // real
            else val[n] = make_double2(0.0, (q & 1) ? h : -h);               // conj(+-i t/2)
            ++n;
        }
    }
    // insertion sort by column
    for (int a = 1; a < n; ++a) {
        int32_t kc = col[a];
        double2 kv = val[a];
        int b = a - 1;
        while (b >= 0 && col[b] > kc) {
            col[b + 1] = col[b];
            val[b + 1] = val[b];
            --b;
        }
        col[b + 1] = kc;
        val[b + 1] = kv;
    }
    return n;
}

template <typename C> __device__ inline C to_prec(double2 z);
template <> __device__ inline double2 to_prec<double2>(double2 z) { return z; }
template <> __device__ inline float2 to_prec<float2>(double2 z) {
    return make_float2(__double2float_rn(z.x), __double2float_rn(z.y));
}

// One thread per window of sigma canonical rows: stable counting sort by
// decreasing row length; perm[window start + rank] = canonical row.
__global__ void k_sigma_sort(Lattice g, int sigma, int32_t *perm) {
    int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t r0 = w * sigma;
    if (r0 >= g.n_rows) return;
    int64_t r1 = min(r0 + (int64_t)sigma, g.n_rows);
    int cnt[TOPI_MAX_ROW + 1];
    for (int k = 0; k <= TOPI_MAX_ROW; ++k) cnt[k] = 0;
    for (int64_t i = r0; i < r1; ++i) ++cnt[topi_row_len(g.row0 + i, g)];
    int start[TOPI_MAX_ROW + 1];
    int run = 0;
    for (int k = TOPI_MAX_ROW; k >= 0; --k) {
        start[k] = run;
        run += cnt[k];
    }
    for (int64_t i = r0; i < r1; ++i) perm[r0 + start[topi_row_len(g.row0 + i, g)]++] = (int32_t)i;
}

// Slots per row of each chunk: the longest row's length, or for packed
// values the most real entries (low 16 bits) and the most imaginary entries
// (high 16 bits) of any row.
__global__ void k_chunk_len(Lattice g, int log2C, int64_t n_chunks, const int32_t *perm, bool packed,
                            int32_t *chunk_len, int64_t *slots) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    int C = 1 << log2C;
    int mx = 0, mre = 0, mim = 0;
    for (int rr = 0; rr < C; ++rr) {
        int64_t r = (c << log2C) + rr;
        if (r >= g.n_rows) break;
        int64_t i = g.row0 + (perm ? perm[r] : r);
        mx = max(mx, topi_row_len(i, g));
        int a, b;
        topi_row_counts(i, g, &a, &b);
        mre = max(mre, a);
        mim = max(mim, b);
    }
    chunk_len[c] = packed ? (mre | (mim << 16)) : mx;
    slots[c] = (int64_t)(packed ? mre + mim : mx) << log2C;
}

template <typename C>
__global__ void k_fill(Lattice g, TopiValues v, int log2C, int64_t n_chunks, const int32_t *perm,
                       const int64_t *chunk_ptr, const int32_t *chunk_len, int32_t *col, C *val) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= (n_chunks << log2C)) return;
    int64_t c = r >> log2C;
    int64_t rr = r & ((1 << log2C) - 1);
    int64_t base = chunk_ptr[c] + rr;
    int len = chunk_len[c];
    int32_t ec[TOPI_MAX_ROW];
    double2 ev[TOPI_MAX_ROW];
    int n = 0;
    if (r < g.n_rows) n = topi_row(g.row0 + (perm ? perm[r] : r), g, v, ec, ev);
    for (int k = 0; k < n; ++k) ec[k] = (int32_t)local_col(ec[k], g);
    for (int k = 0; k < len; ++k) {
        int64_t at = base + ((int64_t)k << log2C);
        if (k < n) {
            col[at] = ec[k];
            val[at] = to_prec<C>(ev[k]);
        } else {
            col[at] = -1;
            val[at] = to_prec<C>(make_double2(0.0, 0.0));
        }
    }
}

// Packed fill: one real scalar per slot; each row stores its real entries in
// slots [0, n_re) and its imaginary entries (their imaginary parts) in
// [n_re, n_re + n_im), both in ascending column order, with n_re, n_im the
// chunk's maxima (every Topi entry is purely real or purely imaginary).
template <typename S>
__global__ void k_fill_packed(Lattice g, TopiValues v, int log2C, int64_t n_chunks, const int32_t *perm,
                              const int64_t *chunk_ptr, const int32_t *chunk_len, int32_t *col, S *val) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= (n_chunks << log2C)) return;
    int64_t c = r >> log2C;
    int64_t rr = r & ((1 << log2C) - 1);
    int64_t base = chunk_ptr[c] + rr;
    const int n_re = chunk_len[c] & 0xffff, n_im = chunk_len[c] >> 16;
    int32_t ec[TOPI_MAX_ROW];
    double2 ev[TOPI_MAX_ROW];
    int n = 0;
    if (r < g.n_rows) n = topi_row(g.row0 + (perm ? perm[r] : r), g, v, ec, ev);
    for (int k = 0; k < n; ++k) ec[k] = (int32_t)local_col(ec[k], g);
    int kre = 0, kim = n_re;
    for (int k = 0; k < n; ++k) {
        bool im = ev[k].y != 0.0;
        int64_t at = base + ((int64_t)(im ? kim++ : kre++) << log2C);
        col[at] = ec[k];
        val[at] = (S)(im ? ev[k].y : ev[k].x);
    }
    for (; kre < n_re; ++kre) {
        col[base + ((int64_t)kre << log2C)] = -1;
        val[base + ((int64_t)kre << log2C)] = (S)0;
    }
    for (; kim < n_re + n_im; ++kim) {
        col[base + ((int64_t)kim << log2C)] = -1;
        val[base + ((int64_t)kim << log2C)] = (S)0;
    }
}

// CSR export: row lengths of canonical rows, then entries.
__global__ void k_csr_len(int64_t n_rows, int log2C, const int64_t *chunk_ptr,
                          const int32_t *chunk_len, const int32_t *perm, const int32_t *col, bool packed,
                          int64_t *rowlen) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    int64_t c = r >> log2C;
    int64_t base = chunk_ptr[c] + (r & ((1 << log2C) - 1));
    const int len = packed ? (chunk_len[c] & 0xffff) + (chunk_len[c] >> 16) : chunk_len[c];
    int n = 0;
    for (int k = 0; k < len; ++k)
        if (col[base + ((int64_t)k << log2C)] != -1) ++n;
    rowlen[perm ? perm[r] : r] = n;
}

template <typename C>
__global__ void k_csr_fill(int64_t n_rows, int log2C, const int64_t *chunk_ptr,
                           const int32_t *chunk_len, const int32_t *perm, const int32_t *col,
                           const C *val, const int64_t *rowptr, int32_t *ocol, C *oval) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    int64_t c = r >> log2C;
    int64_t base = chunk_ptr[c] + (r & ((1 << log2C) - 1));
    int64_t o = rowptr[perm ? perm[r] : r];
    for (int k = 0; k < chunk_len[c]; ++k) {
        int64_t at = base + ((int64_t)k << log2C);
        int32_t cc = col[at];
        if (cc >= 0) {
            ocol[o] = cc;
            oval[o] = val[at];
            ++o;
        }
    }
}

// Packed rows back to complex CSR: merge the ascending real and imaginary
// groups into one ascending row.
template <typename S, typename C>
__global__ void k_csr_fill_packed(int64_t n_rows, int log2C, const int64_t *chunk_ptr, const int32_t *chunk_len,
                                  const int32_t *perm, const int32_t *col, const S *val, const int64_t *rowptr,
                                  int32_t *ocol, C *oval) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    int64_t c = r >> log2C;
    int64_t base = chunk_ptr[c] + (r & ((1 << log2C) - 1));
    int64_t o = rowptr[perm ? perm[r] : r];
    const int n_re = chunk_len[c] & 0xffff, n_im = chunk_len[c] >> 16;
    int a = 0, b = n_re;
    while (true) {
        int32_t ca = a < n_re ? col[base + ((int64_t)a << log2C)] : -1;
        int32_t cb = b < n_re + n_im ? col[base + ((int64_t)b << log2C)] : -1;
        if (ca < 0 && cb < 0) break;
        C z;
        if (cb < 0 || (ca >= 0 && ca < cb)) {
            z.x = val[base + ((int64_t)a << log2C)];
            z.y = (S)0;
            ocol[o] = ca;
            ++a;
        } else {
            z.x = (S)0;
            z.y = val[base + ((int64_t)b << log2C)];
            ocol[o] = cb;
            ++b;
        }
        oval[o] = z;
        ++o;
    }
}

cfd_status check_params(const cfd_topi_params *p, int C, int sigma, int prec) {
    if (!p) return fail(CFD_ERR_ARG, "params is NULL");
    int L[3] = {p->Nx, p->Ny, p->Nz};
    int per[3] = {p->periodic_x, p->periodic_y, p->periodic_z};
    for (int j = 0; j < 3; ++j) {
        if (L[j] < 1) return fail(CFD_ERR_ARG, "lattice extent %d < 1", L[j]);
        if (per[j] && L[j] < 3) return fail(CFD_ERR_ARG, "periodic axis needs >= 3 sites");
    }
    double n = 4.0 * p->Nx * (double)p->Ny * p->Nz;
    if (n > 2147483647.0) return fail(CFD_ERR_ARG, "N = %.0f exceeds 32-bit column indices", n);
    if (C < 4 || C > 128 || (C & (C - 1))) return fail(CFD_ERR_ARG, "C=%d must be a power of two in 4..128", C);
    if (sigma < 1 || sigma > 65536 || (sigma > 1 && sigma % C))
        return fail(CFD_ERR_ARG, "sigma=%d must be 1 or a multiple of C up to 65536", sigma);
    if (prec != CFD_C128 && prec != CFD_C64) return fail(CFD_ERR_ARG, "prec %d invalid", prec);
    return CFD_OK;
}

// Host replica of the chunk lengths (for sizes, no GPU work): rows sorted
// stably by decreasing length inside each sigma window, then per chunk the
// longest row (complex values) or the most real plus the most imaginary
// entries (packed values).
int64_t host_slots(const Lattice &g, int C, int sigma, bool packed) {
    int64_t slots = 0;
    std::vector<int64_t> order;
    for (int64_t r0 = 0; r0 < g.n_rows; r0 += (sigma > 1 ? sigma : g.n_rows)) {
        int64_t r1 = sigma > 1 ? std::min<int64_t>(r0 + sigma, g.n_rows) : g.n_rows;
        order.clear();
        if (sigma > 1) {
            for (int k = TOPI_MAX_ROW; k >= 0; --k)
                for (int64_t i = r0; i < r1; ++i)
                    if (topi_row_len(g.row0 + i, g) == k) order.push_back(i);
        }
        for (int64_t a = r0; a < r1; a += C) {
            int mx = 0, mre = 0, mim = 0;
            for (int64_t q = a; q < std::min<int64_t>(a + C, r1); ++q) {
                int64_t i = g.row0 + (sigma > 1 ? order[q - r0] : q);
                mx = std::max(mx, topi_row_len(i, g));
                int x, y;
                topi_row_counts(i, g, &x, &y);
                mre = std::max(mre, x);
                mim = std::max(mim, y);
            }
            slots += (int64_t)(packed ? mre + mim : mx) * C;
        }
    }
    return slots;
}

// After building realisation r into its slice of a batch with local indices:
// shift chunk pointers by the slice's first slot, columns and the sorting
// permutation by its first row, pad rows permute to themselves, and tag the
// slice's chunks with r.
__global__ void k_batch_fixup(int r, int64_t row_off, int64_t slot_off, int64_t n_chunks_r, int64_t n_rows_r,
                              int64_t padded_r, int64_t slots_r, int64_t *chunk_ptr, int32_t *chunk_rid,
                              int32_t *perm, int32_t *col) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < slots_r; e += stride)
        if (col[e] >= 0) col[e] += (int32_t)row_off;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= n_chunks_r; e += stride) {
        chunk_ptr[e] += slot_off;
        if (e < n_chunks_r) chunk_rid[e] = r;
    }
    if (perm)
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < padded_r; e += stride)
            perm[e] = (int32_t)(row_off + (e < n_rows_r ? perm[e] : e));
}

struct BatchLayout {
    std::vector<int64_t> row_off, slot_off, slots, chunk_off;
    int64_t nnz = 0, work = 0;
};

int64_t batch_pad(int C, int sigma) { return std::max<int64_t>(std::max(C, sigma), 32); }

cfd_status batch_layout(const cfd_topi_params *p, int R, int C, int sigma, int prec, bool packed, BatchLayout &L) {
    if (!p || R < 1) return fail(CFD_ERR_ARG, "empty batch");
    const int64_t P = batch_pad(C, sigma);
    L.row_off.assign(R + 1, 0);
    L.slot_off.assign(R + 1, 0);
    L.slots.assign(R, 0);
    L.chunk_off.assign(R + 1, 0);
    for (int r = 0; r < R; ++r) {
        CFD_TRY(check_params(p + r, C, sigma, prec));
        Lattice g = lattice_of(p + r);
        int64_t padded = (g.n_rows + P - 1) / P * P;
        L.row_off[r + 1] = L.row_off[r] + padded;
        L.chunk_off[r + 1] = L.row_off[r + 1] / C;
        L.slots[r] = host_slots(g, C, sigma, packed);
        L.slot_off[r + 1] = L.slot_off[r] + L.slots[r];
        for (int64_t i = 0; i < g.n_rows; i += 4) L.nnz += 4 * topi_row_len(i, g);
        int64_t nch = padded / C;
        L.work = std::max<int64_t>(L.work, (int64_t)(round_up((size_t)nch * 8, 256) + scan_workspace(nch)));
    }
    if (L.row_off[R] > 2147483647LL) return fail(CFD_ERR_ARG, "batch exceeds 32-bit column indices");
    return CFD_OK;
}

// Sizes of the SELL arrays for the rows of g.
void query_sizes(const Lattice &g, int C, int sigma, int prec_arg, cfd_matrix_sizes *out) {
    const bool packed = (prec_arg & CFD_PACK_RI) != 0;
    const int prec = prec_arg & ~CFD_PACK_RI;
    int64_t nnz = 0;
    for (int64_t i = 0; i < g.n_rows; i += 4) nnz += 4 * topi_row_len(g.row0 + i, g);
    int64_t n_chunks = (g.n_rows + C - 1) / C;
    int64_t slots = host_slots(g, C, sigma, packed);
    size_t sv = packed ? ((prec == CFD_C128) ? 8 : 4) : ((prec == CFD_C128) ? 16 : 8);
    out->n_rows = g.n_rows;
    out->nnz = nnz;
    out->n_chunks = n_chunks;
    out->n_slots = slots;
    out->bytes_val = (int64_t)round_up((size_t)slots * sv, 256);
    out->bytes_col = (int64_t)round_up((size_t)slots * 4, 256);
    out->bytes_chunk_ptr = (int64_t)round_up((size_t)(n_chunks + 1) * 8, 256);
    out->bytes_chunk_len = (int64_t)round_up((size_t)n_chunks * 4, 256);
    out->bytes_perm = sigma > 1 ? (int64_t)round_up((size_t)g.n_rows * 4, 256) : 0;
    out->bytes_work = (int64_t)(round_up((size_t)n_chunks * 8, 256) + scan_workspace(n_chunks));
}

// Build the rows of g into SELL-C-sigma (sizes sz from query_sizes).
cfd_status build_impl(const Lattice &g, const cfd_topi_params *p, int C, int sigma, int prec_arg,
                      const cfd_matrix_sizes &sz, const cfd_matrix_buffers *buf, cfd_matrix *out,
                      cudaStream_t stream) {
    const bool packed = (prec_arg & CFD_PACK_RI) != 0;
    const int prec = prec_arg & ~CFD_PACK_RI;
    if (!buf || !out) return fail(CFD_ERR_ARG, "buffers or out is NULL");
    if (!buf->val || !buf->col || !buf->chunk_ptr || !buf->chunk_len || !buf->work ||
        (sigma > 1 && !buf->perm))
        return fail(CFD_ERR_ARG, "a required matrix buffer is NULL");
    if (!aligned16(buf->val) || !aligned16(buf->col) || !aligned16(buf->chunk_ptr) ||
        !aligned16(buf->chunk_len) || !aligned16(buf->work) || (buf->perm && !aligned16(buf->perm)))
        return fail(CFD_ERR_ARG, "matrix buffers must be 16-byte aligned");
    TopiValues v{p->t, p->m, p->gamma, p->seed};
    int log2C = 0;
    while ((1 << log2C) < C) ++log2C;
    int32_t *perm = sigma > 1 ? static_cast<int32_t *>(buf->perm) : nullptr;
    int32_t *chunk_len = static_cast<int32_t *>(buf->chunk_len);
    int64_t *chunk_ptr = static_cast<int64_t *>(buf->chunk_ptr);
    Carve w(buf->work, (size_t)sz.bytes_work);
    int64_t *slots = w.take<int64_t>((size_t)sz.n_chunks);
    void *scan_work = w.take<char>(scan_workspace(sz.n_chunks));
    const int T = 256;
    if (perm) {
        int64_t windows = (g.n_rows + sigma - 1) / sigma;
        k_sigma_sort<<<(unsigned)((windows + T - 1) / T), T, 0, stream>>>(g, sigma, perm);
        CFD_COUNT_LAUNCH();
    }
    k_chunk_len<<<(unsigned)((sz.n_chunks + T - 1) / T), T, 0, stream>>>(g, log2C, sz.n_chunks, perm, packed,
                                                                          chunk_len, slots);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    CFD_TRY(exclusive_scan_i64(slots, chunk_ptr, sz.n_chunks, scan_work, stream));
    int64_t rows_pad = sz.n_chunks << log2C;
    unsigned grid = (unsigned)((rows_pad + T - 1) / T);
    if (packed && prec == CFD_C128)
        k_fill_packed<double><<<grid, T, 0, stream>>>(g, v, log2C, sz.n_chunks, perm, chunk_ptr, chunk_len,
                                                      static_cast<int32_t *>(buf->col),
                                                      static_cast<double *>(buf->val));
    else if (packed)
        k_fill_packed<float><<<grid, T, 0, stream>>>(g, v, log2C, sz.n_chunks, perm, chunk_ptr, chunk_len,
                                                     static_cast<int32_t *>(buf->col), static_cast<float *>(buf->val));
    else if (prec == CFD_C128)
        k_fill<double2><<<grid, T, 0, stream>>>(g, v, log2C, sz.n_chunks, perm, chunk_ptr, chunk_len,
                                                static_cast<int32_t *>(buf->col),
                                                static_cast<double2 *>(buf->val));
    else
        k_fill<float2><<<grid, T, 0, stream>>>(g, v, log2C, sz.n_chunks, perm, chunk_ptr, chunk_len,
                                               static_cast<int32_t *>(buf->col),
                                               static_cast<float2 *>(buf->val));
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    out->n_rows = sz.n_rows;
    out->nnz = sz.nnz;
    out->n_chunks = sz.n_chunks;
    out->n_slots = sz.n_slots;
    out->C = C;
    out->sigma = sigma;
    out->prec = prec;
    out->flags = (packed ? CFD_MATRIX_PACKED : 0) | (TOPI_MAX_ROW << CFD_MATRIX_SLOTS_SHIFT);
    out->val = buf->val;
    out->col = static_cast<int32_t *>(buf->col);
    out->chunk_ptr = chunk_ptr;
    out->chunk_len = chunk_len;
    out->perm = perm;
    return CFD_OK;
}

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" {

// ------------------------------------------------ z-slab distribution --

cfd_status cfd_slab_plan(const cfd_topi_params *p, int nranks, int rank, cfd_slab *out) {
    clear_error();
    CFD_TRY(check_params(p, 32, 1, CFD_C128));
    if (!out) return fail(CFD_ERR_ARG, "out is NULL");
    if (nranks < 1 || rank < 0 || rank >= nranks) return fail(CFD_ERR_ARG, "rank %d of %d invalid", rank, nranks);
    if (nranks > p->Nz) return fail(CFD_ERR_ARG, "%d ranks for %d z-planes: every rank needs a plane", nranks, p->Nz);
    const int64_t plane = 4LL * p->Nx * p->Ny;
    const int Nz = p->Nz;
    cfd_slab s;
    s.nranks = nranks;
    s.rank = rank;
    s.z0 = (int32_t)((int64_t)rank * Nz / nranks);
    s.z1 = (int32_t)((int64_t)(rank + 1) * Nz / nranks);
    s.row0 = plane * s.z0;
    s.n_local = plane * (s.z1 - s.z0);
    s.plane = plane;
    s.lo_rank = s.hi_rank = -1;
    s.lo_base = s.hi_base = -1;
    if (nranks > 1) {
        if (s.z0 > 0) { s.lo_rank = rank - 1; s.lo_base = plane * (s.z0 - 1); }
        else if (p->periodic_z) { s.lo_rank = nranks - 1; s.lo_base = plane * (Nz - 1); }
        if (s.z1 < Nz) { s.hi_rank = rank + 1; s.hi_base = plane * s.z1; }
        else if (p->periodic_z) { s.hi_rank = 0; s.hi_base = 0; }
    }
    *out = s;
    return CFD_OK;
}

int64_t cfd_slab_local_col(const cfd_slab *s, int64_t col) {
    if (!s) return -1;
    Lattice g;
    g.n_rows = s->n_local;
    g.row0 = s->row0;
    g.slab = 1;
    g.plane = s->plane;
    g.lo_base = s->lo_base;
    g.hi_base = s->hi_base;
    return local_col(col, g);
}

cfd_status cfd_slab_query_size(const cfd_topi_params *p, const cfd_slab *slab, int C, int sigma, int prec_arg,
                               cfd_matrix_sizes *out) {
    clear_error();
    const int prec = prec_arg & ~CFD_PACK_RI;
    CFD_TRY(check_params(p, C, sigma, prec));
    if (!slab || !out) return fail(CFD_ERR_ARG, "slab or out is NULL");
    if (slab->n_local < 1 || slab->plane != 4LL * p->Nx * p->Ny || slab->row0 + slab->n_local > 4LL * p->Nx * p->Ny * p->Nz)
        return fail(CFD_ERR_ARG, "slab does not fit the lattice (use cfd_slab_plan)");
    query_sizes(lattice_of_slab(p, slab), C, sigma, prec_arg, out);
    return CFD_OK;
}

cfd_status cfd_build_matrix_slab(const cfd_topi_params *p, const cfd_slab *slab, int C, int sigma, int prec_arg,
                                 const cfd_matrix_buffers *buf, cfd_matrix *out, cudaStream_t stream) {
    cfd_matrix_sizes sz;
    CFD_TRY(cfd_slab_query_size(p, slab, C, sigma, prec_arg, &sz));
    return build_impl(lattice_of_slab(p, slab), p, C, sigma, prec_arg, sz, buf, out, stream);
}


cfd_status cfd_matrix_query_size(const cfd_topi_params *p, int C, int sigma, int prec_arg,
                                 cfd_matrix_sizes *out) {
    clear_error();
    const int prec = prec_arg & ~CFD_PACK_RI;
    CFD_TRY(check_params(p, C, sigma, prec));
    if (!out) return fail(CFD_ERR_ARG, "out is NULL");
    query_sizes(lattice_of(p), C, sigma, prec_arg, out);
    return CFD_OK;
}

cfd_status cfd_build_matrix(const cfd_topi_params *p, int C, int sigma, int prec_arg,
                            const cfd_matrix_buffers *buf, cfd_matrix *out, cudaStream_t stream) {
    cfd_matrix_sizes sz;
    CFD_TRY(cfd_matrix_query_size(p, C, sigma, prec_arg, &sz));
    return build_impl(lattice_of(p), p, C, sigma, prec_arg, sz, buf, out, stream);
}

cfd_status cfd_batch_query_size(const cfd_topi_params *p, int R, int C, int sigma, int prec_arg,
                                cfd_matrix_sizes *out, int64_t *row_off) {
    clear_error();
    const bool packed = (prec_arg & CFD_PACK_RI) != 0;
    const int prec = prec_arg & ~CFD_PACK_RI;
    if (!out) return fail(CFD_ERR_ARG, "out is NULL");
    BatchLayout L;
    CFD_TRY(batch_layout(p, R, C, sigma, prec, packed, L));
    size_t s = packed ? ((prec == CFD_C128) ? 8 : 4) : ((prec == CFD_C128) ? 16 : 8);
    int64_t N = L.row_off[R], n_chunks = N / C, slots = L.slot_off[R];
    out->n_rows = N;
    out->nnz = L.nnz;
    out->n_chunks = n_chunks;
    out->n_slots = slots;
    out->bytes_val = (int64_t)round_up((size_t)slots * s, 256);
    out->bytes_col = (int64_t)round_up((size_t)slots * 4, 256);
    out->bytes_chunk_ptr = (int64_t)round_up((size_t)(n_chunks + 1) * 8, 256);
    out->bytes_chunk_len = (int64_t)round_up((size_t)n_chunks * 4, 256);
    out->bytes_perm = sigma > 1 ? (int64_t)round_up((size_t)N * 4, 256) : 0;
    out->bytes_work = L.work;
    if (row_off)
        for (int r = 0; r <= R; ++r) row_off[r] = L.row_off[r];
    return CFD_OK;
}

cfd_status cfd_build_batch(const cfd_topi_params *p, int R, int C, int sigma, int prec_arg,
                           const cfd_matrix_buffers *buf, int32_t *chunk_rid, cfd_matrix *out,
                           cudaStream_t stream) {
    clear_error();
    cfd_matrix_sizes sz;
    CFD_TRY(cfd_batch_query_size(p, R, C, sigma, prec_arg, &sz, nullptr));
    const bool packed = (prec_arg & CFD_PACK_RI) != 0;
    const int prec = prec_arg & ~CFD_PACK_RI;
    if (!buf || !out || !chunk_rid) return fail(CFD_ERR_ARG, "buffers, chunk_rid or out is NULL");
    if (!buf->val || !buf->col || !buf->chunk_ptr || !buf->chunk_len || !buf->work || (sigma > 1 && !buf->perm))
        return fail(CFD_ERR_ARG, "a required matrix buffer is NULL");
    if (!aligned16(buf->val) || !aligned16(buf->col) || !aligned16(buf->chunk_ptr) || !aligned16(buf->work))
        return fail(CFD_ERR_ARG, "matrix buffers must be 16-byte aligned");
    BatchLayout L;
    CFD_TRY(batch_layout(p, R, C, sigma, prec, packed, L));
    int log2C = 0;
    while ((1 << log2C) < C) ++log2C;
    int32_t *perm_all = sigma > 1 ? static_cast<int32_t *>(buf->perm) : nullptr;
    int32_t *chunk_len = static_cast<int32_t *>(buf->chunk_len);
    int64_t *chunk_ptr = static_cast<int64_t *>(buf->chunk_ptr);
    int32_t *col = static_cast<int32_t *>(buf->col);
    const int T = 256;
    for (int r = 0; r < R; ++r) {
        Lattice g = lattice_of(p + r);
        TopiValues v{p[r].t, p[r].m, p[r].gamma, p[r].seed};
        const int64_t padded = L.row_off[r + 1] - L.row_off[r];
        const int64_t nch = padded / C, c0 = L.chunk_off[r], s0 = L.slot_off[r];
        Carve w(buf->work, (size_t)sz.bytes_work);
        int64_t *slots = w.take<int64_t>((size_t)nch);
        void *scan_work = w.take<char>(scan_workspace(nch));
        int32_t *perm = perm_all ? perm_all + L.row_off[r] : nullptr;
        if (perm) {
            int64_t windows = (g.n_rows + sigma - 1) / sigma;
            k_sigma_sort<<<(unsigned)((windows + T - 1) / T), T, 0, stream>>>(g, sigma, perm);
            CFD_COUNT_LAUNCH();
        }
        k_chunk_len<<<(unsigned)((nch + T - 1) / T), T, 0, stream>>>(g, log2C, nch, perm, packed, chunk_len + c0,
                                                                     slots);
        CFD_COUNT_LAUNCH();
        CFD_LAUNCH_CHECK();
        CFD_TRY(exclusive_scan_i64(slots, chunk_ptr + c0, nch, scan_work, stream));
        unsigned grid = (unsigned)((padded + T - 1) / T);
        if (packed && prec == CFD_C128)
            k_fill_packed<double><<<grid, T, 0, stream>>>(g, v, log2C, nch, perm, chunk_ptr + c0, chunk_len + c0,
                                                          col + s0, static_cast<double *>(buf->val) + s0);
        else if (packed)
            k_fill_packed<float><<<grid, T, 0, stream>>>(g, v, log2C, nch, perm, chunk_ptr + c0, chunk_len + c0,
                                                         col + s0, static_cast<float *>(buf->val) + s0);
        else if (prec == CFD_C128)
            k_fill<double2><<<grid, T, 0, stream>>>(g, v, log2C, nch, perm, chunk_ptr + c0, chunk_len + c0, col + s0,
                                                    static_cast<double2 *>(buf->val) + s0);
        else
            k_fill<float2><<<grid, T, 0, stream>>>(g, v, log2C, nch, perm, chunk_ptr + c0, chunk_len + c0, col + s0,
                                                   static_cast<float2 *>(buf->val) + s0);
        CFD_COUNT_LAUNCH();
        int64_t span = std::max(std::max(L.slots[r], nch + 1), padded);
        k_batch_fixup<<<(unsigned)std::min<int64_t>((span + T - 1) / T, 4096), T, 0, stream>>>(
            r, L.row_off[r], s0, nch, g.n_rows, padded, L.slots[r], chunk_ptr + c0, chunk_rid + c0, perm, col + s0);
        CFD_COUNT_LAUNCH();
        CFD_LAUNCH_CHECK();
    }
    out->n_rows = sz.n_rows;
    out->nnz = sz.nnz;
    out->n_chunks = sz.n_chunks;
    out->n_slots = sz.n_slots;
    out->C = C;
    out->sigma = sigma;
    out->prec = prec;
    out->flags = ((prec_arg & CFD_PACK_RI) ? CFD_MATRIX_PACKED : 0) | (TOPI_MAX_ROW << CFD_MATRIX_SLOTS_SHIFT);
    out->val = buf->val;
    out->col = col;
    out->chunk_ptr = chunk_ptr;
    out->chunk_len = chunk_len;
    out->perm = perm_all;
    return CFD_OK;
}

size_t cfd_export_csr_workspace(const cfd_matrix *H) {
    if (!H || H->n_rows < 1) return 0;
    return round_up((size_t)H->n_rows * 8, 256) + scan_workspace(H->n_rows);
}

cfd_status cfd_matrix_export_csr(const cfd_matrix *H, int64_t *rowptr, int32_t *col, void *val,
                                 void *work, size_t work_bytes, cudaStream_t stream) {
    clear_error();
    CFD_TRY(check_matrix(H));
    if (!rowptr || !col || !val || !work) return fail(CFD_ERR_ARG, "export buffer is NULL");
    if (work_bytes < cfd_export_csr_workspace(H)) return fail(CFD_ERR_OOM, "export workspace too small");
    int log2C = 0;
    while ((1 << log2C) < H->C) ++log2C;
    Carve w(work, work_bytes);
    int64_t *rowlen = w.take<int64_t>((size_t)H->n_rows);
    void *scan_work = w.take<char>(scan_workspace(H->n_rows));
    const int T = 256;
    unsigned grid = (unsigned)((H->n_rows + T - 1) / T);
    k_csr_len<<<grid, T, 0, stream>>>(H->n_rows, log2C, H->chunk_ptr, H->chunk_len, H->perm, H->col,
                                      (H->flags & CFD_MATRIX_PACKED) != 0, rowlen);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    CFD_TRY(exclusive_scan_i64(rowlen, rowptr, H->n_rows, scan_work, stream));
    const bool packed = (H->flags & CFD_MATRIX_PACKED) != 0;
    if (packed && H->prec == CFD_C128)
        k_csr_fill_packed<double, double2><<<grid, T, 0, stream>>>(H->n_rows, log2C, H->chunk_ptr, H->chunk_len,
                                                                   H->perm, H->col,
                                                                   static_cast<const double *>(H->val), rowptr, col,
                                                                   static_cast<double2 *>(val));
    else if (packed)
        k_csr_fill_packed<float, float2><<<grid, T, 0, stream>>>(H->n_rows, log2C, H->chunk_ptr, H->chunk_len,
                                                                 H->perm, H->col, static_cast<const float *>(H->val),
                                                                 rowptr, col, static_cast<float2 *>(val));
    else if (H->prec == CFD_C128)
        k_csr_fill<double2><<<grid, T, 0, stream>>>(H->n_rows, log2C, H->chunk_ptr, H->chunk_len,
                                                    H->perm, H->col, static_cast<const double2 *>(H->val),
                                                    rowptr, col, static_cast<double2 *>(val));
    else
        k_csr_fill<float2><<<grid, T, 0, stream>>>(H->n_rows, log2C, H->chunk_ptr, H->chunk_len,
                                                   H->perm, H->col, static_cast<const float2 *>(H->val),
                                                   rowptr, col, static_cast<float2 *>(val));
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

}  // extern "C"
