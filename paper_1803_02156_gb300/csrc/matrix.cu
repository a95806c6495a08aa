// Topological-insulator Hamiltonian (Sect. 2.1) built on the device directly
// into SELL-C-sigma, and canonical CSR export.
#include <vector>

#include "common.cuh"

namespace cfd {
namespace {

constexpr int TOPI_MAX_ROW = 13;

struct Lattice {
    int32_t L[3];
    int32_t per[3];
    int64_t n_rows;
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
    for (int64_t i = r0; i < r1; ++i) ++cnt[topi_row_len(i, g)];
    int start[TOPI_MAX_ROW + 1];
    int run = 0;
    for (int k = TOPI_MAX_ROW; k >= 0; --k) {
        start[k] = run;
        run += cnt[k];
    }
    for (int64_t i = r0; i < r1; ++i) perm[r0 + start[topi_row_len(i, g)]++] = (int32_t)i;
}

__global__ void k_chunk_len(Lattice g, int log2C, int64_t n_chunks, const int32_t *perm,
                            int32_t *chunk_len, int64_t *slots) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    int C = 1 << log2C;
    int mx = 0;
    for (int rr = 0; rr < C; ++rr) {
        int64_t r = (c << log2C) + rr;
        if (r >= g.n_rows) break;
        int64_t i = perm ? perm[r] : r;
        mx = max(mx, topi_row_len(i, g));
    }
    chunk_len[c] = mx;
    slots[c] = (int64_t)mx << log2C;
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
    if (r < g.n_rows) n = topi_row(perm ? perm[r] : r, g, v, ec, ev);
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

// CSR export: row lengths of canonical rows, then entries.
__global__ void k_csr_len(int64_t n_rows, int log2C, const int64_t *chunk_ptr,
                          const int32_t *chunk_len, const int32_t *perm, const int32_t *col,
                          int64_t *rowlen) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    int64_t c = r >> log2C;
    int64_t base = chunk_ptr[c] + (r & ((1 << log2C) - 1));
    int n = 0;
    for (int k = 0; k < chunk_len[c]; ++k)
        if (col[base + ((int64_t)k << log2C)] >= 0) ++n;
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

// Host replica of the chunk lengths (for sizes, no GPU work): after the
// stable descending sort inside each window, chunk c's length is that of its
// first row.
int64_t host_slots(const Lattice &g, int C, int sigma) {
    int64_t n_chunks = (g.n_rows + C - 1) / C;
    int64_t slots = 0;
    if (sigma == 1) {
        for (int64_t c = 0; c < n_chunks; ++c) {
            int mx = 0;
            for (int64_t i = c * C; i < std::min<int64_t>((c + 1) * C, g.n_rows); ++i)
                mx = std::max(mx, topi_row_len(i, g));
            slots += (int64_t)mx * C;
        }
        return slots;
    }
    std::vector<int> sorted;
    for (int64_t r0 = 0; r0 < g.n_rows; r0 += sigma) {
        int64_t r1 = std::min<int64_t>(r0 + sigma, g.n_rows);
        int cnt[TOPI_MAX_ROW + 1] = {0};
        for (int64_t i = r0; i < r1; ++i) ++cnt[topi_row_len(i, g)];
        sorted.clear();
        for (int k = TOPI_MAX_ROW; k >= 0; --k)
            for (int q = 0; q < cnt[k]; ++q) sorted.push_back(k);
        for (size_t a = 0; a < sorted.size(); a += C) slots += (int64_t)sorted[a] * C;
    }
    return slots;
}

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" {

cfd_status cfd_matrix_query_size(const cfd_topi_params *p, int C, int sigma, int prec,
                                 cfd_matrix_sizes *out) {
    clear_error();
    CFD_TRY(check_params(p, C, sigma, prec));
    if (!out) return fail(CFD_ERR_ARG, "out is NULL");
    Lattice g = lattice_of(p);
    int64_t nnz = 0;
    for (int64_t i = 0; i < g.n_rows; i += 4) nnz += 4 * topi_row_len(i, g);
    int64_t n_chunks = (g.n_rows + C - 1) / C;
    int64_t slots = host_slots(g, C, sigma);
    size_t s = (prec == CFD_C128) ? 16 : 8;
    out->n_rows = g.n_rows;
    out->nnz = nnz;
    out->n_chunks = n_chunks;
    out->n_slots = slots;
    out->bytes_val = (int64_t)round_up((size_t)slots * s, 256);
    out->bytes_col = (int64_t)round_up((size_t)slots * 4, 256);
    out->bytes_chunk_ptr = (int64_t)round_up((size_t)(n_chunks + 1) * 8, 256);
    out->bytes_chunk_len = (int64_t)round_up((size_t)n_chunks * 4, 256);
    out->bytes_perm = sigma > 1 ? (int64_t)round_up((size_t)g.n_rows * 4, 256) : 0;
    out->bytes_work = (int64_t)(round_up((size_t)n_chunks * 8, 256) + scan_workspace(n_chunks));
    return CFD_OK;
}

cfd_status cfd_build_matrix(const cfd_topi_params *p, int C, int sigma, int prec,
                            const cfd_matrix_buffers *buf, cfd_matrix *out, cudaStream_t stream) {
    cfd_matrix_sizes sz;
    CFD_TRY(cfd_matrix_query_size(p, C, sigma, prec, &sz));
    if (!buf || !out) return fail(CFD_ERR_ARG, "buffers or out is NULL");
    if (!buf->val || !buf->col || !buf->chunk_ptr || !buf->chunk_len || !buf->work ||
        (sigma > 1 && !buf->perm))
        return fail(CFD_ERR_ARG, "a required matrix buffer is NULL");
    if (!aligned16(buf->val) || !aligned16(buf->col) || !aligned16(buf->chunk_ptr) ||
        !aligned16(buf->chunk_len) || !aligned16(buf->work) || (buf->perm && !aligned16(buf->perm)))
        return fail(CFD_ERR_ARG, "matrix buffers must be 16-byte aligned");
    Lattice g = lattice_of(p);
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
    }
    k_chunk_len<<<(unsigned)((sz.n_chunks + T - 1) / T), T, 0, stream>>>(g, log2C, sz.n_chunks, perm,
                                                                          chunk_len, slots);
    CFD_LAUNCH_CHECK();
    CFD_TRY(exclusive_scan_i64(slots, chunk_ptr, sz.n_chunks, scan_work, stream));
    int64_t rows_pad = sz.n_chunks << log2C;
    unsigned grid = (unsigned)((rows_pad + T - 1) / T);
    if (prec == CFD_C128)
        k_fill<double2><<<grid, T, 0, stream>>>(g, v, log2C, sz.n_chunks, perm, chunk_ptr, chunk_len,
                                                static_cast<int32_t *>(buf->col),
                                                static_cast<double2 *>(buf->val));
    else
        k_fill<float2><<<grid, T, 0, stream>>>(g, v, log2C, sz.n_chunks, perm, chunk_ptr, chunk_len,
                                               static_cast<int32_t *>(buf->col),
                                               static_cast<float2 *>(buf->val));
    CFD_LAUNCH_CHECK();
    out->n_rows = sz.n_rows;
    out->nnz = sz.nnz;
    out->n_chunks = sz.n_chunks;
    out->n_slots = sz.n_slots;
    out->C = C;
    out->sigma = sigma;
    out->prec = prec;
    out->reserved = 0;
    out->val = buf->val;
    out->col = static_cast<int32_t *>(buf->col);
    out->chunk_ptr = chunk_ptr;
    out->chunk_len = chunk_len;
    out->perm = perm;
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
                                      rowlen);
    CFD_LAUNCH_CHECK();
    CFD_TRY(exclusive_scan_i64(rowlen, rowptr, H->n_rows, scan_work, stream));
    if (H->prec == CFD_C128)
        k_csr_fill<double2><<<grid, T, 0, stream>>>(H->n_rows, log2C, H->chunk_ptr, H->chunk_len,
                                                    H->perm, H->col, static_cast<const double2 *>(H->val),
                                                    rowptr, col, static_cast<double2 *>(val));
    else
        k_csr_fill<float2><<<grid, T, 0, stream>>>(H->n_rows, log2C, H->chunk_ptr, H->chunk_len,
                                                   H->perm, H->col, static_cast<const float2 *>(H->val),
                                                   rowptr, col, static_cast<float2 *>(val));
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

}  // extern "C"
