// Status strings, per-thread error messages, device queries, prefix scan.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>

#include "common.cuh"

namespace cfd {

static thread_local char g_last_error[512] = {0};
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

cfd_status fail(cfd_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

void clear_error() { g_last_error[0] = 0; }

int sm_count() {
    static std::atomic<int> cached[64] = {};   // per device, 0 until first asked
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int n = cached[dev].load();
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
        cached[dev].store(n);
    }
    return n;
}

cfd_status check_matrix(const cfd_matrix *H) {
    if (!H) return fail(CFD_ERR_ARG, "matrix is NULL");
    if (H->n_rows < 1 || H->n_chunks < 1 || !H->val || !H->col || !H->chunk_ptr || !H->chunk_len)
        return fail(CFD_ERR_ARG, "matrix is not built");
    if (H->C < 4 || H->C > 128 || (H->C & (H->C - 1)))
        return fail(CFD_ERR_ARG, "matrix chunk height C=%d invalid", H->C);
    if (H->prec != CFD_C128 && H->prec != CFD_C64)
        return fail(CFD_ERR_ARG, "matrix precision %d invalid", H->prec);
    if (H->sigma > 1 && !H->perm) return fail(CFD_ERR_ARG, "sigma > 1 needs perm");
    return CFD_OK;
}

// ------------------------------------------------------------------ scan --

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide inclusive scan of one value per thread (Hillis-Steele in smem).
__device__ int64_t block_inclusive_scan(int64_t v, int64_t *sm) {
    int t = threadIdx.x;
    sm[t] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_THREADS; off <<= 1) {
        int64_t a = (t >= off) ? sm[t - off] : 0;
        __syncthreads();
        sm[t] += a;
        __syncthreads();
    }
    int64_t r = sm[t];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_tile_sums(const int64_t *in, int64_t n,
                                                               int64_t *tile_sum) {
    __shared__ int64_t sm[SCAN_THREADS];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) s += in[base + k];
    int64_t inc = block_inclusive_scan(s, sm);
    if (threadIdx.x == SCAN_THREADS - 1) tile_sum[blockIdx.x] = inc;
}

// One CTA: exclusive scan of the tile sums in place (any count, carried).
__global__ void __launch_bounds__(SCAN_THREADS) scan_tile_offsets(int64_t *tile_sum, int64_t n_tiles) {
    __shared__ int64_t sm[SCAN_THREADS];
    __shared__ int64_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t start = 0; start < n_tiles; start += SCAN_THREADS) {
        int64_t i = start + threadIdx.x;
        int64_t v = (i < n_tiles) ? tile_sum[i] : 0;
        int64_t inc = block_inclusive_scan(v, sm);
        int64_t carry = carry_s;
        if (i < n_tiles) tile_sum[i] = carry + inc - v;
        __syncthreads();
        if (threadIdx.x == SCAN_THREADS - 1) carry_s = carry + inc;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_apply(const int64_t *in, int64_t n,
                                                           const int64_t *tile_off, int64_t *out) {
    __shared__ int64_t sm[SCAN_THREADS];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int64_t inc = block_inclusive_scan(s, sm);
    int64_t run = tile_off[blockIdx.x] + inc - s;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
        if (base + k == n - 1) out[n] = run;
    }
}

size_t scan_workspace(int64_t n) {
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return round_up((size_t)(tiles + 1) * sizeof(int64_t), 256);
}

cfd_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, void *work,
                              cudaStream_t stream) {
    if (n <= 0) {
        CFD_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), stream));
        return CFD_OK;
    }
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int64_t *ts = static_cast<int64_t *>(work);
    scan_tile_sums<<<(unsigned)tiles, SCAN_THREADS, 0, stream>>>(in, n, ts);
    CFD_COUNT_LAUNCH();
    scan_tile_offsets<<<1, SCAN_THREADS, 0, stream>>>(ts, tiles);
    CFD_COUNT_LAUNCH();
    scan_apply<<<(unsigned)tiles, SCAN_THREADS, 0, stream>>>(in, n, ts, out);
    CFD_COUNT_LAUNCH();
    CFD_LAUNCH_CHECK();
    return CFD_OK;
}

}  // namespace cfd

extern "C" {

const char *cfd_status_string(int status) {
    switch (status) {
    case CFD_OK: return "CFD_OK";
    case CFD_ERR_ARG: return "CFD_ERR_ARG";
    case CFD_ERR_CUDA: return "CFD_ERR_CUDA";
    case CFD_ERR_OOM: return "CFD_ERR_OOM";
    case CFD_ERR_BOUNDS: return "CFD_ERR_BOUNDS";
    case CFD_ERR_TIMEOUT: return "CFD_ERR_TIMEOUT";
    case CFD_ERR_NOCONV: return "CFD_ERR_NOCONV";
    case CFD_ERR_INTERNAL: return "CFD_ERR_INTERNAL";
    default: return "CFD_ERR_UNKNOWN";
    }
}

const char *cfd_last_error(void) { return cfd::g_last_error; }

const char *cfd_version(void) { return "1.0.0"; }

unsigned long long cfd_launch_count(void) { return cfd::g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
