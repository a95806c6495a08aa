// Shared internals of libcfd: error reporting, complex helpers, SELL view.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "../../include/cfd.h"

namespace cfd {

// ---------------------------------------------------------------- errors --

// Records a message for cfd_last_error() on the calling thread and returns st.
cfd_status fail(cfd_status st, const char *fmt, ...);
void clear_error();

#define CFD_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return ::cfd::fail(CFD_ERR_CUDA, "%s failed: %s (%s:%d)", #call,         \
                               cudaGetErrorString(e_), __FILE__, __LINE__);         \
    } while (0)

#define CFD_LAUNCH_CHECK()                                                          \
    do {                                                                            \
        cudaError_t e_ = cudaGetLastError();                                        \
        if (e_ != cudaSuccess)                                                      \
            return ::cfd::fail(CFD_ERR_CUDA, "kernel launch failed: %s (%s:%d)",    \
                               cudaGetErrorString(e_), __FILE__, __LINE__);         \
    } while (0)

#define CFD_TRY(expr)                                                               \
    do {                                                                            \
        cfd_status s_ = (expr);                                                     \
        if (s_ != CFD_OK) return s_;                                                \
    } while (0)

// Every kernel the library launches is counted (cfd_launch_count()).
void count_launch();
// Adds n (negative: removes) kernels to the count; the current count.
void count_launches(long long n);
unsigned long long launch_count();
#define CFD_COUNT_LAUNCH() ::cfd::count_launch()

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over a caller-provided scratch buffer (256-byte aligned
// sub-buffers).  Used to carve workspaces; never allocates.
// CUDA events timing the phases of a solve iteration, created once and
// destroyed on every exit path (error returns included).
struct PhaseEvents {
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaError_t create() {
        for (auto &x : e) {
            cudaError_t st = cudaEventCreate(&x);
            if (st != cudaSuccess) return st;
        }
        return cudaSuccess;
    }
    float ms(int a, int b) const {
        float t = 0.f;
        cudaEventElapsedTime(&t, e[a], e[b]);
        return t;
    }
    PhaseEvents() = default;
    PhaseEvents(const PhaseEvents &) = delete;
    PhaseEvents &operator=(const PhaseEvents &) = delete;
    ~PhaseEvents() {
        for (auto x : e)
            if (x) cudaEventDestroy(x);
    }
};

struct Carve {
    char *base;
    size_t cap, off = 0;
    Carve(void *b, size_t c) : base(static_cast<char *>(b)), cap(c) {}
    template <typename T>
    T *take(size_t count) {
        off = round_up(off, 256);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
    bool fits() const { return off <= cap; }
};

// Number of SMs of the current device (cached per device).
int sm_count();

// ----------------------------------------------------------- complex math --

template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };
template <typename T> using cplx_t = typename cplx<T>::type;

template <typename T>
__device__ __forceinline__ cplx_t<T> cmake(T re, T im) {
    cplx_t<T> z;
    z.x = re;
    z.y = im;
    return z;
}

// acc += h * v (complex), four fused multiply-adds.
template <typename C>
__device__ __forceinline__ void cfma(C &acc, const C h, const C v) {
    acc.x = fma(h.x, v.x, acc.x);
    acc.x = fma(-h.y, v.y, acc.x);
    acc.y = fma(h.x, v.y, acc.y);
    acc.y = fma(h.y, v.x, acc.y);
}

// ------------------------------------------------------------ SELL view --

template <typename T>
struct SellView {
    const cplx_t<T> *val;     // complex values (packed == false)
    const T *pval;            // packed: one real scalar per slot (packed == true)
    bool packed;
    const int32_t *col;
    const int64_t *chunk_ptr;
    const int32_t *chunk_len;  // packed: real slot count | imaginary slot count << 16
    const int32_t *perm;  // sorted row -> canonical row, nullptr when sigma == 1
    int64_t n_rows;
    int log2C;
    int slots_bound;          // upper bound on slots per row of any chunk (0: unknown)
};

template <typename T>
inline SellView<T> sell_view(const cfd_matrix *H) {
    SellView<T> v;
    v.packed = (H->flags & CFD_MATRIX_PACKED) != 0;
    v.val = v.packed ? nullptr : static_cast<const cplx_t<T> *>(H->val);
    v.pval = v.packed ? static_cast<const T *>(H->val) : nullptr;
    v.col = H->col;
    v.chunk_ptr = H->chunk_ptr;
    v.chunk_len = H->chunk_len;
    v.perm = H->perm;
    v.n_rows = H->n_rows;
    int l = 0;
    while ((1 << l) < H->C) ++l;
    v.log2C = l;
    v.slots_bound = (H->flags >> CFD_MATRIX_SLOTS_SHIFT) & 0xff;
    return v;
}

cfd_status check_matrix(const cfd_matrix *H);

// Exclusive scan of n int64 values into n + 1 outputs: out[0] = 0,
// out[i + 1] = sum in[0..i].  in and out must not overlap.
// work: scan_workspace(n) bytes.
size_t scan_workspace(int64_t n);
cfd_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, void *work,
                              cudaStream_t stream);

}  // namespace cfd
