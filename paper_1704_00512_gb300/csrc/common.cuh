// Shared internals of libcheb.so: error state, launch checks, small device helpers.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/cheb.h"

namespace cheb {

constexpr int BS = 4;   // basis functions per atom = block edge
constexpr int BB = 16;  // elements per block

// Thread-local message of the last failure, returned by cheb_last_error().
std::string &last_error();

int fail(int code, const char *fmt, ...);

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Checks the launch(es) that just happened on this thread and counts them
// (cheb_launch_count).
int check_launch(const char *what, int n_launches = 1);

#define CHEB_CUDA(call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return ::cheb::fail(CHEB_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define CHEB_TRY(expr)             \
    do {                           \
        int rc_ = (expr);          \
        if (rc_ != CHEB_OK) return rc_; \
    } while (0)

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Bump allocator over caller-provided workspace.
struct Carve {
    char *base;
    size_t cap;
    size_t off = 0;
    Carve(void *b, size_t c) : base(static_cast<char *>(b)), cap(c) {}
    template <typename T>
    T *take(size_t n) {
        off = align_up(off);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += n * sizeof(T);
        return p;
    }
    bool fits() const { return off <= cap; }
};

// ---------------------------------------------------------------------------
// device helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed tree), result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT / 32; ++i) r += sh[i];
    }
    __syncthreads();
    return r;
}

// Index of block (row, col) in a sorted block-CSR row, or -1.
__device__ __forceinline__ int64_t find_in_row(const int64_t *rp, const int32_t *ci, int64_t row,
                                               int32_t col) {
    int64_t lo = rp[row], hi = rp[row + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        int32_t c = ci[mid];
        if (c == col) return mid;
        if (c < col) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// Block row of block index b (binary search in row_ptr).
__device__ __forceinline__ int64_t row_of(const int64_t *rp, int64_t nbr, int64_t b) {
    int64_t lo = 0, hi = nbr - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (rp[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace cheb
