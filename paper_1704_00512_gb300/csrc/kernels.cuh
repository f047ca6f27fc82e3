// Device helpers shared by the recursion kernels (expand.cu, resident.cu).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace cheb {

constexpr int MAX_F = 8;  // accumulators (functions / mu values) per expansion

// ---------------------------------------------------------------------------
// Double-float: a value carried as the unevaluated sum hi + lo of two floats
// (|lo| <= ulp(hi)/2 when normalised), about 48 significant bits, with every
// operation on the FP32 pipe.  Building blocks: Knuth's TwoSum (the exact
// rounding error of a + b in six additions, no ordering needed), the fast
// two-sum for |a| >= |b| (Dekker 1971, three additions) and the exact product
// error fma(a, b, -a*b).  GB300 runs FP64 FMA at 1/64 of the FP32 rate, so
// FP64-accurate block products are cheaper this way.
struct __align__(8) dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ dfl(int v) : hi((float)v), lo(0.f) {}
    __device__ __forceinline__ dfl(double v) {
        hi = __double2float_rn(v);
        lo = __double2float_rn(v - (double)hi);
    }
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return dfl(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
    const float s = a + b;
    return dfl(s, b - (s - a));
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const dfl s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));  // lo * lo (2^-48 relative) dropped
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfl &operator+=(dfl &a, dfl b) { return a = a + b; }

// acc + h x for the long sums of the block products: the product's exact
// error and cross terms and the sum's TwoSum error collect in lo, which is
// left unnormalised (the next TwoSum on hi is exact for any magnitudes); the
// row-end additions normalise.
__device__ __forceinline__ dfl mac(dfl h, dfl x, dfl acc) {
    const float p = h.hi * x.hi;
    float e = fmaf(h.hi, x.hi, -p);
    e = fmaf(h.hi, x.lo, fmaf(h.lo, x.hi, e));
    const dfl s = df_two_sum(acc.hi, p);
    return dfl(s.hi, s.lo + (acc.lo + e));
}
__device__ __forceinline__ float mac(float h, float x, float acc) { return fmaf(h, x, acc); }
__device__ __forceinline__ double mac(double h, double x, double acc) { return fma(h, x, acc); }

__device__ __forceinline__ float shfl_xor_t(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double shfl_xor_t(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ dfl shfl_xor_t(dfl v, int m) {
    return dfl(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

// two consecutive double-floats <-> one 16-byte vector
__device__ __forceinline__ void df_unpack(dfl &a, dfl &b, float4 v) {
    a = dfl(v.x, v.y);
    b = dfl(v.z, v.w);
}
__device__ __forceinline__ float4 df_pack(dfl a, dfl b) { return make_float4(a.hi, a.lo, b.hi, b.lo); }

template <typename T>
__device__ __forceinline__ void load16(T (&h)[16], const T *p);
template <>
__device__ __forceinline__ void load16<float>(float (&h)[16], const float *p) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float4 v = __ldg(q + i);
        h[4 * i] = v.x; h[4 * i + 1] = v.y; h[4 * i + 2] = v.z; h[4 * i + 3] = v.w;
    }
}
template <>
__device__ __forceinline__ void load16<double>(double (&h)[16], const double *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        double2 v = __ldg(q + i);
        h[2 * i] = v.x; h[2 * i + 1] = v.y;
    }
}

template <>
__device__ __forceinline__ void load16<dfl>(dfl (&h)[16], const dfl *p) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < 8; ++i) df_unpack(h[2 * i], h[2 * i + 1], __ldg(q + i));
}

template <typename T>
__device__ __forceinline__ void lds4(T (&x)[4], const T *p);
template <>
__device__ __forceinline__ void lds4<float>(float (&x)[4], const float *p) {
    float4 v = *reinterpret_cast<const float4 *>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
template <>
__device__ __forceinline__ void lds4<double>(double (&x)[4], const double *p) {
    double2 a = *reinterpret_cast<const double2 *>(p);
    double2 b = *reinterpret_cast<const double2 *>(p + 2);
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
}

template <>
__device__ __forceinline__ void lds4<dfl>(dfl (&x)[4], const dfl *p) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    df_unpack(x[0], x[1], q[0]);
    df_unpack(x[2], x[3], q[1]);
}

// 16-byte asynchronous global->shared copy (sm_80+ cp.async, L2 only).
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T>
__device__ __forceinline__ void lds16(T (&h)[16], const T *p);
template <>
__device__ __forceinline__ void lds16<float>(float (&h)[16], const float *p) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 v = reinterpret_cast<const float4 *>(p)[i];
        h[4 * i] = v.x; h[4 * i + 1] = v.y; h[4 * i + 2] = v.z; h[4 * i + 3] = v.w;
    }
}
template <>
__device__ __forceinline__ void lds16<double>(double (&h)[16], const double *p) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const double2 v = reinterpret_cast<const double2 *>(p)[i];
        h[2 * i] = v.x; h[2 * i + 1] = v.y;
    }
}

__device__ __forceinline__ int rank_of(const uint2 *bits, int K) {
    const uint2 w = bits[K >> 5];
    const unsigned bit = 1u << (K & 31);
    if (!(w.x & bit)) return -1;
    return (int)w.y + __popc(w.x & (bit - 1u));
}

// Exclusive block scan of one int per thread; returns the prefix, *total = sum.
template <int NW>
__device__ __forceinline__ int block_excl_scan(int v, int *wsum, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int x = lane < NW ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int n = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += n;
        }
        if (lane < NW) wsum[lane] = x;
    }
    __syncthreads();
    const int excl = incl - v + (warp > 0 ? wsum[warp - 1] : 0);
    *total = wsum[NW - 1];
    __syncthreads();
    return excl;
}

template <int NV>
struct Moments {
    double v[NV];    // this thread's partial sums
    double *dst[NV];  // device scalars receiving the totals (NULL = not wanted)
};

// Deterministic sum of the per-block partials by the last block to finish.
template <int NT, int NV>
__device__ __forceinline__ void finish_moments(double *part, int32_t *counter, const Moments<NV> m, double *red) {
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double w = warp_sum(m.v[i]);
        if (lane == 0) red[warp * NV + i] = w;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += red[w * NV + i];
            part[(int64_t)blockIdx.x * NV + i] = s;
        }
        __threadfence();
        const int prev = atomicAdd(counter, 1);
        s_last = prev == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += NT) {
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += __ldcg(part + (int64_t)b * NV + i);
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double w = warp_sum(acc[i]);
        if (lane == 0) red[warp * NV + i] = w;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += red[w * NV + i];
            if (m.dst[i]) *m.dst[i] = s;
        }
        *counter = 0;
        __threadfence();
    }
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    static __device__ __forceinline__ void ld(float (&v)[4], const float *p) {
        float4 a = *reinterpret_cast<const float4 *>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    static __device__ __forceinline__ void ldg(float (&v)[4], const float *p) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    static __device__ __forceinline__ void st(float *p, const float (&v)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct Vec4<double> {
    static __device__ __forceinline__ void ld(double (&v)[4], const double *p) {
        double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void ldg(double (&v)[4], const double *p) {
        double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p + 2));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void st(double *p, const double (&v)[4]) {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
    }
};

template <>
struct Vec4<dfl> {
    static __device__ __forceinline__ void ld(dfl (&v)[4], const dfl *p) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
        df_unpack(v[0], v[1], q[0]);
        df_unpack(v[2], v[3], q[1]);
    }
    static __device__ __forceinline__ void ldg(dfl (&v)[4], const dfl *p) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
        df_unpack(v[0], v[1], __ldg(q));
        df_unpack(v[2], v[3], __ldg(q + 1));
    }
    static __device__ __forceinline__ void st(dfl *p, const dfl (&v)[4]) {
        float4 *q = reinterpret_cast<float4 *>(p);
        q[0] = df_pack(v[0], v[1]);
        q[1] = df_pack(v[2], v[3]);
    }
};

// N = 1, 2 or 4 consecutive elements at p (aligned to N elements): plain load,
// read-only load and store.
template <typename T, int N>
__device__ __forceinline__ void ldn(T (&v)[N], const T *p) {
    if constexpr (N == 4) {
        Vec4<T>::ld(v, p);
    } else if constexpr (N == 2 && std::is_same_v<T, dfl>) {
        df_unpack(v[0], v[1], *reinterpret_cast<const float4 *>(p));
    } else if constexpr (N == 2) {
        if constexpr (sizeof(T) == 4) {
            const float2 a = *reinterpret_cast<const float2 *>(p);
            v[0] = a.x; v[1] = a.y;
        } else {
            const double2 a = *reinterpret_cast<const double2 *>(p);
            v[0] = a.x; v[1] = a.y;
        }
    } else {
        v[0] = *p;
    }
}
template <typename T, int N>
__device__ __forceinline__ void ldgn(T (&v)[N], const T *p) {
    if constexpr (N == 4) {
        Vec4<T>::ldg(v, p);
    } else if constexpr (N == 2 && std::is_same_v<T, dfl>) {
        df_unpack(v[0], v[1], __ldg(reinterpret_cast<const float4 *>(p)));
    } else if constexpr (N == 1 && std::is_same_v<T, dfl>) {
        const float2 a = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = dfl(a.x, a.y);
    } else if constexpr (N == 2) {
        if constexpr (sizeof(T) == 4) {
            const float2 a = __ldg(reinterpret_cast<const float2 *>(p));
            v[0] = a.x; v[1] = a.y;
        } else {
            const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
            v[0] = a.x; v[1] = a.y;
        }
    } else {
        v[0] = __ldg(p);
    }
}
template <typename T, int N>
__device__ __forceinline__ void stn(T *p, const T (&v)[N]) {
    if constexpr (N == 4) {
        Vec4<T>::st(p, v);
    } else if constexpr (N == 2 && std::is_same_v<T, dfl>) {
        *reinterpret_cast<float4 *>(p) = df_pack(v[0], v[1]);
    } else if constexpr (N == 2) {
        if constexpr (sizeof(T) == 4)
            *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
        else
            *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    } else {
        *p = v[0];
    }
}

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

// Byte offset of 16-byte chunk c of panel block b (XOR-swizzled inside its
// 128-byte line so 32 lanes reading chunk c of 32 blocks spread over the banks).
template <typename T>
__device__ __forceinline__ int rchunk(int b, int c);
template <>
__device__ __forceinline__ int rchunk<float>(int b, int c) {
    const int line = b >> 1;
    return line * 128 + ((((b & 1) << 2) | c) ^ (line & 7)) * 16;
}
template <>
__device__ __forceinline__ int rchunk<double>(int b, int c) {
    return b * 128 + ((c ^ b) & 7) * 16;
}

template <>
__device__ __forceinline__ int rchunk<dfl>(int b, int c) {
    return b * 128 + ((c ^ b) & 7) * 16;
}

template <typename T>
__device__ __forceinline__ void r_ld(T (&x)[16], const unsigned char *B, int b);
template <>
__device__ __forceinline__ void r_ld<float>(float (&x)[16], const unsigned char *B, int b) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 v = *reinterpret_cast<const float4 *>(B + rchunk<float>(b, c));
        x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
    }
}
template <>
__device__ __forceinline__ void r_ld<double>(double (&x)[16], const unsigned char *B, int b) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const double2 v = *reinterpret_cast<const double2 *>(B + rchunk<double>(b, c));
        x[2 * c] = v.x; x[2 * c + 1] = v.y;
    }
}

template <>
__device__ __forceinline__ void r_ld<dfl>(dfl (&x)[16], const unsigned char *B, int b) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
        df_unpack(x[2 * c], x[2 * c + 1], *reinterpret_cast<const float4 *>(B + rchunk<dfl>(b, c)));
}

}  // namespace cheb
