// The whole Chebyshev expansion in one launch: every thread block owns a panel
// of block columns and runs all recursion steps for it with T_k and T_{k-1}
// resident in shared memory.
//
// Column J of T_{k+1} = 2 M~ T_k - T_{k-1} needs only column J of T_k and
// T_{k-1} (Sec. "Expansion in Chebyshev polynomials": the columns of the
// Chebyshev matrix polynomials follow their own recursion), so a panel never
// needs data another thread block writes: there is no grid-wide barrier and no
// wait of any kind.  Per step the panel reads only the operator M~ (its union
// rows, from L2/HBM) and read-modify-writes its blocks of the FP64 accumulators;
// T_k never goes to HBM.  Systems of a block-diagonal batch are panels with
// their own term count and coefficients, so one launch expands them all.
//
// Per thread block:
//   A. the union of the panel's row lists (bitmap + prefix popcounts), the
//      position of every panel block, and its global slot;
//   B. T_0 = I and T_1 = M~ on the panel's blocks, accumulators
//      c_0/2 T_0 + c_1 T_1, moments of terms 0 and 1;
//   C. for k = 1 .. n-2: masked products of the union rows with the panel's
//      T_k (lanes: P panel columns x 32/P K-groups, 4x4 block products,
//      butterfly over K-groups) giving T_{k+1} = 2 M~ T_k - T_{k-1} in place of
//      T_{k-1}; then every panel block adds c_j[k+1] T_{k+1} to accumulator j
//      and the moments Tr T_{k+1}, <T_{k+1}, G> are written per panel and step;
//   D. a second kernel sums the per-panel moments of each system and step in
//      a fixed order (deterministic).
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "plan.cuh"

namespace cheb {

template <typename T>
struct ResArgs {
    int64_t nw;
    int32_t ucap, bcap;
    const int64_t *rp;
    const int32_t *ci;
    const int32_t *tperm;
    const int32_t *panels;
    const int32_t *panel_sys;
    const int64_t *Lrp;
    const int32_t *Lci;
    const T *Lv;
    const int32_t *n_terms;  // per system, or NULL: n_single for every panel
    int32_t n_single;
    const double *coef;       // coef[coef_off[sys] + f * coef_stride + k]
    const int64_t *coef_off;  // per system, or NULL (offset 0)
    int32_t coef_stride;
    int32_t nf;
    double *acc[MAX_F];
    const double *G;
    double *part;  // [panel][kmax][2] moment partials
    int32_t kmax;
    // operator row lists of the resident panels (NULL: rank the operator rows)
    const int64_t *lrow_base;
    const int32_t *lrow_ptr;
    const uint32_t *lent;
    int32_t round_bf16;  // CHEB_BF16: every stored T_{k+1} rounded to bfloat16
};

__device__ __forceinline__ float res_round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ double res_round_bf16(double x) { return x; }
__device__ __forceinline__ dfl res_round_bf16(dfl x) { return x; }

template <typename T>
__device__ __forceinline__ void r_st(unsigned char *B, int b, const T (&x)[16]);
template <>
__device__ __forceinline__ void r_st<float>(unsigned char *B, int b, const float (&x)[16]) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<float4 *>(B + rchunk<float>(b, c)) = make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
}
template <>
__device__ __forceinline__ void r_st<double>(unsigned char *B, int b, const double (&x)[16]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) *reinterpret_cast<double2 *>(B + rchunk<double>(b, c)) = make_double2(x[2 * c], x[2 * c + 1]);
}
template <>
__device__ __forceinline__ void r_st<dfl>(unsigned char *B, int b, const dfl (&x)[16]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) *reinterpret_cast<float4 *>(B + rchunk<dfl>(b, c)) = df_pack(x[2 * c], x[2 * c + 1]);
}
// element i of panel block b
template <typename T>
__device__ __forceinline__ T *r_el(unsigned char *B, int b, int i) {
    constexpr int PER = 16 / sizeof(T);
    return reinterpret_cast<T *>(B + rchunk<T>(b, i / PER)) + (i % PER);
}
// row r (4 elements) of panel block b
template <typename T>
__device__ __forceinline__ void r_row(T (&y)[4], const unsigned char *B, int b, int r);
template <>
__device__ __forceinline__ void r_row<float>(float (&y)[4], const unsigned char *B, int b, int r) {
    const float4 v = *reinterpret_cast<const float4 *>(B + rchunk<float>(b, r));
    y[0] = v.x; y[1] = v.y; y[2] = v.z; y[3] = v.w;
}
template <>
__device__ __forceinline__ void r_row<double>(double (&y)[4], const unsigned char *B, int b, int r) {
    const double2 u = *reinterpret_cast<const double2 *>(B + rchunk<double>(b, 2 * r));
    const double2 v = *reinterpret_cast<const double2 *>(B + rchunk<double>(b, 2 * r + 1));
    y[0] = u.x; y[1] = u.y; y[2] = v.x; y[3] = v.y;
}
template <>
__device__ __forceinline__ void r_row<dfl>(dfl (&y)[4], const unsigned char *B, int b, int r) {
    df_unpack(y[0], y[1], *reinterpret_cast<const float4 *>(B + rchunk<dfl>(b, 2 * r)));
    df_unpack(y[2], y[3], *reinterpret_cast<const float4 *>(B + rchunk<dfl>(b, 2 * r + 1)));
}

// Deterministic thread-block sum of two values, written to dst[0..1] by thread 0.
template <int NT>
__device__ __forceinline__ void block_sum2(double t, double g, double *red, double *dst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    t = warp_sum(t);
    g = warp_sum(g);
    if (lane == 0) {
        red[2 * warp] = t;
        red[2 * warp + 1] = g;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double st = 0.0, sg = 0.0;
        for (int w = 0; w < NT / 32; ++w) {
            st += red[2 * w];
            sg += red[2 * w + 1];
        }
        dst[0] = st;
        dst[1] = sg;
    }
    __syncthreads();
}

template <typename T, int P, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_resident(const ResArgs<T> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int wsum[32];
    __shared__ int s_cb[P + 1];
    constexpr int NT = NW * 32;
    constexpr int KG = 32 / P;
    constexpr int NU = 32 / KG;
    constexpr int EPL = KG >= 16 ? 1 : 16 / KG;
    const ResLayout lay = res_layout(a.nw, a.ucap, a.bcap, P, sizeof(T), NW);
    uint2 *bits = reinterpret_cast<uint2 *>(smem + lay.off_bits);
    int32_t *ulist = reinterpret_cast<int32_t *>(smem + lay.off_ulist);
    int16_t *pos = reinterpret_cast<int16_t *>(smem + lay.off_pos);
    uint32_t *gslot = reinterpret_cast<uint32_t *>(smem + lay.off_gslot);
    int2 *wlist = reinterpret_cast<int2 *>(smem + lay.off_wl);
    unsigned char *Xb = smem + lay.off_x;
    unsigned char *Yb = smem + lay.off_y;
    double *red = reinterpret_cast<double *>(smem + lay.off_red);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int panel = blockIdx.x;
    const int sys = a.panel_sys[panel];
    const int n = a.n_terms ? a.n_terms[sys] : a.n_single;
    const double *coef = a.coef + (a.coef_off ? a.coef_off[sys] : 0);
    const int j0 = a.panels[2 * panel], ncols = a.panels[2 * panel + 1];
    double *part = a.part + (int64_t)panel * a.kmax * 2;

    // A. union of the panel's row lists
    for (int64_t w = tid; w < a.nw; w += NT) bits[w] = make_uint2(0u, 0u);
    if (tid == 0) {
        int c = 0;
        for (int q = 0; q < P; ++q) {
            s_cb[q] = c;
            if (q < ncols) c += (int)(a.rp[j0 + q + 1] - a.rp[j0 + q]);
        }
        s_cb[P] = c;
    }
    __syncthreads();
    for (int q = 0; q < ncols; ++q) {
        const int64_t b = a.rp[j0 + q], e = a.rp[j0 + q + 1];
        for (int64_t p = b + tid; p < e; p += NT) {
            const int K = a.ci[p];
            atomicOr(&bits[K >> 5].x, 1u << (K & 31));
        }
    }
    __syncthreads();
    const int64_t chunk = (a.nw + NT - 1) / NT;
    const int64_t wb = min(a.nw, (int64_t)tid * chunk), we = min(a.nw, wb + chunk);
    int cnt = 0;
    for (int64_t w = wb; w < we; ++w) cnt += __popc(bits[w].x);
    int total;
    int run = block_excl_scan<NW>(cnt, wsum, &total);
    for (int64_t w = wb; w < we; ++w) {
        unsigned m = bits[w].x;
        bits[w].y = (unsigned)run;
        while (m) {
            const int bpos = __ffs(m) - 1;
            ulist[run++] = (int)(w * 32 + bpos);
            m &= m - 1u;
        }
    }
    const int nu = total;
    const int nblk = s_cb[P];
    if (nu > a.ucap || nblk > a.bcap) return;  // cannot happen for a plan-built launch (uniform exit)
    for (int i = tid; i < nu * P; i += NT) pos[i] = -1;
    __syncthreads();

    // B. T_0 (in Y), T_1 (in X), accumulators and moments of terms 0 and 1
    {
        double c0[MAX_F], c1[MAX_F];
#pragma unroll
        for (int f = 0; f < MAX_F; ++f) {
            c0[f] = f < a.nf ? coef[(int64_t)f * a.coef_stride] : 0.0;
            c1[f] = f < a.nf ? coef[(int64_t)f * a.coef_stride + 1] : 0.0;
        }
        double t0 = 0.0, t1 = 0.0, g0 = 0.0, g1 = 0.0;
        for (int q = 0; q < ncols; ++q) {
            const int J = j0 + q;
            const int64_t pb = a.rp[J];
            for (int64_t p = pb + tid; p < a.rp[J + 1]; p += NT) {
                const int K = a.ci[p];
                const int e = (int)(p - pb);
                const int b = s_cb[q] + e;
                pos[rank_of(bits, K) * P + q] = (int16_t)e;
                const uint32_t gs = (uint32_t)a.tperm[p];
                gslot[b] = gs | (K == J ? 0x80000000u : 0u);
                const int64_t la = find_in_row(a.Lrp, a.Lci, K, J);
                T v0[16], v1[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    v0[i] = (K == J && (i % 5) == 0) ? T(1) : T(0);
                    v1[i] = la >= 0 ? a.Lv[la * BB + i] : T(0);
                }
                r_st<T>(Yb, b, v0);
                r_st<T>(Xb, b, v1);
                const int64_t idx = (int64_t)gs * BB;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const double d0 = (double)v0[i], d1 = (double)v1[i];
#pragma unroll
                    for (int f = 0; f < MAX_F; ++f)
                        if (f < a.nf) a.acc[f][idx + i] = 0.5 * c0[f] * d0 + c1[f] * d1;
                    if (a.G) {
                        g0 += a.G[idx + i] * d0;
                        g1 += a.G[idx + i] * d1;
                    }
                    if (K == J && (i % 5) == 0) {
                        t0 += d0;
                        t1 += d1;
                    }
                }
            }
        }
        block_sum2<NT>(t0, g0, red, part);
        block_sum2<NT>(t1, g1, red, part + 2);
    }

    // C. the recursion
    const int q = lane % P, kg = lane / P;
    const unsigned lt = (1u << lane) - 1u;
    int2 *wl = wlist + warp * 64;
    // With the plan's operator row lists the in-union entries of a row are read
    // from its list (the same entries in the same order as ranking gives);
    // otherwise the row's column indices are ranked against the bitmap.
    const int32_t *rptr = a.lrow_ptr ? a.lrow_ptr + a.lrow_base[panel] : nullptr;
    for (int k = 1; k + 1 < n; ++k) {
        for (int s = warp; s < nu; s += NW) {
            const int I = ulist[s];
            const int64_t a0 = a.Lrp[I], a1 = a.Lrp[I + 1];
            T acc[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = T(0);
            int pending = 0;
            int64_t base = rptr ? (int64_t)rptr[s] : a0;
            const int64_t end = rptr ? (int64_t)rptr[s + 1] : a1;
            int Knext = (!rptr && a0 + lane < a1) ? a.Lci[a0 + lane] : -1;
            uint32_t wnext = (rptr && base + lane < end) ? a.lent[base + lane] : 0u;
            while (true) {
                if (base < end) {
                    if (rptr) {
                        const int nn = end - base < 32 ? (int)(end - base) : 32;
                        const uint32_t w = wnext;
                        wnext = (base + 32 + lane < end) ? a.lent[base + 32 + lane] : 0u;
                        if (lane < nn) wl[pending + lane] = make_int2((int)(a0 + (w >> 16)), (int)(w & 0xffffu));
                        pending += nn;
                    } else {
                        const int K = Knext;
                        Knext = (base + 32 + lane < a1) ? a.Lci[base + 32 + lane] : -1;
                        const int s2 = K >= 0 ? rank_of(bits, K) : -1;
                        const unsigned vm = __ballot_sync(0xffffffffu, s2 >= 0);
                        if (s2 >= 0) wl[pending + __popc(vm & lt)] = make_int2((int)(base + lane), s2);
                        pending += __popc(vm);
                    }
                    base += 32;
                    __syncwarp();
                }
                const bool raw_done = base >= end;
                if (pending >= 32 || (raw_done && pending > 0)) {
                    const int nb = pending < 32 ? pending : 32;
                    int2 en[NU];
                    T h[NU][16];
#pragma unroll
                    for (int u = 0; u < NU; ++u) {
                        const int e = u * KG + kg;
                        en[u] = make_int2(-1, -1);
                        if (e < nb) {
                            const int2 w = wl[e];
                            const int eq = q < ncols ? pos[w.y * P + q] : -1;
                            if (eq >= 0) {
                                en[u] = make_int2(w.x, s_cb[q] + eq);
                                load16<T>(h[u], a.Lv + (int64_t)w.x * BB);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < NU; ++u) {
                        if (en[u].x < 0) continue;
                        T x[16];
                        r_ld<T>(x, Xb, en[u].y);
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int m = 0; m < 4; ++m)
#pragma unroll
                                for (int c = 0; c < 4; ++c)
                                    acc[4 * r + c] = mac(h[u][4 * r + m], x[4 * m + c], acc[4 * r + c]);
                    }
                    __syncwarp();
                    const int rest = pending - nb;
                    const int2 keep = lane < rest ? wl[nb + lane] : make_int2(0, 0);
                    __syncwarp();
                    if (lane < rest) wl[lane] = keep;
                    pending = rest;
                    __syncwarp();
                }
                if (raw_done && pending == 0) break;
            }
#pragma unroll
            for (int o = P; o < 32; o <<= 1)
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] += shfl_xor_t(acc[i], o);
            // T_{k+1} = 2 (M~ T_k) - T_{k-1}, in place of T_{k-1}, for the panel's blocks only
            if (q < ncols && kg * EPL < 16) {
                const int e = pos[s * P + q];
                if (e >= 0) {
                    const int b = s_cb[q] + e;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (i / EPL == kg) {
                            T *yp = r_el<T>(Yb, b, i);
                            const T v = T(2) * acc[i] - *yp;
                            *yp = a.round_bf16 ? res_round_bf16(v) : v;
                        }
                }
            }
        }
        __syncthreads();
        // accumulators and moments of term k+1
        double cf[MAX_F];
#pragma unroll
        for (int f = 0; f < MAX_F; ++f) cf[f] = f < a.nf ? coef[(int64_t)f * a.coef_stride + k + 1] : 0.0;
        double tp = 0.0, gp = 0.0;
        for (int t = tid; t < nblk * 4; t += NT) {
            const int b = t >> 2, r = t & 3;
            T y[4];
            r_row<T>(y, Yb, b, r);
            const uint32_t gs = gslot[b];
            const int64_t idx = (int64_t)(gs & 0x7fffffffu) * BB + 4 * r;
            double yd[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) yd[c] = (double)y[c];
#pragma unroll
            for (int f = 0; f < MAX_F; ++f) {
                if (f < a.nf) {
                    double v[4];
                    Vec4<double>::ld(v, a.acc[f] + idx);
#pragma unroll
                    for (int c = 0; c < 4; ++c) v[c] += cf[f] * yd[c];
                    Vec4<double>::st(a.acc[f] + idx, v);
                }
            }
            if (a.G) {
                double gv[4];
                Vec4<double>::ldg(gv, a.G + idx);
#pragma unroll
                for (int c = 0; c < 4; ++c) gp += gv[c] * yd[c];
            }
            if (gs & 0x80000000u) tp += yd[r];
        }
        block_sum2<NT>(tp, gp, red, part + (int64_t)(k + 1) * 2);
        unsigned char *tmp = Xb;
        Xb = Yb;
        Yb = tmp;
    }
}

// mom[sys_off + k] = sum over the system's panels of the partials (fixed order).
__global__ void k_res_moments(const double *part, int kmax, const int32_t *sys_panel, const int32_t *n_terms,
                              int n_single, int nsys, int mom_stride, double *mom, double *gmom) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int sy = blockIdx.y;
    if (sy >= nsys) return;
    const int n = n_terms ? n_terms[sy] : n_single;
    if (k >= n) return;
    double t = 0.0, g = 0.0;
    for (int p = sys_panel[sy]; p < sys_panel[sy + 1]; ++p) {
        t += part[((int64_t)p * kmax + k) * 2];
        g += part[((int64_t)p * kmax + k) * 2 + 1];
    }
    if (mom) mom[(int64_t)sy * mom_stride + k] = t;
    if (gmom) gmom[(int64_t)sy * mom_stride + k] = g;
}

__global__ void k_to_dfl_res(const double *in, dfl *out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = dfl(in[i]);
}

__global__ void k_to_f32_res(const double *in, float *out, int64_t n, int round_bf16) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = round_bf16 ? __bfloat162float(__float2bfloat16_rn(in[i])) : (float)in[i];
}

template <typename T, int P, int NW, int MINB>
int launch_resident(const cheb_plan *plan, const ResArgs<T> &a, cudaStream_t s) {
    const ResLayout lay = res_layout(a.nw, a.ucap, a.bcap, P, sizeof(T), NW);
    auto fn = k_resident<T, P, NW, MINB>;
    CHEB_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    fn<<<(unsigned)plan->n_rpanels, NW * 32, lay.total, s>>>(a);
    return check_launch("k_resident");
}

template <typename T>
int run_resident(const cheb_plan *plan, const ResArgs<T> &a, cudaStream_t s);
#define CHEB_RES_CASE(T, TABLE, i) \
    case i: return launch_resident<T, TABLE[i].P, TABLE[i].NW, TABLE[i].MINB>(plan, a, s);
template <>
int run_resident<double>(const cheb_plan *plan, const ResArgs<double> &a, cudaStream_t s) {
    static_assert(N_TILES_F64 == 5, "tile table size");
    switch (plan->tile) {
        CHEB_RES_CASE(double, TILES_F64, 0)
        CHEB_RES_CASE(double, TILES_F64, 1)
        CHEB_RES_CASE(double, TILES_F64, 2)
        CHEB_RES_CASE(double, TILES_F64, 3)
        CHEB_RES_CASE(double, TILES_F64, 4)
        default: return fail(CHEB_ERR_INVALID, "bad FP64 tile %d", plan->tile);
    }
}
template <>
int run_resident<dfl>(const cheb_plan *plan, const ResArgs<dfl> &a, cudaStream_t s) {
    switch (plan->tile) {
        CHEB_RES_CASE(dfl, TILES_F64, 0)
        CHEB_RES_CASE(dfl, TILES_F64, 1)
        CHEB_RES_CASE(dfl, TILES_F64, 2)
        CHEB_RES_CASE(dfl, TILES_F64, 3)
        CHEB_RES_CASE(dfl, TILES_F64, 4)
        default: return fail(CHEB_ERR_INVALID, "bad FP64 tile %d", plan->tile);
    }
}
template <>
int run_resident<float>(const cheb_plan *plan, const ResArgs<float> &a, cudaStream_t s) {
    static_assert(N_TILES_F32 == 6, "tile table size");
    switch (plan->tile) {
        CHEB_RES_CASE(float, TILES_F32, 0)
        CHEB_RES_CASE(float, TILES_F32, 1)
        CHEB_RES_CASE(float, TILES_F32, 2)
        CHEB_RES_CASE(float, TILES_F32, 3)
        CHEB_RES_CASE(float, TILES_F32, 4)
        CHEB_RES_CASE(float, TILES_F32, 5)
        default: return fail(CHEB_ERR_INVALID, "bad FP32 tile %d", plan->tile);
    }
}
#undef CHEB_RES_CASE

size_t resident_ws(const cheb_plan *plan, int64_t nnzL, int precision, int kmax) {
    size_t b = 0;
    if (precision != CHEB_F64) b += align_up(nnzL * BB * (precision == CHEB_F64X ? 8 : 4));
    b += align_up((size_t)plan->n_rpanels * kmax * 2 * sizeof(double));
    return b + 256;
}

template <typename T>
int resident_impl(const cheb_plan *plan, const cheb_bsr *Mt, int kmax, const int32_t *n_terms_dev, int n_single,
                  const double *coeffs, const int64_t *coef_off, int32_t stride, int32_t nf, double *const *acc,
                  double *moments, const double *G, double *gmoments, int mom_stride, void *ws, size_t ws_bytes,
                  cudaStream_t s, int round_bf16 = 0) {
    Carve cv(ws, ws_bytes);
    const T *Lv;
    const int64_t n = Mt->nnzb * BB;
    if constexpr (std::is_same_v<T, double>) {
        Lv = reinterpret_cast<const T *>(Mt->vals);
    } else if constexpr (std::is_same_v<T, dfl>) {
        dfl *lv = cv.take<dfl>(n);
        if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_expand: workspace too small");
        k_to_dfl_res<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double *)Mt->vals, lv, n);
        CHEB_TRY(check_launch("k_to_dfl"));
        Lv = lv;
    } else {
        float *lv = cv.take<float>(n);
        if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_expand: workspace too small");
        k_to_f32_res<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double *)Mt->vals, lv, n, round_bf16);
        CHEB_TRY(check_launch("k_to_f32"));
        Lv = reinterpret_cast<const T *>(lv);
    }
    double *part = cv.take<double>((size_t)plan->n_rpanels * kmax * 2);
    if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_expand: workspace too small");
    ResArgs<T> a{};
    a.nw = (plan->nbr + 31) / 32;
    a.ucap = plan->max_union_res;
    a.bcap = plan->max_nblk_res;
    a.rp = plan->rp;
    a.ci = plan->ci;
    a.tperm = plan->d_tperm;
    a.panels = plan->d_rpanels;
    a.panel_sys = plan->d_rpanel_sys;
    a.Lrp = Mt->row_ptr;
    a.Lci = Mt->col_idx;
    a.Lv = Lv;
    if (plan->op_bound && plan->op_rp == Mt->row_ptr && plan->op_ci == Mt->col_idx && plan->rlists.d_ptr) {
        a.lrow_base = plan->rlists.d_base;
        a.lrow_ptr = plan->rlists.d_ptr;
        a.lent = plan->rlists.d_ent;
    }
    a.n_terms = n_terms_dev;
    a.n_single = n_single;
    a.coef = coeffs;
    a.coef_off = coef_off;
    a.coef_stride = stride;
    a.nf = nf;
    for (int f = 0; f < nf; ++f) a.acc[f] = acc[f];
    a.G = G;
    a.part = part;
    a.kmax = kmax;
    a.round_bf16 = round_bf16;
    CHEB_TRY(run_resident<T>(plan, a, s));
    if (moments || gmoments) {
        const dim3 g((kmax + 127) / 128, plan->nsys);
        k_res_moments<<<g, 128, 0, s>>>(part, kmax, plan->d_sys_rpanel, n_terms_dev, n_single, plan->nsys, mom_stride,
                                        moments, G ? gmoments : nullptr);
        CHEB_TRY(check_launch("k_res_moments"));
    }
    return CHEB_OK;
}

}  // namespace cheb

using namespace cheb;

static int check_res_operator(const cheb_plan *plan, const cheb_bsr *Mt) {
    if (!plan || !plan->bound) return fail(CHEB_ERR_INVALID, "plan is NULL or not bound");
    if (!Mt || Mt->nbr != plan->nbr || !Mt->row_ptr || !Mt->col_idx || !Mt->vals || Mt->dtype != CHEB_F64)
        return fail(CHEB_ERR_INVALID, "operator must be FP64 with the plan's block rows");
    return CHEB_OK;
}

extern "C" int cheb_expand_workspace_size(const cheb_plan *plan, const cheb_bsr *Mt, int32_t precision,
                                          int32_t max_terms, size_t *bytes) {
    if (!plan || !Mt || !bytes || max_terms < 2)
        return fail(CHEB_ERR_INVALID, "cheb_expand_workspace_size: bad arguments");
    *bytes = resident_ws(plan, Mt->nnzb, precision, max_terms);
    return CHEB_OK;
}

extern "C" int cheb_expand(const cheb_plan *plan, const cheb_bsr *Mt, int32_t n_terms, const double *coeffs,
                           int32_t coeff_stride, int32_t n_f, double *const *acc, double *moments, const double *G,
                           double *gmoments, int32_t precision, void *ws, size_t ws_bytes, void *stream) {
    CHEB_TRY(check_res_operator(plan, Mt));
    if (plan->nsys != 1) return fail(CHEB_ERR_INVALID, "cheb_expand: batched plan; use cheb_expand_batched");
    if (n_terms < 2 || n_f < 0 || n_f > MAX_F || (n_f > 0 && (!acc || !coeffs)) || (n_f > 0 && coeff_stride < n_terms))
        return fail(CHEB_ERR_INVALID, "cheb_expand: bad n_terms / n_f / coefficients");
    for (int f = 0; f < n_f; ++f)
        if (!acc[f]) return fail(CHEB_ERR_INVALID, "cheb_expand: accumulator %d is NULL", f);
    if (precision != plan->precision) return fail(CHEB_ERR_INVALID, "cheb_expand: plan precision differs");
    const size_t need = resident_ws(plan, Mt->nnzb, precision, n_terms);
    if (!ws || ws_bytes < need) return fail(CHEB_ERR_NOSPACE, "cheb_expand: workspace %zu < %zu", ws_bytes, need);
    cudaStream_t s = as_stream(stream);
    const double *cf = coeffs;  // never read when n_f == 0
    if (precision == CHEB_F64)
        return resident_impl<double>(plan, Mt, n_terms, nullptr, n_terms, cf, nullptr, coeff_stride, n_f, acc, moments,
                                     G, gmoments, n_terms, ws, ws_bytes, s);
    if (precision == CHEB_F64X)
        return resident_impl<dfl>(plan, Mt, n_terms, nullptr, n_terms, cf, nullptr, coeff_stride, n_f, acc, moments,
                                  G, gmoments, n_terms, ws, ws_bytes, s);
    if (precision == CHEB_F32 || precision == CHEB_BF16)
        return resident_impl<float>(plan, Mt, n_terms, nullptr, n_terms, cf, nullptr, coeff_stride, n_f, acc, moments,
                                    G, gmoments, n_terms, ws, ws_bytes, s, precision == CHEB_BF16);
    return fail(CHEB_ERR_INVALID, "cheb_expand: unsupported precision %d", precision);
}

extern "C" int cheb_expand_batched(const cheb_plan *plan, const cheb_bsr *Mt, int32_t max_terms,
                                   const int32_t *n_terms, const double *coeffs, const int64_t *coeff_offset,
                                   int32_t coeff_stride, int32_t n_f, double *const *acc, double *moments,
                                   const double *G, double *gmoments, int32_t moment_stride, int32_t precision,
                                   void *ws, size_t ws_bytes, void *stream) {
    CHEB_TRY(check_res_operator(plan, Mt));
    if (max_terms < 2 || !n_terms || n_f < 0 || n_f > MAX_F || (n_f > 0 && (!acc || !coeffs || !coeff_offset)) ||
        ((moments || gmoments) && moment_stride < max_terms))
        return fail(CHEB_ERR_INVALID, "cheb_expand_batched: bad arguments");
    for (int f = 0; f < n_f; ++f)
        if (!acc[f]) return fail(CHEB_ERR_INVALID, "cheb_expand_batched: accumulator %d is NULL", f);
    if (precision != plan->precision) return fail(CHEB_ERR_INVALID, "cheb_expand_batched: plan precision differs");
    const size_t need = resident_ws(plan, Mt->nnzb, precision, max_terms);
    if (!ws || ws_bytes < need) return fail(CHEB_ERR_NOSPACE, "cheb_expand_batched: workspace %zu < %zu", ws_bytes, need);
    cudaStream_t s = as_stream(stream);
    const double *cf = coeffs;  // never read when n_f == 0
    if (precision == CHEB_F64)
        return resident_impl<double>(plan, Mt, max_terms, n_terms, 0, cf, n_f > 0 ? coeff_offset : nullptr,
                                     coeff_stride, n_f, acc, moments, G, gmoments, moment_stride, ws, ws_bytes, s);
    if (precision == CHEB_F64X)
        return resident_impl<dfl>(plan, Mt, max_terms, n_terms, 0, cf, n_f > 0 ? coeff_offset : nullptr,
                                  coeff_stride, n_f, acc, moments, G, gmoments, moment_stride, ws, ws_bytes, s);
    if (precision == CHEB_F32 || precision == CHEB_BF16)
        return resident_impl<float>(plan, Mt, max_terms, n_terms, 0, cf, n_f > 0 ? coeff_offset : nullptr,
                                    coeff_stride, n_f, acc, moments, G, gmoments, moment_stride, ws, ws_bytes, s,
                                    precision == CHEB_BF16);
    return fail(CHEB_ERR_INVALID, "cheb_expand_batched: unsupported precision %d", precision);
}
