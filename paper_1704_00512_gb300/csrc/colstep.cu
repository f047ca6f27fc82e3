// The FP32 / BF16 recursion step in column order: one step of the masked
// Chebyshev recursion (Eq. 3) fused with the accumulation of several
// expansions (Eq. 1) and the moments Tr T_{k+1}, <T_{k+1}, G>.
//
// Column J of T_{k+1} needs only column J of T_k and T_{k-1} (Sec. "Expansion
// in Chebyshev polynomials").  The recursion therefore keeps T_k in *column
// order*: the blocks (K, J) of column J are stored contiguously, at the BCSR
// positions of row J of the symmetric output pattern (block (K, J) at the
// position of (J, K); its 16 values stay row-major).  A panel of consecutive
// block columns is then one contiguous range, read and written with
// coalesced 64-byte block accesses.  The accumulators and G stay in the
// caller's BCSR order; block b of the column order is block tperm[b] there.
//
// One thread block per panel (the plan's column panels):
//   1. the panel's T_k blocks go to shared memory X[slot][4][4P] (slot = rank
//      of the block row in the union of the panel's row lists, precomputed;
//      zero where a column has no block in that row); rows of a slot's
//      block are XOR-swizzled by the slot so that the K-groups of a quarter
//      warp read distinct banks;
//   2. each warp takes union rows I; lane = (panel column q, K-group); the
//      operator blocks L_IK of row I with K in the union are the row's
//      precomputed entries, taken KG at a time (one chunk, one per K-group)
//      and copied by cp.async into a per-warp ring of stages, several chunks
//      ahead of the multiplication (across row ends); the entry words of a
//      whole row are fetched one row ahead and handed out by shuffles;
//   3. at the end of a row a reduce-scatter over the K-groups leaves each lane
//      16/KG elements of the block (I, J_q), and the lane finishes them:
//      T_{k+1} = alpha (M~ T_k) + beta T_{k-1}, acc_j += c_j[k+1] T_{k+1},
//      and its parts of Tr T_{k+1} and <T_{k+1}, G> -- with the operands of
//      that epilogue (T_{k-1}, G, accumulators) loaded at the start of the
//      row, so their latency hides under the row's products;
//   4. the last thread block to finish sums the per-block moment partials in
//      a fixed order (deterministic).
#include <cuda_bf16.h>

#include <algorithm>
#include <numeric>
#include <thread>

#include "common.cuh"
#include "kernels.cuh"
#include "plan.cuh"

namespace cheb {

struct ColArgs {
    const int32_t *panels;  // (first column, column count, union rows, 0) per thread block
    const int32_t *wchunk;  // [panels][NW + 1] chunk range of each warp
    const int32_t *wrow;    // [panels][NW + 1] row-list range of each warp
    const uint32_t *rows;   // union slot | chunk count << COL_SLOT_BITS, per warp row
    const uint32_t *ent;    // [chunks][KG] operator block << COL_SLOT_BITS | union slot
    const uint16_t *slot;
    const int64_t *rp;     // P_out row_ptr = column starts in column order
    const int32_t *ci;     // row of each column-order block
    const int32_t *tperm;  // BCSR position of each column-order block
    const float *Lv;       // operator values (FP32 copy, one zero block appended), BCSR order
    const float *R;        // T_k (column order)
    const float *Rm;       // T_{k-1} (column order) or NULL
    float *C;              // T_{k+1} (column order)
    float alpha, beta;
    int32_t nf;
    double *acc[MAX_F];   // the caller's FP64 accumulators (BCSR order): init and final kernels
    float *accp[MAX_F];   // the accumulators during the expansion: (hi, lo) float pairs, column order
    const double *coef;
    int32_t coef_stride;
    int32_t term;
    const double *G;      // the caller's G (BCSR order): init kernel
    const float *Gp;      // G as (hi, lo) float pairs in column order, or NULL
    double *mom, *gmom, *part;  // moment scalars of term k+1 (terms k-1, k at [-2], [-1])
    int32_t *counter;
    int32_t round_bf16;
    // Terms accumulated (and their moments taken) by this launch: bit 0 term
    // k+1 (the T_{k+1} it forms), bit 1 term k (T_k, in shared memory), bit 2
    // term k-1 (T_{k-1}, read for the recursion anyway).  Grouping three
    // terms per update cuts the accumulator and G traffic threefold and sums
    // in the same order as one term per step.
    int32_t grp;
};

// Double-float arithmetic (a value is an unevaluated sum hi + lo of two
// floats, about 48 significant bits): GB300 issues FP64 at 1/64 of the FP32
// rate, so the per-step FP64 accumulation of Eq. 1 and the trace functional
// are carried on the FP32 pipe with error-free transformations (Knuth's
// two-sum, the FMA product error) and converted to FP64 once per expansion.
__device__ __forceinline__ void ff_add_prod(float &hi, float &lo, float y, float ch, float cl) {
    // (hi, lo) += y * (ch + cl)
    const float p = __fmul_rn(y, ch);
    float pe = __fmaf_rn(y, ch, -p);
    pe = __fmaf_rn(y, cl, pe);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    const float t = __fadd_rn(__fadd_rn(lo, pe), e);
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
}
__host__ __device__ inline void ff_split(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// L2 policies: the operator (read by every panel whose union holds its
// blocks) is kept, the streams read once per step are evicted first.
__device__ __forceinline__ uint64_t policy_keep() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_stream() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 16 floats of an operator block, read once per panel: no L1 allocation.
__device__ __forceinline__ void ld_op(float (&h)[16], const float *p, uint64_t pol) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float4 v;
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "l"(p + 4 * i), "l"(pol));
        h[4 * i] = v.x; h[4 * i + 1] = v.y; h[4 * i + 2] = v.z; h[4 * i + 3] = v.w;
    }
}
__device__ __forceinline__ void cp_async16_hint(void *dst_smem, const void *src, uint64_t pol) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "l"(pol)
                 : "memory");
}
// Streamed loads and stores with an L2 policy (the EPL = 1 or 2 elements a
// lane finishes; 16 floats of a T_k block).
template <int N>
__device__ __forceinline__ void ldh(float (&v)[N], const float *p, uint64_t pol) {
    if constexpr (N == 2) {
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;"
                     : "=f"(v[0]), "=f"(v[1]) : "l"(p), "l"(pol));
    } else {
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v[0]) : "l"(p), "l"(pol));
    }
}
template <int N>
__device__ __forceinline__ void ldh(double (&v)[N], const double *p, uint64_t pol) {
    if constexpr (N == 2) {
        asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
                     : "=d"(v[0]), "=d"(v[1]) : "l"(p), "l"(pol));
    } else {
        asm volatile("ld.global.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v[0]) : "l"(p), "l"(pol));
    }
}
template <int N>
__device__ __forceinline__ void sth(float *p, const float (&v)[N], uint64_t pol) {
    if constexpr (N == 2) {
        asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1,%2}, %3;" ::"l"(p), "f"(v[0]), "f"(v[1]), "l"(pol)
                     : "memory");
    } else {
        asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v[0]), "l"(pol) : "memory");
    }
}
template <int N>
__device__ __forceinline__ void sth(double *p, const double (&v)[N], uint64_t pol) {
    if constexpr (N == 2) {
        asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1,%2}, %3;" ::"l"(p), "d"(v[0]), "d"(v[1]), "l"(pol)
                     : "memory");
    } else {
        asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v[0]), "l"(pol) : "memory");
    }
}
// EPL consecutive (hi, lo) pairs: 2 * EPL floats
template <int N>
__device__ __forceinline__ void ldh_pairs(float (&v)[2 * N], const float *p, uint64_t pol) {
    if constexpr (N == 2) {
        asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p), "l"(pol));
    } else {
        asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;"
                     : "=f"(v[0]), "=f"(v[1]) : "l"(p), "l"(pol));
    }
}
template <int N>
__device__ __forceinline__ void sth_pairs(float *p, const float (&v)[2 * N], uint64_t pol) {
    if constexpr (N == 2) {
        asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "f"(v[0]), "f"(v[1]),
                     "f"(v[2]), "f"(v[3]), "l"(pol)
                     : "memory");
    } else {
        asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1,%2}, %3;" ::"l"(p), "f"(v[0]), "f"(v[1]), "l"(pol)
                     : "memory");
    }
}
template <int N>
__device__ __forceinline__ void ldg_pairs(float (&v)[2 * N], const float *p, uint64_t pol) {
    if constexpr (N == 2) {
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p), "l"(pol));
    } else {
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;"
                     : "=f"(v[0]), "=f"(v[1]) : "l"(p), "l"(pol));
    }
}

__device__ __forceinline__ void ldh16(float (&h)[16], const float *p, uint64_t pol) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=f"(h[4 * i]), "=f"(h[4 * i + 1]), "=f"(h[4 * i + 2]), "=f"(h[4 * i + 3])
                     : "l"(p + 4 * i), "l"(pol));
}

__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t *p, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

template <int P, int NW, int NFP>
__global__ void __launch_bounds__(NW * 32, 1) k_colstep(const ColArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int D = COL_STAGES;     // operator stages per warp
    constexpr int NT = NW * 32;
    constexpr int KG = 32 / P;        // K-groups per warp
    constexpr int LKG = ilog2(KG);
    constexpr int EPL = 16 / KG;      // elements of a block per lane after the reduce-scatter
    constexpr int RQ = 8 / P;         // K-groups per quarter warp
    constexpr int CPL = 4 / P;        // 16-byte chunks of a staged block copied per lane
    constexpr uint32_t SM = (1u << COL_SLOT_BITS) - 1u;
    static_assert(P == 4, "panel width 4 (rows of at most two columns run on paired lane quads)");
    __shared__ int64_t s_cb[P + 1];
    __shared__ int s_dslot[P];
    __shared__ float s_ch[3][MAX_F], s_cl[3][MAX_F];  // coefficients of terms k-1, k, k+1
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int pid = blockIdx.x;
    const int j0 = a.panels[4 * pid], nc = a.panels[4 * pid + 1], nu = a.panels[4 * pid + 2];
    const ColLayout lay = col_layout(nu, P, NW);
    float *X = reinterpret_cast<float *>(smem + lay.off_x);
    int32_t *opos = reinterpret_cast<int32_t *>(smem + lay.off_pos);
    double *red = reinterpret_cast<double *>(smem + lay.off_red);

    const uint64_t pkeep = policy_keep(), pstream = policy_stream();
    // 1. gather the panel's columns of T_k
    if (tid <= P) s_cb[tid] = a.rp[j0 + min(tid, nc)];
    if (tid < P) s_dslot[tid] = -1;
    if (tid < 3 * MAX_F) {
        const int j = tid / MAX_F, f = tid % MAX_F;  // term k-1+j
        const int term = a.term - 2 + j;
        ff_split(f < a.nf && term >= 0 ? a.coef[(int64_t)f * a.coef_stride + term] : 0.0, s_ch[j][f], s_cl[j][f]);
    }
    {
        float4 *x4 = reinterpret_cast<float4 *>(X);
        for (int i = tid; i < nu * 4 * P; i += NT) x4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = tid; i < nu * P; i += NT) opos[i] = -1;
    }
    __syncthreads();
    {
        const int64_t cb0 = s_cb[0], cb1 = s_cb[nc];
        for (int64_t b = cb0 + tid; b < cb1; b += NT) {
            int q = 0;
#pragma unroll
            for (int qq = 1; qq < P; ++qq)
                if (qq < nc && b >= s_cb[qq]) q = qq;
            const int s = a.slot[b];
            float v[16];
            ldh16(v, a.R + b * BB, pstream);
            float *xs = X + (size_t)s * 16 * P + 4 * q;
            const int sw = s & (RQ - 1);
#pragma unroll
            for (int m = 0; m < 4; ++m)
                *reinterpret_cast<float4 *>(xs + (m ^ sw) * 4 * P) =
                    make_float4(v[4 * m], v[4 * m + 1], v[4 * m + 2], v[4 * m + 3]);
            opos[s * P + q] = (int32_t)b;
            if (a.ci[b] == j0 + q) s_dslot[q] = s;
        }
    }
    __syncthreads();

    // Tr T and <T, G> of terms k-1, k, k+1, double-float partial sums
    float th[3] = {0.f, 0.f, 0.f}, tl[3] = {0.f, 0.f, 0.f};
    float gh[3] = {0.f, 0.f, 0.f}, gl[3] = {0.f, 0.f, 0.f};
    const int q = lane % P, kg = lane / P;
    const int i0 = kg * EPL;
    // 16-byte chunk c of a staged block of K-group kg sits at chunk c ^ skw, so
    // that the K-groups' blocks spread over all banks
    const int skw = (kg >> 1) & 3;

    // 2. the warp's chunks.  The plan lays out every warp's work as one stream
    // of chunks (CW = EK * KG entries, EK per K-group; each row padded with
    // zero-block entries to whole chunks) and a list of its rows (union slot,
    // chunk count).  Operator blocks go through a ring of D stages: the copies
    // of chunk n + D - 1 are issued (cp.async) before chunk n is multiplied.
    // The entry words come in windows of 32 (32/CW chunks), one word per lane,
    // four windows deep, and are handed to the K-groups by shuffles.
    constexpr int EK = COL_EK;        // entries of a K-group per chunk
    constexpr int CW = EK * KG;       // entries (words, staged blocks) per chunk
    float *stg = reinterpret_cast<float *>(smem + lay.off_stage) + (size_t)warp * D * CW * 16;
    const int64_t c0 = a.wchunk[pid * (NW + 1) + warp], c1 = a.wchunk[pid * (NW + 1) + warp + 1];
    const int r0 = a.wrow[pid * (NW + 1) + warp], r1 = a.wrow[pid * (NW + 1) + warp + 1];
    const int nch = (int)(c1 - c0);
    if (nch > 0) {
        constexpr int WC = 32 / CW;  // chunks per window
        // Chunk n is always in win0 and chunk n + D - 1, whose operator blocks
        // are issued while chunk n is multiplied, always in win1, both at
        // window offset jo = n - n0 (n0: first chunk of win0), so that a
        // word's source lane is jo * CW + e * KG + kg with no window select.
        static_assert(D - 1 == WC, "the producer runs exactly one window ahead");
        const uint32_t *ew = a.ent + c0 * CW;  // words of the warp's chunks
        const int nw = nch * CW;
        uint32_t win0 = lane < nw ? ld_stream_u32(ew + lane, pstream) : 0u;
        uint32_t win1 = 32 + lane < nw ? ld_stream_u32(ew + 32 + lane, pstream) : 0u;
        uint32_t win2 = 64 + lane < nw ? ld_stream_u32(ew + 64 + lane, pstream) : 0u;
        uint32_t win3 = 96 + lane < nw ? ld_stream_u32(ew + 96 + lane, pstream) : 0u;
        // the lane's part of stage st for the chunk whose words are in window
        // value win at source lanes lb + e * KG: 16-byte chunk c of block
        // (e, kg) at chunk c ^ skw, so that the K-groups' blocks spread over
        // all banks
        auto produce = [&](uint32_t win, int lb, int st, bool live) {
            uint32_t words[EK];
#pragma unroll
            for (int e = 0; e < EK; ++e) words[e] = __shfl_sync(0xffffffffu, win, lb + e * KG);
            if (live) {
                float *dst = stg + st * CW * 16;
#pragma unroll
                for (int e = 0; e < EK; ++e) {
                    const float *src = a.Lv + (int64_t)(words[e] >> COL_SLOT_BITS) * BB;
#pragma unroll
                    for (int i = 0; i < CPL; ++i)
                        cp_async16_hint(dst + (e * KG + kg) * 16 + 4 * ((q * CPL + i) ^ skw), src + 4 * (q * CPL + i),
                                        pkeep);
                }
            }
            cp_async_commit();
        };
#pragma unroll
        for (int i = 0; i < D - 1; ++i) produce(win0, i * CW + kg, i, i < nch);
        // Rows: union slot s, chunks left cl.  A row with blocks in at most two
        // of the panel's columns ("half" row) runs with each column on two
        // lane quads: lane (q, kg) takes column cols[q & 1] and only entry
        // e = q >> 1 of each chunk (16 K-groups per column), so its chunks
        // cost half the products.  Lane's column col, its output position pos
        // (-1: no output from this lane), and the same for the next row.
        auto row_col = [&](uint32_t w, int &col, int &p) {
            const int sl = (int)(w & SM);
            const bool hf = (w >> COL_SLOT_BITS) & 1u;
            const int ca = (int)((w >> (COL_SLOT_BITS + 1)) & 3u), cb = (int)((w >> (COL_SLOT_BITS + 3)) & 3u);
            col = hf ? ((q & 1) ? cb : ca) : q;
            p = opos[sl * P + col];
            if (hf && ((q >> 1) != 0 || ((q & 1) && cb == ca))) p = -1;
        };
        int r = r0;
        uint32_t rw = a.rows[r], rwn = r + 1 < r1 ? a.rows[r + 1] : 0u, rwm = r + 2 < r1 ? a.rows[r + 2] : 0u;
        int s = (int)(rw & SM), cl = (int)(rw >> COL_ROW_SHIFT);
        bool half = (rw >> COL_SLOT_BITS) & 1u;
        int col, pos, coln = 0, posn = -1;
        row_col(rw, col, pos);
        if (r + 1 < r1) row_col(rwn, coln, posn);
        float tm[EPL], gv[2 * EPL], av[NFP > 0 ? NFP : 1][2 * EPL];
        auto prefetch_epilogue = [&]() {
#pragma unroll
            for (int j = 0; j < EPL; ++j) tm[j] = 0.f;
#pragma unroll
            for (int j = 0; j < 2 * EPL; ++j) gv[j] = 0.f;
            if (pos >= 0) {
                if (a.Rm) ldh<EPL>(tm, a.Rm + (int64_t)pos * BB + i0, pstream);
                if (a.grp) {
                    if (a.Gp) ldg_pairs<EPL>(gv, a.Gp + ((int64_t)pos * BB + i0) * 2, pstream);
#pragma unroll
                    for (int f = 0; f < NFP; ++f)
                        if (f < a.nf) ldh_pairs<EPL>(av[f], a.accp[f] + ((int64_t)pos * BB + i0) * 2, pstream);
                }
            }
        };
        prefetch_epilogue();
        float acc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = 0.f;
        // acc += L_IK X[K][col] for staged block b of stage st and slot tc.
        // Row m of slot tc's block sits at row m ^ (tc & 1): even rows at
        // m * 4P + d, odd rows at m * 4P - d, d = (tc & 1) * 4P.
        static_assert(RQ == 2, "slot swizzle of one bit");
        const float *xcol = X + 4 * col;  // follows col from row to row
        auto multiply = [&](const float *hs, uint32_t tc) {
            float hc[16];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float4 v = *reinterpret_cast<const float4 *>(hs + 4 * (c ^ skw));
                hc[4 * c] = v.x; hc[4 * c + 1] = v.y; hc[4 * c + 2] = v.z; hc[4 * c + 3] = v.w;
            }
            const int d = (int)(tc & 1u) * 4 * P;
            const float *xe = xcol + tc * (16 * P) + d, *xo = xcol + tc * (16 * P) - d;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float4 x = *reinterpret_cast<const float4 *>((m & 1 ? xo : xe) + m * 4 * P);
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    acc[4 * rr + 0] = fmaf(hc[4 * rr + m], x.x, acc[4 * rr + 0]);
                    acc[4 * rr + 1] = fmaf(hc[4 * rr + m], x.y, acc[4 * rr + 1]);
                    acc[4 * rr + 2] = fmaf(hc[4 * rr + m], x.z, acc[4 * rr + 2]);
                    acc[4 * rr + 3] = fmaf(hc[4 * rr + m], x.w, acc[4 * rr + 3]);
                }
            }
        };
        // n0: first chunk of win0; lb = (n - n0) * CW + kg; sc, ps: stages of
        // chunks n and n + D - 1
        int n0 = 0, lb = kg, sc = 0, ps = D - 1;
        for (int n = 0; n < nch; ++n) {
            produce(win1, lb, ps, n + D - 1 < nch);
            cp_async_wait<D - 1>();
            __syncwarp();
            const float *st = stg + sc * CW * 16 + kg * 16;
            if (!half) {
#pragma unroll
                for (int e = 0; e < EK; ++e)
                    multiply(st + e * KG * 16, __shfl_sync(0xffffffffu, win0, lb + e * KG) & SM);
            } else {
                const int e = q >> 1;
                const uint32_t wv = __shfl_sync(0xffffffffu, win0, lb + e * KG);
                multiply(st + e * KG * 16, wv & SM);
            }
            __syncwarp();
            sc = sc + 1 == D ? 0 : sc + 1;
            ps = ps + 1 == D ? 0 : ps + 1;
            lb += CW;
            if (n + 1 - n0 == WC) {
                // the next window: shift, and fetch the one three windows ahead
                n0 += WC;
                lb = kg;
                win0 = win1;
                win1 = win2;
                win2 = win3;
                const int e = (n0 + 3 * WC) * CW + lane;
                win3 = e < nw ? ld_stream_u32(ew + e, pstream) : 0u;
            }
            if (--cl == 0) {
                // 3. the row is done: combine the K-groups (a half row's two
                // lane quads per column first), reduce-scatter, then finish
                // the lane's elements of block (row s, column col).  The
                // accumulators NFP, NFP + 1 (not prefetched at the row's start)
                // are loaded first, so that the reduce-scatter's shuffles
                // cover part of their latency.
                constexpr int NL = NFP > 0 ? 1 : 0;
                float lv[NL > 0 ? NL : 1][2 * EPL];
                if (NL > 0 && a.grp && pos >= 0) {
#pragma unroll
                    for (int f = 0; f < NL; ++f)
                        if (NFP + f < a.nf)
                            ldh_pairs<EPL>(lv[f], a.accp[NFP + f] + ((int64_t)pos * BB + i0) * 2, pstream);
                }
                if (half) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], P / 2);
                }
#pragma unroll
                for (int l = 0; l < LKG; ++l) {
                    const int nn = 8 >> l;
                    const int off = P << (LKG - 1 - l);
                    const bool hi = (kg >> (LKG - 1 - l)) & 1;
#pragma unroll
                    for (int j = 0; j < nn; ++j) {
                        const float mine = hi ? acc[nn + j] : acc[j], other = hi ? acc[j] : acc[nn + j];
                        acc[j] = mine + __shfl_xor_sync(0xffffffffu, other, off);
                    }
                }
                if (pos >= 0) {
                    float y[EPL];
#pragma unroll
                    for (int j = 0; j < EPL; ++j) {
                        y[j] = a.Rm ? a.alpha * acc[j] + a.beta * tm[j] : a.alpha * acc[j];
                        if (a.round_bf16) y[j] = bf16r(y[j]);
                    }
                    sth<EPL>(a.C + (int64_t)pos * BB + i0, y, pstream);
                    if (a.grp) {
                        // the group's terms in order: T_{k-1} (tm), T_k (the
                        // panel's copy in shared memory), T_{k+1} (y)
                        float tv[3][EPL];
                        {
                            const int rr = i0 / 4, sws = s & (RQ - 1);
                            const float *xk = X + (size_t)s * 16 * P + (rr ^ sws) * 4 * P + 4 * col + (i0 % 4);
#pragma unroll
                            for (int j = 0; j < EPL; ++j) {
                                tv[0][j] = tm[j];
                                tv[1][j] = xk[j];
                                tv[2][j] = y[j];
                            }
                        }
#pragma unroll
                        for (int f = 0; f < MAX_F; ++f) {
                            if (f < a.nf) {
                                float v[2 * EPL];
                                float *pa = a.accp[f] + ((int64_t)pos * BB + i0) * 2;
                                if (f < NFP) {
#pragma unroll
                                    for (int j = 0; j < 2 * EPL; ++j) v[j] = av[f < NFP ? f : 0][j];
                                } else if (f < NFP + NL) {
#pragma unroll
                                    for (int j = 0; j < 2 * EPL; ++j) v[j] = lv[f < NFP + NL ? f - NFP : 0][j];
                                } else {
                                    ldh_pairs<EPL>(v, pa, pstream);
                                }
#pragma unroll
                                for (int t3 = 0; t3 < 3; ++t3)
                                    if ((a.grp >> (2 - t3)) & 1) {
#pragma unroll
                                        for (int j = 0; j < EPL; ++j)
                                            ff_add_prod(v[2 * j], v[2 * j + 1], tv[t3][j], s_ch[t3][f], s_cl[t3][f]);
                                    }
                                sth_pairs<EPL>(pa, v, pstream);
                            }
                        }
                        const bool diag = s == s_dslot[col];
#pragma unroll
                        for (int t3 = 0; t3 < 3; ++t3)
                            if ((a.grp >> (2 - t3)) & 1) {
#pragma unroll
                                for (int j = 0; j < EPL; ++j) {
                                    ff_add_prod(gh[t3], gl[t3], tv[t3][j], gv[2 * j], gv[2 * j + 1]);
                                    // diagonal elements 0, 5, 10, 15 of a diagonal block
                                    if (diag && (i0 + j) % 5 == 0) ff_add_prod(th[t3], tl[t3], tv[t3][j], 1.f, 0.f);
                                }
                            }
                    }
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] = 0.f;
                // the next row of this warp
                if (++r < r1) {
                    // row words are fetched two rows ahead, so that the next
                    // row's output position is known without waiting
                    rw = rwn;
                    rwn = rwm;
                    rwm = r + 2 < r1 ? a.rows[r + 2] : 0u;
                    s = (int)(rw & SM);
                    cl = (int)(rw >> COL_ROW_SHIFT);
                    half = (rw >> COL_SLOT_BITS) & 1u;
                    col = coln;
                    xcol = X + 4 * col;
                    pos = posn;
                    if (r + 1 < r1) row_col(rwn, coln, posn);
                    else posn = -1;
                    prefetch_epilogue();
                }
            }
        }
        cp_async_wait<0>();
    }
    // 4. the moment partials of the panel
    if (a.grp && (a.mom || a.gmom)) {
        auto on = [&](int t3) { return (a.grp >> (2 - t3)) & 1; };
        Moments<6> mm{{(double)th[0] + (double)tl[0], (double)th[1] + (double)tl[1], (double)th[2] + (double)tl[2],
                       (double)gh[0] + (double)gl[0], (double)gh[1] + (double)gl[1], (double)gh[2] + (double)gl[2]},
                      {a.mom && on(0) ? a.mom - 2 : nullptr, a.mom && on(1) ? a.mom - 1 : nullptr,
                       a.mom && on(2) ? a.mom : nullptr, a.gmom && on(0) ? a.gmom - 2 : nullptr,
                       a.gmom && on(1) ? a.gmom - 1 : nullptr, a.gmom && on(2) ? a.gmom : nullptr}};
        finish_moments<NT, 6>(a.part, a.counter, mm, red);
    }
}

// Terms 0 and 1 in column order: T_0 = I and T_1 = M~ (FP32, bfloat16-rounded
// in BF16 mode), the accumulators c_0/2 T_0 + c_1 T_1 as (hi, lo) pairs in
// column order, G as pairs in column order, moments of both terms.
template <int NT>
__global__ void __launch_bounds__(NT) k_colinit(const int64_t *rp, const int32_t *ci, const int32_t *tperm,
                                               int64_t nbr, int64_t nnzb, const int64_t *Lrp, const int32_t *Lci,
                                               const double *Mt, float *T0, float *T1, int32_t nf, ColArgs a,
                                               float *Gp, double *mom, double *gmom) {
    __shared__ double red[(NT / 32) * 4];
    double c0[MAX_F], c1[MAX_F];
#pragma unroll
    for (int f = 0; f < MAX_F; ++f) {
        c0[f] = f < nf ? a.coef[(int64_t)f * a.coef_stride + 0] : 0.0;
        c1[f] = f < nf ? a.coef[(int64_t)f * a.coef_stride + 1] : 0.0;
    }
    double t0 = 0.0, t1 = 0.0, g0 = 0.0, g1 = 0.0;
    for (int64_t b = blockIdx.x * (int64_t)NT + threadIdx.x; b < nnzb; b += (int64_t)gridDim.x * NT) {
        const int64_t J = row_of(rp, nbr, b);  // column of column-order block b
        const int K = ci[b];                   // its row
        const int64_t la = find_in_row(Lrp, Lci, K, (int32_t)J);
        const int64_t o = (int64_t)tperm[b] * BB;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float v0 = (K == J && (i % 5) == 0) ? 1.f : 0.f;
            float v1 = la >= 0 ? (float)Mt[la * BB + i] : 0.f;
            if (a.round_bf16) v1 = bf16r(v1);
            T0[b * BB + i] = v0;
            T1[b * BB + i] = v1;
            const double d0 = (double)v0, d1 = (double)v1;
#pragma unroll
            for (int f = 0; f < MAX_F; ++f)
                if (f < nf) {
                    float hi, lo;
                    ff_split(0.5 * c0[f] * d0 + c1[f] * d1, hi, lo);
                    a.accp[f][(b * BB + i) * 2] = hi;
                    a.accp[f][(b * BB + i) * 2 + 1] = lo;
                }
            if (a.G) {
                const double gval = a.G[o + i];
                g0 += gval * d0;
                g1 += gval * d1;
                float hi, lo;
                ff_split(gval, hi, lo);
                Gp[(b * BB + i) * 2] = hi;
                Gp[(b * BB + i) * 2 + 1] = lo;
            }
            if (K == J && (i % 5) == 0) {
                t0 += d0;
                t1 += d1;
            }
        }
    }
    Moments<4> mm{{t0, t1, g0, g1}, {mom, mom ? mom + 1 : nullptr, gmom, gmom ? gmom + 1 : nullptr}};
    finish_moments<NT, 4>(a.part, a.counter, mm, red);
}

// The accumulators back to the caller: acc_f (BCSR order, FP64) = hi + lo.
__global__ void k_colfinal(const int32_t *tperm, int64_t nnzb, int32_t nf, ColArgs a) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // element of a column-order block
    if (e >= nnzb * BB) return;
    const int64_t b = e / BB, i = e % BB;
    const int64_t o = (int64_t)tperm[b] * BB + i;
    for (int f = 0; f < nf; ++f) a.acc[f][o] = (double)a.accp[f][2 * e] + (double)a.accp[f][2 * e + 1];
}

constexpr int COLINIT_BLOCKS = 1024;

template <int NFP>
static int launch_colstep(const cheb_plan *plan, const ColArgs &a, cudaStream_t s) {
    const ColLists &c = plan->col;
    const ColLayout lay = col_layout(c.max_union, COL_P, COL_NW);
    auto fn = k_colstep<COL_P, COL_NW, NFP>;
    CHEB_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    fn<<<(unsigned)c.n_panels, COL_NW * 32, lay.total, s>>>(a);
    return check_launch("k_colstep");
}

static int run_colstep(const cheb_plan *plan, const ColArgs &a, cudaStream_t s) {
    if (a.nf == 0) return launch_colstep<0>(plan, a, s);
    if (a.nf == 1) return launch_colstep<1>(plan, a, s);
    return launch_colstep<2>(plan, a, s);
}

bool col_usable(const cheb_plan *plan, const cheb_bsr *Mt) {
    return plan->precision != CHEB_F64 && plan->col.bound && plan->op_rp == Mt->row_ptr &&
           plan->op_ci == Mt->col_idx;
}

size_t col_expand_ws(const cheb_plan *plan, int64_t nnzL) {
    size_t b = 3 * align_up(plan->nnzb * BB * 4) + align_up((nnzL + 1) * BB * 4);
    b += (MAX_F + 1) * align_up(plan->nnzb * BB * 8);  // accumulators and G as float pairs
    b += align_up((size_t)std::max<int64_t>(plan->col.n_panels, COLINIT_BLOCKS) * 6 * sizeof(double)) + align_up(64);
    return b + 256;
}

__global__ void k_to_f32_col(const double *in, float *out, int64_t n, int round_bf16) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = round_bf16 ? __bfloat162float(__float2bfloat16_rn(in[i])) : (float)in[i];
}

int col_expand(const cheb_plan *plan, const cheb_bsr *Mt, int32_t n_terms, const double *coeffs, int32_t stride,
               int32_t nf, double *const *acc, double *moments, const double *G, double *gmoments, void *ws,
               size_t ws_bytes, cudaStream_t s, int round_bf16) {
    if (ws_bytes < col_expand_ws(plan, Mt->nnzb))
        return fail(CHEB_ERR_NOSPACE, "cheb_expand_stepwise: workspace %zu < %zu", ws_bytes,
                    col_expand_ws(plan, Mt->nnzb));
    Carve cv(ws, ws_bytes);
    float *buf[3];
    for (int i = 0; i < 3; ++i) buf[i] = cv.take<float>(plan->nnzb * BB);
    float *lv = cv.take<float>((Mt->nnzb + 1) * BB);  // + the zero block of the padding entries
    float *accp[MAX_F];
    for (int f = 0; f < MAX_F; ++f) accp[f] = cv.take<float>(plan->nnzb * BB * 2);
    float *Gp = cv.take<float>(plan->nnzb * BB * 2);
    double *part = cv.take<double>((size_t)std::max<int64_t>(plan->col.n_panels, COLINIT_BLOCKS) * 6);
    int32_t *counter = cv.take<int32_t>(16);
    if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_expand_stepwise: workspace too small");
    {
        const int64_t n = Mt->nnzb * BB;
        k_to_f32_col<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double *)Mt->vals, lv, n, round_bf16);
        CHEB_TRY(check_launch("k_to_f32_col"));
        CHEB_CUDA(cudaMemsetAsync(lv + n, 0, BB * sizeof(float), s));
    }
    CHEB_CUDA(cudaMemsetAsync(counter, 0, 64, s));
    const ColLists &c = plan->col;
    ColArgs a{};
    a.panels = c.d_panels;
    a.wchunk = c.d_wchunk;
    a.wrow = c.d_wrow;
    a.rows = c.d_rows;
    a.ent = c.d_ent;
    a.slot = c.d_slot;
    a.rp = plan->rp;
    a.ci = plan->ci;
    a.tperm = plan->d_tperm;
    a.Lv = lv;
    a.nf = nf;
    for (int f = 0; f < nf; ++f) {
        a.acc[f] = acc[f];
        a.accp[f] = accp[f];
    }
    a.coef = coeffs;
    a.coef_stride = stride;
    a.G = G;
    a.part = part;
    a.counter = counter;
    a.round_bf16 = round_bf16;
    k_colinit<256><<<COLINIT_BLOCKS, 256, 0, s>>>(plan->rp, plan->ci, plan->d_tperm, plan->nbr, plan->nnzb,
                                                  Mt->row_ptr, Mt->col_idx, (const double *)Mt->vals, buf[0],
                                                  buf[1], nf, a, Gp, moments, gmoments);
    CHEB_TRY(check_launch("k_colinit"));
    a.Gp = G ? Gp : nullptr;
    a.alpha = 2.f;
    a.beta = -1.f;
    // terms 2.. n-1 are accumulated three at a time: the launch forming term
    // t adds (t-2, t-1, t) when t = 4, 7, 10, ..., and the last launch adds
    // the terms left after the last such group
    int done = 1;  // last term accumulated (terms 0 and 1: k_colinit)
    for (int k = 1; k + 1 < n_terms; ++k) {
        const int t = k + 1;
        a.R = buf[k % 3];
        a.Rm = buf[(k - 1) % 3];
        a.C = buf[(k + 1) % 3];
        a.term = t;
        a.grp = 0;
        if ((t >= 4 && (t - 1) % 3 == 0) || t == n_terms - 1) {
            for (int u = done + 1; u <= t; ++u) a.grp |= 1 << (t - u);
            done = t;
        }
        a.mom = moments ? moments + t : nullptr;
        a.gmom = (gmoments && G) ? gmoments + t : nullptr;
        CHEB_TRY(run_colstep(plan, a, s));
    }
    if (nf > 0) {
        const int64_t n = plan->nnzb * BB;
        k_colfinal<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(plan->d_tperm, plan->nnzb, nf, a);
        CHEB_TRY(check_launch("k_colfinal"));
    }
    return CHEB_OK;
}

// ---------------------------------------------------------------------------
// Host: the column kernel's panels and work streams for operator pattern
// (lrp, lci).  Per panel: the union of its columns' rows (slot = rank); per
// union row its operator entries with K in the union (dealt round-robin over
// the slot residues modulo the K-groups of a quarter warp, so those K-groups
// read different shared-memory banks), padded with zero-block entries to
// whole chunks of KG; rows dealt to the NW warps by decreasing chunk count,
// each to the warp with the least work so far; per warp its rows' chunks in
// one stream and its row list.

struct ColCounts {
    std::vector<int64_t> chunks, rows;
    std::vector<int32_t> max_row;
};

static void col_fill(const ColLists &c, const std::vector<int64_t> &rp, const std::vector<int32_t> &ci,
                     const std::vector<int64_t> &lrp, const std::vector<int32_t> &lci, int64_t nbr, int64_t p0,
                     int64_t p1, bool count_only, ColCounts &cnt, const std::vector<int64_t> &chunk_off,
                     const std::vector<int64_t> &row_off, std::vector<int32_t> &pan, std::vector<int32_t> &wchunk,
                     std::vector<int32_t> &wrow, std::vector<uint32_t> &rows, std::vector<uint32_t> &ent,
                     std::vector<uint16_t> &slot) {
    const int KG = 32 / c.P, CW = COL_EK * KG, NW = c.NW, rq = 8 / c.P;
    const uint32_t zero_word = (uint32_t)lci.size() << COL_SLOT_BITS;  // the appended zero block, slot 0
    std::vector<int32_t> stamp(nbr, -1), slot_of(nbr, -1), uni;
    std::vector<std::vector<uint32_t>> cls(rq), rent;
    std::vector<int32_t> order, wl;
    std::vector<uint8_t> cmask;
    std::vector<int64_t> load(NW);
    std::vector<std::vector<int32_t>> wrows(NW);
    for (int64_t p = p0; p < p1; ++p) {
        const int32_t j0 = c.h_panels[4 * p], nc = c.h_panels[4 * p + 1];
        uni.clear();
        for (int32_t q = 0; q < nc; ++q)
            for (int64_t e = rp[j0 + q]; e < rp[j0 + q + 1]; ++e)
                if (stamp[ci[e]] != (int32_t)p) {
                    stamp[ci[e]] = (int32_t)p;
                    uni.push_back(ci[e]);
                }
        std::sort(uni.begin(), uni.end());
        const int nu = (int)uni.size();
        for (int u = 0; u < nu; ++u) slot_of[uni[u]] = u;
        // the entries of every union row, interleaved and padded
        rent.assign(nu, {});
        int32_t mr = 0;
        for (int u = 0; u < nu; ++u) {
            const int32_t I = uni[u];
            for (auto &v : cls) v.clear();
            for (int64_t e = lrp[I]; e < lrp[I + 1]; ++e)
                if (stamp[lci[e]] == (int32_t)p) {
                    const int32_t sl = slot_of[lci[e]];
                    cls[sl % rq].push_back(((uint32_t)e << COL_SLOT_BITS) | (uint32_t)sl);
                }
            // position p of a chunk (8 K-groups x 2 entries) takes slot residue
            // (p ^ (p >> 3)) mod 2, so that the two K-groups of a quarter warp
            // differ in it both for the entries e = 0, 1 of a full row and for
            // the pair (p, p + 8) that a half row's lane quads read together;
            // when one residue runs out the other fills in
            std::vector<uint32_t> &r = rent[u];
            std::vector<size_t> at(rq, 0);
            size_t left = 0;
            for (auto &v : cls) left += v.size();
            for (size_t pos = 0; left > 0; ++pos) {
                const int p = (int)(pos % (size_t)CW);
                int k = ((p ^ (p >> 3)) & 1) % rq;
                if (at[k] >= cls[k].size())
                    for (int kk = 0; kk < rq; ++kk)
                        if (at[kk] < cls[kk].size()) {
                            k = kk;
                            break;
                        }
                r.push_back(cls[k][at[k]++]);
                --left;
            }
            mr = std::max(mr, (int32_t)r.size());
            const size_t padded = std::max<size_t>(1, (r.size() + CW - 1) / CW) * CW;
            r.resize(padded, zero_word);
        }
        // the columns of the panel in which each union row has a block
        std::vector<uint8_t> &cm = cmask;
        cm.assign(nu, 0);
        for (int32_t q = 0; q < nc; ++q)
            for (int64_t e = rp[j0 + q]; e < rp[j0 + q + 1]; ++e) cm[slot_of[ci[e]]] |= (uint8_t)(1u << q);
        // rows to warps: decreasing chunk count (a chunk's copies, waits and
        // bookkeeping cost about as much as its products), each to the warp
        // with the fewest chunks so far
        auto work = [&](int32_t u) { return (int64_t)(rent[u].size() / CW); };
        order.resize(nu);
        for (int u = 0; u < nu; ++u) order[u] = u;
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return work(x) > work(y); });
        std::fill(load.begin(), load.end(), 0);
        for (auto &v : wrows) v.clear();
        int64_t total = 0;
        for (const int32_t u : order) {
            const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            load[w] += work(u);
            wrows[w].push_back(u);
            total += (int64_t)rent[u].size() / CW;
        }
        if (count_only) {
            cnt.chunks[p] = total;
            cnt.rows[p] = nu;
            cnt.max_row[p] = mr;
            continue;
        }
        pan[4 * p] = j0;
        pan[4 * p + 1] = nc;
        pan[4 * p + 2] = nu;
        pan[4 * p + 3] = 0;
        for (int32_t q = 0; q < nc; ++q)
            for (int64_t e = rp[j0 + q]; e < rp[j0 + q + 1]; ++e) slot[e] = (uint16_t)slot_of[ci[e]];
        int64_t ch = chunk_off[p], ro = row_off[p];
        for (int w = 0; w < NW; ++w) {
            wchunk[p * (NW + 1) + w] = (int32_t)ch;
            wrow[p * (NW + 1) + w] = (int32_t)ro;
            std::sort(wrows[w].begin(), wrows[w].end());
            for (const int32_t u : wrows[w]) {
                const std::vector<uint32_t> &r = rent[u];
                // half row: blocks in at most two columns (ca, cb; cb = ca for one)
                const uint32_t m = cm[u];
                const int pc = __builtin_popcount(m);
                uint32_t hw = 0;
                if (pc <= 2) {
                    const uint32_t ca = (uint32_t)__builtin_ctz(m);
                    const uint32_t cb = pc == 2 ? (uint32_t)(31 - __builtin_clz(m)) : ca;
                    hw = 1u | (ca << 1) | (cb << 3);
                }
                rows[ro++] = (uint32_t)u | (hw << COL_SLOT_BITS) | ((uint32_t)(r.size() / CW) << COL_ROW_SHIFT);
                std::copy(r.begin(), r.end(), ent.begin() + ch * CW);
                ch += (int64_t)r.size() / CW;
            }
        }
        wchunk[p * (NW + 1) + NW] = (int32_t)ch;
        wrow[p * (NW + 1) + NW] = (int32_t)ro;
    }
}

// Union rows a panel of the column kernel may hold: shared memory, and slots
// below 2^COL_SLOT_BITS.
int32_t col_ucap() {
    int lo = 0, hi = 65535;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (col_layout(mid, COL_P, COL_NW).total <= (size_t)CHEB_MAX_DYN_SMEM - 1024) lo = mid; else hi = mid - 1;
    }
    return std::min(lo, (1 << COL_SLOT_BITS) - 1);
}

int col_build(cheb_plan *plan, const std::vector<int64_t> &rp, const std::vector<int32_t> &ci,
              const std::vector<int64_t> &lrp, const std::vector<int32_t> &lci) {
    ColLists c;
    c.P = COL_P;
    c.NW = COL_NW;
    const int CW = COL_EK * 32 / c.P;  // entries per chunk
    const int64_t nbr = plan->nbr, nnzb = plan->nnzb;
    c.ucap = col_ucap();
    // entries pack the operator block index (the appended zero block included)
    // above the union slot
    if ((int64_t)lci.size() + 1 >= ((int64_t)1 << (32 - COL_SLOT_BITS))) return CHEB_ERR_NOSPACE;
    // panels: greedy along the columns while the union fits
    std::vector<int32_t> stamp(nbr, -1);
    {
        int64_t j = 0, panel = 0;
        while (j < nbr) {
            int32_t cnt = 0, ncols = 0;
            const int64_t j0 = j;
            while (j < nbr && ncols < c.P) {
                int32_t add = 0;
                for (int64_t p = rp[j]; p < rp[j + 1]; ++p) add += stamp[ci[p]] != (int32_t)panel;
                if (cnt + add > c.ucap) break;
                for (int64_t p = rp[j]; p < rp[j + 1]; ++p) stamp[ci[p]] = (int32_t)panel;
                cnt += add;
                ++ncols;
                ++j;
            }
            if (ncols == 0) return CHEB_ERR_NOSPACE;  // a single column does not fit: no column kernel
            c.h_panels.insert(c.h_panels.end(), {(int32_t)j0, ncols, cnt, 0});
            c.max_union = std::max(c.max_union, cnt);
            ++panel;
        }
        c.n_panels = panel;
    }
    const int64_t np = c.n_panels;
    ColCounts cnt;
    cnt.chunks.assign(np, 0);
    cnt.rows.assign(np, 0);
    cnt.max_row.assign(np, 0);
    std::vector<int64_t> chunk_off(np + 1, 0), row_off(np + 1, 0);
    std::vector<int32_t> pan(4 * np), wchunk(np * (c.NW + 1)), wrow(np * (c.NW + 1));
    std::vector<uint32_t> rows, ent;
    std::vector<uint16_t> slot(nnzb);
    const int nth = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)std::thread::hardware_concurrency(), 16, np}));
    auto run = [&](bool count_only) {
        std::vector<std::thread> th;
        for (int t = 0; t < nth; ++t) {
            const int64_t p0 = np * t / nth, p1 = np * (t + 1) / nth;
            th.emplace_back([&, p0, p1] {
                col_fill(c, rp, ci, lrp, lci, nbr, p0, p1, count_only, cnt, chunk_off, row_off, pan, wchunk, wrow,
                         rows, ent, slot);
            });
        }
        for (auto &x : th) x.join();
    };
    run(true);
    for (int64_t p = 0; p < np; ++p) {
        chunk_off[p + 1] = chunk_off[p] + cnt.chunks[p];
        row_off[p + 1] = row_off[p] + cnt.rows[p];
        c.max_row = std::max(c.max_row, cnt.max_row[p]);
    }
    if (chunk_off[np] * CW >= (int64_t)INT32_MAX) return CHEB_ERR_NOSPACE;
    c.n_entries = chunk_off[np] * CW;
    rows.resize(row_off[np]);
    ent.resize(chunk_off[np] * CW);
    run(false);
    c.h_panels.swap(pan);
    c.h_wchunk.swap(wchunk);
    c.h_wrow.swap(wrow);
    c.h_rows.swap(rows);
    c.h_ent.swap(ent);
    c.h_slot.swap(slot);
    c.n_rows = (int64_t)c.h_rows.size();
    c.n_slot = (int64_t)c.h_slot.size();
    c.built = true;
    plan->col = std::move(c);
    return CHEB_OK;
}

int col_bind(ColLists &c, Carve &cv, cudaStream_t s) {
    if (!c.built) return CHEB_OK;
    if (c.device) {
        // lists built on the device: one copy of their block into the workspace
        // (the same carve order, so every array keeps its offset)
        char *dst = cv.take<char>(c.bytes());
        if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_plan_bind_operator: workspace too small");
        CHEB_CUDA(cudaMemcpyAsync(dst, c.tmp, c.bytes(), cudaMemcpyDeviceToDevice, s));
        const ptrdiff_t d = dst - static_cast<char *>(c.tmp);
        c.d_panels = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(c.d_panels) + d);
        c.d_wchunk = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(c.d_wchunk) + d);
        c.d_wrow = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(c.d_wrow) + d);
        c.d_rows = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(c.d_rows) + d);
        c.d_ent = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(c.d_ent) + d);
        c.d_slot = reinterpret_cast<uint16_t *>(reinterpret_cast<char *>(c.d_slot) + d);
        return CHEB_OK;
    }
    c.d_panels = cv.take<int32_t>(c.h_panels.size());
    c.d_wchunk = cv.take<int32_t>(c.h_wchunk.size());
    c.d_wrow = cv.take<int32_t>(c.h_wrow.size());
    c.d_rows = cv.take<uint32_t>(std::max<size_t>(c.h_rows.size(), 1));
    c.d_ent = cv.take<uint32_t>(std::max<size_t>(c.h_ent.size(), 1));
    c.d_slot = cv.take<uint16_t>(c.h_slot.size());
    if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_plan_bind_operator: workspace too small");
    CHEB_CUDA(cudaMemcpyAsync(c.d_panels, c.h_panels.data(), c.h_panels.size() * 4, cudaMemcpyHostToDevice, s));
    CHEB_CUDA(cudaMemcpyAsync(c.d_wchunk, c.h_wchunk.data(), c.h_wchunk.size() * 4, cudaMemcpyHostToDevice, s));
    CHEB_CUDA(cudaMemcpyAsync(c.d_wrow, c.h_wrow.data(), c.h_wrow.size() * 4, cudaMemcpyHostToDevice, s));
    if (!c.h_rows.empty())
        CHEB_CUDA(cudaMemcpyAsync(c.d_rows, c.h_rows.data(), c.h_rows.size() * 4, cudaMemcpyHostToDevice, s));
    if (!c.h_ent.empty())
        CHEB_CUDA(cudaMemcpyAsync(c.d_ent, c.h_ent.data(), c.h_ent.size() * 4, cudaMemcpyHostToDevice, s));
    CHEB_CUDA(cudaMemcpyAsync(c.d_slot, c.h_slot.data(), c.h_slot.size() * 2, cudaMemcpyHostToDevice, s));
    return CHEB_OK;
}

void col_free(ColLists &c) {
    if (c.tmp) cudaFree(c.tmp);
    c.tmp = nullptr;
}

void col_release_host(ColLists &c) {
    col_free(c);  // (after the stream has been synchronised)
    std::vector<int32_t>().swap(c.h_wchunk);
    std::vector<int32_t>().swap(c.h_wrow);
    std::vector<uint32_t>().swap(c.h_rows);
    std::vector<uint32_t>().swap(c.h_ent);
    std::vector<uint16_t>().swap(c.h_slot);
    c.bound = c.built;
}

}  // namespace cheb
