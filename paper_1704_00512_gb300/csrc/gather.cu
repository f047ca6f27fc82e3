// Gather plan of the column-order step kernel built on the device (Eq. 3
// restricted to the pattern; column independence, Sec. "Expansion in
// Chebyshev polynomials"): from the device block-CSR patterns of P_out and of
// the operator, with the same panels, row order, warp streams and entry words
// as the host builder in colstep.cu (bit for bit).
//
//   k_gp_panels  one thread block walks the block columns in order and closes a
//                panel when COL_P columns are in it or the next column's new
//                rows would overflow the union capacity (a stamp per row marks
//                the rows already in the open panel);
//   k_gp_rows    one thread block per panel: the union of the panel's
//                columns' rows as a bitmap with ranks (slot = rank), per union
//                row the count of operator entries whose column is in the union,
//                and -- in the fill pass -- the rows dealt to the NW warps by
//                decreasing chunk count (each to the warp with the least work so
//                far, ties to the lowest warp), the row words, the entry streams
//                interleaved by slot parity and padded with zero-block entries,
//                and the union slot of every P_out block of the panel;
//   k_gp_scan    offsets of the panels' chunks and rows.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "plan.cuh"

namespace cheb {

constexpr int GP_NT = 512;
constexpr int GP_NWARP = GP_NT / 32;
constexpr int GP_MAXU = 1 << COL_SLOT_BITS;  // union slots
constexpr int GP_HMAX = 4096;                // chunk counts of a row (rows hold <= 65536 blocks)
static_assert(GP_NWARP == COL_NW, "one warp of the builder per warp stream of the step kernel");

// Block-wide integer sum, returned to every thread.
__device__ __forceinline__ int64_t gp_block_sum(int64_t v, int64_t *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    int64_t r = 0;
#pragma unroll
    for (int i = 0; i < GP_NWARP; ++i) r += sh[i];
    __syncthreads();
    return r;
}
__device__ __forceinline__ int gp_block_max(int v, int *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    int r = 0;
#pragma unroll
    for (int i = 0; i < GP_NWARP; ++i) r = max(r, sh[i]);
    __syncthreads();
    return r;
}

// The panel walk shared by every panel set: within each system [sys_col[s],
// sys_col[s+1]) (one system 0..nbr when sys_col is NULL) the block columns are
// taken in order, and a panel is closed when P columns are in it or the next
// column would take its union of rows above ucap or its blocks above bcap.
// panels: (first column, columns, union rows, 0) per panel; aux (or NULL):
// (blocks, system) per panel.  out[0] = panels, out[1] = largest union, out[2]
// = 1 if a single column does not fit, out[3] = most blocks of a panel.
// stamp: int32[nbr] set to -1.
__global__ void __launch_bounds__(GP_NT) k_gp_panels(const int64_t *rp, const int32_t *ci, int64_t nbr, int P,
                                                     int64_t ucap, int64_t bcap, const int64_t *sys_col, int nsys,
                                                     int32_t *stamp, int32_t *panels, int32_t *aux, int64_t *out) {
    __shared__ int64_t sh[GP_NWARP];
    const int tid = threadIdx.x;
    int32_t panel = 0;
    int64_t mu = 0, mb = 0;
    for (int sy = 0; sy < nsys; ++sy) {
        int64_t j = sys_col ? sys_col[sy] : 0;
        const int64_t end = sys_col ? sys_col[sy + 1] : nbr;
        while (j < end) {
            int64_t cnt = 0, nblk = 0;
            int ncols = 0;
            const int64_t j0 = j;
            while (j < end && ncols < P) {
                const int64_t len = rp[j + 1] - rp[j];
                int64_t add = 0;
                for (int64_t e = rp[j] + tid; e < rp[j + 1]; e += GP_NT) add += stamp[ci[e]] != panel;
                add = gp_block_sum(add, sh);  // reads of column j all happen before this barrier
                if (cnt + add > ucap || nblk + len > bcap) break;
                for (int64_t e = rp[j] + tid; e < rp[j + 1]; e += GP_NT) stamp[ci[e]] = panel;
                __syncthreads();
                cnt += add;
                nblk += len;
                ++ncols;
                ++j;
            }
            if (ncols == 0) {
                if (tid == 0) out[2] = 1;
                return;
            }
            if (tid == 0) {
                panels[4 * panel] = (int32_t)j0;
                panels[4 * panel + 1] = ncols;
                panels[4 * panel + 2] = (int32_t)cnt;
                panels[4 * panel + 3] = 0;
                if (aux) {
                    aux[2 * panel] = (int32_t)nblk;
                    aux[2 * panel + 1] = sy;
                }
            }
            mu = max(mu, cnt);
            mb = max(mb, nblk);
            ++panel;
        }
    }
    if (tid == 0) {
        out[0] = panel;
        out[1] = mu;
        out[2] = 0;
        out[3] = mb;
    }
}

struct GpArgs {
    const int64_t *rp;
    const int32_t *ci;
    int64_t nbr;
    const int64_t *lrp;
    const int32_t *lci;
    int64_t nnzL;
    const int32_t *panels;
    // count pass
    int64_t *cnt_chunks, *cnt_rows;
    int32_t *cnt_maxrow;
    // fill pass
    const int64_t *chunk_off, *row_off;
    int32_t *wchunk, *wrow;
    uint32_t *rows, *ent;
    uint16_t *slot;
    int32_t *err;
};

template <bool FILL>
__global__ void __launch_bounds__(GP_NT) k_gp_rows(const GpArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ int ulist[GP_MAXU];
    __shared__ int work[GP_MAXU];
    __shared__ int cm[GP_MAXU];
    __shared__ int row_ch[GP_MAXU];
    __shared__ int row_ro[GP_MAXU];
    __shared__ int16_t order[GP_MAXU];
    __shared__ uint8_t wsel[GP_MAXU];
    __shared__ int wsum[32];
    __shared__ int64_t sh[GP_NWARP];
    __shared__ int shi[GP_NWARP];
    __shared__ int64_t bin_ch[COL_NW + 1];
    __shared__ int bin_ro[COL_NW + 1];
    constexpr int CW = COL_EK * 32 / COL_P;  // entries per chunk
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t p = blockIdx.x;
    const int j0 = a.panels[4 * p], nc = a.panels[4 * p + 1], nu_plan = a.panels[4 * p + 2];
    const int64_t nw = (a.nbr + 31) / 32;
    uint2 *bits = reinterpret_cast<uint2 *>(dsm);

    // 1. union bitmap of the panel's columns' rows, ranks, sorted union list
    for (int64_t w = tid; w < nw; w += GP_NT) bits[w] = make_uint2(0u, 0u);
    __syncthreads();
    for (int q = 0; q < nc; ++q)
        for (int64_t e = a.rp[j0 + q] + tid; e < a.rp[j0 + q + 1]; e += GP_NT) {
            const int K = a.ci[e];
            atomicOr(&bits[K >> 5].x, 1u << (K & 31));
        }
    __syncthreads();
    const int64_t chunk = (nw + GP_NT - 1) / GP_NT;
    const int64_t wb = min(nw, (int64_t)tid * chunk), we = min(nw, wb + chunk);
    int cnt = 0;
    for (int64_t w = wb; w < we; ++w) cnt += __popc(bits[w].x);
    int total;
    int run = block_excl_scan<GP_NWARP>(cnt, wsum, &total);
    const int nu = total;
    if (nu != nu_plan || nu > GP_MAXU) {  // uniform
        if (tid == 0) atomicExch(a.err, 1);
        return;
    }
    for (int64_t w = wb; w < we; ++w) {
        unsigned m = bits[w].x;
        bits[w].y = (unsigned)run;
        while (m) {
            const int b = __ffs(m) - 1;
            ulist[run++] = (int)(w * 32 + b);
            m &= m - 1u;
        }
    }
    for (int u = tid; u < nu; u += GP_NT) cm[u] = 0;
    __syncthreads();

    // 2. the panel columns holding a block of each union row; slots of the
    // panel's P_out blocks
    for (int q = 0; q < nc; ++q)
        for (int64_t e = a.rp[j0 + q] + tid; e < a.rp[j0 + q + 1]; e += GP_NT) {
            const int sl = rank_of(bits, a.ci[e]);
            atomicOr(&cm[sl], 1 << q);
            if (FILL) a.slot[e] = (uint16_t)sl;
        }

    // 3. per union row: operator entries in the union, chunks
    int mymax = 0;
    int64_t mych = 0;
    for (int u = tid; u < nu; u += GP_NT) {
        const int I = ulist[u];
        int n = 0;
        for (int64_t e = a.lrp[I]; e < a.lrp[I + 1]; ++e) n += rank_of(bits, a.lci[e]) >= 0;
        const int wk = max(1, (n + CW - 1) / CW);
        work[u] = wk;
        mymax = max(mymax, n);
        mych += wk;
    }
    const int64_t chunks = gp_block_sum(mych, sh);  // (barrier: work[], cm[] complete)
    const int maxrow = gp_block_max(mymax, shi);
    if (!FILL) {
        if (tid == 0) {
            a.cnt_chunks[p] = chunks;
            a.cnt_rows[p] = nu;
            a.cnt_maxrow[p] = maxrow;
        }
        return;
    }

    // 4. rows to warps: decreasing chunk count (stable), each to the warp
    // with the fewest chunks so far (the lowest such warp)
    if (tid == 0) {
        int *hist = reinterpret_cast<int *>(dsm + (((size_t)nw * sizeof(uint2) + 15) & ~(size_t)15));
        int maxw = 0;
        for (int u = 0; u < nu; ++u) maxw = max(maxw, work[u]);
        if (maxw > GP_HMAX) {
            atomicExch(a.err, 2);
            maxw = GP_HMAX;  // the lists are not used after an error; keep the writes in bounds
        }
        for (int v = 0; v <= maxw; ++v) hist[v] = 0;
        for (int u = 0; u < nu; ++u) ++hist[min(work[u], maxw)];
        int at = 0;
        for (int v = maxw; v >= 0; --v) {
            const int t = hist[v];
            hist[v] = at;
            at += t;
        }
        for (int u = 0; u < nu; ++u) order[hist[min(work[u], maxw)]++] = (int16_t)u;
        int64_t load[COL_NW];
        int nrow[COL_NW];
#pragma unroll
        for (int w = 0; w < COL_NW; ++w) {
            load[w] = 0;
            nrow[w] = 0;
        }
        for (int i = 0; i < nu; ++i) {
            const int u = order[i];
            int best = 0;
#pragma unroll
            for (int w = 1; w < COL_NW; ++w)
                if (load[w] < load[best]) best = w;
#pragma unroll
            for (int w = 0; w < COL_NW; ++w)
                if (w == best) {
                    load[w] += work[u];
                    ++nrow[w];
                }
            wsel[u] = (uint8_t)best;
        }
        int64_t ch = 0;
        int ro = 0;
#pragma unroll
        for (int w = 0; w < COL_NW; ++w) {
            bin_ch[w] = ch;
            bin_ro[w] = ro;
            ch += load[w];
            ro += nrow[w];
        }
        bin_ch[COL_NW] = ch;
        bin_ro[COL_NW] = ro;
    }
    __syncthreads();

    // 5. warp w lays out the rows of stream w in increasing union slot
    {
        const int w = warp;
        const unsigned lt = (1u << lane) - 1u;
        int ro = bin_ro[w];
        int64_t ch = bin_ch[w];
        for (int base = 0; base < nu; base += 32) {
            const int u = base + lane;
            const bool sel = u < nu && wsel[u] == w;
            const unsigned m = __ballot_sync(0xffffffffu, sel);
            const int wk = sel ? work[u] : 0;
            int incl = wk;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int n = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += n;
            }
            if (sel) {
                row_ro[u] = ro + __popc(m & lt);
                row_ch[u] = (int)(ch + incl - wk);
            }
            ro += __popc(m);
            ch += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            a.wchunk[p * (COL_NW + 1) + w] = (int32_t)(a.chunk_off[p] + bin_ch[w]);
            a.wrow[p * (COL_NW + 1) + w] = (int32_t)(a.row_off[p] + bin_ro[w]);
            if (w == 0) {
                a.wchunk[p * (COL_NW + 1) + COL_NW] = (int32_t)(a.chunk_off[p] + bin_ch[COL_NW]);
                a.wrow[p * (COL_NW + 1) + COL_NW] = (int32_t)(a.row_off[p] + bin_ro[COL_NW]);
            }
        }
    }
    __syncthreads();

    // 6. row words and entry streams.  Position t of a chunk takes an entry
    // whose slot has parity (t ^ (t >> 3)) & 1, so that the two K-groups of a
    // quarter warp read different banks; when one parity runs out the other
    // fills in.  Entries of one parity keep the operator row's order.
    const uint32_t zero_word = (uint32_t)a.nnzL << COL_SLOT_BITS;
    for (int u = tid; u < nu; u += GP_NT) {
        const int I = ulist[u];
        const unsigned m = (unsigned)cm[u];
        const int pc = __popc(m);
        uint32_t hw = 0;
        if (pc <= 2) {
            const uint32_t ca = (uint32_t)(__ffs(m) - 1);
            const uint32_t cb = pc == 2 ? (uint32_t)(31 - __clz(m)) : ca;
            hw = 1u | (ca << 1) | (cb << 3);
        }
        a.rows[a.row_off[p] + row_ro[u]] = (uint32_t)u | (hw << COL_SLOT_BITS) | ((uint32_t)work[u] << COL_ROW_SHIFT);
        uint32_t *out = a.ent + (a.chunk_off[p] + row_ch[u]) * CW;
        const int64_t e0 = a.lrp[I], e1 = a.lrp[I + 1];
        int n0 = 0, n1 = 0;
        for (int64_t e = e0; e < e1; ++e) {
            const int sl = rank_of(bits, a.lci[e]);
            if (sl >= 0) {
                if (sl & 1) ++n1; else ++n0;
            }
        }
        int64_t c0 = e0, c1 = e0;
        int t0 = 0, t1 = 0;
        const int n = n0 + n1;
        for (int pos = 0; pos < n; ++pos) {
            const int t = pos % CW;
            int k = (t ^ (t >> 3)) & 1;
            if (k == 0 ? t0 >= n0 : t1 >= n1) k ^= 1;
            int64_t &c = k ? c1 : c0;
            int sl = -1;
            while (c < e1) {
                sl = rank_of(bits, a.lci[c]);
                if (sl >= 0 && (sl & 1) == k) break;
                ++c;
            }
            if (c >= e1) {  // cannot happen with the counts above; never emit a bad block index
                atomicExch(a.err, 3);
                out[pos] = zero_word;
            } else {
                out[pos] = ((uint32_t)c << COL_SLOT_BITS) | (uint32_t)sl;
            }
            ++c;
            if (k) ++t1; else ++t0;
        }
        for (int pos = n; pos < work[u] * CW; ++pos) out[pos] = zero_word;
    }
}

// off[i] = sum of v[0..i), off[n] = total (one thread block of 1024)
__global__ void __launch_bounds__(1024) k_gp_scan(const int64_t *v, int64_t n, int64_t *off) {
    __shared__ int64_t part[1024];
    const int tid = threadIdx.x;
    const int64_t per = (n + 1023) / 1024, b = min(n, (int64_t)tid * per), e = min(n, b + per);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += v[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int64_t run = 0;
        for (int i = 0; i < 1024; ++i) {
            const int64_t t = part[i];
            part[i] = run;
            run += t;
        }
        off[n] = run;
    }
    __syncthreads();
    int64_t run = part[tid];
    for (int64_t i = b; i < e; ++i) {
        off[i] = run;
        run += v[i];
    }
}

// ---------------------------------------------------------------------------
// The plan of P_out itself, on the device: checks, transposition map, the
// longest block row.

// first[0]: first row whose row_ptr range is decreasing or leaves [0, nnzb];
// first[1]: first row with a column out of range; first[2]: first row whose
// columns do not strictly ascend; first[3]: first row without its diagonal
// block (nbr where none).  *maxlen: the longest row.
__global__ void k_pc_check(const int64_t *rp, const int32_t *ci, int64_t nbr, int64_t nnzb, int64_t *first,
                           int32_t *maxlen) {
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= nbr) return;
    const int64_t a = rp[I], b = rp[I + 1];
    if (a < 0 || b > nnzb || b < a) {
        atomicMin(reinterpret_cast<long long *>(first), (long long)I);
        return;
    }
    atomicMax(maxlen, (int32_t)(b - a < (int64_t)INT32_MAX ? b - a : (int64_t)INT32_MAX));
    bool diag = false;
    for (int64_t p = a; p < b; ++p) {
        const int32_t c = ci[p];
        if (c < 0 || c >= nbr) {
            atomicMin(reinterpret_cast<long long *>(first + 1), (long long)I);
            return;
        }
        if (p > a && c <= ci[p - 1]) {
            atomicMin(reinterpret_cast<long long *>(first + 2), (long long)I);
            return;
        }
        diag |= c == I;
    }
    if (!diag) atomicMin(reinterpret_cast<long long *>(first + 3), (long long)I);
}

// tperm[p] = position of block (J, I) for block p = (I, J); *bad = the first
// block without a transpose (nnzb where none).  Runs on a checked pattern.
__global__ void k_pc_tperm(const int64_t *rp, const int32_t *ci, int64_t nbr, int64_t nnzb, int32_t *tperm,
                           int64_t *bad) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nnzb) return;
    const int64_t I = row_of(rp, nbr, p);
    const int64_t q = find_in_row(rp, ci, ci[p], (int32_t)I);
    if (q < 0)
        atomicMin(reinterpret_cast<long long *>(bad), (long long)p);
    else
        tperm[p] = (int32_t)q;
}

// Checks of an operator pattern (n blocks): first[0] rows decreasing or out of
// [0, n] or longer than 65536 blocks; first[1] a column out of range.
__global__ void k_op_check(const int64_t *rp, const int32_t *ci, int64_t nbr, int64_t n, int64_t *first) {
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= nbr) return;
    const int64_t a = rp[I], b = rp[I + 1];
    if (a < 0 || b > n || b < a || b - a > 65536) {
        atomicMin(reinterpret_cast<long long *>(first), (long long)I);
        return;
    }
    for (int64_t p = a; p < b; ++p)
        if (ci[p] < 0 || ci[p] >= nbr) {
            atomicMin(reinterpret_cast<long long *>(first + 1), (long long)I);
            return;
        }
}

// Row lists of one panel set (the FP64 step kernel's and the resident
// kernel's): per panel (pairs[2p], pairs[2p+1] = first column, columns), per
// union row in increasing order, the operator row's blocks whose column is in
// the union as (offset in the operator row << 16 | union slot).  Count pass:
// cnt[p] entries, nrow[p] = union rows + 1.  Fill pass: row pointers from
// row_base[p] (global entry offsets from ent_off[p]) and the entries.
template <bool FILL>
__global__ void __launch_bounds__(GP_NT) k_rl_rows(const int64_t *rp, const int32_t *ci, int64_t nbr,
                                                   const int64_t *lrp, const int32_t *lci, const int32_t *pairs,
                                                   int maxu, int64_t *cnt, int64_t *nrow, const int64_t *ent_off,
                                                   const int64_t *row_base, int32_t *lrow_ptr, uint32_t *lent,
                                                   int32_t *err) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ int wsum[32];
    const int tid = threadIdx.x;
    const int64_t p = blockIdx.x;
    const int j0 = pairs[2 * p], nc = pairs[2 * p + 1];
    const int64_t nw = (nbr + 31) / 32;
    uint2 *bits = reinterpret_cast<uint2 *>(dsm);
    int *ulist = reinterpret_cast<int *>(dsm + (((size_t)nw * sizeof(uint2) + 15) & ~(size_t)15));
    for (int64_t w = tid; w < nw; w += GP_NT) bits[w] = make_uint2(0u, 0u);
    __syncthreads();
    for (int q = 0; q < nc; ++q)
        for (int64_t e = rp[j0 + q] + tid; e < rp[j0 + q + 1]; e += GP_NT) {
            const int K = ci[e];
            atomicOr(&bits[K >> 5].x, 1u << (K & 31));
        }
    __syncthreads();
    const int64_t chunk = (nw + GP_NT - 1) / GP_NT;
    const int64_t wb = min(nw, (int64_t)tid * chunk), we = min(nw, wb + chunk);
    int c = 0;
    for (int64_t w = wb; w < we; ++w) c += __popc(bits[w].x);
    int nu;
    int run = block_excl_scan<GP_NWARP>(c, wsum, &nu);
    if (nu > maxu) {  // uniform
        if (tid == 0) atomicExch(err, 1);
        return;
    }
    for (int64_t w = wb; w < we; ++w) {
        unsigned m = bits[w].x;
        bits[w].y = (unsigned)run;
        while (m) {
            const int b = __ffs(m) - 1;
            ulist[run++] = (int)(w * 32 + b);
            m &= m - 1u;
        }
    }
    __syncthreads();
    // thread t takes union rows [u0, u1) in order; a block scan gives offsets
    const int rch = (nu + GP_NT - 1) / GP_NT, u0 = min(nu, tid * rch), u1 = min(nu, u0 + rch);
    int mine = 0;
    for (int u = u0; u < u1; ++u) {
        const int I = ulist[u];
        for (int64_t a = lrp[I]; a < lrp[I + 1]; ++a) mine += rank_of(bits, lci[a]) >= 0;
    }
    int total;
    int off = block_excl_scan<GP_NWARP>(mine, wsum, &total);
    if (!FILL) {
        if (tid == 0) {
            cnt[p] = total;
            nrow[p] = nu + 1;
        }
        return;
    }
    const int64_t e0 = ent_off[p], r0 = row_base[p];
    for (int u = u0; u < u1; ++u) {
        const int I = ulist[u];
        lrow_ptr[r0 + u] = (int32_t)(e0 + off);
        for (int64_t a = lrp[I]; a < lrp[I + 1]; ++a) {
            const int sl = rank_of(bits, lci[a]);
            if (sl >= 0) lent[e0 + off++] = ((uint32_t)(a - lrp[I]) << 16) | (uint32_t)sl;
        }
    }
    if (tid == 0) lrow_ptr[r0 + nu] = (int32_t)(e0 + total);
}

// Dynamic shared memory of k_gp_rows: bitmap words (+ the fill pass's histogram).// Dynamic shared memory of k_gp_rows: bitmap words (+ the fill pass's histogram).
static size_t gp_dyn_smem(int64_t nbr, bool fill) {
    const size_t bits = align_up((size_t)((nbr + 31) / 32) * sizeof(uint2), 16);
    return bits + (fill ? (GP_HMAX + 1) * sizeof(int) : 0);
}

int col_build_device(cheb_plan *plan, const cheb_bsr *L, int32_t ucap, cudaStream_t s) {
    ColLists c;
    c.P = COL_P;
    c.NW = COL_NW;
    c.ucap = ucap;
    constexpr int CW = COL_EK * 32 / COL_P;
    const int64_t nbr = plan->nbr, nnzL = L->nnzb;
    if (nnzL + 1 >= ((int64_t)1 << (32 - COL_SLOT_BITS))) return CHEB_ERR_NOSPACE;
    const size_t dyn_fill = gp_dyn_smem(nbr, true);
    if (dyn_fill + 48 * 1024 > (size_t)CHEB_MAX_DYN_SMEM) return CHEB_ERR_NOSPACE;
    // scratch: stamps, panels (at most one per column), counts and offsets
    const size_t n1 = (size_t)nbr + 1;
    size_t off = 0;
    auto at = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const size_t o_stamp = at(nbr * 4), o_pan = at(4 * nbr * 4), o_out = at(8 * 8), o_chunks = at(nbr * 8),
                 o_rows = at(nbr * 8), o_max = at(nbr * 4), o_choff = at(n1 * 8), o_rooff = at(n1 * 8);
    char *scr = nullptr;
    CHEB_CUDA(cudaMalloc(&scr, off));
    struct Free {
        char *p;
        ~Free() { cudaFree(p); }
    } free_scr{scr};
    int32_t *stamp = reinterpret_cast<int32_t *>(scr + o_stamp), *pan = reinterpret_cast<int32_t *>(scr + o_pan);
    int64_t *out = reinterpret_cast<int64_t *>(scr + o_out);
    int64_t *cnt_chunks = reinterpret_cast<int64_t *>(scr + o_chunks), *cnt_rows = reinterpret_cast<int64_t *>(scr + o_rows);
    int32_t *cnt_max = reinterpret_cast<int32_t *>(scr + o_max);
    int64_t *choff = reinterpret_cast<int64_t *>(scr + o_choff), *rooff = reinterpret_cast<int64_t *>(scr + o_rooff);
    int32_t *err = reinterpret_cast<int32_t *>(out + 4);
    CHEB_CUDA(cudaMemsetAsync(stamp, 0xff, nbr * 4, s));
    CHEB_CUDA(cudaMemsetAsync(out, 0, 8 * 8, s));
    k_gp_panels<<<1, GP_NT, 0, s>>>(plan->rp, plan->ci, nbr, COL_P, ucap, INT64_MAX, nullptr, 1, stamp, pan, nullptr,
                                    out);
    CHEB_TRY(check_launch("k_gp_panels"));
    int64_t h_out[3];
    CHEB_CUDA(cudaMemcpyAsync(h_out, out, sizeof(h_out), cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    if (h_out[2]) return CHEB_ERR_NOSPACE;  // a single column does not fit: no column kernel
    const int64_t np = h_out[0];
    c.n_panels = np;
    c.max_union = (int32_t)h_out[1];
    GpArgs a{};
    a.rp = plan->rp;
    a.ci = plan->ci;
    a.nbr = nbr;
    a.lrp = L->row_ptr;
    a.lci = L->col_idx;
    a.nnzL = nnzL;
    a.panels = pan;
    a.cnt_chunks = cnt_chunks;
    a.cnt_rows = cnt_rows;
    a.cnt_maxrow = cnt_max;
    a.err = err;
    const size_t dyn_count = gp_dyn_smem(nbr, false);
    CHEB_CUDA(cudaFuncSetAttribute(k_gp_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_count));
    CHEB_CUDA(cudaFuncSetAttribute(k_gp_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_fill));
    k_gp_rows<false><<<(unsigned)np, GP_NT, dyn_count, s>>>(a);
    CHEB_TRY(check_launch("k_gp_rows count"));
    k_gp_scan<<<1, 1024, 0, s>>>(cnt_chunks, np, choff);
    k_gp_scan<<<1, 1024, 0, s>>>(cnt_rows, np, rooff);
    CHEB_TRY(check_launch("k_gp_scan", 2));
    std::vector<int32_t> h_max(np);
    int64_t tot[2];
    int32_t h_err = 0;
    CHEB_CUDA(cudaMemcpyAsync(h_max.data(), cnt_max, np * 4, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(&tot[0], choff + np, 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(&tot[1], rooff + np, 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    if (h_err) return fail(CHEB_ERR_INVALID, "gather plan: inconsistent panel union (code %d)", h_err);
    if (tot[0] * CW >= (int64_t)INT32_MAX) return CHEB_ERR_NOSPACE;
    for (const int32_t m : h_max) c.max_row = std::max(c.max_row, m);
    c.n_entries = tot[0] * CW;
    c.n_rows = tot[1];
    c.n_slot = plan->nnzb;
    // the lists, in device memory of their own until cheb_plan_bind_operator
    // copies them into the operator workspace
    c.built = true;  // (sizes complete: bytes() counts them from here on)
    const size_t nbytes = c.bytes();
    CHEB_CUDA(cudaMalloc(&c.tmp, nbytes));
    struct FreeOnError {
        ColLists &c;
        bool armed = true;
        ~FreeOnError() {
            if (armed) col_free(c);
        }
    } guard{c};
    Carve cv(c.tmp, nbytes);
    c.d_panels = cv.take<int32_t>(4 * np);
    c.d_wchunk = cv.take<int32_t>(np * (COL_NW + 1));
    c.d_wrow = cv.take<int32_t>(np * (COL_NW + 1));
    c.d_rows = cv.take<uint32_t>(std::max<int64_t>(c.n_rows, 1));
    c.d_ent = cv.take<uint32_t>(std::max<int64_t>(c.n_entries, 1));
    c.d_slot = cv.take<uint16_t>(c.n_slot);
    CHEB_CUDA(cudaMemcpyAsync(c.d_panels, pan, 4 * np * 4, cudaMemcpyDeviceToDevice, s));
    a.chunk_off = choff;
    a.row_off = rooff;
    a.wchunk = c.d_wchunk;
    a.wrow = c.d_wrow;
    a.rows = c.d_rows;
    a.ent = c.d_ent;
    a.slot = c.d_slot;
    k_gp_rows<true><<<(unsigned)np, GP_NT, dyn_fill, s>>>(a);
    CHEB_TRY(check_launch("k_gp_rows fill"));
    CHEB_CUDA(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    if (h_err) return fail(CHEB_ERR_INVALID, "gather plan: inconsistent row lists (code %d)", h_err);
    c.device = true;
    guard.armed = false;
    plan->col = std::move(c);
    return CHEB_OK;
}

}  // namespace cheb

namespace cheb {

// ---------------------------------------------------------------------------
// Host-side launchers of the plan kernels (plan.cu drives them).

int gp_check_pattern(const int64_t *rp, const int32_t *ci, int64_t nbr, int64_t nnzb, int64_t first[4],
                     int32_t *maxlen, cudaStream_t s) {
    int64_t *d = nullptr;
    CHEB_CUDA(cudaMallocAsync(&d, 5 * 8, s));
    const int64_t init[5] = {nbr, nbr, nbr, nbr, 0};
    CHEB_CUDA(cudaMemcpyAsync(d, init, sizeof(init), cudaMemcpyHostToDevice, s));
    k_pc_check<<<(unsigned)((nbr + 255) / 256), 256, 0, s>>>(rp, ci, nbr, nnzb, d,
                                                           reinterpret_cast<int32_t *>(d + 4));
    const int rc = check_launch("k_pc_check");
    int64_t h[5] = {0, 0, 0, 0, 0};
    if (rc == CHEB_OK) CHEB_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaFreeAsync(d, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    CHEB_TRY(rc);
    for (int i = 0; i < 4; ++i) first[i] = h[i];
    int32_t ml;
    std::memcpy(&ml, &h[4], 4);
    *maxlen = ml;
    return CHEB_OK;
}

int gp_tperm(const int64_t *rp, const int32_t *ci, int64_t nbr, int64_t nnzb, int32_t *tperm, int64_t *bad,
             cudaStream_t s) {
    int64_t *d = nullptr;
    CHEB_CUDA(cudaMallocAsync(&d, 8, s));
    CHEB_CUDA(cudaMemcpyAsync(d, &nnzb, 8, cudaMemcpyHostToDevice, s));
    k_pc_tperm<<<(unsigned)((nnzb + 255) / 256), 256, 0, s>>>(rp, ci, nbr, nnzb, tperm, d);
    const int rc = check_launch("k_pc_tperm");
    if (rc == CHEB_OK) CHEB_CUDA(cudaMemcpyAsync(bad, d, 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaFreeAsync(d, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    return rc;
}

int gp_walk(const int64_t *rp, const int32_t *ci, int64_t nbr, int P, int64_t ucap, int64_t bcap,
            const std::vector<int64_t> &sys_col, std::vector<int32_t> &panels4, std::vector<int32_t> &aux,
            int64_t out[4], cudaStream_t s) {
    const int nsys = (int)sys_col.size() - 1;
    size_t off = 0;
    auto at = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const size_t o_stamp = at(nbr * 4), o_pan = at(4 * nbr * 4), o_aux = at(2 * nbr * 4), o_out = at(4 * 8),
                 o_sys = at(sys_col.size() * 8);
    char *scr = nullptr;
    CHEB_CUDA(cudaMalloc(&scr, off));
    struct Free {
        char *p;
        ~Free() { cudaFree(p); }
    } free_scr{scr};
    int32_t *stamp = reinterpret_cast<int32_t *>(scr + o_stamp), *pan = reinterpret_cast<int32_t *>(scr + o_pan),
            *ax = reinterpret_cast<int32_t *>(scr + o_aux);
    int64_t *dout = reinterpret_cast<int64_t *>(scr + o_out), *dsys = reinterpret_cast<int64_t *>(scr + o_sys);
    CHEB_CUDA(cudaMemsetAsync(stamp, 0xff, nbr * 4, s));
    CHEB_CUDA(cudaMemsetAsync(dout, 0, 4 * 8, s));
    CHEB_CUDA(cudaMemcpyAsync(dsys, sys_col.data(), sys_col.size() * 8, cudaMemcpyHostToDevice, s));
    k_gp_panels<<<1, GP_NT, 0, s>>>(rp, ci, nbr, P, ucap, bcap, dsys, nsys, stamp, pan, ax, dout);
    CHEB_TRY(check_launch("k_gp_panels"));
    CHEB_CUDA(cudaMemcpyAsync(out, dout, 4 * 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    if (out[2]) return CHEB_OK;  // the caller reports the column that does not fit
    panels4.resize(4 * out[0]);
    aux.resize(2 * out[0]);
    CHEB_CUDA(cudaMemcpyAsync(panels4.data(), pan, panels4.size() * 4, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(aux.data(), ax, aux.size() * 4, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    return CHEB_OK;
}

int gp_check_operator(const cheb_bsr *L, int64_t nbr, int64_t first[2], cudaStream_t s) {
    int64_t *d = nullptr;
    CHEB_CUDA(cudaMallocAsync(&d, 2 * 8, s));
    const int64_t init[2] = {nbr, nbr};
    CHEB_CUDA(cudaMemcpyAsync(d, init, sizeof(init), cudaMemcpyHostToDevice, s));
    k_op_check<<<(unsigned)((nbr + 255) / 256), 256, 0, s>>>(L->row_ptr, L->col_idx, nbr, L->nnzb, d);
    const int rc = check_launch("k_op_check");
    if (rc == CHEB_OK) CHEB_CUDA(cudaMemcpyAsync(first, d, 2 * 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaFreeAsync(d, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    return rc;
}

int row_lists_device(const int64_t *rp, const int32_t *ci, int64_t nbr, const cheb_bsr *L, const int32_t *pairs,
                     int64_t np, int maxu, RowLists &out, cudaStream_t s) {
    if (np == 0) return CHEB_OK;
    const size_t dyn = (((size_t)((nbr + 31) / 32) * sizeof(uint2) + 15) & ~(size_t)15) + (size_t)maxu * 4;
    if (dyn > (size_t)CHEB_MAX_DYN_SMEM - 2048)
        return fail(CHEB_ERR_NOSPACE, "cheb_plan_attach_operator: %zu bytes of panel bitmap and union", dyn);
    CHEB_CUDA(cudaFuncSetAttribute(k_rl_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    CHEB_CUDA(cudaFuncSetAttribute(k_rl_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int64_t *scr = nullptr;  // cnt, nrow [np]; ent_off, row_base [np + 1]; error flag
    CHEB_CUDA(cudaMalloc(&scr, (4 * np + 3) * 8));
    struct Free {
        int64_t *p;
        ~Free() { cudaFree(p); }
    } free_scr{scr};
    int64_t *cnt = scr, *nrow = scr + np, *ent_off = scr + 2 * np, *row_base = scr + 3 * np + 1;
    int32_t *err = reinterpret_cast<int32_t *>(scr + 4 * np + 2);
    CHEB_CUDA(cudaMemsetAsync(err, 0, 4, s));
    k_rl_rows<false><<<(unsigned)np, GP_NT, dyn, s>>>(rp, ci, nbr, L->row_ptr, L->col_idx, pairs, maxu, cnt, nrow,
                                                      nullptr, nullptr, nullptr, nullptr, err);
    k_gp_scan<<<1, 1024, 0, s>>>(cnt, np, ent_off);
    k_gp_scan<<<1, 1024, 0, s>>>(nrow, np, row_base);
    CHEB_TRY(check_launch("row lists count", 3));
    int64_t tot[2];
    int32_t h_err = 0;
    CHEB_CUDA(cudaMemcpyAsync(&tot[0], ent_off + np, 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(&tot[1], row_base + np, 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    if (h_err) return fail(CHEB_ERR_INVALID, "cheb_plan_attach_operator: panel union above the plan's maximum");
    if (tot[0] >= (int64_t)INT32_MAX)
        return fail(CHEB_ERR_NOSPACE, "cheb_plan_attach_operator: %lld list entries exceed the int32 offsets",
                    (long long)tot[0]);
    out.device = true;
    out.n_base = np;
    out.n_ptr = tot[1];
    out.n_ent = tot[0];
    CHEB_CUDA(cudaMalloc(&out.tmp, out.bytes()));
    Carve cv(out.tmp, out.bytes());
    out.d_base = cv.take<int64_t>(np);
    out.d_ptr = cv.take<int32_t>(std::max<int64_t>(out.n_ptr, 1));
    out.d_ent = cv.take<uint32_t>(std::max<int64_t>(out.n_ent, 1));
    CHEB_CUDA(cudaMemcpyAsync(out.d_base, row_base, np * 8, cudaMemcpyDeviceToDevice, s));
    k_rl_rows<true><<<(unsigned)np, GP_NT, dyn, s>>>(rp, ci, nbr, L->row_ptr, L->col_idx, pairs, maxu, nullptr,
                                                     nullptr, ent_off, row_base, out.d_ptr, out.d_ent, err);
    CHEB_TRY(check_launch("row lists fill"));
    CHEB_CUDA(cudaStreamSynchronize(s));
    return CHEB_OK;
}

}  // namespace cheb
