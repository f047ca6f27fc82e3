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

// out[0] = panels, out[1] = largest union, out[2] = 1 if a single column does
// not fit (no column kernel for this pattern).  stamp: int32[nbr] set to -1.
__global__ void __launch_bounds__(GP_NT) k_gp_panels(const int64_t *rp, const int32_t *ci, int64_t nbr, int P,
                                                     int ucap, int32_t *stamp, int32_t *panels, int64_t *out) {
    __shared__ int64_t sh[GP_NWARP];
    const int tid = threadIdx.x;
    int64_t j = 0;
    int32_t panel = 0, mu = 0;
    while (j < nbr) {
        int cnt = 0, ncols = 0;
        const int64_t j0 = j;
        while (j < nbr && ncols < P) {
            int64_t add = 0;
            for (int64_t e = rp[j] + tid; e < rp[j + 1]; e += GP_NT) add += stamp[ci[e]] != panel;
            add = gp_block_sum(add, sh);  // reads of column j all happen before this barrier
            if (cnt + add > ucap) break;
            for (int64_t e = rp[j] + tid; e < rp[j + 1]; e += GP_NT) stamp[ci[e]] = panel;
            __syncthreads();
            cnt += (int)add;
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
            panels[4 * panel + 2] = cnt;
            panels[4 * panel + 3] = 0;
        }
        mu = max(mu, cnt);
        ++panel;
    }
    if (tid == 0) {
        out[0] = panel;
        out[1] = mu;
        out[2] = 0;
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

// Dynamic shared memory of k_gp_rows: bitmap words (+ the fill pass's histogram).
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
    k_gp_panels<<<1, GP_NT, 0, s>>>(plan->rp, plan->ci, nbr, COL_P, ucap, stamp, pan, out);
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
