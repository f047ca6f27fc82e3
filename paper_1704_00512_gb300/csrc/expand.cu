// The hot path: one step of the masked Chebyshev recursion (Eq. 3) fused with
// the accumulation of several expansions (Eq. 1) and the moments that feed the
// penalty check (Eq. 5) and the mu search.
//
// Data flow of one step (one thread block per column panel, see plan.cu):
//   1. mark the rows of the panel's block columns in a shared bitmap and rank
//      them (prefix popcounts): the union of the columns' row lists;
//   2. gather the panel's columns of T_k into shared memory X[slot][4][4P]
//      (zero where a column has no block in that row);
//   3. each warp takes union rows I; its 32 lanes split into P column lanes x
//      32/P K-groups; a lane accumulates the full 4x4 block sum over K of
//      M~_IK X[K] for its column -- the masked product restricted to the
//      panel's columns (columns are independent, Sec. "Expansion in Chebyshev
//      polynomials").  The operator blocks M~_IK with K in the union come from
//      the plan's per-panel row lists, or from ranking the operator row's
//      column indices against the union bitmap;
//   4. when a row is done the K-groups' sums are combined by a reduce-scatter;
//      for the blocks of P_out only (the truncation, Sec. "Sparsity and
//      truncation") T_{k+1} = alpha * (M~ T_k) + beta * T_{k-1} is formed,
//      c_j[k+1] T_{k+1} added to every FP64 accumulator j, and Tr T_{k+1} and
//      <T_{k+1}, G> summed -- by each lane for its elements as soon as the row
//      is done (FP64), or in a pass over the panel's blocks after all rows
//      (FP32, whose latency-bound rows gain from many loads in flight);
//   5. the last thread block to finish sums the per-block moment partials in
//      a fixed order (deterministic) and resets the completion counter.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "plan.cuh"

namespace cheb {

template <typename T>
struct StepArgs {
    int64_t nw;  // bitmap words
    int32_t ucap;
    const int64_t *rp;
    const int32_t *ci;
    const int32_t *tperm;
    const int32_t *panels;
    const int64_t *Lrp;
    const int32_t *Lci;
    const T *Lv;
    const T *R;
    const T *Rm;
    T *C;
    T alpha, beta;
    int32_t nf;
    double *acc[MAX_F];
    const double *coef;
    int32_t coef_stride;
    int32_t term;
    const double *G;
    double *mom;   // device scalar for Tr T_{k+1} (or NULL)
    double *gmom;  // device scalar for <T_{k+1}, G> (or NULL)
    double *part;  // per-block partials
    int32_t *counter;
    int32_t round_bf16;  // store T_{k+1} rounded to bfloat16 (CHEB_BF16 mode)
    // operator row lists of the plan (NULL: rank the operator's rows each step)
    const int64_t *lrow_base;
    const int32_t *lrow_ptr;
    const uint32_t *lent;
};

// x rounded to the nearest bfloat16 (ties to even), returned as float
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ double bf16_round(double x) { return x; }
__device__ __forceinline__ dfl bf16_round(dfl x) { return x; }

template <typename T, int P, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_step(const StepArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int wsum[32];
    constexpr int NT = NW * 32;
    constexpr int KG = 32 / P;                  // K-groups per warp
    constexpr int BT = step_batch(P);          // operator blocks per staged batch
    constexpr int NU = BT / KG;                 // staged entries per K-group per batch
    constexpr int EPL = KG >= 16 ? 1 : 16 / KG;  // elements of a block sum per lane
    // FP64 rows are bound by the FMA pipe, which hides the memory latency of
    // finishing each row at once; FP32 rows are latency-bound and finish in a
    // separate pass over the panel's blocks with many loads in flight.
    constexpr bool FUSE = sizeof(T) == 8;
    const StepLayout lay = step_layout(a.nw, a.ucap, P, sizeof(T), NW);
    uint2 *bits = reinterpret_cast<uint2 *>(smem + lay.off_bits);
    int32_t *ulist = reinterpret_cast<int32_t *>(smem + lay.off_ulist);
    int32_t *oslot = reinterpret_cast<int32_t *>(smem + lay.off_pos);
    int2 *wlist = reinterpret_cast<int2 *>(smem + lay.off_wl);
    int *bslot = reinterpret_cast<int *>(smem + lay.off_bslot);
    T *hbuf = reinterpret_cast<T *>(smem + lay.off_hbuf);
    T *X = reinterpret_cast<T *>(smem + lay.off_x);
    double *red = reinterpret_cast<double *>(smem + lay.off_red);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j0 = a.panels[2 * blockIdx.x], ncols = a.panels[2 * blockIdx.x + 1];

    // 1. bitmap of the rows present in the panel's columns, ranks, union list
    for (int64_t w = tid; w < a.nw; w += NT) bits[w] = make_uint2(0u, 0u);
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
    if (nu > a.ucap) return;  // cannot happen for a plan-built launch (uniform exit)
    // 2. gather the panel's columns of T_k into X[slot][4][4P] (zero elsewhere)
    {
        uint4 *x4 = reinterpret_cast<uint4 *>(X);
        const int64_t n4 = (int64_t)nu * BB * P * sizeof(T) / 16;
        for (int64_t i = tid; i < n4; i += NT) x4[i] = make_uint4(0u, 0u, 0u, 0u);
        for (int64_t i = tid; i < (int64_t)nu * P; i += NT) oslot[i] = -1;
    }
    __syncthreads();
    for (int q = 0; q < ncols; ++q) {
        const int64_t b = a.rp[j0 + q], e = a.rp[j0 + q + 1];
        for (int64_t p = b + tid; p < e; p += NT) {
            const int K = a.ci[p];
            const int s = rank_of(bits, K);
            T v[16];
            const int32_t o = a.tperm[p];
            load16<T>(v, a.R + (int64_t)o * BB);
            T *xs = X + (int64_t)s * BB * P + 4 * q;
            const int sw = s & 1;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const T r4[4] = {v[4 * m], v[4 * m + 1], v[4 * m + 2], v[4 * m + 3]};
                Vec4<T>::st(xs + (m ^ sw) * 4 * P, r4);
            }
            oslot[s * P + q] = o;
        }
    }
    __syncthreads();

    double coefv[MAX_F];
#pragma unroll
    for (int f = 0; f < MAX_F; ++f) coefv[f] = f < a.nf ? a.coef[(int64_t)f * a.coef_stride + a.term] : 0.0;
    double tpart = 0.0, gpart = 0.0;

    // 3. union rows: masked block products M~_I. X for the panel's columns.
    // Each warp takes union rows s = warp, warp + NW, ...; the in-union
    // operator blocks of its rows form one stream of batches of up to BT.  A
    // batch's operator blocks are copied to shared memory with asynchronous
    // copies (cp.async) while the batch before it is multiplied; a row's last
    // batch may be followed by the next row's first, so the next row's blocks
    // are in flight while the current row is finished.  A batch never spans
    // two rows.  In a batch each of the 32/P K-groups takes every (32/P)-th
    // entry; a lane multiplies the 4x4 operator block by the panel block of
    // its column q.  The batch's entries come either from the plan's operator
    // row lists (precomputed per panel and union row) or, without lists, from
    // ranking the operator row's column indices against the union bitmap.
    {
        const int q = lane % P, kg = lane / P;
        // two batches of BT staged blocks, chunks XOR-swizzled like the panel blocks
        unsigned char *hb = reinterpret_cast<unsigned char *>(hbuf + (size_t)warp * 2 * BT * BB);
        int *bs = bslot + warp * 64;  // union slots of the staged blocks
        // batch entry of this lane: operator block index, union slot
        auto issue = [&](int buf, int n, int64_t blk, int slot) {
            if (lane < n) {
                bs[buf * BT + lane] = slot;
                const T *src = a.Lv + blk * BB;
                const int b = buf * BT + lane;
#pragma unroll
                for (int c = 0; c < (int)(BB * sizeof(T) / 16); ++c)
                    cp_async16(hb + rchunk<T>(b, c), src + c * (16 / sizeof(T)));
            }
            cp_async_commit();
        };
        auto compute = [&](T(&acc)[16], int buf, int n) {
#pragma unroll
            for (int u = 0; u < NU; ++u) {
                const int e = u * KG + kg;
                if (e >= n) continue;
                T h[16];
                r_ld<T>(h, hb, buf * BT + e);
                const int s2 = bs[buf * BT + e];
                const T *xs = X + s2 * (BB * P) + 4 * q;
                const int sw = s2 & 1;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    T x[4];
                    lds4<T>(x, xs + (m ^ sw) * 4 * P);
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[4 * r + c] = mac(h[4 * r + m], x[c], acc[4 * r + c]);
                }
            }
        };
        // A finished row: the K-groups' partial 4x4 sums are combined by a
        // reduce-scatter -- plain butterflies over K-group bits beyond 16
        // groups, then halving exchanges from the highest K-group bit down --
        // after which the lane holds elements i0 .. i0+EPL-1 of the block sum,
        // i0 = (kg >> EX) * EPL, of the output block (row ulist[s], column
        // j0 + q) if P_out has it.  With FUSE the lane finishes them at once:
        // T_{k+1} = alpha * (M~ T_k) + beta * T_{k-1}, every FP64 accumulator
        // += c_j[k+1] T_{k+1}, and its parts of Tr T_{k+1} and <T_{k+1}, G>;
        // otherwise it stores the raw sum for the epilogue pass (step 4).
        constexpr int LKG = ilog2(KG), EX = LKG > 4 ? LKG - 4 : 0, LV = LKG - EX;
        auto finish_row = [&](T(&acc)[16], int s) {
#pragma unroll
            for (int t = 0; t < EX; ++t)
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] += shfl_xor_t(acc[i], P << t);
#pragma unroll
            for (int l = 0; l < LV; ++l) {
                const int bit = LKG - 1 - l, n = 16 >> (l + 1);
                const bool hi = (kg >> bit) & 1;
#pragma unroll
                for (int j = 0; j < n; ++j) {
                    const T mine = hi ? acc[n + j] : acc[j], other = hi ? acc[j] : acc[n + j];
                    acc[j] = mine + shfl_xor_t(other, P << bit);
                }
            }
            const int o = q < ncols && (kg & ((1 << EX) - 1)) == 0 ? oslot[s * P + q] : -1;
            if (!FUSE && o >= 0) {
                // raw product; the epilogue pass below finishes the block
                T y[EPL];
#pragma unroll
                for (int j = 0; j < EPL; ++j) y[j] = acc[j];
                stn<T, EPL>(a.C + (int64_t)o * BB + (kg >> EX) * EPL, y);
            }
            if (FUSE && o >= 0) {
                const int i0 = (kg >> EX) * EPL;
                const int64_t idx = (int64_t)o * BB + i0;
                T y[EPL];
                if (a.Rm) {
                    T m[EPL];
                    ldgn<T, EPL>(m, a.Rm + idx);
#pragma unroll
                    for (int j = 0; j < EPL; ++j) y[j] = a.alpha * acc[j] + a.beta * m[j];
                } else {
#pragma unroll
                    for (int j = 0; j < EPL; ++j) y[j] = a.alpha * acc[j];
                }
                if (a.round_bf16) {
#pragma unroll
                    for (int j = 0; j < EPL; ++j) y[j] = bf16_round(y[j]);
                }
                stn<T, EPL>(a.C + idx, y);
                double yd[EPL];
#pragma unroll
                for (int j = 0; j < EPL; ++j) yd[j] = (double)y[j];
                // all accumulators are loaded before any is written back, so
                // their loads are in flight together
                double av[MAX_F][EPL];
#pragma unroll
                for (int f = 0; f < MAX_F; ++f)
                    if (f < a.nf) ldn<double, EPL>(av[f], a.acc[f] + idx);
#pragma unroll
                for (int f = 0; f < MAX_F; ++f) {
                    if (f < a.nf) {
#pragma unroll
                        for (int j = 0; j < EPL; ++j) av[f][j] += coefv[f] * yd[j];
                        stn<double, EPL>(a.acc[f] + idx, av[f]);
                    }
                }
                if (a.G) {
                    double gv[EPL];
                    ldgn<double, EPL>(gv, a.G + idx);
#pragma unroll
                    for (int j = 0; j < EPL; ++j) gpart += gv[j] * yd[j];
                }
                if (ulist[s] == j0 + q) {
#pragma unroll
                    for (int j = 0; j < EPL; ++j)
                        if ((i0 + j) % 5 == 0) tpart += yd[j];  // diagonal elements 0, 5, 10, 15
                }
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = T(0);
        };
        // consumer: the batch in flight, its row slot and whether it ends the row
        T acc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = T(0);
        int inflight = -1, n_inflight = 0, row_inflight = 0, last_inflight = 0, nb = 0;
        auto consume = [&](bool got) {
            if (inflight < 0) return;
            if (got)
                cp_async_wait<1>();
            else
                cp_async_wait<0>();
            __syncwarp();
            compute(acc, inflight, n_inflight);
            if (last_inflight) finish_row(acc, row_inflight);
            __syncwarp();
        };
        auto advance = [&](int n, int prow, int plast) {
            inflight = nb;
            n_inflight = n;
            row_inflight = prow;
            last_inflight = plast;
            nb ^= 1;
        };
        if (a.lrow_ptr) {
            // Operator row lists: entries [rptr[s], rptr[s+1]) of union row s,
            // each (offset of the block in the operator row << 16 | union slot).
            // The entry words of a row's next batch are loaded one batch ahead;
            // the following row's range, operator row start and first words one
            // row ahead, and the range of the row after it two rows ahead.
            const int32_t *rptr = a.lrow_ptr + a.lrow_base[blockIdx.x];
            int ps = warp;
            int64_t e = 0, e1 = 0, ab = 0, ne0 = 0, ne1 = 0, nab = 0, me0 = 0, me1 = 0, mab = 0;
            if (ps < nu) {
                e = rptr[ps];
                e1 = rptr[ps + 1];
                ab = a.Lrp[ulist[ps]];
            }
            uint32_t wcur = (ps < nu && lane < BT && e + lane < e1) ? a.lent[e + lane] : 0u;
            if (ps + NW < nu) {
                ne0 = rptr[ps + NW];
                ne1 = rptr[ps + NW + 1];
                nab = a.Lrp[ulist[ps + NW]];
            }
            uint32_t wnext = (ps + NW < nu && lane < BT && ne0 + lane < ne1) ? a.lent[ne0 + lane] : 0u;
            if (ps + 2 * NW < nu) {
                me0 = rptr[ps + 2 * NW];
                me1 = rptr[ps + 2 * NW + 1];
                mab = a.Lrp[ulist[ps + 2 * NW]];
            }
            while (true) {
                const bool got = ps < nu;
                int n = 0, prow = ps, plast = 0;
                if (got) {
                    // an empty row issues one empty batch, so that its zero product is stored
                    n = (int)(e1 - e < BT ? e1 - e : BT);
                    issue(nb, n, ab + (int64_t)(wcur >> 16), (int)(wcur & 0xffffu));
                    e += n;
                    if (e >= e1) {
                        plast = 1;
                        ps += NW;
                        e = ne0;
                        e1 = ne1;
                        ab = nab;
                        wcur = wnext;
                        ne0 = me0;
                        ne1 = me1;
                        nab = mab;
                        wnext = (ps + NW < nu && lane < BT && ne0 + lane < ne1) ? a.lent[ne0 + lane] : 0u;
                        if (ps + 2 * NW < nu) {
                            me0 = rptr[ps + 2 * NW];
                            me1 = rptr[ps + 2 * NW + 1];
                            mab = a.Lrp[ulist[ps + 2 * NW]];
                        }
                    } else {
                        wcur = (lane < BT && e + lane < e1) ? a.lent[e + lane] : 0u;
                    }
                }
                consume(got);
                if (!got) break;
                advance(n, prow, plast);
            }
        } else {
            // Ranking: the row's column indices are ranked 32 at a time (one per
            // lane) against the union bitmap; those in the union go to the
            // warp's staging ring wl, from which batches of BT are issued.
            const unsigned lt = (1u << lane) - 1u;
            int2 *wl = wlist + warp * 64;
            // producer: row slot ps being staged, its unranked range [base, a1)
            // and its next 64 column indices (two chunks); the following row's
            // bounds and first 64 indices, and the bounds of the row after it,
            // are fetched ahead.
            int ps = warp;
            int64_t base = 0, a1 = 0, na0 = 0, na1 = 0, ma0 = 0, ma1 = 0;
            if (ps < nu) {
                const int I0 = ulist[ps];
                base = a.Lrp[I0];
                a1 = a.Lrp[I0 + 1];
            }
            int Kq1 = (ps < nu && base + lane < a1) ? a.Lci[base + lane] : -1;
            int Kq2 = (ps < nu && base + 32 + lane < a1) ? a.Lci[base + 32 + lane] : -1;
            if (ps + NW < nu) {
                const int I1 = ulist[ps + NW];
                na0 = a.Lrp[I1];
                na1 = a.Lrp[I1 + 1];
            }
            int Kn1 = (ps + NW < nu && na0 + lane < na1) ? a.Lci[na0 + lane] : -1;
            int Kn2 = (ps + NW < nu && na0 + 32 + lane < na1) ? a.Lci[na0 + 32 + lane] : -1;
            if (ps + 2 * NW < nu) {
                const int I2 = ulist[ps + 2 * NW];
                ma0 = a.Lrp[I2];
                ma1 = a.Lrp[I2 + 1];
            }
            int pending = 0, row_issued = 0;
            while (true) {
                int n = 0, prow = 0, plast = 0;
                bool got = false;
                while (ps < nu) {
                    if (base < a1 && pending < BT) {
                        const int K = Kq1;
                        Kq1 = Kq2;
                        Kq2 = (base + 64 + lane < a1) ? a.Lci[base + 64 + lane] : -1;
                        const int s2 = K >= 0 ? rank_of(bits, K) : -1;
                        const unsigned vm = __ballot_sync(0xffffffffu, s2 >= 0);
                        if (s2 >= 0) wl[pending + __popc(vm & lt)] = make_int2((int)(base + lane), s2);
                        pending += __popc(vm);
                        base += 32;
                        __syncwarp();
                        continue;
                    }
                    // pending >= BT, or every raw entry of the row is ranked.  A
                    // row with no operator block in the union issues one empty
                    // batch, so that its (zero) product is still stored.
                    n = pending < BT ? pending : BT;
                    prow = ps;
                    if (n > 0 || !row_issued) {
                        const int2 w = lane < n ? wl[lane] : make_int2(0, 0);
                        issue(nb, n, (int64_t)w.x, w.y);
                        __syncwarp();
                        const int rest = pending - n;
                        const int2 keep = lane < rest ? wl[n + lane] : make_int2(0, 0);
                        __syncwarp();
                        if (lane < rest) wl[lane] = keep;
                        pending = rest;
                        __syncwarp();
                        got = true;
                        row_issued = 1;
                    }
                    if (base >= a1 && pending == 0) {  // row fully staged: advance
                        // the row's last batch: the one just issued, or (when the
                        // row's remaining raw entries were all outside the union)
                        // the one in flight, which is always this row's latest
                        if (got)
                            plast = 1;
                        else
                            last_inflight = 1;
                        row_issued = 0;
                        ps += NW;
                        base = na0;
                        a1 = na1;
                        Kq1 = Kn1;
                        Kq2 = Kn2;
                        na0 = ma0;
                        na1 = ma1;
                        Kn1 = (ps + NW < nu && na0 + lane < na1) ? a.Lci[na0 + lane] : -1;
                        Kn2 = (ps + NW < nu && na0 + 32 + lane < na1) ? a.Lci[na0 + 32 + lane] : -1;
                        if (ps + 2 * NW < nu) {
                            const int I2 = ulist[ps + 2 * NW];
                            ma0 = a.Lrp[I2];
                            ma1 = a.Lrp[I2 + 1];
                        }
                    }
                    if (got) break;
                }
                consume(got);
                if (!got) break;
                advance(n, prow, plast);
            }
        }
    }
    __syncthreads();

    // 4. without FUSE, the epilogue pass over the panel's output blocks, one
    // block row (4 elements) per thread in column order: T_{k+1} = alpha *
    // (M~ T_k) + beta * T_{k-1}, accumulators, Tr T_{k+1} and <T_{k+1}, G>.
    if constexpr (!FUSE) {
        // cumulative block counts of the panel's columns (indexed by constants only)
        int cum[5];
        cum[0] = 0;
        int nblk = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            cum[q + 1] = cum[q] + (q < ncols ? (int)(a.rp[j0 + q + 1] - a.rp[j0 + q]) : 0);
            if (q < ncols) nblk = cum[q + 1];
        }
        for (int t = tid; t < nblk * 4; t += NT) {
            const int b = t >> 2, r = t & 3;
            int q = 0, base = 0;
#pragma unroll
            for (int qq = 1; qq < 4; ++qq)
                if (qq < ncols && b >= cum[qq]) {
                    q = qq;
                    base = cum[qq];
                }
            const int J = j0 + q;
            const int64_t p = a.rp[J] + (b - base);
            const int K = a.ci[p];
            const int64_t idx = (int64_t)a.tperm[p] * BB + 4 * r;
            T y[4];
            Vec4<T>::ld(y, a.C + idx);
            if (a.Rm) {
                T m4[4];
                Vec4<T>::ldg(m4, a.Rm + idx);
#pragma unroll
                for (int c = 0; c < 4; ++c) y[c] = a.alpha * y[c] + a.beta * m4[c];
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) y[c] = a.alpha * y[c];
            }
            if (a.round_bf16) {
#pragma unroll
                for (int c = 0; c < 4; ++c) y[c] = bf16_round(y[c]);
            }
            Vec4<T>::st(a.C + idx, y);
            double yd[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) yd[c] = (double)y[c];
            // all accumulator rows are loaded before any is written back, so
            // their loads are in flight together
            double av[MAX_F][4];
#pragma unroll
            for (int f = 0; f < MAX_F; ++f)
                if (f < a.nf) Vec4<double>::ld(av[f], a.acc[f] + idx);
#pragma unroll
            for (int f = 0; f < MAX_F; ++f) {
                if (f < a.nf) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) av[f][c] += coefv[f] * yd[c];
                    Vec4<double>::st(a.acc[f] + idx, av[f]);
                }
            }
            if (a.G) {
                double gv[4];
                Vec4<double>::ldg(gv, a.G + idx);
#pragma unroll
                for (int c = 0; c < 4; ++c) gpart += gv[c] * yd[c];
            }
            if (K == J) tpart += yd[r];
        }
    }
    // 5. the moment partials of the panel
    if (a.mom || a.gmom) {
        Moments<2> mm{{tpart, gpart}, {a.mom, a.gmom}};
        finish_moments<NT, 2>(a.part, a.counter, mm, red);
    }
}

// Terms 0 and 1: T_0 = I and T_1 = M~ on P_out, accumulators c_0/2 T_0 + c_1 T_1,
// moments of both.  Same panel grid as the step kernel, so the partial buffer and
// completion counter are shared.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_init(const int64_t *rp, const int32_t *ci, const int32_t *tperm,
                                             const int32_t *panels, const int64_t *Lrp, const int32_t *Lci,
                                             const double *Mt, T *T0, T *T1, int32_t nf, StepArgs<T> a,
                                             double *mom, double *gmom) {
    __shared__ double red[(NT / 32) * 4];
    const int j0 = panels[2 * blockIdx.x], ncols = panels[2 * blockIdx.x + 1];
    double c0[MAX_F], c1[MAX_F];
#pragma unroll
    for (int f = 0; f < MAX_F; ++f) {
        c0[f] = f < nf ? a.coef[(int64_t)f * a.coef_stride + 0] : 0.0;
        c1[f] = f < nf ? a.coef[(int64_t)f * a.coef_stride + 1] : 0.0;
    }
    double t0 = 0.0, t1 = 0.0, g0 = 0.0, g1 = 0.0;
    for (int q = 0; q < ncols; ++q) {
        const int J = j0 + q;
        for (int64_t p = rp[J] + threadIdx.x; p < rp[J + 1]; p += NT) {
            const int K = ci[p];  // block (K, J) of the column
            const int64_t slot = (int64_t)tperm[p] * BB;
            const int64_t la = find_in_row(Lrp, Lci, K, J);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const T v0 = (K == J && (i % 5) == 0) ? T(1) : T(0);
                T v1 = la >= 0 ? (T)Mt[la * BB + i] : T(0);
                if (a.round_bf16) v1 = bf16_round(v1);
                T0[slot + i] = v0;
                T1[slot + i] = v1;
                const double d0 = (double)v0, d1 = (double)v1;
#pragma unroll
                for (int f = 0; f < MAX_F; ++f)
                    if (f < nf) a.acc[f][slot + i] = 0.5 * c0[f] * d0 + c1[f] * d1;
                if (a.G) {
                    g0 += a.G[slot + i] * d0;
                    g1 += a.G[slot + i] * d1;
                }
                if (K == J && (i % 5) == 0) {
                    t0 += d0;
                    t1 += d1;
                }
            }
        }
    }
    Moments<4> mm{{t0, t1, g0, g1}, {mom, mom ? mom + 1 : nullptr, gmom, gmom ? gmom + 1 : nullptr}};
    finish_moments<NT, 4>(a.part, a.counter, mm, red);
}

// FP64 values split into double-floats (hi = the nearest float, lo = the
// nearest float to the remainder)
__global__ void k_to_dfl(const double *in, dfl *out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = dfl(in[i]);
}

__global__ void k_to_f32(const double *in, float *out, int64_t n, int round_bf16) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = round_bf16 ? __bfloat162float(__float2bfloat16_rn(in[i])) : (float)in[i];
}

template <typename T, int P, int NW, int MINB>
int launch_step(const cheb_plan *plan, const StepArgs<T> &a, cudaStream_t s) {
    const StepLayout lay = step_layout(a.nw, a.ucap, P, sizeof(T), NW);
    auto fn = k_step<T, P, NW, MINB>;
    CHEB_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    fn<<<(unsigned)plan->n_panels, NW * 32, lay.total, s>>>(a);
    return check_launch("k_step");
}

template <typename T>
StepArgs<T> base_args(const cheb_plan *plan, const cheb_bsr *L, const T *Lv) {
    StepArgs<T> a{};
    a.nw = (plan->nbr + 31) / 32;
    a.ucap = plan->max_union;
    a.rp = plan->rp;
    a.ci = plan->ci;
    a.tperm = plan->d_tperm;
    a.panels = plan->d_panels;
    a.Lrp = L->row_ptr;
    a.Lci = L->col_idx;
    a.Lv = Lv;
    if (plan->op_bound && plan->op_rp == L->row_ptr && plan->op_ci == L->col_idx) {
        a.lrow_base = plan->lists.d_base;
        a.lrow_ptr = plan->lists.d_ptr;
        a.lent = plan->lists.d_ent;
    }
    return a;
}

template <typename T>
int run_step(const cheb_plan *plan, const StepArgs<T> &a, cudaStream_t s);
#define CHEB_TILE_CASE(T, TABLE, i) \
    case i: return launch_step<T, TABLE[i].P, TABLE[i].NW, TABLE[i].MINB>(plan, a, s);
template <>
int run_step<double>(const cheb_plan *plan, const StepArgs<double> &a, cudaStream_t s) {
    static_assert(N_TILES_F64 == 5, "tile table size");
    switch (plan->tile) {
        CHEB_TILE_CASE(double, TILES_F64, 0)
        CHEB_TILE_CASE(double, TILES_F64, 1)
        CHEB_TILE_CASE(double, TILES_F64, 2)
        CHEB_TILE_CASE(double, TILES_F64, 3)
        CHEB_TILE_CASE(double, TILES_F64, 4)
        default: return fail(CHEB_ERR_INVALID, "bad FP64 tile %d", plan->tile);
    }
}
template <>
int run_step<dfl>(const cheb_plan *plan, const StepArgs<dfl> &a, cudaStream_t s) {
    // FP64-accurate plans share the FP64 tile shapes (8-byte elements)
    switch (plan->tile) {
        CHEB_TILE_CASE(dfl, TILES_F64, 0)
        CHEB_TILE_CASE(dfl, TILES_F64, 1)
        CHEB_TILE_CASE(dfl, TILES_F64, 2)
        CHEB_TILE_CASE(dfl, TILES_F64, 3)
        CHEB_TILE_CASE(dfl, TILES_F64, 4)
        default: return fail(CHEB_ERR_INVALID, "bad FP64 tile %d", plan->tile);
    }
}
template <>
int run_step<float>(const cheb_plan *plan, const StepArgs<float> &a, cudaStream_t s) {
    static_assert(N_TILES_F32 == 6, "tile table size");
    switch (plan->tile) {
        CHEB_TILE_CASE(float, TILES_F32, 0)
        CHEB_TILE_CASE(float, TILES_F32, 1)
        CHEB_TILE_CASE(float, TILES_F32, 2)
        CHEB_TILE_CASE(float, TILES_F32, 3)
        CHEB_TILE_CASE(float, TILES_F32, 4)
        CHEB_TILE_CASE(float, TILES_F32, 5)
        default: return fail(CHEB_ERR_INVALID, "bad FP32 tile %d", plan->tile);
    }
}
#undef CHEB_TILE_CASE

size_t expand_ws(const cheb_plan *plan, int64_t nnzL, int precision) {
    const size_t esz = (precision == CHEB_F64 || precision == CHEB_F64X) ? 8 : 4;
    size_t b = 3 * align_up(plan->nnzb * BB * esz);
    if (precision != CHEB_F64) b += align_up(nnzL * BB * esz);
    b += align_up(plan->n_panels * 4 * sizeof(double)) + align_up(64);
    b += 256;
    if ((precision == CHEB_F32 || precision == CHEB_BF16) && plan->col.built)
        b = std::max(b, col_expand_ws(plan, nnzL));
    return b;
}

template <typename T>
int expand_impl(const cheb_plan *plan, const cheb_bsr *Mt, int32_t n_terms, const double *coeffs,
                int32_t stride, int32_t nf, double *const *acc, double *moments, const double *G,
                double *gmoments, void *ws, size_t ws_bytes, cudaStream_t s, int round_bf16 = 0) {
    Carve cv(ws, ws_bytes);
    T *buf[3];
    for (int i = 0; i < 3; ++i) buf[i] = cv.take<T>(plan->nnzb * BB);
    const T *Lv;
    const int64_t nL = Mt->nnzb * BB;
    if constexpr (std::is_same_v<T, double>) {
        Lv = reinterpret_cast<const T *>(Mt->vals);
    } else if constexpr (std::is_same_v<T, dfl>) {
        dfl *lv = cv.take<dfl>(nL);
        if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_expand_stepwise: workspace too small");
        k_to_dfl<<<(unsigned)((nL + 255) / 256), 256, 0, s>>>((const double *)Mt->vals, lv, nL);
        CHEB_TRY(check_launch("k_to_dfl"));
        Lv = lv;
    } else {
        float *lv = cv.take<float>(nL);
        if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_expand_stepwise: workspace too small");
        k_to_f32<<<(unsigned)((nL + 255) / 256), 256, 0, s>>>((const double *)Mt->vals, lv, nL, round_bf16);
        CHEB_TRY(check_launch("k_to_f32"));
        Lv = reinterpret_cast<const T *>(lv);
    }
    double *part = cv.take<double>(plan->n_panels * 4);
    int32_t *counter = cv.take<int32_t>(16);
    if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_expand_stepwise: workspace too small");
    CHEB_CUDA(cudaMemsetAsync(counter, 0, 64, s));
    StepArgs<T> a = base_args<T>(plan, Mt, Lv);
    a.nf = nf;
    for (int f = 0; f < nf; ++f) a.acc[f] = acc[f];
    a.coef = coeffs;
    a.coef_stride = stride;
    a.G = G;
    a.part = part;
    a.counter = counter;
    a.round_bf16 = round_bf16;
    k_init<T, 256><<<(unsigned)plan->n_panels, 256, 0, s>>>(plan->rp, plan->ci, plan->d_tperm, plan->d_panels,
                                                          Mt->row_ptr, Mt->col_idx, (const double *)Mt->vals,
                                                          buf[0], buf[1], nf, a, moments, gmoments);
    CHEB_TRY(check_launch("k_init"));
    a.alpha = T(2);
    a.beta = T(-1);
    for (int k = 1; k + 1 < n_terms; ++k) {
        a.R = buf[k % 3];
        a.Rm = buf[(k - 1) % 3];
        a.C = buf[(k + 1) % 3];
        a.term = k + 1;
        a.mom = moments ? moments + k + 1 : nullptr;
        a.gmom = (gmoments && G) ? gmoments + k + 1 : nullptr;
        CHEB_TRY(run_step<T>(plan, a, s));
    }
    return CHEB_OK;
}

}  // namespace cheb

using namespace cheb;

static int check_operator(const cheb_plan *plan, const cheb_bsr *Mt) {
    if (!plan || !plan->bound) return fail(CHEB_ERR_INVALID, "plan is NULL or not bound");
    if (!Mt || Mt->nbr != plan->nbr || !Mt->row_ptr || !Mt->col_idx || !Mt->vals || Mt->dtype != CHEB_F64)
        return fail(CHEB_ERR_INVALID, "operator must be FP64 with the plan's block rows");
    return CHEB_OK;
}

extern "C" int cheb_expand_stepwise_workspace_size(const cheb_plan *plan, const cheb_bsr *Mt, int32_t precision,
                                                   size_t *bytes) {
    if (!plan || !Mt || !bytes) return fail(CHEB_ERR_INVALID, "cheb_expand_stepwise_workspace_size: NULL argument");
    *bytes = expand_ws(plan, Mt->nnzb, precision);
    return CHEB_OK;
}

extern "C" int cheb_expand_stepwise(const cheb_plan *plan, const cheb_bsr *Mt, int32_t n_terms, const double *coeffs,
                           int32_t coeff_stride, int32_t n_f, double *const *acc, double *moments,
                           const double *G, double *gmoments, int32_t precision, void *ws, size_t ws_bytes,
                           void *stream) {
    CHEB_TRY(check_operator(plan, Mt));
    if (n_terms < 2 || n_f < 0 || n_f > MAX_F || (n_f > 0 && (!acc || !coeffs)) || coeff_stride < n_terms)
        return fail(CHEB_ERR_INVALID, "cheb_expand_stepwise: bad n_terms / n_f / coefficients");
    for (int f = 0; f < n_f; ++f)
        if (!acc[f]) return fail(CHEB_ERR_INVALID, "cheb_expand_stepwise: accumulator %d is NULL", f);
    if (precision != plan->precision) return fail(CHEB_ERR_INVALID, "cheb_expand_stepwise: plan precision differs");
    if (!ws || ws_bytes < expand_ws(plan, Mt->nnzb, precision))
        return fail(CHEB_ERR_NOSPACE, "cheb_expand_stepwise: workspace %zu < %zu", ws_bytes,
                    expand_ws(plan, Mt->nnzb, precision));
    cudaStream_t s = as_stream(stream);
    if (precision == CHEB_F64)
        return expand_impl<double>(plan, Mt, n_terms, coeffs, coeff_stride, n_f, acc, moments, G, gmoments, ws,
                                   ws_bytes, s);
    if (precision == CHEB_F64X)
        return expand_impl<dfl>(plan, Mt, n_terms, coeffs, coeff_stride, n_f, acc, moments, G, gmoments, ws,
                                ws_bytes, s);
    if ((precision == CHEB_F32 || precision == CHEB_BF16) && col_usable(plan, Mt))
        return col_expand(plan, Mt, n_terms, coeffs, coeff_stride, n_f, acc, moments, G, gmoments, ws, ws_bytes, s,
                          precision == CHEB_BF16);
    if (precision == CHEB_F32 || precision == CHEB_BF16)
        return expand_impl<float>(plan, Mt, n_terms, coeffs, coeff_stride, n_f, acc, moments, G, gmoments, ws,
                                  ws_bytes, s, precision == CHEB_BF16);
    return fail(CHEB_ERR_INVALID, "cheb_expand_stepwise: unsupported precision %d", precision);
}

extern "C" int cheb_masked_product(const cheb_plan *plan, const cheb_bsr *L, const double *R, double alpha,
                                   const double *D, double beta, double *C, void *stream) {
    CHEB_TRY(check_operator(plan, L));
    if (plan->precision != CHEB_F64) return fail(CHEB_ERR_INVALID, "cheb_masked_product: needs an FP64 plan");
    if (!R || !C || C == R || (D && C == D)) return fail(CHEB_ERR_INVALID, "cheb_masked_product: bad pointers");
    StepArgs<double> a = base_args<double>(plan, L, (const double *)L->vals);
    a.R = R;
    a.Rm = D;
    a.C = C;
    a.alpha = alpha;
    a.beta = D ? beta : 0.0;
    a.nf = 0;
    return run_step<double>(plan, a, as_stream(stream));
}

extern "C" int cheb_newton_schulz(const cheb_plan *plan, const cheb_bsr *S, const double *X0, double *X1,
                                  double *tmp, void *stream) {
    if (!S || !X0 || !X1 || !tmp || X1 == X0 || X1 == tmp || tmp == X0)
        return fail(CHEB_ERR_INVALID, "cheb_newton_schulz: bad pointers");
    CHEB_TRY(cheb_masked_product(plan, S, X0, 1.0, nullptr, 0.0, tmp, stream));
    if (!plan) return CHEB_ERR_INVALID;
    cheb_bsr Xb{plan->nbr, plan->nnzb, plan->rp, plan->ci, const_cast<double *>(X0), CHEB_F64};
    return cheb_masked_product(plan, &Xb, tmp, -1.0, X0, 2.0, X1, stream);
}

extern "C" int cheb_newton_schulz_isqrt(const cheb_plan *plan, const cheb_bsr *S, const double *Z0, double *Z1,
                                        double *tmp1, double *tmp2, void *stream) {
    if (!plan || !S || !Z0 || !Z1 || !tmp1 || !tmp2 || Z1 == Z0 || Z1 == tmp1 || Z1 == tmp2 || tmp1 == tmp2 ||
        tmp1 == Z0 || tmp2 == Z0)
        return fail(CHEB_ERR_INVALID, "cheb_newton_schulz_isqrt: bad pointers");
    cheb_bsr Zb{plan->nbr, plan->nnzb, plan->rp, plan->ci, const_cast<double *>(Z0), CHEB_F64};
    // tmp1 = P(Z0 Z0); tmp2 = P(S tmp1); Z1 = 1.5 Z0 - 0.5 P(Z0 tmp2)
    CHEB_TRY(cheb_masked_product(plan, &Zb, Z0, 1.0, nullptr, 0.0, tmp1, stream));
    CHEB_TRY(cheb_masked_product(plan, S, tmp1, 1.0, nullptr, 0.0, tmp2, stream));
    return cheb_masked_product(plan, &Zb, tmp2, -0.5, Z0, 1.5, Z1, stream);
}
