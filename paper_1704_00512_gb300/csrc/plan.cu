// Plan creation (host C++): checks the output pattern, builds the block
// transposition map and groups block columns into panels.
//
// Columns of the Chebyshev recursion are independent (Sec. "Expansion in
// Chebyshev polynomials": each column of T_{k+1} needs only the same column of
// T_k and T_{k-1}), so one thread block can advance a panel of P neighbouring
// block columns with their row lists gathered in shared memory.  The panels are
// formed greedily along the column order: a column joins the current panel while
// the panel has fewer than P columns and the union of the panel's row lists
// still fits the shared-memory budget.
#include <algorithm>
#include <thread>

#include "common.cuh"
#include "plan.cuh"

using namespace cheb;

static int union_capacity(int64_t nbr, int P, int esz, int nwarps, size_t budget) {
    int64_t nw = (nbr + 31) / 32;
    // largest ucap with step_layout(nw, ucap, P, esz, nwarps).total <= budget
    int lo = 0, hi = 1 << 16;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (step_layout(nw, mid, P, esz, nwarps).total <= budget) lo = mid; else hi = mid - 1;
    }
    return std::min(lo, 32767);
}

extern "C" int cheb_tile_count(int32_t precision) {
    if (precision < CHEB_F64 || precision > CHEB_F64X) return 0;
    return n_tiles(precision);
}

extern "C" int cheb_tile_info(int32_t precision, int32_t tile, int32_t *panel_width, int32_t *warps,
                              int32_t *blocks_per_sm) {
    if (precision < CHEB_F64 || precision > CHEB_F64X || tile < 0 ||
        tile >= n_tiles(precision))
        return fail(CHEB_ERR_INVALID, "cheb_tile_info: no tile %d for precision %d", tile, precision);
    const TileCfg c = tile_cfg(precision, tile);
    if (panel_width) *panel_width = c.P;
    if (warps) *warps = c.NW;
    if (blocks_per_sm) *blocks_per_sm = c.MINB;
    return CHEB_OK;
}

// 0: plans and lists built by device kernels (gather.cu); 1: on host threads
// (the reference builders, bit-identical)
static int32_t g_plan_host = 0;

extern "C" int cheb_set_plan_builder(int32_t host) {
    if (host != 0 && host != 1) return fail(CHEB_ERR_INVALID, "cheb_set_plan_builder: 0 (device) or 1 (host)");
    g_plan_host = host;
    return CHEB_OK;
}

static void free_row_lists(RowLists &l) {
    if (l.tmp) cudaFree(l.tmp);
    l.tmp = nullptr;
}

// cheb_plan_create on the device: checks, transposition map and the two panel
// walks run as kernels on P_out's device arrays; only the panel tables (a few
// integers per panel) come back to the host.
static int plan_create_device(cheb_plan *plan, const std::vector<int64_t> &sys_col, const TileCfg &cfg,
                              int esz, size_t budget, cudaStream_t s) {
    const int64_t nbr = plan->nbr, nnzb = plan->nnzb;
    int64_t ends[2];
    CHEB_CUDA(cudaMemcpyAsync(&ends[0], plan->rp, 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(&ends[1], plan->rp + nbr, 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    if (ends[0] != 0 || ends[1] != nnzb) return fail(CHEB_ERR_INVALID, "cheb_plan_create: row_ptr does not span nnzb");
    int64_t first[4];
    int32_t maxlen = 1;
    CHEB_TRY(gp_check_pattern(plan->rp, plan->ci, nbr, nnzb, first, &maxlen, s));
    if (first[0] < nbr) return fail(CHEB_ERR_INVALID, "row_ptr not monotone at row %lld", (long long)first[0]);
    if (first[1] < nbr) return fail(CHEB_ERR_INVALID, "col_idx out of range in row %lld", (long long)first[1]);
    if (first[2] < nbr) return fail(CHEB_ERR_INVALID, "col_idx not strictly ascending in row %lld", (long long)first[2]);
    if (first[3] < nbr) return fail(CHEB_ERR_INVALID, "diagonal block missing in row %lld", (long long)first[3]);
    CHEB_CUDA(cudaMalloc(&plan->tmp_tperm, std::max<int64_t>(nnzb, 1) * 4));
    int64_t bad = nnzb;
    CHEB_TRY(gp_tperm(plan->rp, plan->ci, nbr, nnzb, plan->tmp_tperm, &bad, s));
    if (bad < nnzb) return fail(CHEB_ERR_INVALID, "pattern not symmetric: block %lld has no transpose", (long long)bad);
    maxlen = std::max<int32_t>(maxlen, 1);
    // step-kernel panels
    std::vector<int32_t> pan4, aux;
    int64_t out[4];
    CHEB_TRY(gp_walk(plan->rp, plan->ci, nbr, plan->P, plan->ucap, INT64_MAX, {0, nbr}, pan4, aux, out, s));
    if (out[2]) return fail(CHEB_ERR_NOSPACE, "a column does not fit the shared-memory panel of %d rows", plan->ucap);
    plan->n_panels = out[0];
    plan->max_union = (int32_t)out[1];
    plan->h_panels.resize(2 * out[0]);
    for (int64_t p = 0; p < out[0]; ++p) {
        plan->h_panels[2 * p] = pan4[4 * p];
        plan->h_panels[2 * p + 1] = pan4[4 * p + 1];
    }
    // resident panels, as in the host builder
    const int64_t nw = (nbr + 31) / 32;
    const int P = plan->P;
    auto bcap_for = [&](int64_t ucap) {
        int64_t lo = 0, hi = (int64_t)P * maxlen;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (res_layout(nw, ucap, mid, P, esz, cfg.NW).total <= budget) lo = mid; else hi = mid - 1;
        }
        return lo;
    };
    int64_t Ucap = std::min<int64_t>(2 * (int64_t)maxlen, 32767);
    int64_t Bcap = bcap_for(Ucap);
    while (Bcap < maxlen && Ucap > maxlen) {
        Ucap = std::max<int64_t>(maxlen, Ucap * 3 / 4);
        Bcap = bcap_for(Ucap);
    }
    if (Bcap < maxlen) return fail(CHEB_ERR_NOSPACE, "a column of %d blocks does not fit a resident panel", maxlen);
    CHEB_TRY(gp_walk(plan->rp, plan->ci, nbr, P, Ucap, Bcap, sys_col, pan4, aux, out, s));
    if (out[2]) return fail(CHEB_ERR_NOSPACE, "a column does not fit a resident panel");
    const int64_t nr = out[0];
    plan->h_rpanels.resize(2 * nr);
    plan->h_rpanel_sys.resize(nr);
    for (int64_t p = 0; p < nr; ++p) {
        plan->h_rpanels[2 * p] = pan4[4 * p];
        plan->h_rpanels[2 * p + 1] = pan4[4 * p + 1];
        plan->h_rpanel_sys[p] = aux[2 * p + 1];
    }
    const int nsys = (int)sys_col.size() - 1;
    plan->h_sys_rpanel.assign(nsys + 1, (int32_t)nr);
    for (int64_t p = nr - 1; p >= 0; --p) plan->h_sys_rpanel[plan->h_rpanel_sys[p]] = (int32_t)p;
    plan->n_rpanels = nr;
    plan->max_union_res = (int32_t)out[1];
    plan->max_nblk_res = (int32_t)out[3];
    return CHEB_OK;
}

static int plan_create_impl(const cheb_bsr *P_out, int32_t precision, int32_t tile, int32_t nsys,
                            const int64_t *sys_row_start, cheb_plan **out, size_t *plan_ws_bytes, void *stream) {
    if (!out || !plan_ws_bytes) return fail(CHEB_ERR_INVALID, "cheb_plan_create: NULL output");
    *out = nullptr;
    if (!P_out || P_out->nbr < 1 || P_out->nnzb < P_out->nbr || !P_out->row_ptr || !P_out->col_idx)
        return fail(CHEB_ERR_INVALID, "cheb_plan_create: bad pattern");
    if (precision < CHEB_F64 || precision > CHEB_F64X)
        return fail(CHEB_ERR_INVALID, "cheb_plan_create: precision must be CHEB_F64, CHEB_F32, CHEB_BF16 or CHEB_F64X");
    if (P_out->nnzb >= (int64_t)INT32_MAX) return fail(CHEB_ERR_INVALID, "cheb_plan_create: too many blocks");
    if (tile < 0) tile = 0;
    if (tile >= n_tiles(precision)) return fail(CHEB_ERR_INVALID, "cheb_plan_create: no tile %d", tile);
    if (nsys < 1) return fail(CHEB_ERR_INVALID, "cheb_plan_create: nsys < 1");
    const int64_t nbr = P_out->nbr, nnzb = P_out->nnzb;
    std::vector<int64_t> sys_col(nsys + 1);
    if (sys_row_start) {
        for (int i = 0; i <= nsys; ++i) sys_col[i] = sys_row_start[i];
        if (sys_col[0] != 0 || sys_col[nsys] != nbr)
            return fail(CHEB_ERR_INVALID, "cheb_plan_create: system row starts must span 0..nbr");
        for (int i = 0; i < nsys; ++i)
            if (sys_col[i + 1] <= sys_col[i]) return fail(CHEB_ERR_INVALID, "cheb_plan_create: empty system %d", i);
    } else {
        if (nsys != 1) return fail(CHEB_ERR_INVALID, "cheb_plan_create: system row starts missing");
        sys_col[0] = 0;
        sys_col[1] = nbr;
    }
    cudaStream_t s = as_stream(stream);
    auto plan_ws = [](const cheb_plan *pl) {
        return align_up(pl->nnzb * 4) + align_up(pl->h_panels.size() * 4) + align_up(64) +
               align_up(pl->h_rpanels.size() * 4) + align_up(pl->h_rpanel_sys.size() * 4) +
               align_up(pl->h_sys_rpanel.size() * 4);
    };
    if (!g_plan_host) {
        auto plan = new cheb_plan();
        plan->nbr = nbr;
        plan->nnzb = nnzb;
        plan->rp = P_out->row_ptr;
        plan->ci = P_out->col_idx;
        plan->precision = precision;
        plan->nsys = nsys;
        plan->h_sys_col = sys_col;
        plan->gather_host = 0;
        const TileCfg cfg = tile_cfg(precision, tile);
        const int esz = (precision == CHEB_F64 || precision == CHEB_F64X) ? 8 : 4;
        plan->tile = tile;
        plan->P = cfg.P;
        plan->NW = cfg.NW;
        plan->minb = cfg.MINB;
        const size_t budget = smem_budget(cfg.MINB);
        plan->ucap = union_capacity(nbr, cfg.P, esz, cfg.NW, budget);
        const int rc = plan_create_device(plan, sys_col, cfg, esz, budget, s);
        if (rc != CHEB_OK) {
            if (plan->tmp_tperm) cudaFree(plan->tmp_tperm);
            delete plan;
            return rc;
        }
        plan->ws_bytes = plan_ws(plan);
        *plan_ws_bytes = plan->ws_bytes;
        *out = plan;
        return CHEB_OK;
    }
    std::vector<int64_t> rp(nbr + 1);
    std::vector<int32_t> ci(nnzb);
    CHEB_CUDA(cudaMemcpyAsync(rp.data(), P_out->row_ptr, (nbr + 1) * 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(ci.data(), P_out->col_idx, nnzb * 4, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    if (rp[0] != 0 || rp[nbr] != nnzb) return fail(CHEB_ERR_INVALID, "cheb_plan_create: row_ptr does not span nnzb");
    for (int64_t I = 0; I < nbr; ++I) {
        if (rp[I + 1] < rp[I]) return fail(CHEB_ERR_INVALID, "row_ptr not monotone at row %lld", (long long)I);
        bool diag = false;
        for (int64_t p = rp[I]; p < rp[I + 1]; ++p) {
            if (ci[p] < 0 || ci[p] >= nbr) return fail(CHEB_ERR_INVALID, "col_idx out of range in row %lld", (long long)I);
            if (p > rp[I] && ci[p] <= ci[p - 1]) return fail(CHEB_ERR_INVALID, "col_idx not strictly ascending in row %lld", (long long)I);
            diag |= ci[p] == I;
        }
        if (!diag) return fail(CHEB_ERR_INVALID, "diagonal block missing in row %lld", (long long)I);
    }
    auto plan = new cheb_plan();
    plan->nbr = nbr;
    plan->nnzb = nnzb;
    plan->rp = P_out->row_ptr;
    plan->ci = P_out->col_idx;
    plan->precision = precision;
    plan->nsys = nsys;
    plan->h_sys_col = sys_col;
    plan->gather_host = 1;
    plan->h_tperm.resize(nnzb);
    for (int64_t I = 0; I < nbr; ++I) {
        for (int64_t p = rp[I]; p < rp[I + 1]; ++p) {
            const int32_t J = ci[p];
            auto b = ci.begin() + rp[J], e = ci.begin() + rp[J + 1];
            auto it = std::lower_bound(b, e, (int32_t)I);
            if (it == e || *it != I) {
                delete plan;
                return fail(CHEB_ERR_INVALID, "pattern not symmetric: (%lld,%d) present, transpose missing",
                            (long long)I, J);
            }
            plan->h_tperm[p] = (int32_t)(it - ci.begin());
        }
    }
    const TileCfg cfg = tile_cfg(precision, tile);
    const int P = cfg.P;
    const int esz = (precision == CHEB_F64 || precision == CHEB_F64X) ? 8 : 4;
    plan->tile = tile;
    plan->P = P;
    plan->NW = cfg.NW;
    plan->minb = cfg.MINB;
    const size_t budget = smem_budget(cfg.MINB);
    plan->ucap = union_capacity(nbr, P, esz, cfg.NW, budget);
    const int64_t nw = (nbr + 31) / 32;
    std::vector<int32_t> stamp(nbr, -1);
    // step-kernel panels: greedy along the columns while the union fits
    {
        int64_t j = 0, panel = 0;
        int32_t max_union = 0;
        while (j < nbr) {
            int32_t cnt = 0, ncols = 0;
            const int64_t j0 = j;
            while (j < nbr && ncols < P) {
                int32_t add = 0;
                for (int64_t p = rp[j]; p < rp[j + 1]; ++p) add += stamp[ci[p]] != (int32_t)panel;
                if (ncols > 0 && cnt + add > plan->ucap) break;
                if (cnt + add > plan->ucap) {
                    delete plan;
                    return fail(CHEB_ERR_NOSPACE, "column %lld has %d rows, shared-memory panel holds %d",
                                (long long)j, add, plan->ucap);
                }
                for (int64_t p = rp[j]; p < rp[j + 1]; ++p) stamp[ci[p]] = (int32_t)panel;
                cnt += add;
                ++ncols;
                ++j;
            }
            plan->h_panels.push_back((int32_t)j0);
            plan->h_panels.push_back(ncols);
            max_union = std::max(max_union, cnt);
            ++panel;
        }
        plan->n_panels = panel;
        plan->max_union = max_union;
    }
    // resident panels: greedy within each system while the panel's union and
    // block count stay under caps (Ucap, Bcap) whose layout fits the budget,
    // so that the launch (sized by the maxima over panels) fits as well
    {
        int32_t maxlen = 1;
        for (int64_t j = 0; j < nbr; ++j) maxlen = std::max(maxlen, (int32_t)(rp[j + 1] - rp[j]));
        auto bcap_for = [&](int64_t ucap) {
            int64_t lo = 0, hi = (int64_t)P * maxlen;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) / 2;
                if (res_layout(nw, ucap, mid, P, esz, cfg.NW).total <= budget) lo = mid; else hi = mid - 1;
            }
            return lo;
        };
        int64_t Ucap = std::min<int64_t>(2 * (int64_t)maxlen, 32767);
        int64_t Bcap = bcap_for(Ucap);
        while (Bcap < maxlen && Ucap > maxlen) {
            Ucap = std::max<int64_t>(maxlen, Ucap * 3 / 4);
            Bcap = bcap_for(Ucap);
        }
        if (Bcap < maxlen) {
            delete plan;
            return fail(CHEB_ERR_NOSPACE, "a column of %d blocks does not fit a resident panel", maxlen);
        }
        std::fill(stamp.begin(), stamp.end(), -1);
        int64_t panel = 0;
        int32_t max_union = 0, max_nblk = 0;
        for (int sy = 0; sy < nsys; ++sy) {
            plan->h_sys_rpanel.push_back((int32_t)panel);
            int64_t j = sys_col[sy];
            while (j < sys_col[sy + 1]) {
                int32_t cnt = 0, ncols = 0, nblk = 0;
                const int64_t j0 = j;
                while (j < sys_col[sy + 1] && ncols < P) {
                    int32_t add = 0;
                    const int32_t len = (int32_t)(rp[j + 1] - rp[j]);
                    for (int64_t p = rp[j]; p < rp[j + 1]; ++p) add += stamp[ci[p]] != (int32_t)panel;
                    if (ncols > 0 && (cnt + add > Ucap || nblk + len > Bcap)) break;
                    for (int64_t p = rp[j]; p < rp[j + 1]; ++p) stamp[ci[p]] = (int32_t)panel;
                    cnt += add;
                    nblk += len;
                    ++ncols;
                    ++j;
                }
                plan->h_rpanels.push_back((int32_t)j0);
                plan->h_rpanels.push_back(ncols);
                plan->h_rpanel_sys.push_back(sy);
                max_union = std::max(max_union, cnt);
                max_nblk = std::max(max_nblk, nblk);
                ++panel;
            }
        }
        plan->h_sys_rpanel.push_back((int32_t)panel);
        plan->n_rpanels = panel;
        plan->max_union_res = max_union;
        plan->max_nblk_res = max_nblk;
    }
    plan->ws_bytes = plan_ws(plan);
    *plan_ws_bytes = plan->ws_bytes;
    *out = plan;
    return CHEB_OK;
}

extern "C" int cheb_plan_create(const cheb_bsr *P_out, int32_t precision, int32_t tile, cheb_plan **out,
                                size_t *plan_ws_bytes, void *stream) {
    return plan_create_impl(P_out, precision, tile, 1, nullptr, out, plan_ws_bytes, stream);
}

extern "C" int cheb_plan_create_batched(const cheb_bsr *P_out, int32_t precision, int32_t tile, int32_t nsys,
                                        const int64_t *sys_row_start, cheb_plan **out, size_t *plan_ws_bytes,
                                        void *stream) {
    if (!sys_row_start) return fail(CHEB_ERR_INVALID, "cheb_plan_create_batched: sys_row_start is NULL");
    return plan_create_impl(P_out, precision, tile, nsys, sys_row_start, out, plan_ws_bytes, stream);
}

extern "C" int cheb_plan_bind(cheb_plan *plan, void *ws, size_t ws_bytes, void *stream) {
    if (!plan) return fail(CHEB_ERR_INVALID, "cheb_plan_bind: NULL plan");
    if (!ws || ws_bytes < plan->ws_bytes)
        return fail(CHEB_ERR_NOSPACE, "cheb_plan_bind: workspace %zu < %zu", ws_bytes, plan->ws_bytes);
    if (((uintptr_t)ws) % 256) return fail(CHEB_ERR_INVALID, "cheb_plan_bind: workspace not 256-byte aligned");
    Carve cv(ws, ws_bytes);
    plan->d_tperm = cv.take<int32_t>(plan->nnzb);
    plan->d_panels = cv.take<int32_t>(plan->h_panels.size());
    plan->d_counter = cv.take<int32_t>(16);
    plan->d_rpanels = cv.take<int32_t>(plan->h_rpanels.size());
    plan->d_rpanel_sys = cv.take<int32_t>(plan->h_rpanel_sys.size());
    plan->d_sys_rpanel = cv.take<int32_t>(plan->h_sys_rpanel.size());
    cudaStream_t s = as_stream(stream);
    if (plan->tmp_tperm)
        CHEB_CUDA(cudaMemcpyAsync(plan->d_tperm, plan->tmp_tperm, plan->nnzb * 4, cudaMemcpyDeviceToDevice, s));
    else
        CHEB_CUDA(cudaMemcpyAsync(plan->d_tperm, plan->h_tperm.data(), plan->nnzb * 4, cudaMemcpyHostToDevice, s));
    CHEB_CUDA(cudaMemcpyAsync(plan->d_panels, plan->h_panels.data(), plan->h_panels.size() * 4,
                              cudaMemcpyHostToDevice, s));
    CHEB_CUDA(cudaMemsetAsync(plan->d_counter, 0, 64, s));
    CHEB_CUDA(cudaMemcpyAsync(plan->d_rpanels, plan->h_rpanels.data(), plan->h_rpanels.size() * 4,
                              cudaMemcpyHostToDevice, s));
    CHEB_CUDA(cudaMemcpyAsync(plan->d_rpanel_sys, plan->h_rpanel_sys.data(), plan->h_rpanel_sys.size() * 4,
                              cudaMemcpyHostToDevice, s));
    CHEB_CUDA(cudaMemcpyAsync(plan->d_sys_rpanel, plan->h_sys_rpanel.data(), plan->h_sys_rpanel.size() * 4,
                              cudaMemcpyHostToDevice, s));
    // The host vectors are read by the async copies: finish them before returning.
    CHEB_CUDA(cudaStreamSynchronize(s));
    if (plan->tmp_tperm) {
        cudaFree(plan->tmp_tperm);
        plan->tmp_tperm = nullptr;
    }
    plan->bound = true;
    return CHEB_OK;
}

extern "C" int cheb_plan_info(const cheb_plan *plan, int64_t *n_panels, int32_t *panel_width,
                              int32_t *max_union) {
    if (!plan) return fail(CHEB_ERR_INVALID, "cheb_plan_info: NULL plan");
    if (n_panels) *n_panels = plan->n_panels;
    if (panel_width) *panel_width = plan->P;
    if (max_union) *max_union = plan->max_union;
    return CHEB_OK;
}

extern "C" int cheb_plan_resident_info(const cheb_plan *plan, int64_t *n_panels, int32_t *max_union,
                                       int32_t *max_blocks) {
    if (!plan) return fail(CHEB_ERR_INVALID, "cheb_plan_resident_info: NULL plan");
    if (n_panels) *n_panels = plan->n_rpanels;
    if (max_union) *max_union = plan->max_union_res;
    if (max_blocks) *max_blocks = plan->max_nblk_res;
    return CHEB_OK;
}

extern "C" int cheb_plan_col_info(const cheb_plan *plan, int64_t *n_panels, int32_t *max_union,
                                  int64_t *n_entries) {
    if (!plan) return fail(CHEB_ERR_INVALID, "cheb_plan_col_info: NULL plan");
    const bool on = plan->col.built;
    if (n_panels) *n_panels = on ? plan->col.n_panels : 0;
    if (max_union) *max_union = on ? plan->col.max_union : 0;
    if (n_entries) *n_entries = on ? plan->col.n_entries : 0;
    return CHEB_OK;
}

extern "C" int cheb_plan_destroy(cheb_plan *plan) {
    if (plan) {
        col_free(plan->col);
        free_row_lists(plan->lists);
        free_row_lists(plan->rlists);
        if (plan->tmp_tperm) cudaFree(plan->tmp_tperm);
    }
    delete plan;
    return CHEB_OK;
}

extern "C" int cheb_plan_set_gather_builder(cheb_plan *plan, int32_t host) {
    if (!plan || (host != 0 && host != 1)) return fail(CHEB_ERR_INVALID, "cheb_plan_set_gather_builder: bad arguments");
    plan->gather_host = host;
    return CHEB_OK;
}

extern "C" int cheb_plan_lists_copy(const cheb_plan *plan, int32_t which, void *dst, size_t dst_bytes,
                                    size_t *bytes, void *stream) {
    if (!plan || !bytes || which < 0 || which > 16) return fail(CHEB_ERR_INVALID, "cheb_plan_lists_copy: bad arguments");
    if (!plan->bound) return fail(CHEB_ERR_INVALID, "cheb_plan_lists_copy: plan not bound");
    const ColLists &c = plan->col;
    if (which <= 5 && !(c.built && c.bound))
        return fail(CHEB_ERR_INVALID, "cheb_plan_lists_copy: no bound column-kernel lists");
    if (which >= 11 && !plan->op_bound) return fail(CHEB_ERR_INVALID, "cheb_plan_lists_copy: no bound row lists");
    const int64_t np = c.n_panels;
    const RowLists &a = plan->lists, &b = plan->rlists;
    const void *src[17] = {c.d_panels, c.d_wchunk, c.d_wrow, c.d_rows, c.d_ent, c.d_slot,
                           plan->d_tperm, plan->d_panels, plan->d_rpanels, plan->d_rpanel_sys, plan->d_sys_rpanel,
                           a.d_base, a.d_ptr, a.d_ent, b.d_base, b.d_ptr, b.d_ent};
    const size_t n[17] = {(size_t)np * 16, (size_t)np * (c.NW + 1) * 4, (size_t)np * (c.NW + 1) * 4,
                          (size_t)c.n_rows * 4, (size_t)c.n_entries * 4, (size_t)c.n_slot * 2,
                          (size_t)plan->nnzb * 4, plan->h_panels.size() * 4, plan->h_rpanels.size() * 4,
                          plan->h_rpanel_sys.size() * 4, plan->h_sys_rpanel.size() * 4,
                          (size_t)a.n_base * 8, (size_t)a.n_ptr * 4, (size_t)a.n_ent * 4,
                          (size_t)b.n_base * 8, (size_t)b.n_ptr * 4, (size_t)b.n_ent * 4};
    *bytes = n[which];
    if (!dst) return CHEB_OK;
    if (dst_bytes < n[which]) return fail(CHEB_ERR_NOSPACE, "cheb_plan_lists_copy: %zu < %zu bytes", dst_bytes, n[which]);
    cudaStream_t s = as_stream(stream);
    if (n[which]) CHEB_CUDA(cudaMemcpyAsync(dst, src[which], n[which], cudaMemcpyDeviceToDevice, s));
    return CHEB_OK;
}

// Panels [p0, p1) of a panel set's operator row lists: with count_only, the
// number of list entries of each panel; otherwise the row pointers and
// entries, written at the panel offsets the counts gave.
static void build_row_lists(int64_t nbr, const std::vector<int32_t> &panels, const std::vector<int64_t> &rp,
                            const std::vector<int32_t> &ci, const std::vector<int64_t> &lrp,
                            const std::vector<int32_t> &lci, int64_t p0, int64_t p1, bool count_only,
                            std::vector<int64_t> &cnt, std::vector<int64_t> &nrow, const std::vector<int64_t> &ent_off,
                            std::vector<int32_t> &lrow_ptr, std::vector<int64_t> &lrow_base,
                            std::vector<uint32_t> &lent) {
    std::vector<int32_t> stamp(nbr, -1), slot_of(nbr, -1), uni;
    for (int64_t p = p0; p < p1; ++p) {
        const int32_t j0 = panels[2 * p], nc = panels[2 * p + 1];
        uni.clear();
        for (int32_t q = 0; q < nc; ++q)
            for (int64_t e = rp[j0 + q]; e < rp[j0 + q + 1]; ++e)
                if (stamp[ci[e]] != (int32_t)p) {
                    stamp[ci[e]] = (int32_t)p;
                    uni.push_back(ci[e]);
                }
        std::sort(uni.begin(), uni.end());
        for (size_t u = 0; u < uni.size(); ++u) slot_of[uni[u]] = (int32_t)u;
        if (count_only) {
            int64_t c = 0;
            for (const int32_t I : uni)
                for (int64_t a = lrp[I]; a < lrp[I + 1]; ++a) c += stamp[lci[a]] == (int32_t)p;
            cnt[p] = c;
            nrow[p] = (int64_t)uni.size() + 1;
            continue;
        }
        int64_t w = ent_off[p], r = lrow_base[p];
        for (const int32_t I : uni) {
            lrow_ptr[r++] = (int32_t)w;
            for (int64_t a = lrp[I]; a < lrp[I + 1]; ++a)
                if (stamp[lci[a]] == (int32_t)p)
                    lent[w++] = ((uint32_t)(a - lrp[I]) << 16) | (uint32_t)slot_of[lci[a]];
        }
        lrow_ptr[r] = (int32_t)w;
    }
}

// The row lists of one panel set (np panels), built on host threads.
static int make_row_lists(int64_t nbr, const std::vector<int32_t> &panels, int64_t np, const std::vector<int64_t> &rp,
                          const std::vector<int32_t> &ci, const std::vector<int64_t> &lrp,
                          const std::vector<int32_t> &lci, RowLists &out) {
    std::vector<int64_t> cnt(np), nrow(np), ent_off(np + 1), lrow_base(np + 1);
    std::vector<int32_t> lrow_ptr;
    std::vector<uint32_t> lent;
    const int nth = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)std::thread::hardware_concurrency(), 16, np}));
    auto run = [&](bool count_only) {
        std::vector<std::thread> th;
        for (int t = 0; t < nth; ++t) {
            const int64_t p0 = np * t / nth, p1 = np * (t + 1) / nth;
            th.emplace_back([&, p0, p1] {
                build_row_lists(nbr, panels, rp, ci, lrp, lci, p0, p1, count_only, cnt, nrow, ent_off, lrow_ptr,
                                lrow_base, lent);
            });
        }
        for (auto &x : th) x.join();
    };
    run(true);
    ent_off[0] = lrow_base[0] = 0;
    for (int64_t p = 0; p < np; ++p) {
        ent_off[p + 1] = ent_off[p] + cnt[p];
        lrow_base[p + 1] = lrow_base[p] + nrow[p];
    }
    if (ent_off[np] >= (int64_t)INT32_MAX)
        return fail(CHEB_ERR_NOSPACE, "cheb_plan_attach_operator: %lld list entries exceed the int32 offsets",
                    (long long)ent_off[np]);
    lrow_ptr.resize(lrow_base[np]);
    lent.resize(ent_off[np]);
    run(false);
    lrow_base.resize(np);
    out.h_base.swap(lrow_base);
    out.h_ptr.swap(lrow_ptr);
    out.h_ent.swap(lent);
    out.n_base = (int64_t)out.h_base.size();
    out.n_ptr = (int64_t)out.h_ptr.size();
    out.n_ent = (int64_t)out.h_ent.size();
    return CHEB_OK;
}

extern "C" int cheb_plan_attach_operator(cheb_plan *plan, const cheb_bsr *L, size_t *op_ws_bytes, void *stream) {
    if (!plan || !L || !op_ws_bytes || !L->row_ptr || !L->col_idx || L->nbr != plan->nbr)
        return fail(CHEB_ERR_INVALID, "cheb_plan_attach_operator: bad arguments");
    if (plan->ucap > 65535) return fail(CHEB_ERR_INVALID, "cheb_plan_attach_operator: union too large");
    const int64_t nbr = plan->nbr, nnzL = L->nnzb;
    if (nnzL >= (int64_t)INT32_MAX) return fail(CHEB_ERR_INVALID, "cheb_plan_attach_operator: operator too large");
    cudaStream_t s = as_stream(stream);
    free_row_lists(plan->lists);
    free_row_lists(plan->rlists);
    col_free(plan->col);
    plan->lists = RowLists();
    plan->rlists = RowLists();
    plan->col = ColLists();
    plan->op_ws_bytes = 0;
    plan->op_bound = false;
    if (!plan->gather_host) {
        // every list built by device kernels from the device patterns (gather.cu)
        if (!plan->bound) return fail(CHEB_ERR_INVALID, "cheb_plan_attach_operator: bind the plan first");
        int64_t ends[2];
        CHEB_CUDA(cudaMemcpyAsync(&ends[0], L->row_ptr, 8, cudaMemcpyDeviceToHost, s));
        CHEB_CUDA(cudaMemcpyAsync(&ends[1], L->row_ptr + nbr, 8, cudaMemcpyDeviceToHost, s));
        CHEB_CUDA(cudaStreamSynchronize(s));
        if (ends[0] != 0 || ends[1] != nnzL) return fail(CHEB_ERR_INVALID, "cheb_plan_attach_operator: bad row_ptr");
        int64_t first[2];
        CHEB_TRY(gp_check_operator(L, nbr, first, s));
        if (first[0] < nbr)
            return fail(CHEB_ERR_INVALID, "cheb_plan_attach_operator: row_ptr decreasing or row longer than 65536 blocks at row %lld",
                        (long long)first[0]);
        if (first[1] < nbr)
            return fail(CHEB_ERR_INVALID, "cheb_plan_attach_operator: column out of range in row %lld", (long long)first[1]);
        RowLists lists, rlists;
        int rc = row_lists_device(plan->rp, plan->ci, nbr, L, plan->d_panels, plan->n_panels, plan->max_union, lists, s);
        if (rc == CHEB_OK && plan->n_rpanels > 0)
            rc = row_lists_device(plan->rp, plan->ci, nbr, L, plan->d_rpanels, plan->n_rpanels, plan->max_union_res,
                                  rlists, s);
        if (rc != CHEB_OK) {
            free_row_lists(lists);
            free_row_lists(rlists);
            return rc;
        }
        plan->op_rp = L->row_ptr;
        plan->op_ci = L->col_idx;
        plan->lists = std::move(lists);
        plan->rlists = std::move(rlists);
        if (plan->precision == CHEB_F32 || plan->precision == CHEB_BF16) {
            rc = col_build_device(plan, L, col_ucap(), s);
            if (rc != CHEB_OK && rc != CHEB_ERR_NOSPACE) return rc;
        }
        plan->op_ws_bytes = plan->lists.bytes() + plan->rlists.bytes() + plan->col.bytes();
        *op_ws_bytes = plan->op_ws_bytes;
        return CHEB_OK;
    }
    std::vector<int64_t> rp(nbr + 1), lrp(nbr + 1);
    std::vector<int32_t> ci(plan->nnzb), lci(nnzL);
    CHEB_CUDA(cudaMemcpyAsync(rp.data(), plan->rp, (nbr + 1) * 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(ci.data(), plan->ci, plan->nnzb * 4, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(lrp.data(), L->row_ptr, (nbr + 1) * 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(lci.data(), L->col_idx, nnzL * 4, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    if (lrp[0] != 0 || lrp[nbr] != nnzL) return fail(CHEB_ERR_INVALID, "cheb_plan_attach_operator: bad row_ptr");
    for (int64_t I = 0; I < nbr; ++I) {
        if (lrp[I + 1] < lrp[I] || lrp[I + 1] - lrp[I] > 65536)
            return fail(CHEB_ERR_INVALID, "cheb_plan_attach_operator: row_ptr decreasing or row longer than 65536 blocks at row %lld",
                        (long long)I);
        for (int64_t a = lrp[I]; a < lrp[I + 1]; ++a)
            if (lci[a] < 0 || lci[a] >= nbr)
                return fail(CHEB_ERR_INVALID, "cheb_plan_attach_operator: column out of range in row %lld", (long long)I);
    }
    RowLists lists, rlists;
    CHEB_TRY(make_row_lists(nbr, plan->h_panels, plan->n_panels, rp, ci, lrp, lci, lists));
    if (plan->n_rpanels > 0)
        CHEB_TRY(make_row_lists(nbr, plan->h_rpanels, plan->n_rpanels, rp, ci, lrp, lci, rlists));
    plan->op_rp = L->row_ptr;
    plan->op_ci = L->col_idx;
    plan->lists = std::move(lists);
    plan->rlists = std::move(rlists);
    // reduced-precision plans: the column-order step kernel's lists (left
    // unbuilt when a panel column or an operator row does not fit it; the
    // per-step products then use the ranking kernel)
    if (plan->precision == CHEB_F32 || plan->precision == CHEB_BF16) {
        const int rc = col_build(plan, rp, ci, lrp, lci);
        if (rc != CHEB_OK && rc != CHEB_ERR_NOSPACE) return rc;
    }
    plan->op_ws_bytes = plan->lists.bytes() + plan->rlists.bytes() + plan->col.bytes();
    plan->op_bound = false;
    *op_ws_bytes = plan->op_ws_bytes;
    return CHEB_OK;
}

// Device copies of one panel set's lists, carved from the operator workspace.
static int bind_row_lists(RowLists &l, Carve &cv, cudaStream_t s) {
    if (l.n_base == 0) return CHEB_OK;
    if (l.device) {
        char *dst = cv.take<char>(l.bytes());
        if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_plan_bind_operator: workspace too small");
        CHEB_CUDA(cudaMemcpyAsync(dst, l.tmp, l.bytes(), cudaMemcpyDeviceToDevice, s));
        const ptrdiff_t d = dst - static_cast<char *>(l.tmp);
        l.d_base = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(l.d_base) + d);
        l.d_ptr = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(l.d_ptr) + d);
        l.d_ent = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(l.d_ent) + d);
        return CHEB_OK;
    }
    l.d_base = cv.take<int64_t>(l.h_base.size());
    l.d_ptr = cv.take<int32_t>(l.h_ptr.size());
    l.d_ent = cv.take<uint32_t>(std::max<size_t>(l.h_ent.size(), 1));
    if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_plan_bind_operator: workspace too small");
    CHEB_CUDA(cudaMemcpyAsync(l.d_base, l.h_base.data(), l.h_base.size() * 8, cudaMemcpyHostToDevice, s));
    CHEB_CUDA(cudaMemcpyAsync(l.d_ptr, l.h_ptr.data(), l.h_ptr.size() * 4, cudaMemcpyHostToDevice, s));
    if (!l.h_ent.empty())
        CHEB_CUDA(cudaMemcpyAsync(l.d_ent, l.h_ent.data(), l.h_ent.size() * 4, cudaMemcpyHostToDevice, s));
    return CHEB_OK;
}

extern "C" int cheb_plan_bind_operator(cheb_plan *plan, void *ws, size_t ws_bytes, void *stream) {
    if (!plan || plan->op_ws_bytes == 0) return fail(CHEB_ERR_INVALID, "cheb_plan_bind_operator: nothing attached");
    if (!ws || ws_bytes < plan->op_ws_bytes || ((uintptr_t)ws) % 256)
        return fail(CHEB_ERR_NOSPACE, "cheb_plan_bind_operator: workspace %zu < %zu or misaligned", ws_bytes,
                    plan->op_ws_bytes);
    Carve cv(ws, ws_bytes);
    cudaStream_t s = as_stream(stream);
    CHEB_TRY(bind_row_lists(plan->lists, cv, s));
    CHEB_TRY(bind_row_lists(plan->rlists, cv, s));
    CHEB_TRY(col_bind(plan->col, cv, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    col_release_host(plan->col);
    free_row_lists(plan->lists);
    free_row_lists(plan->rlists);
    // the device copies are the only ones needed from here on
    for (RowLists *l : {&plan->lists, &plan->rlists}) {
        std::vector<int32_t>().swap(l->h_ptr);
        std::vector<uint32_t>().swap(l->h_ent);
    }
    plan->op_bound = true;
    return CHEB_OK;
}
