// The plan object: transposition map and column panels of a symmetric output pattern.
#pragma once

#include <algorithm>
#include <vector>

#include "common.cuh"

// Largest dynamic shared memory a block may use on sm_100/sm_103 (227 KB).
#define CHEB_MAX_DYN_SMEM 232448

// Operator row lists of one panel set (see cheb_plan).
struct RowLists {
    std::vector<int64_t> h_base;  // [panels] first row pointer of each panel
    std::vector<int32_t> h_ptr;   // [sum of (union + 1) over panels] entry offsets
    std::vector<uint32_t> h_ent;  // entries
    int64_t n_base = 0, n_ptr = 0, n_ent = 0;  // sizes of the three arrays
    int64_t *d_base = nullptr;
    int32_t *d_ptr = nullptr;
    uint32_t *d_ent = nullptr;
    // built by the device kernels: the d_ arrays live in tmp until bound
    bool device = false;
    void *tmp = nullptr;
    size_t bytes() const {
        return n_base == 0 ? 0
                           : ::cheb::align_up((size_t)n_base * 8) + ::cheb::align_up((size_t)std::max<int64_t>(n_ptr, 1) * 4) +
                                 ::cheb::align_up((size_t)std::max<int64_t>(n_ent, 1) * 4);
    }
};

// Data of the column-order step kernel (colstep.cu) for one operator pattern:
// its own panels (at most COL_P columns whose union fits shared memory), in
// column order, as (first column, column count, union rows, 0); per panel and
// warp a range of chunks and of rows; per warp row a word (union slot, a flag
// for rows with blocks in at most two of the panel's columns and those
// columns, chunk count); the chunks' entry words (index of the block L_IK in the
// operator << COL_SLOT_BITS | union slot of K; COL_EK * 32/COL_P words per
// chunk, word e * 32/COL_P + g for K-group g); and
// the union slot of every P_out block in column order.
struct ColLists {
    int32_t P = 0, NW = 0;
    int32_t ucap = 0, max_union = 0, max_row = 0;
    int64_t n_panels = 0;
    int64_t n_entries = 0;  // padded, in whole chunks
    std::vector<int32_t> h_panels;
    std::vector<int32_t> h_wchunk;  // [panels][NW + 1]
    std::vector<int32_t> h_wrow;    // [panels][NW + 1]
    std::vector<uint32_t> h_rows;
    std::vector<uint32_t> h_ent;
    std::vector<uint16_t> h_slot;
    int32_t *d_panels = nullptr;
    int32_t *d_wchunk = nullptr;
    int32_t *d_wrow = nullptr;
    uint32_t *d_rows = nullptr;
    uint32_t *d_ent = nullptr;
    uint16_t *d_slot = nullptr;
    int64_t n_rows = 0, n_slot = 0;  // row words; P_out blocks (one slot each)
    bool built = false, bound = false;
    // built by the gather-plan kernels (gather.cu): the d_ arrays live in tmp
    // (device memory of their own) until cheb_plan_bind_operator copies them
    bool device = false;
    void *tmp = nullptr;
    size_t bytes() const {
        if (!built) return 0;
        return ::cheb::align_up((size_t)n_panels * 16) + 2 * ::cheb::align_up((size_t)n_panels * (NW + 1) * 4) +
               ::cheb::align_up((size_t)std::max<int64_t>(n_rows, 1) * 4) +
               ::cheb::align_up((size_t)std::max<int64_t>(n_entries, 1) * 4) + ::cheb::align_up((size_t)n_slot * 2);
    }
};

struct cheb_plan {
    int64_t nbr = 0;
    int64_t nnzb = 0;
    const int64_t *rp = nullptr;  // device, caller-owned pattern of P_out
    const int32_t *ci = nullptr;
    int32_t precision = CHEB_F64;
    int32_t tile = 0;       // index into the tile table of this precision
    int32_t P = 1;          // panel width (block columns advanced by one thread block)
    int32_t NW = 8;         // warps per thread block
    int32_t minb = 1;       // thread blocks per SM the shared-memory budget allows
    int64_t n_panels = 0;
    int32_t max_union = 0;  // largest union of row lists over a panel
    int32_t ucap = 0;       // union rows that fit in shared memory
    std::vector<int32_t> h_tperm;   // slot of (J,I) for each slot (I,J)
    int32_t *tmp_tperm = nullptr;   // the same, built on the device, until cheb_plan_bind
    std::vector<int32_t> h_panels;  // pairs (first column, column count)
    // panels of the resident kernel (whole expansion per thread block); they
    // never straddle two systems of a block-diagonal batch
    int32_t nsys = 1;
    std::vector<int64_t> h_sys_col;     // first block column of each system (+ end)
    std::vector<int32_t> h_rpanels;     // pairs (first column, column count)
    std::vector<int32_t> h_rpanel_sys;  // system of each resident panel
    std::vector<int32_t> h_sys_rpanel;  // first resident panel of each system (+ end)
    int64_t n_rpanels = 0;
    int32_t max_union_res = 0;  // largest union of row lists over a resident panel
    int32_t max_nblk_res = 0;   // most blocks held by a resident panel
    // device copies after cheb_plan_bind
    bool bound = false;
    int32_t *d_tperm = nullptr;
    int32_t *d_panels = nullptr;
    int32_t *d_counter = nullptr;  // grid-completion counter used by the step kernel
    int32_t *d_rpanels = nullptr;
    int32_t *d_rpanel_sys = nullptr;
    int32_t *d_sys_rpanel = nullptr;
    size_t ws_bytes = 0;
    // Operator row lists (cheb_plan_attach_operator): for every panel and each
    // of its union rows (ascending block row), the operator row's blocks whose
    // column lies in the union, as (offset of the block in the operator row
    // << 16 | union slot of the column).  One set for the per-step panels, one
    // for the resident panels.  Valid for the operator pattern (op_rp, op_ci).
    const int64_t *op_rp = nullptr;
    const int32_t *op_ci = nullptr;
    RowLists lists, rlists;
    ColLists col;  // FP32 / BF16 plans: the column-order step kernel's lists
    int32_t gather_host = 0;  // 1: build them on host threads (the reference builder)
    size_t op_ws_bytes = 0;
    bool op_bound = false;
};

namespace cheb {

// Shared-memory layout of the step kernel for a panel of width P over a union of
// ucap rows, element size esz, nw bitmap words, nwarps warps.
// Operator blocks per staged batch of the step kernel: 16 for panels of two or
// more columns (a multiple of the 32/P K-groups of a warp), 32 for one column.
__host__ __device__ constexpr int step_batch(int P) { return P >= 2 ? 16 : 32; }

struct StepLayout {
    size_t off_bits, off_ulist, off_pos, off_wl, off_bslot, off_hbuf, off_x, off_red, total;
};

__host__ __device__ inline StepLayout step_layout(int64_t nw, int64_t ucap, int P, int esz, int nwarps) {
    StepLayout L;
    size_t o = 0;
    L.off_bits = o;
    o += (size_t)nw * 8;  // uint2 {bitmap word, prefix count}
    o = (o + 15) / 16 * 16;
    L.off_ulist = o;
    o += (size_t)ucap * 4;
    o = (o + 15) / 16 * 16;
    L.off_pos = o;
    o += (size_t)ucap * P * 4;  // output block index of (union row, panel column), -1 if absent
    o = (o + 15) / 16 * 16;
    L.off_wl = o;
    o += (size_t)nwarps * 64 * 8;  // per-warp ring of staged (block index, union slot) pairs
    L.off_bslot = o;
    o += (size_t)nwarps * 64 * 4;  // union slots of the two staged batches
    o = (o + 127) / 128 * 128;
    L.off_hbuf = o;
    o += (size_t)nwarps * 2 * step_batch(P) * BB * esz;  // two staged batches of operator blocks per warp
    o = (o + 15) / 16 * 16;
    L.off_x = o;
    o += (size_t)ucap * BB * P * esz;  // the gathered panel of T_k
    o = (o + 15) / 16 * 16;
    L.off_red = o;
    o += 128 * 8;  // per-warp moment partials (<= 32 warps x 4)
    L.total = o;
    return L;
}

// Shared-memory layout of the resident kernel: the union bookkeeping of the
// panel, the global slot of each of its nblk blocks, and two nblk-block buffers
// (T_k and T_{k-1} / T_{k+1}) that stay in shared memory for the whole expansion.
struct ResLayout {
    size_t off_bits, off_ulist, off_pos, off_gslot, off_wl, off_x, off_y, off_red, total;
};

__host__ __device__ inline ResLayout res_layout(int64_t nw, int64_t ucap, int64_t bcap, int P, int esz, int nwarps) {
    ResLayout L;
    size_t o = 0;
    L.off_bits = o;
    o += (size_t)nw * 8;
    o = (o + 15) / 16 * 16;
    L.off_ulist = o;
    o += (size_t)ucap * 4;
    o = (o + 15) / 16 * 16;
    L.off_pos = o;
    o += (size_t)ucap * P * 2;
    o = (o + 15) / 16 * 16;
    L.off_gslot = o;
    o += (size_t)bcap * 4;
    o = (o + 15) / 16 * 16;
    L.off_wl = o;
    o += (size_t)nwarps * 64 * 8;
    o = (o + 127) / 128 * 128;
    const size_t xb = ((size_t)bcap * BB * esz + 127) / 128 * 128;
    L.off_x = o;
    o += xb;
    L.off_y = o;
    o += xb;
    L.off_red = o;
    o += 128 * 8;
    L.total = o;
    return L;
}

// Column-order step kernel (colstep.cu): panel width, warps, operator stages
// per warp, and its shared-memory layout for a union of ucap rows: the warps'
// stages of operator blocks, the panel's T_k blocks X[slot][4][4P] (FP32),
// the column-order position of each (union row, panel column) block, the
// moment partials of the warps.
constexpr int COL_P = 4;
constexpr int COL_NW = 16;
constexpr int COL_STAGES = 3;
constexpr int COL_EK = 2;  // operator entries of each K-group per chunk
constexpr int COL_SLOT_BITS = 10;  // union slots < 1024; operator blocks < 2^22
// a row word: union slot | half-row flag << 10 | its two columns << 11, << 13
// | chunk count << COL_ROW_SHIFT
constexpr int COL_ROW_SHIFT = COL_SLOT_BITS + 5;
struct ColLayout {
    size_t off_x, off_pos, off_stage, off_red, total;
};
__host__ __device__ inline ColLayout col_layout(int64_t ucap, int P, int nwarps) {
    ColLayout L;
    const int kg = 32 / P;
    size_t o = 0;
    L.off_stage = o;  // per warp: COL_STAGES chunks of COL_EK * 32/P operator blocks
    o += (size_t)nwarps * COL_STAGES * COL_EK * kg * 64;
    L.off_x = o;
    o += (size_t)ucap * 64 * P;
    L.off_pos = o;
    o += (size_t)ucap * P * 4;
    o = (o + 15) / 16 * 16;
    L.off_red = o;
    o += (size_t)nwarps * 6 * 8;  // moment partials: 6 per warp
    L.total = o;
    return L;
}

// Tile shapes of the step kernel: panel width P, warps per block NW, blocks per
// SM MINB (the shared-memory budget of a block is the SM's share for MINB).
struct TileCfg {
    int P, NW, MINB;
};
constexpr TileCfg TILES_F32[] = {{4, 16, 1}, {4, 8, 1}, {4, 12, 1}, {2, 8, 2}, {2, 4, 3}, {1, 8, 3}};
constexpr TileCfg TILES_F64[] = {{2, 8, 1}, {2, 4, 2}, {1, 8, 2}, {1, 4, 3}, {2, 16, 1}};
constexpr int N_TILES_F32 = sizeof(TILES_F32) / sizeof(TileCfg);
constexpr int N_TILES_F64 = sizeof(TILES_F64) / sizeof(TileCfg);
// F32 and BF16 share the FP32 shapes, F64X (8-byte double-floats) the FP64 ones
inline bool wide_elements(int precision) { return precision == CHEB_F64 || precision == CHEB_F64X; }
inline int n_tiles(int precision) { return wide_elements(precision) ? N_TILES_F64 : N_TILES_F32; }
inline TileCfg tile_cfg(int precision, int tile) {
    return wide_elements(precision) ? TILES_F64[tile] : TILES_F32[tile];
}
// Dynamic shared memory one block may use when MINB blocks share an SM
// (228 KB per SM, 1 KB reserved per block, a little static shared memory).
inline size_t smem_budget(int minb) {
    size_t per = 233472 / (size_t)minb - 1024 - 512;
    return per < (size_t)CHEB_MAX_DYN_SMEM ? per : (size_t)CHEB_MAX_DYN_SMEM;
}

// Column-order step kernel (colstep.cu): host build and binding of its lists,
// and the expansion through it.
int32_t col_ucap();
int col_build(cheb_plan *plan, const std::vector<int64_t> &rp, const std::vector<int32_t> &ci,
              const std::vector<int64_t> &lrp, const std::vector<int32_t> &lci);
// the same lists built by device kernels from the device patterns (gather.cu)
int col_build_device(cheb_plan *plan, const cheb_bsr *L, int32_t ucap, cudaStream_t s);
void col_free(ColLists &c);
// the plan of P_out and the row lists on the device (gather.cu)
int gp_check_pattern(const int64_t *rp, const int32_t *ci, int64_t nbr, int64_t nnzb, int64_t first[4],
                     int32_t *maxlen, cudaStream_t s);
int gp_tperm(const int64_t *rp, const int32_t *ci, int64_t nbr, int64_t nnzb, int32_t *tperm, int64_t *bad,
             cudaStream_t s);
int gp_walk(const int64_t *rp, const int32_t *ci, int64_t nbr, int P, int64_t ucap, int64_t bcap,
            const std::vector<int64_t> &sys_col, std::vector<int32_t> &panels4, std::vector<int32_t> &aux,
            int64_t out[4], cudaStream_t s);
int gp_check_operator(const cheb_bsr *L, int64_t nbr, int64_t first[2], cudaStream_t s);
int row_lists_device(const int64_t *rp, const int32_t *ci, int64_t nbr, const cheb_bsr *L, const int32_t *pairs,
                     int64_t np, int maxu, RowLists &out, cudaStream_t s);
int col_bind(ColLists &c, Carve &cv, cudaStream_t s);
void col_release_host(ColLists &c);
bool col_usable(const cheb_plan *plan, const cheb_bsr *Mt);
size_t col_expand_ws(const cheb_plan *plan, int64_t nnzL);
int col_expand(const cheb_plan *plan, const cheb_bsr *Mt, int32_t n_terms, const double *coeffs, int32_t stride,
               int32_t nf, double *const *acc, double *moments, const double *G, double *gmoments, void *ws,
               size_t ws_bytes, cudaStream_t s, int round_bf16);

}  // namespace cheb
