/*
 * cheb.h -- C ABI of libcheb.so: sparse Chebyshev matrix functions on one GB300.
 *
 * The library evaluates f(M) ~ p(M) = c_0/2 I + sum_{k>=1} c_k T_k(M~) (Eq. 1)
 * for a 4x4-block-sparse symmetric M, with the spectrum mapped into [-1, 1]
 * (Eq. 2), the Chebyshev matrices from the three-term recursion (Eq. 3), each
 * product truncated to a fixed output sparsity pattern with buffer regions
 * (Sec. "Sparsity and truncation"), and the coefficients from Eq. 4 with the
 * degree picked by Eq. 6.  On top of it: Fermi-operator expansion with the
 * S^-1/2 transformation and the mu search on Tr(KS) = N (Sec. "Fermi Operator
 * Expansion"), matrix powers (Sec. "Matrix powers"), selected eigenvalues
 * (Sec. "Extraction of selected eigenvalues") and bound checks (Eq. 5).
 *
 * Conventions (all calls):
 *  - Every function returns int: CHEB_OK or one of the CHEB_ERR_* codes; the
 *    message of the last failure in the calling thread is cheb_last_error().
 *  - Matrices are block-CSR with 4x4 row-major blocks (cheb_bsr).  row_ptr is
 *    int64[nbr+1], col_idx int32[nnzb] sorted ascending within each row, vals
 *    nnzb*16 elements.  Unless stated otherwise every pointer is DEVICE memory
 *    owned by the caller; the library never frees it.
 *  - The library allocates no device memory.  Scratch memory comes from the
 *    caller through a workspace argument; each call documents how to size it.
 *    Host memory is allocated only for plan objects (cheb_plan_create).
 *  - Every call takes a cudaStream_t (passed as void*, NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless documented as
 *    "host-returning", in which case they synchronise the stream before they
 *    return their host outputs.
 *  - Output patterns must be symmetric and contain every diagonal block.
 */
#ifndef CHEB_H
#define CHEB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    CHEB_OK = 0,
    CHEB_ERR_INVALID = 1,       /* bad argument, size or pattern */
    CHEB_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
    CHEB_ERR_NOT_SPD = 3,       /* lower spectral bound <= 0 where a positive one is required */
    CHEB_ERR_BOUNDS = 4,        /* penalty check (Eq. 5) says the bounds do not hold */
    CHEB_ERR_NOT_CONVERGED = 5, /* iteration cap reached (mu bisection, degree search) */
    CHEB_ERR_TIMEOUT = 6,       /* a device-side wait gave up after its time limit */
    CHEB_ERR_NOSPACE = 7        /* workspace too small, or a pattern too wide for the kernels */
};

/* Element types of matrix values. */
enum { CHEB_F64 = 0, CHEB_F32 = 1, CHEB_BF16 = 2, CHEB_F64X = 3 };

/* Function kinds for cheb_func.kind (all in the unscaled variable x). */
enum {
    CHEB_FERMI = 0,    /* 1/(1+exp((x-mu)/kT)), Eq. 7 with beta = 1/kT */
    CHEB_ERFC = 1,     /* 0.5*erfc((x-mu)/kT), Eq. 9 with beta = 1/kT */
    CHEB_POWER = 2,    /* x^a, Sec. "Matrix powers" (x > 0 on the interval) */
    CHEB_INTERVAL = 3, /* Fermi(x; mu=hi) - Fermi(x; mu=lo): states in [lo, hi] */
    CHEB_PENALTY = 4   /* Eq. 5 in the scaled variable xs in [-1,1]:
                          exp(-|a|(xs+1)) - exp(|a|(xs-1)) */
};

typedef struct cheb_bsr {
    int64_t nbr;            /* block rows (= block columns) */
    int64_t nnzb;           /* stored 4x4 blocks */
    const int64_t *row_ptr; /* device, int64[nbr+1] */
    const int32_t *col_idx; /* device, int32[nnzb], ascending within each row */
    void *vals;             /* device, nnzb*16 elements of type dtype (may be NULL for a pattern) */
    int32_t dtype;          /* CHEB_F64 / CHEB_F32 / CHEB_BF16 */
} cheb_bsr;

typedef struct cheb_func {
    int32_t kind; /* CHEB_FERMI ... */
    double mu;    /* chemical potential (FERMI, ERFC) */
    double kT;    /* smearing width (FERMI, ERFC, INTERVAL) */
    double a;     /* exponent (POWER) or alpha (PENALTY) */
    double lo;    /* interval ends (INTERVAL) */
    double hi;
} cheb_func;

/* Message of the last failure in this thread ("" if none).  Never NULL. */
const char *cheb_last_error(void);

/* Number of kernel launches this process has made through the library (all
 * threads, all devices).  For accounting only; never resets. */
uint64_t cheb_launch_count(void);

/* ---------------------------------------------------------------------------
 * Sparsity patterns.  Sec. "Sparsity and truncation": the library works on a
 * fixed pattern; the output pattern is a larger "buffer" pattern.  Both are
 * built here from atom positions by a distance cutoff, as in the paper's tests
 * (Sec. "Performance").
 *
 * cheb_pattern_build: block pattern {(I,J) : minimum-image distance <= r_cut}
 * (inclusive, diagonal always present) for n_atoms atoms in a periodic cube
 * of edge box_L.  xyz: device double[n_atoms][3], coordinates in [0, box_L).
 * The distance test is done in float64 without fused multiply-add:
 * dx = x_J - x_I wrapped once by +-box_L when |dx| > box_L/2, then
 * (dx*dx + dy*dy) + dz*dz <= r_cut*r_cut.
 * Two calls: with col_idx == NULL it writes row_ptr (device int64[n_atoms+1])
 * and returns the block count in *nnzb (host-returning); with col_idx != NULL
 * (device int32[*nnzb]) and the row_ptr of the first call it fills the sorted
 * column lists (asynchronous).  Errors: CHEB_ERR_INVALID for n_atoms < 1,
 * box_L <= 0 or r_cut < 0.
 */
int cheb_pattern_build(const double *xyz, int64_t n_atoms, double box_L, double r_cut,
                       int64_t *row_ptr, int32_t *col_idx, int64_t *nnzb, void *stream);

/* ---------------------------------------------------------------------------
 * Plans.  A plan holds what the masked products need to know about the output
 * pattern P_out (symmetric): the transposition map of its blocks and the
 * grouping of its block columns into panels that one thread block advances
 * together (columns are independent under Eq. 3, Sec. "Expansion in Chebyshev
 * polynomials").  precision (CHEB_F64 / CHEB_F32) selects the panel width.
 *
 * The step kernel comes in several tile shapes per precision (panel width,
 * warps per block, blocks per SM); cheb_tile_count / cheb_tile_info list them.
 *
 * cheb_plan_create (host-returning): checks P_out (device row_ptr/col_idx:
 * symmetry, sortedness, diagonal blocks; CHEB_ERR_INVALID otherwise), builds
 * its transposition map and groups columns into panels for tile shape `tile`
 * (-1 = the default shape of the precision) -- with device kernels unless
 * cheb_set_plan_builder(1) asked for the host builders, see below -- and
 * returns a host-allocated plan and the device workspace it needs in
 * *plan_ws_bytes.
 * cheb_plan_bind copies the plan tables into caller device memory plan_ws
 * (>= plan_ws_bytes, 256-byte aligned); the plan then refers to that memory,
 * which must stay valid until cheb_plan_destroy.  P_out's row_ptr/col_idx
 * pointers are remembered by the plan and must stay valid too.
 * cheb_plan_info reports (n_panels, panel width, max panel union rows) of the
 * per-step kernel; cheb_plan_resident_info (n_panels, max union rows, max
 * blocks per panel) of the resident expansion kernel.  A CHEB_BF16 plan uses
 * the FP32 tile shapes.
 */
typedef struct cheb_plan cheb_plan;

int cheb_tile_count(int32_t precision);
int cheb_tile_info(int32_t precision, int32_t tile, int32_t *panel_width, int32_t *warps,
                   int32_t *blocks_per_sm);
int cheb_plan_create(const cheb_bsr *P_out, int32_t precision, int32_t tile, cheb_plan **plan,
                     size_t *plan_ws_bytes, void *stream);
int cheb_plan_bind(cheb_plan *plan, void *plan_ws, size_t plan_ws_bytes, void *stream);
int cheb_plan_info(const cheb_plan *plan, int64_t *n_panels, int32_t *panel_width,
                   int32_t *max_union);

/* Operator row lists (optional, for the per-step kernel; the gather plan of the
 * masked product restricted to each panel).  For the operator pattern L (the
 * M~ of the recursion), cheb_plan_attach_operator (host-returning) precomputes
 * for every panel and each row I of the union of its columns' row lists the
 * blocks L_IK whose column K lies in that union, as 32-bit words (offset of
 * the block within row I of L) << 16 | (rank of K in the union); rows of L
 * must hold at most 65536 blocks.  *op_ws_bytes receives the device memory
 * the lists need (about 4 bytes per entry, plus 4 per (panel, union row) and
 * 8 per panel).  After cheb_plan_bind_operator copies them into caller memory
 * op_ws (256-byte aligned, kept valid until cheb_plan_destroy or the next
 * attach), every per-step product whose operator has exactly these
 * row_ptr/col_idx pointers reads its entries from the lists instead of
 * ranking the operator's rows at every step; other operators use the ranking
 * path.  Both paths multiply the same blocks in the same order, so results
 * are bit-identical.  Attaching again replaces the lists.  The lists are
 * built by device kernels from the device arrays of P_out and L (the plan
 * must be bound first) unless the host builders were chosen (see "Builders"
 * below). */
int cheb_plan_attach_operator(cheb_plan *plan, const cheb_bsr *L, size_t *op_ws_bytes, void *stream);

/* Column-order step kernel of reduced-precision plans.  For a CHEB_F32 or
 * CHEB_BF16 plan, cheb_plan_attach_operator also builds the gather plan of a
 * second per-step kernel that keeps T_k in column order (the blocks of each
 * block column contiguous; columns are independent under Eq. 3, Sec.
 * "Expansion in Chebyshev polynomials"): panels of up to 4 block columns
 * whose union of row lists fits shared memory (at most 1023 rows), in column
 * order; per union row its operator entries with K in the union (32-bit
 * words: index of the operator block << 10 | union slot), padded to whole
 * chunks of 8 with entries naming a zero block; the union rows of a panel
 * dealt to the thread block's warps to balance their chunks, each warp's
 * chunks stored as one stream; and the union slot of every P_out block (2
 * bytes each).  After cheb_plan_bind_operator, cheb_expand_stepwise with
 * that operator and an FP32/BF16 precision runs this kernel; it sums each
 * block product in a different order from the ranking kernel, so results
 * agree to rounding, and are bitwise reproducible run to run.  It is not
 * built (and the ranking kernel runs) when one column's rows do not fit it
 * or the operator has 2^22 - 1 blocks or more.  cheb_plan_col_info reports
 * its panel count (0 when not built), largest union and total operator
 * entries (padding included).
 *
 * This gather plan is built by device kernels from the device patterns of
 * P_out and the operator (a sequential panel walk in one thread block, then
 * one thread block per panel: union bitmap and ranks, per-row entry counts, the
 * rows dealt to the warps by decreasing chunk count, each to the warp with the
 * fewest chunks so far, and the entry streams; a few scalars and per-panel
 * maxima come back to the host to size the lists).  It uses device memory of
 * its own until cheb_plan_bind_operator copies the lists into the operator
 * workspace.
 *
 * Builders.  By default cheb_plan_create and cheb_plan_attach_operator build
 * everything with device kernels from the device arrays (pattern checks, the
 * transposition map, the panel walks, the operator row lists of both panel
 * sets and the column kernel's lists); only the panel tables -- a few integers
 * per panel -- and sizes come back to the host, and cheb_plan_attach_operator
 * then needs a bound plan.  The device builders take scratch device memory
 * with cudaMalloc during the call (and hold the built tables in it until
 * cheb_plan_bind / cheb_plan_bind_operator copy them into the caller's
 * workspace); they are setup calls, not for stream capture.  cheb_set_plan_builder(1) makes later plans use the
 * host threads instead (a copy of the patterns on the host: the reference
 * builders, bit-identical), cheb_set_plan_builder(0) restores the device;
 * cheb_plan_set_gather_builder(plan, host) picks the builder of one plan's
 * next attach.  cheb_plan_lists_copy copies bound table `which` into device
 * memory dst (dst_bytes); *bytes receives its size (dst NULL: size only):
 * 0 column-kernel panels int32[4 per panel], 1 its warp chunk starts and 2
 * warp row starts int32[panels][17], 3 row words, 4 entry words uint32, 5
 * slots uint16[nnzb]; 6 the transposition map int32[nnzb]; 7 step panels and
 * 8 resident panels int32[2 per panel]; 9 the system of each resident panel,
 * 10 the first resident panel of each system (+ end); 11-13 the step panels'
 * operator row lists (first row pointer per panel int64, row pointers int32,
 * entries uint32), 14-16 the resident panels' ones.  Asynchronous. */
int cheb_plan_col_info(const cheb_plan *plan, int64_t *n_panels, int32_t *max_union, int64_t *n_entries);
int cheb_set_plan_builder(int32_t host);
int cheb_plan_set_gather_builder(cheb_plan *plan, int32_t host);
int cheb_plan_lists_copy(const cheb_plan *plan, int32_t which, void *dst, size_t dst_bytes, size_t *bytes,
                         void *stream);
int cheb_plan_bind_operator(cheb_plan *plan, void *op_ws, size_t op_ws_bytes, void *stream);
int cheb_plan_destroy(cheb_plan *plan);

/* ---------------------------------------------------------------------------
 * Eq. 2: M~ = sigma (M - tau I), sigma = 2/(emax-emin), tau = (emin+emax)/2.
 * M: FP64 matrix with every diagonal block present; out: device double[nnzb*16]
 * on M's pattern (may alias M->vals).  Asynchronous.
 */
int cheb_scale(const cheb_bsr *M, double emin, double emax, double *out, void *stream);

/* ---------------------------------------------------------------------------
 * Spectral bounds (Sec. "Determination of the eigenvalue bounds ..."): k steps
 * of plain Lanczos on the FP64 matrix M from start vector v0 (device
 * double[4*nbr]; NULL means the default v_i = 1 + u_i/2, u_i = (top 53 bits
 * of splitmix64(i)) / 2^53, i = 0..4 nbr - 1: positive, with a component along
 * every eigenvector of structured matrices), stopping early at a breakdown
 * (beta_j <= 1e-12 (|alpha_j| + beta_{j-1}): an invariant Krylov space), then
 * the extreme eigenvalues
 * theta_min/max of the Lanczos tridiagonal and the residuals
 * beta_k |s| of their Ritz pairs.  *emin = theta_min - m_lo, *emax = theta_max
 * + m_hi with m = max(2*residual, margin_frac*(theta_max - theta_min)).
 * Host-returning.  theta (host double[2], may be NULL) receives theta_min/max.
 * Workspace: cheb_bounds_workspace_size.  Errors: CHEB_ERR_INVALID for k < 1
 * or k > 512.
 */
int cheb_bounds_workspace_size(int64_t nbr, int32_t k, size_t *bytes);
int cheb_bounds(const cheb_bsr *M, int32_t k, const double *v0, double margin_frac,
                double *emin, double *emax, double *theta, void *ws, size_t ws_bytes,
                void *stream);

/* Warm start (Sec. "Determination of the eigenvalue bounds and polynomial
 * degree": in a self-consistent loop the bounds of the previous step are a
 * good guess, checked on the fly by the penalty trace).  As cheb_bounds, with
 * the result the hull of warm = [lo, hi] (host double[2], lo < hi) and the
 * Lanczos interval: Ritz values always lie within the spectrum, so a warm
 * bound that falls inside the Lanczos interval is widened to it, and a warm
 * interval that already contains it is kept (few Lanczos steps suffice).
 * Host-returning; same workspace as cheb_bounds.  Errors: as cheb_bounds, and
 * CHEB_ERR_INVALID for a NULL or empty warm interval. */
int cheb_bounds_warm(const cheb_bsr *M, int32_t k, const double *v0, double margin_frac,
                     const double *warm, double *emin, double *emax, double *theta, void *ws,
                     size_t ws_bytes, void *stream);

/* Bounds of an SPD matrix for the matrix powers (Sec. "Matrix powers"): as
 * cheb_bounds, then CHEB_ERR_NOT_SPD if the lowest Ritz value is <= 0, and the
 * lower bound raised to at least half the lowest Ritz value (the paper's
 * rescaling near zero is not specified; this keeps x^a finite on the
 * interval).  Host-returning; same workspace as cheb_bounds. */
int cheb_bounds_spd(const cheb_bsr *S, int32_t k, const double *v0, double margin_frac,
                    double *emin, double *emax, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Coefficients (Eq. 4) and degree (Eq. 6).  For each of the n_f functions
 * (host array funcs) on the interval [emin, emax]:
 *   c_j = (2/n) sum_{k<n} f(cos(pi(k+1/2)/n)/sigma + tau) cos(pi j (k+1/2)/n).
 * If tol > 0 the term count n is the smallest entry of the ladder
 * {m * 2^e : 8 <= m <= 15, e >= 1} in [16, n_max] whose maximum fit error
 * |p_n - f| over 8193 uniform points plus the 2n+1 extrema of T_{2n} is below
 * tol (divided by max|f| when rel != 0), taken as the largest such n over the
 * n_f functions; if tol <= 0, n = n_max.  coeffs: device double[n_f][n_max],
 * entries j >= n set to 0.  *n_out (host) receives n.  Host-returning.
 * Errors: CHEB_ERR_NOT_CONVERGED if no ladder entry <= n_max reaches tol;
 * CHEB_ERR_INVALID for n_f < 1, n_max < 16, emax <= emin.
 */
int cheb_coeffs_workspace_size(int32_t n_f, int32_t n_max, size_t *bytes);
int cheb_coeffs(const cheb_func *funcs, int32_t n_f, double emin, double emax, double tol,
                int32_t rel, int32_t n_max, int32_t *n_out, double *coeffs, void *ws,
                size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * The fused recursion (Eq. 1 + Eq. 3).  Mt: the scaled operator (FP64, pattern
 * P_L with every diagonal block, P_L contained in the plan's P_out, nbr equal).
 * For k = 0..n_terms-1 it forms T_0 = I, T_1 = Mt, T_{k+1} = 2 P_out(Mt T_k)
 * - T_{k-1} (left multiplication, no symmetrisation) and, fused into the same
 * pass, acc_j += coeffs[j][k] T_k for every j < n_f (c_0 halved, Eq. 1),
 * moments[k] = Tr T_k and gmoments[k] = <T_k, G> (sum over P_out of
 * elementwise products) when G is given.
 *   coeffs: device double[n_f][coeff_stride]; acc: host array of n_f device
 *   pointers, each double[nnzb(P_out)*16] in BCSR order on P_out (overwritten);
 *   moments, gmoments: device double[n_terms] or NULL; G: device double on
 *   P_out or NULL.  precision: CHEB_F64 (T_k and products in FP64), CHEB_F32
 *   (Mt rounded to FP32, T_k stored and multiplied in FP32, accumulators and
 *   moments in FP64) or CHEB_BF16 with a CHEB_BF16 plan (as CHEB_F32, with Mt
 *   and every stored T_k rounded to bfloat16, round to nearest even: bfloat16
 *   block products summed in FP32).  Results are bitwise reproducible run to
 *   run.
 *
 * cheb_expand runs the whole expansion in one kernel launch: every thread
 * block owns a panel of block columns (columns are independent under Eq. 3)
 * and keeps its T_k, T_{k-1} in shared memory for all steps; there is no
 * inter-block synchronisation.  Asynchronous, graph-capturable (no host
 * copies).  Workspace: cheb_expand_workspace_size with max_terms >= n_terms.
 * Errors: CHEB_ERR_INVALID (n_terms < 2, n_f < 0 or > 8, plan precision !=
 * precision, batched plan), CHEB_ERR_NOSPACE (workspace too small).
 */
int cheb_expand_workspace_size(const cheb_plan *plan, const cheb_bsr *Mt, int32_t precision,
                               int32_t max_terms, size_t *bytes);
int cheb_expand(const cheb_plan *plan, const cheb_bsr *Mt, int32_t n_terms,
                const double *coeffs, int32_t coeff_stride, int32_t n_f, double *const *acc,
                double *moments, const double *G, double *gmoments, int32_t precision,
                void *ws, size_t ws_bytes, void *stream);

/* The same expansion as one kernel launch per step (T_k in HBM, three
 * P_out-sized buffers in the workspace).  Same arguments and results up to
 * rounding order; kept as an independent second implementation and for
 * plans whose panels do not fit the resident kernel.  It also takes
 * precision CHEB_BF16 (with a CHEB_BF16 plan): Mt and every stored T_k are
 * rounded to bfloat16 (round to nearest even) while the block products are
 * summed in FP32 and the accumulators/moments kept in FP64 -- bfloat16 block
 * products with FP32 accumulation. */
int cheb_expand_stepwise_workspace_size(const cheb_plan *plan, const cheb_bsr *Mt,
                                        int32_t precision, size_t *bytes);
int cheb_expand_stepwise(const cheb_plan *plan, const cheb_bsr *Mt, int32_t n_terms,
                         const double *coeffs, int32_t coeff_stride, int32_t n_f,
                         double *const *acc, double *moments, const double *G, double *gmoments,
                         int32_t precision, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Batched expansion: many independent systems of uneven size in one launch.
 * The caller concatenates the systems block-diagonally (block rows of system
 * i are sys_row_start[i] .. sys_row_start[i+1]-1, each system's operator
 * already scaled with its own bounds) and creates the plan with
 * cheb_plan_create_batched so that no panel straddles two systems.  System i
 * runs n_terms[i] terms (device int32[nsys], max_terms >= all of them) with
 * coefficients coeffs + coeff_offset[i] (device int64[nsys]; layout
 * [n_f][coeff_stride] per system); moments of system i go to
 * moments/gmoments + i*moment_stride.  acc / G are on the concatenated P_out.
 * One kernel launch for all systems and all steps (plus one moment reduction);
 * asynchronous and graph-capturable.
 */
int cheb_plan_create_batched(const cheb_bsr *P_out, int32_t precision, int32_t tile,
                             int32_t nsys, const int64_t *sys_row_start, cheb_plan **plan,
                             size_t *plan_ws_bytes, void *stream);
int cheb_plan_resident_info(const cheb_plan *plan, int64_t *n_panels, int32_t *max_union,
                            int32_t *max_blocks);
int cheb_expand_batched(const cheb_plan *plan, const cheb_bsr *Mt, int32_t max_terms,
                        const int32_t *n_terms, const double *coeffs,
                        const int64_t *coeff_offset, int32_t coeff_stride, int32_t n_f,
                        double *const *acc, double *moments, const double *G, double *gmoments,
                        int32_t moment_stride, int32_t precision, void *ws, size_t ws_bytes,
                        void *stream);

/* ---------------------------------------------------------------------------
 * One masked product (the building block of Eq. 3 outside the recursion):
 *   C = alpha P_out(L R) + beta D
 * L: FP64 BCSR with nbr rows (any pattern); R, D, C: FP64 values on the plan's
 * P_out (BCSR order).  D may be NULL (beta ignored).  C must not alias R or D.
 * The plan must be an FP64 plan.  Asynchronous; no workspace.
 */
int cheb_masked_product(const cheb_plan *plan, const cheb_bsr *L, const double *R, double alpha,
                        const double *D, double beta, double *C, void *stream);

/* Block transpose on the plan's symmetric pattern: out = A^T.  FP64; out must
 * not alias A.  Asynchronous. */
int cheb_transpose(const cheb_plan *plan, const double *A, double *out, void *stream);

/* Block-diagonal concatenation (setup of a batched expansion; not in the
 * paper).  parts: host array of nsys BCSR descriptors (device pointers).
 * out_row_ptr: device int64[sum of nbr + 1] = each part's row pointers shifted
 * by the blocks of the parts before it; out_col_idx: device int32[sum of nnzb]
 * = each part's column indices shifted by the rows of the parts before it;
 * out_vals (device, may be NULL): the parts' values in order, elem_bytes (4 or
 * 8) per element, 16 elements per block.  Asynchronous.  Errors:
 * CHEB_ERR_INVALID for nsys < 1, NULL or inconsistent parts, more than
 * INT32_MAX block rows. */
int cheb_block_diag(int32_t nsys, const cheb_bsr *parts, int64_t *out_row_ptr, int32_t *out_col_idx,
                    void *out_vals, int32_t elem_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Locality relabelling of a system (the paper has no counterpart: the column
 * kernel takes panels of consecutive block columns, which column independence
 * (Sec. "Expansion in Chebyshev polynomials") allows, and atoms that lie
 * close together give panels with small unions of rows, so fewer operator
 * entries per step).  A system is relabelled by building its patterns from the
 * reordered atoms (cheb_pattern_build gives the relabelled patterns exactly)
 * and moving values between the labellings.
 *   locality_order: perm (device int64[n_atoms]) = the atoms in the order of a
 *     3-D Hilbert curve through the periodic box of edge box (J. Skilling,
 *     AIP Conf. Proc. 707, 381 (2004)): cell coordinates floor(1024 frac(x /
 *     box)) per axis, key = the 30-bit Hilbert index, ties by atom index.
 *     perm[i'] = the old index of new atom i'.  xyz: device double[n_atoms][3].
 *     Workspace: cheb_locality_order_ws(n_atoms) bytes (8 per atom, rounded up
 *     to a power of two).  Asynchronous.
 *   position_map: map (device int64[P_new->nnzb]) = position in P_old of block
 *     (perm[I'], perm[J']) for each block (I', J') of P_new (the same number
 *     of rows and blocks).  Host-returning; CHEB_ERR_INVALID if a block is
 *     missing or perm is not within [0, nbr).  Workspace: 4 bytes.
 *   gather_rows: dst[i][c] = src[map[i]][c], i < n, c < width (device
 *     doubles); rows whose map is outside [0, n_src) are written as 0.
 *   scatter_rows: dst[map[i]][c] = src[i][c]; rows whose map is outside
 *     [0, n_dst) are skipped.  Both asynchronous; src must not alias dst.
 */
size_t cheb_locality_order_ws(int64_t n_atoms);
int cheb_locality_order(const double *xyz, int64_t n_atoms, double box, int64_t *perm, void *ws,
                        size_t ws_bytes, void *stream);
int cheb_position_map(const cheb_bsr *P_new, const cheb_bsr *P_old, const int64_t *perm, int64_t *map,
                      void *ws, size_t ws_bytes, void *stream);
int cheb_gather_rows(const double *src, int64_t n_src, const int64_t *map, int64_t n, int32_t width,
                     double *dst, void *stream);
int cheb_scatter_rows(const double *src, const int64_t *map, int64_t n, int32_t width, double *dst,
                      int64_t n_dst, void *stream);

/* Keep the blocks of A (FP64 on pattern PA) that lie in pattern P: out = device
 * double[P->nnzb*16]; blocks of P outside PA are written as zero.
 * Asynchronous. */
int cheb_restrict(const cheb_bsr *A, const cheb_bsr *P, double *out, void *stream);

/* ---------------------------------------------------------------------------
 * Trace (Sec. "Fermi Operator Expansion": Tr(KS) = N).  out (device double[1])
 * = sum over the blocks (i,j) of B's pattern of A_ij * B_ij, which is Tr(A B)
 * for symmetric B; blocks of B outside A's pattern count as zero.  FP64.
 * Asynchronous.  Workspace: cheb_trace_workspace_size.
 */
int cheb_trace_workspace_size(const cheb_bsr *B, size_t *bytes);
int cheb_trace(const cheb_bsr *A, const cheb_bsr *B, double *out, void *ws, size_t ws_bytes,
               void *stream);

/* ---------------------------------------------------------------------------
 * Penalty check, Eq. 5: out (device double[1]) = c^p_0/2 t_0 + sum_k c^p_k t_k
 * with c^p from Eq. 4 for CHEB_PENALTY with parameter alpha, n_terms = length
 * of the moment vector t (device).  The bounds hold when |out| is below a
 * threshold chosen by the caller.  Asynchronous.  Workspace: 8*n_terms bytes.
 */
int cheb_penalty_trace(const double *moments, int32_t n_terms, double alpha, double *out,
                       void *ws, size_t ws_bytes, void *stream);

/* A re-summed trace: out (device double[1]) = coeffs[0]/2 moments[0] +
 * sum_{k>=1} coeffs[k] moments[k] (device arrays of n_terms).  With the
 * moments <T_k, G_H> of the energy functional and the coefficients of an
 * occupation function it is E = Tr(K H) for that function without new
 * products -- the energy comparison that chooses beta (Sec. "Fermi Operator
 * Expansion": K and K' differ only in their coefficients).  Asynchronous. */
int cheb_series_value(const double *coeffs, const double *moments, int32_t n_terms, double *out,
                      void *stream);

/* The same trace as a decision on the solve path (host-returning): *value
 * (host, may be NULL) = the penalty trace of the first n_terms (>= 3)
 * moments; *verdict (host) = 0 when |value| < threshold; otherwise the side
 * that fails, read from the last two moments: a level outside [-1, 1]
 * dominates them as T_k grows like cosh(k acosh|x~|), with alternating signs
 * below -1 (verdict -1: the lower bound is too high) and one sign above +1
 * (verdict +1: the upper bound is too low) -- the sign of the trace itself
 * does not tell, because the penalty polynomial grows outside the interval
 * too; 2 when the trace or those moments are not finite (the recursion
 * overflowed; no side named).  The threshold and alpha are the caller's (the
 * paper leaves both open); |alpha| is capped at 0.4*n_terms, so that the
 * penalty polynomial of n_terms terms resolves the exponential's decay.
 * Workspace: 8*n_terms + 8 bytes. */
int cheb_penalty_check(const double *moments, int32_t n_terms, double alpha, double threshold,
                       double *value, int32_t *verdict, void *ws, size_t ws_bytes, void *stream);

/* The bound a penalty verdict names, moved out (Eq. 5 and the penalty passage
 * of Sec. "Determination of the eigenvalue bounds and polynomial degree": the
 * failing bound has to be adjusted).  bounds: host double[2] (emin < emax),
 * updated in place: verdict -1 lowers emin, +1 raises emax, 2 (non-finite
 * trace, side unknown) does both, by frac * (emax - emin); 0 leaves them.
 * Host only, synchronous; CHEB_ERR_INVALID for a bad verdict, frac < 0 or an
 * empty interval. */
int cheb_widen_bounds(double *bounds, int32_t verdict, double frac);

/* ---------------------------------------------------------------------------
 * mu search (Sec. "Fermi Operator Expansion": adjust mu until Tr(KS) = N, by
 * re-summing the expansion with new coefficients).  gmoments: device
 * double[n_terms], g_k = Tr(post(T_k) S).  N(mu) = c_0(mu) g_0/2 +
 * sum_k c_k(mu) g_k with c(mu) from Eq. 4 for kind (CHEB_FERMI or CHEB_ERFC)
 * and width kT on [emin, emax].  Bisection on the bracket (lo, hi) (host
 * double[2]; NULL = [emin, emax]): mid = (lo+hi)/2 in float64, decision bit =
 * [N(mid) > N_e] (then hi = mid, else lo = mid), stop when |N(mid) - N_e| <=
 * tol_N or after max_iter (<= 128) iterations.
 * result: device buffer of 4 doubles + 2 uint64 = 48 bytes:
 *   [0] mu, [1] N(mu), [2] iterations, [3] 1.0 if converged else 0.0,
 *   then bits[2] (bit i of the 128-bit word = decision of iteration i).
 * Asynchronous.  Workspace: 8*n_terms bytes.
 */
int cheb_mu_search(const double *gmoments, int32_t n_terms, double emin, double emax,
                   int32_t kind, double kT, double N_e, double tol_N, int32_t max_iter,
                   const double *bracket, void *result, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * mu search without a workspace.  The paper has no counterpart: this is a
 * library convenience.  It computes exactly what cheb_mu_search computes (same
 * kernels, same arguments and result layout) for callers that cannot hand the
 * library device memory -- e.g. a host loop that must not call cudaMalloc or
 * cudaFree between steps (those calls can synchronise the whole device and
 * stall the work of other streams), or a C caller with no device allocator at
 * hand.  The call itself allocates nothing.
 *
 * Scratch: a fixed array of CHEB_MU_SEARCH_NOALLOC_MAX_TERMS doubles (128 KiB)
 * in the library's own static device memory, one per device.  n_terms above
 * that limit fails with CHEB_ERR_INVALID before anything is launched; use
 * cheb_mu_search with a workspace for longer expansions.  Nothing in the
 * scratch needs to start at zero: every one of the n_terms weights is written
 * before it is read.
 *
 * Device: the current device of the calling thread; stream must belong to it.
 * The first call on a device looks up the scratch's address there (a one-time
 * set-up per device, guarded by a host mutex); make that first call before any
 * stream capture.
 *
 * Overlap: all calls on one device share its scratch, so two calls whose work
 * can overlap (different streams without an ordering between them, or
 * different host threads) race and may return wrong results.  Calls issued to
 * one stream, or otherwise ordered, are safe.  The result buffer is the
 * caller's (device, 48 bytes, as in cheb_mu_search).  Asynchronous.
 */
#define CHEB_MU_SEARCH_NOALLOC_MAX_TERMS 16384
int cheb_mu_search_noalloc(const double *gmoments, int32_t n_terms, double emin, double emax,
                           int32_t kind, double kT, double N_e, double tol_N, int32_t max_iter,
                           const double *bracket, void *result, void *stream);

/* ---------------------------------------------------------------------------
 * One FP64 in-pattern Newton-Schulz step for S^-1 (not in the paper; repairs
 * the precision of a reduced-precision expansion):
 *   X1 = 2 X0 - P_out(X0 P_out(S X0)).
 * S: FP64 on P_S (contained in P_out); X0, X1: FP64 on the plan's P_out; tmp:
 * device double[nnzb(P_out)*16] scratch.  X1 must not alias X0 or tmp.
 * Asynchronous.
 */
int cheb_newton_schulz(const cheb_plan *plan, const cheb_bsr *S, const double *X0, double *X1,
                       double *tmp, void *stream);

/* The same kind of correction for S^-1/2 (not in the paper):
 *   Z1 = 1.5 Z0 - 0.5 P_out(Z0 P_out(S P_out(Z0 Z0))),
 * which squares the relative error of a Z0 that commutes with S (one step after
 * a reduced-precision expansion).  tmp1, tmp2: device double[nnzb(P_out)*16];
 * all pointers distinct.  Asynchronous. */
int cheb_newton_schulz_isqrt(const cheb_plan *plan, const cheb_bsr *S, const double *Z0, double *Z1,
                             double *tmp1, double *tmp2, void *stream);

/* ---------------------------------------------------------------------------
 * out = sum_{i<n} weights[i] * x[i], elementwise over len doubles (n <= 8;
 * weights: host array; x: host array of device pointers; out may alias one of
 * them).  Used to interpolate F(mu) between accumulators taken at several mu
 * of one expansion.  Asynchronous.
 */
int cheb_lincomb(int32_t n, const double *weights, const double *const *x, int64_t len, double *out,
                 void *stream);

/* Several mu from one expansion (host arithmetic, no device work): the n
 * Chebyshev points center + half*cos(pi (i+1/2)/n) of a bracket
 * (cheb_mu_nodes), and the Lagrange weights of those points at x
 * (cheb_lagrange_weights: weights[i] = prod_{j != i} (x - n_j)/(n_i - n_j)),
 * so that F(x) ~ sum_i weights[i] F(n_i) through cheb_lincomb.  n <= 64.
 * Errors: CHEB_ERR_INVALID for n out of range, half < 0, repeated nodes. */
int cheb_mu_nodes(double center, double half, int32_t n, double *nodes);
int cheb_lagrange_weights(const double *nodes, int32_t n, double x, double *weights);

/* ---------------------------------------------------------------------------
 * Learned mu proposal (not in the paper).  A 35 -> 128 -> 128 -> 2 ReLU network
 * in FP32 maps low-order moments of the scaled operator, its bounds and the
 * filling to a guess of the scaled Fermi level (output 0) and the log of a
 * bracket half-width in scaled units (output 1).  The plain bisection stays the
 * judge: it runs on the moments of the full expansion, and a mu outside the
 * proposed bracket falls back to a second expansion.
 * Parameters: one flat FP32 vector of cheb_mlp_param_count() = 21378 values,
 * W1[128][35], b1[128], W2[128][128], b2[128], W3[2][128], b3[2].
 *   forward: X device float[batch][35] -> out float[batch][2]; act (device
 *     float[batch*256]) receives the two hidden pre-activations.
 *   loss: with d = (out0 - xstar)/scale and w = exp(out1)/scale (scale =
 *     sigma*kT per sample), L = huber(d) + relu(|d| - w) + 0.01 w, mean over
 *     the batch into *loss (device double, may be NULL); dout = dL/dout.
 *   backward: grad (device float[param_count]) of sum(dout * out); ws device
 *     float[batch*256].
 *   init: Xavier-uniform weights W ~ U(-a, a), a = sqrt(6/(fan_in + fan_out)),
 *     biases 0, into theta (device float[param_count]).  The uniform of
 *     parameter i is u = (top 24 bits of splitmix64((seed * 0xD1B54A32D192ED03)
 *     xor i) + 1/2) / 2^24 (splitmix64: Steele, Lea and Flood, 2014); the
 *     weight a (2u - 1) is formed in FP64 and rounded once to FP32.
 *   adam: one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step t >= 1).
 *   features: the 35 inputs from t_k = Tr T_k (device double[32]): t_k/n_rows,
 *     emin/10, emax/10, N_e/n_rows -> device float[35].
 * All asynchronous; reductions over the batch are sequential per thread
 * (reproducible).
 */
int cheb_mlp_param_count(void);
int cheb_mlp_init(float *theta, uint64_t seed, void *stream);
int cheb_mlp_forward(const float *theta, const float *X, int32_t batch, float *act, float *out,
                     void *stream);
int cheb_mlp_loss(const float *out, const float *xstar, const float *scale, int32_t batch,
                  float *dout, double *loss, void *stream);
int cheb_mlp_backward(const float *theta, const float *X, int32_t batch, const float *act,
                      const float *dout, float *grad, float *ws, void *stream);
int cheb_mlp_adam(float *theta, const float *grad, float *m, float *v, int32_t t, float lr,
                  void *stream);
int cheb_mlp_features(const double *moments, int64_t n_rows, double emin, double emax, double N_e,
                      float *features, void *stream);

/* The bracket one network output proposes, in Ha: out (host float[2], a copy
 * of one row of cheb_mlp_forward's output) holds the scaled mu guess and the
 * log half-width; with the scaling of Eq. 2 on [emin, emax] (sigma = 2/(emax -
 * emin), tau = (emin + emax)/2): *mu_hat = out[0]/sigma + tau, *half =
 * exp(out[1])/sigma clamped to [min_half_kT*kT, max_half_kT*kT].  Host only,
 * synchronous; CHEB_ERR_INVALID for an empty interval, kT <= 0 or
 * min_half_kT > max_half_kT. */
int cheb_mlp_bracket(const float *out, double emin, double emax, double kT, double min_half_kT,
                     double max_half_kT, double *mu_hat, double *half);

/* ---------------------------------------------------------------------------
 * Segment Storage Format (Sec. "Storage format of the sparse matrices"), for
 * callers that hold matrices that way: the nonzeros of the n x n scalar matrix
 * in one value array; the pattern as nseg segments of consecutive entries,
 * keyg[4 s .. 4 s + 3] = (c_s, c_e, r_s, r_e), the first and last column and
 * row of segment s (the (2,2,nseg) descriptor in first-index-fastest order),
 * and keyv[s], the position in the value array where it starts; all indices
 * 1-based.  A segment covers the entries from (r_s, c_s) to (r_e, c_e) in
 * row-major order.
 *   export_size (host-returning): the segment and value counts of the scalar
 *     pattern of A (every entry of a present 4x4 block): one segment per scalar
 *     row and maximal run of consecutive block columns; nnz = 16 nnzb.
 *   export: keyg (device int32[4 nseg]), keyv (device int64[nseg]) and vals
 *     (device double[nnz], row-major) of A (FP64); nseg must be export_size's.
 *     Asynchronous.
 *   import_pattern (host-returning): the 4x4 block pattern holding every entry
 *     of the segments keyg (HOST int32[4 nseg]) of an n x n matrix (n a
 *     multiple of 4) plus every diagonal block: *nnzb; with row_ptr (device
 *     int64[n/4 + 1]) and col_idx (device int32[nnzb]) also the pattern.
 *   import_values (host-returning): A (a pattern from import_pattern, FP64
 *     vals written) = the matrix of keyg, keyv (device) and vals (device
 *     double[nvals]), zero outside the segments.
 * Errors: CHEB_ERR_INVALID for bad sizes, a segment outside the matrix or its
 * values outside vals, or an entry outside A's pattern.
 */
int cheb_ssf_export_size(const cheb_bsr *A, int64_t *nseg, int64_t *nnz, void *stream);
int cheb_ssf_export(const cheb_bsr *A, int64_t nseg, int32_t *keyg, int64_t *keyv, double *vals, void *stream);
int cheb_ssf_import_pattern(int64_t n, int64_t nseg, const int32_t *keyg, int64_t *nnzb, int64_t *row_ptr,
                            int32_t *col_idx, void *stream);
int cheb_ssf_import_values(const cheb_bsr *A, int64_t nseg, const int32_t *keyg, const int64_t *keyv,
                           const double *vals, int64_t nvals, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CHEB_H */
