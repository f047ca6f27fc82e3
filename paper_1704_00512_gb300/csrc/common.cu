// Error state and the small elementwise kernels: scale (Eq. 2), transpose,
// restrict, trace (Tr(KS) = N, Sec. "Fermi Operator Expansion").
#include <atomic>

#include "common.cuh"
#include "plan.cuh"

namespace cheb {

std::string &last_error() {
    static thread_local std::string msg;
    return msg;
}

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    last_error() = buf;
    return code;
}

static std::atomic<unsigned long long> g_launches{0};

int check_launch(const char *what, int n_launches) {
    g_launches.fetch_add((unsigned long long)n_launches, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CHEB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return CHEB_OK;
}

// M~ = sigma (M - tau I) (Eq. 2), one thread per element.
__global__ void k_scale(const int64_t *rp, const int32_t *ci, int64_t nbr, int64_t nnzb,
                        const double *in, double *out, double sigma, double tau) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nnzb * BB) return;
    int64_t b = i / BB;
    int e = (int)(i % BB);
    double v = in[i];
    if ((e % 5) == 0) {
        int64_t I = row_of(rp, nbr, b);
        if (ci[b] == I) v = v - tau;
    }
    out[i] = sigma * v;
}

// out = A^T on a symmetric pattern: block b = (I,J) goes to slot tperm[b] = (J,I), transposed.
__global__ void k_transpose(const int32_t *tperm, int64_t nnzb, const double *in, double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nnzb * BB) return;
    int64_t b = i / BB;
    int e = (int)(i % BB), r = e >> 2, c = e & 3;
    out[(int64_t)tperm[b] * BB + c * 4 + r] = in[i];
}

// out[b] = A block at the position of P's block b; zero where A has no block
// (A is zero outside its pattern).
__global__ void k_restrict(const int64_t *Arp, const int32_t *Aci, const double *A,
                           const int64_t *Prp, const int32_t *Pci, int64_t nbr, int64_t nnzp,
                           double *out) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nnzp) return;
    int64_t I = row_of(Prp, nbr, b);
    int64_t a = find_in_row(Arp, Aci, I, Pci[b]);
#pragma unroll
    for (int e = 0; e < BB; ++e) out[b * BB + e] = a < 0 ? 0.0 : A[a * BB + e];
}

// Per-block partial of sum_{(i,j) in P_B} A_ij B_ij; fixed grid, fixed tree.
template <int NT>
__global__ void k_trace_partial(const int64_t *Arp, const int32_t *Aci, const double *A,
                                const int64_t *Brp, const int32_t *Bci, const double *B,
                                int64_t nbr, int64_t nnzb_B, double *part) {
    __shared__ double sh[NT / 32];
    double s = 0.0;
    for (int64_t b = blockIdx.x * (int64_t)NT + threadIdx.x; b < nnzb_B; b += (int64_t)gridDim.x * NT) {
        int64_t I = row_of(Brp, nbr, b);
        int64_t a = find_in_row(Arp, Aci, I, Bci[b]);
        if (a < 0) continue;  // A is zero outside its pattern
        double d = 0.0;
#pragma unroll
        for (int e = 0; e < BB; ++e) d += A[a * BB + e] * B[b * BB + e];
        s += d;
    }
    double r = block_sum<NT>(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

template <int NT>
__global__ void k_sum_partials(const double *part, int n, double *out) {
    __shared__ double sh[NT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) s += part[i];
    double r = block_sum<NT>(s, sh);
    if (threadIdx.x == 0) *out = r;
}

constexpr int TRACE_GRID = 304;

struct LinComb {
    const double *x[8];
    double w[8];
};

// out = sum_i w_i x_i (elementwise)
__global__ void k_lincomb(LinComb c, int n, int64_t len, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < n) s += c.w[j] * c.x[j][i];
        out[i] = s;
    }
}

}  // namespace cheb

using namespace cheb;

extern "C" const char *cheb_last_error(void) { return last_error().c_str(); }

extern "C" uint64_t cheb_launch_count(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

static int check_bsr(const cheb_bsr *M, const char *name, bool need_vals) {
    if (!M) return fail(CHEB_ERR_INVALID, "%s is NULL", name);
    if (M->nbr < 1 || M->nnzb < 0 || !M->row_ptr || (M->nnzb > 0 && !M->col_idx))
        return fail(CHEB_ERR_INVALID, "%s: bad sizes or pointers", name);
    if (need_vals && (!M->vals || M->dtype != CHEB_F64))
        return fail(CHEB_ERR_INVALID, "%s: FP64 values required", name);
    return CHEB_OK;
}

extern "C" int cheb_scale(const cheb_bsr *M, double emin, double emax, double *out, void *stream) {
    CHEB_TRY(check_bsr(M, "M", true));
    if (!out || !(emax > emin)) return fail(CHEB_ERR_INVALID, "cheb_scale: need out and emax > emin");
    double sigma = 2.0 / (emax - emin), tau = (emin + emax) / 2.0;
    int64_t n = M->nnzb * BB;
    if (n == 0) return CHEB_OK;
    k_scale<<<(unsigned)((n + 255) / 256), 256, 0, as_stream(stream)>>>(
        M->row_ptr, M->col_idx, M->nbr, M->nnzb, (const double *)M->vals, out, sigma, tau);
    return check_launch("k_scale");
}

extern "C" int cheb_transpose(const cheb_plan *plan, const double *A, double *out, void *stream) {
    if (!plan || !plan->bound) return fail(CHEB_ERR_INVALID, "cheb_transpose: plan not bound");
    if (!A || !out || A == out) return fail(CHEB_ERR_INVALID, "cheb_transpose: bad pointers");
    int64_t n = plan->nnzb * BB;
    k_transpose<<<(unsigned)((n + 255) / 256), 256, 0, as_stream(stream)>>>(plan->d_tperm,
                                                                            plan->nnzb, A, out);
    return check_launch("k_transpose");
}

extern "C" int cheb_restrict(const cheb_bsr *A, const cheb_bsr *P, double *out, void *stream) {
    CHEB_TRY(check_bsr(A, "A", true));
    CHEB_TRY(check_bsr(P, "P", false));
    if (!out || A->nbr != P->nbr) return fail(CHEB_ERR_INVALID, "cheb_restrict: bad output or nbr");
    if (P->nnzb == 0) return CHEB_OK;
    k_restrict<<<(unsigned)((P->nnzb + 255) / 256), 256, 0, as_stream(stream)>>>(
        A->row_ptr, A->col_idx, (const double *)A->vals, P->row_ptr, P->col_idx, P->nbr, P->nnzb,
        out);
    return check_launch("k_restrict");
}

extern "C" int cheb_trace_workspace_size(const cheb_bsr *B, size_t *bytes) {
    (void)B;
    if (!bytes) return fail(CHEB_ERR_INVALID, "bytes is NULL");
    *bytes = align_up(TRACE_GRID * sizeof(double)) + 256;
    return CHEB_OK;
}

extern "C" int cheb_trace(const cheb_bsr *A, const cheb_bsr *B, double *out, void *ws,
                          size_t ws_bytes, void *stream) {
    CHEB_TRY(check_bsr(A, "A", true));
    CHEB_TRY(check_bsr(B, "B", true));
    size_t need;
    cheb_trace_workspace_size(B, &need);
    if (!out || A->nbr != B->nbr) return fail(CHEB_ERR_INVALID, "cheb_trace: bad output or nbr");
    if (!ws || ws_bytes < need) return fail(CHEB_ERR_NOSPACE, "cheb_trace: workspace %zu < %zu", ws_bytes, need);
    Carve cv(ws, ws_bytes);
    double *part = cv.take<double>(TRACE_GRID);
    cudaStream_t s = as_stream(stream);
    k_trace_partial<256><<<TRACE_GRID, 256, 0, s>>>(A->row_ptr, A->col_idx, (const double *)A->vals,
                                                    B->row_ptr, B->col_idx, (const double *)B->vals,
                                                    B->nbr, B->nnzb, part);
    CHEB_TRY(check_launch("k_trace_partial"));
    k_sum_partials<256><<<1, 256, 0, s>>>(part, TRACE_GRID, out);
    return check_launch("k_sum_partials");
}

extern "C" int cheb_lincomb(int32_t n, const double *weights, const double *const *x, int64_t len, double *out,
                            void *stream) {
    if (n < 1 || n > 8 || !weights || !x || !out || len < 0) return fail(CHEB_ERR_INVALID, "cheb_lincomb: bad arguments");
    LinComb c{};
    for (int j = 0; j < n; ++j) {
        if (!x[j]) return fail(CHEB_ERR_INVALID, "cheb_lincomb: input %d is NULL", j);
        c.x[j] = x[j];
        c.w[j] = weights[j];
    }
    if (len == 0) return CHEB_OK;
    k_lincomb<<<1216, 256, 0, as_stream(stream)>>>(c, n, len, out);
    return check_launch("k_lincomb");
}

// Block-diagonal concatenation of BCSR matrices (the input of a batched
// expansion): row pointers shifted by the blocks before each part, column
// indices by the rows before it, values copied in order.
namespace cheb {
__global__ void k_shift_i64(const int64_t *in, int64_t n, int64_t add, int64_t *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i] + add;
}
__global__ void k_shift_i32(const int32_t *in, int64_t n, int32_t add, int32_t *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i] + add;
}
}  // namespace cheb

extern "C" int cheb_block_diag(int32_t nsys, const cheb_bsr *parts, int64_t *out_row_ptr, int32_t *out_col_idx,
                               void *out_vals, int32_t elem_bytes, void *stream) {
    if (nsys < 1 || !parts || !out_row_ptr || !out_col_idx)
        return fail(CHEB_ERR_INVALID, "cheb_block_diag: bad arguments");
    if (out_vals && elem_bytes != 4 && elem_bytes != 8)
        return fail(CHEB_ERR_INVALID, "cheb_block_diag: elem_bytes must be 4 or 8");
    int64_t rows = 0, blocks = 0;
    for (int i = 0; i < nsys; ++i) {
        const cheb_bsr &M = parts[i];
        if (M.nbr < 1 || M.nnzb < 0 || !M.row_ptr || (M.nnzb > 0 && !M.col_idx) || (out_vals && M.nnzb > 0 && !M.vals))
            return fail(CHEB_ERR_INVALID, "cheb_block_diag: part %d: bad sizes or pointers", i);
        rows += M.nbr;
        blocks += M.nnzb;
    }
    if (rows >= (int64_t)INT32_MAX) return fail(CHEB_ERR_INVALID, "cheb_block_diag: too many block rows");
    cudaStream_t s = as_stream(stream);
    int64_t r0 = 0, b0 = 0;
    int launches = 0;
    for (int i = 0; i < nsys; ++i) {
        const cheb_bsr &M = parts[i];
        k_shift_i64<<<(unsigned)((M.nbr + 255) / 256), 256, 0, s>>>(M.row_ptr, M.nbr, b0, out_row_ptr + r0);
        ++launches;
        if (M.nnzb > 0) {
            k_shift_i32<<<(unsigned)((M.nnzb + 255) / 256), 256, 0, s>>>(M.col_idx, M.nnzb, (int32_t)r0,
                                                                         out_col_idx + b0);
            ++launches;
            if (out_vals)
                CHEB_CUDA(cudaMemcpyAsync(static_cast<char *>(out_vals) + b0 * BB * elem_bytes, M.vals,
                                          (size_t)M.nnzb * BB * elem_bytes, cudaMemcpyDeviceToDevice, s));
        }
        r0 += M.nbr;
        b0 += M.nnzb;
    }
    // the closing row pointer: the last part's end, shifted like its other rows
    const cheb_bsr &L = parts[nsys - 1];
    k_shift_i64<<<1, 1, 0, s>>>(L.row_ptr + L.nbr, 1, b0 - L.nnzb, out_row_ptr + rows);
    ++launches;
    return check_launch("cheb_block_diag", launches);
}
