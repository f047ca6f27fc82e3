// Spectral bounds from a few Lanczos steps (Sec. "Determination of the
// eigenvalue bounds and polynomial degree" suggests "a few steps of a Lanczos
// method" when no earlier bounds exist).  Plain Lanczos without
// reorthogonalisation on the FP64 block-sparse matrix, all reductions in a
// fixed order; then, on one thread, the extreme eigenvalues of the tridiagonal
// by Sturm-sequence bisection and the last component of their eigenvectors by
// inverse iteration (tridiagonal solve with partial pivoting).
#include <cmath>

#include "common.cuh"

namespace cheb {

constexpr int LZ_GRID = 304;
constexpr int LZ_NT = 256;

struct LzState {
    double alpha[512];
    double beta[512];
    double partial[LZ_GRID];
    double out[8];  // emin, emax, theta_min, theta_max, res_lo, res_hi
    int kk;         // steps actually taken (a zero beta stops early)
};

// y = A x, one warp per block row, lanes over the row's blocks.
__global__ void k_spmv(const int64_t *rp, const int32_t *ci, const double *v, int64_t nbr, const double *x,
                       double *y, const LzState *st, int step) {
    if (st && step >= st->kk) return;
    const int64_t I = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (I >= nbr) return;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t a = rp[I] + lane; a < rp[I + 1]; a += 32) {
        const double *blk = v + a * BB;
        const double *xx = x + (int64_t)ci[a] * BS;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int m = 0; m < 4; ++m) acc[i] += blk[4 * i + m] * xx[m];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        double s = warp_sum(acc[i]);
        if (lane == 0) y[I * BS + i] = s;
    }
}

// mode 0: partial of x.x; mode 1: w -= beta[step-1] vm, partial of w.v;
// mode 2: w -= alpha[step] v, partial of w.w
__global__ void k_lz_vec(int mode, int64_t n, double *w, const double *v, const double *vm, LzState *st,
                         int step) {
    if (step >= st->kk) return;
    __shared__ double sh[LZ_NT / 32];
    double s = 0.0;
    const double b = (mode == 1 && step > 0) ? st->beta[step - 1] : 0.0;
    const double a = mode == 2 ? st->alpha[step] : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)LZ_NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * LZ_NT) {
        double x = w[i];
        if (mode == 1) {
            x = x - b * vm[i];
            w[i] = x;
            s += x * v[i];
        } else if (mode == 2) {
            x = x - a * v[i];
            w[i] = x;
            s += x * x;
        } else {
            s += x * x;
        }
    }
    double r = block_sum<LZ_NT>(s, sh);
    if (threadIdx.x == 0) st->partial[blockIdx.x] = r;
}

// Sum of partials into alpha[step] (what 1), beta[step] = sqrt (what 2), or the
// start-vector norm out[7] (what 0).
__global__ void k_lz_finish(LzState *st, int what, int step) {
    if (step >= st->kk) return;
    __shared__ double sh[LZ_NT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < LZ_GRID; i += LZ_NT) s += st->partial[i];
    double r = block_sum<LZ_NT>(s, sh);
    if (threadIdx.x == 0) {
        if (what == 0) st->out[7] = sqrt(r);
        else if (what == 1) st->alpha[step] = r;
        else {
            // a beta at rounding level of the step's scale is a breakdown: the
            // Krylov space is invariant (e.g. a multiple of the identity), and
            // later steps would only amplify rounding noise
            const double b = sqrt(r);
            st->beta[step] = b;
            const double ref = fabs(st->alpha[step]) + (step > 0 ? st->beta[step - 1] : 0.0);
            if (b == 0.0 || b <= 1e-12 * ref) st->kk = step + 1;
        }
    }
}

// mode 0: v = x / out[7], vm = 0; mode 1: vm = v, v = w / beta[step]
__global__ void k_lz_next(int mode, int64_t n, const double *x, double *v, double *vm, const LzState *st,
                          int step) {
    if (mode == 1 && (step >= st->kk || st->beta[step] == 0.0)) return;
    const double d = mode == 0 ? st->out[7] : st->beta[step];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (mode == 0) {
            v[i] = x[i] / d;
            vm[i] = 0.0;
        } else {
            vm[i] = v[i];
            v[i] = x[i] / d;
        }
    }
}

__global__ void k_fill(double *x, int64_t n, double val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = val;
}

// The default start vector: x_i = 1 + u_i / 2, u_i = (splitmix64(i) >> 11) / 2^53
// (SplitMix64: Steele, Lea and Flood, 2014).  Positive like the all-ones
// vector, but with a component along every eigenvector of a structured matrix
// (the all-ones vector can lie in a small invariant subspace, e.g. of the
// overlap of one atom's basis functions, and Lanczos would then stop inside it).
__device__ __forceinline__ uint64_t lz_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void k_fill_start(double *x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 1.0 + 0.5 * ((double)(lz_splitmix64((uint64_t)i) >> 11) * (1.0 / 9007199254740992.0));
}

// Number of eigenvalues of the tridiagonal (a, b) below x (Sturm sequence).
__device__ int sturm_count(const double *a, const double *b, int k, double x) {
    int c = 0;
    double q = a[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < k; ++i) {
        if (q == 0.0) q = 1e-300;
        q = a[i] - x - b[i - 1] * b[i - 1] / q;
        if (q < 0) ++c;
    }
    return c;
}

// Last component of the unit eigenvector for eigenvalue th (inverse iteration,
// three solves of (T - th I) y = y_prev by Gaussian elimination with partial
// pivoting on the tridiagonal).
__device__ double last_component(const double *a, const double *b, int k, double th, double *dl, double *d,
                                 double *du, double *y) {
    if (k == 1) return 1.0;
    for (int i = 0; i < k; ++i) y[i] = 1.0 / sqrt((double)k);
    for (int it = 0; it < 3; ++it) {
        for (int i = 0; i < k; ++i) d[i] = a[i] - th;
        for (int i = 0; i < k - 1; ++i) {
            dl[i] = b[i];
            du[i] = b[i];
        }
        for (int i = 0; i < k - 1; ++i) {
            if (fabs(d[i]) >= fabs(dl[i])) {
                if (d[i] == 0.0) d[i] = 1e-300;
                const double f = dl[i] / d[i];
                d[i + 1] -= f * du[i];
                y[i + 1] -= f * y[i];
                dl[i] = 0.0;
            } else {
                const double f = d[i] / dl[i];
                d[i] = dl[i];
                const double t = d[i + 1];
                d[i + 1] = du[i] - f * t;
                if (i < k - 2) {
                    dl[i] = du[i + 1];
                    du[i + 1] = -f * dl[i];
                } else {
                    dl[i] = 0.0;
                }
                du[i] = t;
                const double ty = y[i];
                y[i] = y[i + 1];
                y[i + 1] = ty - f * y[i + 1];
            }
        }
        if (d[k - 1] == 0.0) d[k - 1] = 1e-300;
        y[k - 1] = y[k - 1] / d[k - 1];
        y[k - 2] = (y[k - 2] - du[k - 2] * y[k - 1]) / d[k - 2];
        for (int i = k - 3; i >= 0; --i) y[i] = (y[i] - du[i] * y[i + 1] - dl[i] * y[i + 2]) / d[i];
        double nrm = 0.0;
        for (int i = 0; i < k; ++i) nrm += y[i] * y[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < k; ++i) y[i] /= nrm;
    }
    return y[k - 1];
}

__global__ void k_tridiag(LzState *st, double margin_frac, double *scratch) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k = st->kk;
    const double *a = st->alpha, *b = st->beta;
    double lo = a[0], hi = a[0];
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
    double th[2];
    for (int which = 0; which < 2; ++which) {
        double l = lo, h = hi;
        const int target = which == 0 ? 1 : k;
        for (int it = 0; it < 200; ++it) {
            const double m = 0.5 * (l + h);
            if (m <= l || m >= h) break;
            if (sturm_count(a, b, k, m) >= target) h = m; else l = m;
        }
        th[which] = which == 0 ? h : l;
    }
    const double bl = b[k - 1];
    double *dl = scratch, *d = scratch + 512, *du = scratch + 1024, *y = scratch + 1536;
    const double slo = last_component(a, b, k, th[0], dl, d, du, y);
    const double shi = last_component(a, b, k, th[1], dl, d, du, y);
    const double rlo = fabs(bl * slo), rhi = fabs(bl * shi);
    const double width = th[1] - th[0];
    const double mlo = fmax(2.0 * rlo, margin_frac * width), mhi = fmax(2.0 * rhi, margin_frac * width);
    double e0 = th[0] - mlo, e1 = th[1] + mhi;
    // a (near-)degenerate spectrum still gets an interval to scale by: at
    // least 1e-3 of its magnitude (1e-3 around zero), centred on the Ritz values
    const double mag = fmax(fabs(th[0]), fabs(th[1]));
    const double wmin = 1e-3 * (mag > 0.0 ? mag : 1.0);
    if (e1 - e0 < wmin) {
        const double c = 0.5 * (th[0] + th[1]);
        e0 = fmin(e0, c - 0.5 * wmin);
        e1 = fmax(e1, c + 0.5 * wmin);
    }
    st->out[0] = e0;
    st->out[1] = e1;
    st->out[2] = th[0];
    st->out[3] = th[1];
    st->out[4] = rlo;
    st->out[5] = rhi;
}

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_bounds_workspace_size(int64_t nbr, int32_t k, size_t *bytes) {
    if (!bytes || nbr < 1 || k < 1 || k > 512) return fail(CHEB_ERR_INVALID, "cheb_bounds_workspace_size: bad args");
    *bytes = 3 * align_up(nbr * BS * 8) + align_up(sizeof(LzState)) + align_up(2048 * 8) + 256;
    return CHEB_OK;
}

extern "C" int cheb_bounds(const cheb_bsr *M, int32_t k, const double *v0, double margin_frac, double *emin,
                           double *emax, double *theta, void *ws, size_t ws_bytes, void *stream) {
    if (!M || !M->vals || M->dtype != CHEB_F64 || M->nbr < 1 || !emin || !emax)
        return fail(CHEB_ERR_INVALID, "cheb_bounds: bad arguments");
    size_t need;
    CHEB_TRY(cheb_bounds_workspace_size(M->nbr, k, &need));
    if (!ws || ws_bytes < need) return fail(CHEB_ERR_NOSPACE, "cheb_bounds: workspace %zu < %zu", ws_bytes, need);
    const int64_t n = M->nbr * BS;
    Carve cv(ws, ws_bytes);
    double *vm = cv.take<double>(n), *v = cv.take<double>(n), *w = cv.take<double>(n);
    LzState *st = cv.take<LzState>(1);
    double *scratch = cv.take<double>(2048);
    cudaStream_t s = as_stream(stream);
    CHEB_CUDA(cudaMemsetAsync(st, 0, sizeof(LzState), s));
    const int kk = k;
    CHEB_CUDA(cudaMemcpyAsync(&st->kk, &kk, sizeof(int), cudaMemcpyHostToDevice, s));
    // start vector (copied so v0 stays untouched) and its normalisation
    if (v0) CHEB_CUDA(cudaMemcpyAsync(w, v0, n * 8, cudaMemcpyDeviceToDevice, s));
    else {
        k_fill_start<<<LZ_GRID, LZ_NT, 0, s>>>(w, n);
        CHEB_TRY(check_launch("k_fill_start"));
    }
    k_lz_vec<<<LZ_GRID, LZ_NT, 0, s>>>(0, n, w, v, vm, st, 0);
    k_lz_finish<<<1, LZ_NT, 0, s>>>(st, 0, 0);
    k_lz_next<<<LZ_GRID, LZ_NT, 0, s>>>(0, n, w, v, vm, st, 0);
    CHEB_TRY(check_launch("lanczos start", 3));
    const unsigned sg = (unsigned)((M->nbr * 32 + 255) / 256);
    for (int j = 0; j < k; ++j) {
        k_spmv<<<sg, 256, 0, s>>>(M->row_ptr, M->col_idx, (const double *)M->vals, M->nbr, v, w, st, j);
        k_lz_vec<<<LZ_GRID, LZ_NT, 0, s>>>(1, n, w, v, vm, st, j);
        k_lz_finish<<<1, LZ_NT, 0, s>>>(st, 1, j);
        k_lz_vec<<<LZ_GRID, LZ_NT, 0, s>>>(2, n, w, v, vm, st, j);
        k_lz_finish<<<1, LZ_NT, 0, s>>>(st, 2, j);
        k_lz_next<<<LZ_GRID, LZ_NT, 0, s>>>(1, n, w, v, vm, st, j);
        CHEB_TRY(check_launch("lanczos step", 6));
    }
    k_tridiag<<<1, 32, 0, s>>>(st, margin_frac, scratch);
    CHEB_TRY(check_launch("k_tridiag"));
    double out[8];
    CHEB_CUDA(cudaMemcpyAsync(out, st->out, sizeof(out), cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    *emin = out[0];
    *emax = out[1];
    if (theta) {
        theta[0] = out[2];
        theta[1] = out[3];
    }
    return CHEB_OK;
}

extern "C" int cheb_bounds_warm(const cheb_bsr *M, int32_t k, const double *v0, double margin_frac,
                                const double *warm, double *emin, double *emax, double *theta, void *ws,
                                size_t ws_bytes, void *stream) {
    if (!warm || !(warm[0] < warm[1])) return fail(CHEB_ERR_INVALID, "cheb_bounds_warm: warm interval needs lo < hi");
    CHEB_TRY(cheb_bounds(M, k, v0, margin_frac, emin, emax, theta, ws, ws_bytes, stream));
    // Ritz values lie inside the spectrum: a warm interval that misses the
    // Lanczos interval is provably too narrow there and is extended to it
    *emin = std::fmin(*emin, warm[0]);
    *emax = std::fmax(*emax, warm[1]);
    return CHEB_OK;
}
