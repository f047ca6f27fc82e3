// Chebyshev coefficients (Eq. 4), degree selection (Eq. 6), the penalty trace
// (Eq. 5) and the mu bisection on the trace functional (Sec. "Fermi Operator
// Expansion"), all in FP64.
#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace cheb {

constexpr int GRID_UNIFORM = 8193;

struct FuncArr {
    cheb_func f[8];
};

__device__ __forceinline__ double fermi(double x, double mu, double kT) {
    return 1.0 / (1.0 + exp((x - mu) / kT));
}

// f(x) for the unscaled variable x; sigma/tau map x into [-1,1] (Eq. 2).
__device__ double feval(const cheb_func &f, double x, double sigma, double tau) {
    switch (f.kind) {
        case CHEB_FERMI: return fermi(x, f.mu, f.kT);
        case CHEB_ERFC: return 0.5 * erfc((x - f.mu) / f.kT);
        case CHEB_POWER: return pow(x, f.a);
        case CHEB_INTERVAL: return fermi(x, f.hi, f.kT) - fermi(x, f.lo, f.kT);
        case CHEB_PENALTY: {
            const double xs = sigma * (x - tau), al = fabs(f.a);
            return exp(-al * (xs + 1.0)) - exp(al * (xs - 1.0));
        }
        default: return 0.0;
    }
}

// x_k = cos(pi (k+1/2)/n) / sigma + tau: the k-th Chebyshev node mapped back (Eq. 4).
__device__ __forceinline__ double node(int k, int n, double sigma, double tau) {
    return cos(M_PI * (k + 0.5) / n) / sigma + tau;
}

// cos(pi j (k+1/2)/n) with the argument reduced exactly: j(2k+1) mod 4n.
__device__ __forceinline__ double dct_cos(int64_t j, int64_t k, int64_t n) {
    const int64_t idx = (j * (2 * k + 1)) % (4 * n);
    return cos(M_PI * (double)idx / (2.0 * (double)n));
}

// f at the nodes of every (function, candidate) pair: fv[(f*nc + c)*nmax + k].
__global__ void k_nodes(FuncArr F, int nf, const int *cand, int nc, int nmax, double sigma, double tau,
                        double *fv) {
    const int fc = blockIdx.y, f = fc / nc, c = fc % nc;
    const int n = cand[c];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        fv[(int64_t)fc * nmax + k] = feval(F.f[f], node(k, n, sigma, tau), sigma, tau);
}

// Cosine tables cos(pi i / (2n)), i < 4n, for every candidate n (tab + 4*toff[c]).
__global__ void k_cos_table(const int *cand, const int64_t *toff, int nc, double *tab) {
    const int c = blockIdx.y;
    const int64_t n = cand[c];
    double *t = tab + toff[c];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 4 * n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = cos(M_PI * (double)i / (2.0 * (double)n));
}

// c_j = (2/n) sum_k f_k cos(pi j (k+1/2)/n) (Eq. 4), one thread per j; the
// cosine is the table entry j(2k+1) mod 4n (the same value dct_cos computes).
__global__ void k_dct(const double *fv, const int *cand, const int64_t *toff, const double *tab, int nc, int nmax,
                      double *cv) {
    const int fc = blockIdx.y, c = fc % nc;
    const int64_t n = cand[c];
    const double *fk = fv + (int64_t)fc * nmax;
    const double *t = tab + toff[c];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nmax; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        if (j < n) {
            const int64_t step = 2 * (int64_t)j, m = 4 * n;
            int64_t idx = j % m;  // j (2k+1) mod 4n for k = 0
            for (int64_t k = 0; k < n; ++k) {
                s += fk[k] * t[idx];
                idx += step;
                if (idx >= m) idx -= m * (idx / m);
            }
            s = (2.0 / n) * s;
        }
        cv[(int64_t)fc * nmax + j] = s;
    }
}

__device__ __forceinline__ unsigned long long dbits(double v) { return __double_as_longlong(v); }

// max |p_n(x) - f(x)| and max |f(x)| over the degree grid: 8193 uniform points
// on [-1,1] plus the 2n+1 extrema of T_{2n}.  p_n by the scalar recursion
// T_{j+1} = 2 x T_j - T_{j-1} with explicit roundings.  Max over non-negative
// doubles is taken on their bit patterns (order-independent).
__global__ void k_fit_error(FuncArr F, const double *cv, const int *cand, int nc, int nmax, double sigma,
                            double tau, unsigned long long *errmax, unsigned long long *fabsmax) {
    const int fc = blockIdx.y, f = fc / nc, c = fc % nc;
    const int n = cand[c];
    const double *cc = cv + (int64_t)fc * nmax;
    const int npts = GRID_UNIFORM + 2 * n + 1;
    double emax = 0.0, fm = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += gridDim.x * blockDim.x) {
        double x;
        if (i < GRID_UNIFORM) x = -1.0 + i * (2.0 / (GRID_UNIFORM - 1));
        else x = cos(M_PI * (double)(i - GRID_UNIFORM) / (2.0 * n));
        double Tm = 1.0, T = x;
        double p = __dmul_rn(0.5 * cc[0], Tm);
        if (n > 1) p = __dadd_rn(p, __dmul_rn(cc[1], T));
        const double x2 = __dmul_rn(2.0, x);
        for (int j = 2; j < n; ++j) {
            const double Tn = __dsub_rn(__dmul_rn(x2, T), Tm);
            Tm = T;
            T = Tn;
            p = __dadd_rn(p, __dmul_rn(cc[j], T));
        }
        const double fx = feval(F.f[f], x / sigma + tau, sigma, tau);
        emax = fmax(emax, fabs(p - fx));
        fm = fmax(fm, fabs(fx));
    }
    // warp max then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        fm = fmax(fm, __shfl_xor_sync(0xffffffffu, fm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(errmax + fc, dbits(emax));
        atomicMax(fabsmax + fc, dbits(fm));
    }
}

__global__ void k_pick(const double *cv, int nc, int nmax, int ci, int n, int nf, double *out) {
    const int f = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nmax; j += gridDim.x * blockDim.x)
        out[(int64_t)f * nmax + j] = j < n ? cv[((int64_t)f * nc + ci) * nmax + j] : 0.0;
}

// Penalty coefficients at n terms (Eq. 4 for Eq. 5) and their dot with the moments.
__global__ void k_penalty_coeffs(double alpha, int n, double *c) {
    cheb_func f{CHEB_PENALTY, 0, 0, alpha, 0, 0};
    // scaled variable directly: sigma = 1, tau = 0
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += feval(f, node(k, n, 1.0, 0.0), 1.0, 0.0) * dct_cos(j, k, n);
        c[j] = (2.0 / n) * s;
    }
}

template <int NT>
__global__ void k_dot_terms(const double *c, const double *t, int n, double *out) {
    __shared__ double sh[NT / 32];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += NT) s += (k == 0 ? 0.5 * c[0] : c[k]) * t[k];
    double r = block_sum<NT>(s, sh);
    if (threadIdx.x == 0) *out = r;
}

// w_i = (2/n) [g_0/2 + sum_{k>=1} g_k cos(pi k (i+1/2)/n)], so that
// N(mu) = sum_i f(x_i; mu) w_i equals c_0(mu) g_0/2 + sum_k c_k(mu) g_k
// (the two finite sums of Eq. 4 and Eq. 1 swapped).
__global__ void k_count_weights(const double *g, int n, double *w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.5 * g[0];
        for (int k = 1; k < n; ++k) s += g[k] * dct_cos(k, i, n);
        w[i] = (2.0 / n) * s;
    }
}

struct MuResult {
    double mu, N, iters, converged;
    unsigned long long bits[2];
};

template <int NT>
__global__ void k_bisect(const double *w, int n, double emin, double emax, int kind, double kT, double N_e,
                         double tol_N, int max_iter, double lo, double hi, MuResult *res) {
    __shared__ double sh[NT / 32];
    __shared__ double s_N;
    const double sigma = 2.0 / (emax - emin), tau = (emin + emax) / 2.0;
    unsigned long long bits[2] = {0ull, 0ull};
    double mid = 0.5 * (lo + hi), N = 0.0;
    int it = 0, conv = 0;
    cheb_func f{kind, 0.0, kT, 0.0, 0.0, 0.0};
    for (it = 1; it <= max_iter; ++it) {
        mid = 0.5 * (lo + hi);
        f.mu = mid;
        double s = 0.0;
        for (int i = threadIdx.x; i < n; i += NT) s += feval(f, node(i, n, sigma, tau), sigma, tau) * w[i];
        double r = block_sum<NT>(s, sh);
        if (threadIdx.x == 0) s_N = r;
        __syncthreads();
        N = s_N;
        __syncthreads();
        if (fabs(N - N_e) <= tol_N) {
            conv = 1;
            break;
        }
        if (N > N_e) {
            bits[(it - 1) >> 6] |= 1ull << ((it - 1) & 63);
            hi = mid;
        } else {
            lo = mid;
        }
    }
    if (!conv) {
        it = max_iter;
        mid = 0.5 * (lo + hi);
    }
    if (threadIdx.x == 0) {
        res->mu = mid;
        res->N = N;
        res->iters = it;
        res->converged = conv;
        res->bits[0] = bits[0];
        res->bits[1] = bits[1];
    }
}

std::vector<int> ladder(int n_max) {
    std::vector<int> v;
    for (int e = 1; 8 * (1 << e) <= n_max; ++e)
        for (int m = 8; m < 16; ++m) {
            int x = m * (1 << e);
            if (x >= 16 && x <= n_max) v.push_back(x);
        }
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    return v;
}

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_coeffs_workspace_size(int32_t n_f, int32_t n_max, size_t *bytes) {
    if (!bytes || n_f < 1 || n_f > 8 || n_max < 16) return fail(CHEB_ERR_INVALID, "cheb_coeffs_workspace_size: bad args");
    const std::vector<int> lad = ladder(n_max);
    const size_t nc = lad.size() + 1;
    size_t tab = 4 * (size_t)n_max;
    for (int n : lad) tab += 4 * (size_t)n;
    *bytes = 2 * align_up(n_f * nc * (size_t)n_max * 8) + 2 * align_up(n_f * nc * 8) + align_up(nc * 4) +
             align_up(nc * 8) + align_up(tab * 8) + 256;
    return CHEB_OK;
}

extern "C" int cheb_coeffs(const cheb_func *funcs, int32_t n_f, double emin, double emax, double tol, int32_t rel,
                           int32_t n_max, int32_t *n_out, double *coeffs, void *ws, size_t ws_bytes, void *stream) {
    if (!funcs || n_f < 1 || n_f > 8 || n_max < 16 || !(emax > emin) || !coeffs)
        return fail(CHEB_ERR_INVALID, "cheb_coeffs: bad arguments");
    size_t need;
    CHEB_TRY(cheb_coeffs_workspace_size(n_f, n_max, &need));
    if (!ws || ws_bytes < need) return fail(CHEB_ERR_NOSPACE, "cheb_coeffs: workspace %zu < %zu", ws_bytes, need);
    std::vector<int> cand = tol > 0 ? ladder(n_max) : std::vector<int>{n_max};
    if (cand.empty()) return fail(CHEB_ERR_INVALID, "cheb_coeffs: empty degree ladder");
    const int nc = (int)cand.size();
    const double sigma = 2.0 / (emax - emin), tau = (emin + emax) / 2.0;
    FuncArr F{};
    for (int f = 0; f < n_f; ++f) F.f[f] = funcs[f];
    Carve cv(ws, ws_bytes);
    double *fv = cv.take<double>((size_t)n_f * nc * n_max);
    double *cvv = cv.take<double>((size_t)n_f * nc * n_max);
    unsigned long long *errm = cv.take<unsigned long long>((size_t)n_f * nc);
    unsigned long long *fmx = cv.take<unsigned long long>((size_t)n_f * nc);
    int *dcand = cv.take<int>(nc);
    int64_t *dtoff = cv.take<int64_t>(nc);
    std::vector<int64_t> toff(nc);
    int64_t tsum = 0;
    for (int c = 0; c < nc; ++c) {
        toff[c] = tsum;
        tsum += 4 * (int64_t)cand[c];
    }
    double *tab = cv.take<double>(tsum);
    if (!cv.fits()) return fail(CHEB_ERR_NOSPACE, "cheb_coeffs: workspace too small");
    cudaStream_t s = as_stream(stream);
    // host arrays are staged by the copy (pageable memory) before these return
    CHEB_CUDA(cudaMemcpyAsync(dcand, cand.data(), nc * 4, cudaMemcpyHostToDevice, s));
    CHEB_CUDA(cudaMemcpyAsync(dtoff, toff.data(), nc * 8, cudaMemcpyHostToDevice, s));
    const dim3 g0((4 * n_max + 255) / 256, nc);
    k_cos_table<<<g0, 256, 0, s>>>(dcand, dtoff, nc, tab);
    CHEB_TRY(check_launch("k_cos_table"));
    const dim3 g1((n_max + 255) / 256, n_f * nc);
    k_nodes<<<g1, 256, 0, s>>>(F, n_f, dcand, nc, n_max, sigma, tau, fv);
    CHEB_TRY(check_launch("k_nodes"));
    k_dct<<<g1, 256, 0, s>>>(fv, dcand, dtoff, tab, nc, n_max, cvv);
    CHEB_TRY(check_launch("k_dct"));
    int chosen = nc - 1;
    if (tol > 0) {
        CHEB_CUDA(cudaMemsetAsync(errm, 0, n_f * nc * 8, s));
        CHEB_CUDA(cudaMemsetAsync(fmx, 0, n_f * nc * 8, s));
        const int pts = GRID_UNIFORM + 2 * n_max + 1;
        const dim3 g2((pts + 255) / 256, n_f * nc);
        k_fit_error<<<g2, 256, 0, s>>>(F, cvv, dcand, nc, n_max, sigma, tau, errm, fmx);
        CHEB_TRY(check_launch("k_fit_error"));
        std::vector<unsigned long long> he(n_f * nc), hf(n_f * nc);
        CHEB_CUDA(cudaMemcpyAsync(he.data(), errm, n_f * nc * 8, cudaMemcpyDeviceToHost, s));
        CHEB_CUDA(cudaMemcpyAsync(hf.data(), fmx, n_f * nc * 8, cudaMemcpyDeviceToHost, s));
        CHEB_CUDA(cudaStreamSynchronize(s));
        chosen = -1;
        for (int f = 0; f < n_f; ++f) {
            int cf = -1;
            for (int c = 0; c < nc; ++c) {
                double e, m;
                memcpy(&e, &he[f * nc + c], 8);
                memcpy(&m, &hf[f * nc + c], 8);
                if (rel) e = e / m;
                if (e < tol) {
                    cf = c;
                    break;
                }
            }
            if (cf < 0) return fail(CHEB_ERR_NOT_CONVERGED, "cheb_coeffs: function %d needs more than %d terms", f, n_max);
            chosen = std::max(chosen, cf);
        }
    }
    const dim3 g3((n_max + 255) / 256, n_f);
    k_pick<<<g3, 256, 0, s>>>(cvv, nc, n_max, chosen, cand[chosen], n_f, coeffs);
    CHEB_TRY(check_launch("k_pick"));
    if (n_out) {
        *n_out = cand[chosen];
        CHEB_CUDA(cudaStreamSynchronize(s));
    }
    return CHEB_OK;
}

extern "C" int cheb_penalty_trace(const double *moments, int32_t n_terms, double alpha, double *out, void *ws,
                                  size_t ws_bytes, void *stream) {
    if (!moments || !out || n_terms < 1) return fail(CHEB_ERR_INVALID, "cheb_penalty_trace: bad arguments");
    if (!ws || ws_bytes < (size_t)n_terms * 8) return fail(CHEB_ERR_NOSPACE, "cheb_penalty_trace: workspace");
    cudaStream_t s = as_stream(stream);
    double *c = static_cast<double *>(ws);
    k_penalty_coeffs<<<(n_terms + 127) / 128, 128, 0, s>>>(alpha, n_terms, c);
    CHEB_TRY(check_launch("k_penalty_coeffs"));
    k_dot_terms<256><<<1, 256, 0, s>>>(c, moments, n_terms, out);
    return check_launch("k_dot_terms");
}

extern "C" int cheb_mu_search(const double *gmoments, int32_t n_terms, double emin, double emax, int32_t kind,
                              double kT, double N_e, double tol_N, int32_t max_iter, const double *bracket,
                              void *result, void *ws, size_t ws_bytes, void *stream) {
    if (!gmoments || !result || n_terms < 2 || !(emax > emin) || max_iter < 1 || max_iter > 128 || !(kT > 0) ||
        (kind != CHEB_FERMI && kind != CHEB_ERFC))
        return fail(CHEB_ERR_INVALID, "cheb_mu_search: bad arguments");
    if (!ws || ws_bytes < (size_t)n_terms * 8) return fail(CHEB_ERR_NOSPACE, "cheb_mu_search: workspace");
    cudaStream_t s = as_stream(stream);
    double *w = static_cast<double *>(ws);
    k_count_weights<<<(n_terms + 127) / 128, 128, 0, s>>>(gmoments, n_terms, w);
    CHEB_TRY(check_launch("k_count_weights"));
    const double lo = bracket ? bracket[0] : emin, hi = bracket ? bracket[1] : emax;
    k_bisect<256><<<1, 256, 0, s>>>(w, n_terms, emin, emax, kind, kT, N_e, tol_N, max_iter, lo, hi,
                                     static_cast<MuResult *>(result));
    return check_launch("k_bisect");
}

// Workspace-free mu search (no counterpart in the paper).  The count weights
// live in a static device array of the library; its address is looked up once
// per device with that device current and cached under a host mutex.
namespace cheb {

static __device__ __align__(256) double g_mu_noalloc_w[CHEB_MU_SEARCH_NOALLOC_MAX_TERMS];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_mu_noalloc_mx;
static double *g_mu_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

static int mu_noalloc_scratch(double **out) {
    int dev = -1;
    CHEB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return fail(CHEB_ERR_INVALID, "cheb_mu_search_noalloc: device %d beyond the %d supported", dev,
                    NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> lk(g_mu_noalloc_mx);
    if (!g_mu_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_mu_noalloc_w);
        if (e != cudaSuccess || !p)
            return fail(CHEB_ERR_CUDA, "cheb_mu_search_noalloc: scratch address on device %d: %s", dev,
                        cudaGetErrorString(e));
        g_mu_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_mu_noalloc_ptr[dev];
    return CHEB_OK;
}

}  // namespace cheb

extern "C" int cheb_mu_search_noalloc(const double *gmoments, int32_t n_terms, double emin, double emax,
                                      int32_t kind, double kT, double N_e, double tol_N, int32_t max_iter,
                                      const double *bracket, void *result, void *stream) {
    if (!gmoments || !result || n_terms < 2 || !(emax > emin) || max_iter < 1 || max_iter > 128 || !(kT > 0) ||
        (kind != CHEB_FERMI && kind != CHEB_ERFC))
        return fail(CHEB_ERR_INVALID, "cheb_mu_search_noalloc: bad arguments");
    if (n_terms > CHEB_MU_SEARCH_NOALLOC_MAX_TERMS)
        return fail(CHEB_ERR_INVALID,
                    "cheb_mu_search_noalloc: n_terms %d exceeds the static scratch of %d terms; "
                    "use cheb_mu_search with a workspace",
                    n_terms, CHEB_MU_SEARCH_NOALLOC_MAX_TERMS);
    double *w = nullptr;
    CHEB_TRY(mu_noalloc_scratch(&w));
    cudaStream_t s = as_stream(stream);
    k_count_weights<<<(n_terms + 127) / 128, 128, 0, s>>>(gmoments, n_terms, w);
    CHEB_TRY(check_launch("k_count_weights"));
    const double lo = bracket ? bracket[0] : emin, hi = bracket ? bracket[1] : emax;
    k_bisect<256><<<1, 256, 0, s>>>(w, n_terms, emin, emax, kind, kT, N_e, tol_N, max_iter, lo, hi,
                                     static_cast<MuResult *>(result));
    return check_launch("k_bisect");
}

// ---------------------------------------------------------------------------
// Scalar steps of the solve sequences, kept in the library so that the
// binding only moves arguments.

extern "C" int cheb_penalty_check(const double *moments, int32_t n_terms, double alpha, double threshold,
                                  double *value, int32_t *verdict, void *ws, size_t ws_bytes, void *stream) {
    if (!moments || n_terms < 3 || !(threshold > 0) || !verdict)
        return fail(CHEB_ERR_INVALID, "cheb_penalty_check: bad arguments");
    if (!ws || ws_bytes < (size_t)n_terms * 8 + 8) return fail(CHEB_ERR_NOSPACE, "cheb_penalty_check: workspace");
    double *out = static_cast<double *>(ws) + n_terms;
    // |alpha| at most 2/5 of the terms, so that the penalty polynomial of
    // n_terms terms resolves the exponential's decay length
    const double amax = 0.4 * n_terms;
    if (fabs(alpha) > amax) alpha = alpha < 0 ? -amax : amax;
    CHEB_TRY(cheb_penalty_trace(moments, n_terms, alpha, out, ws, (size_t)n_terms * 8, stream));
    double v = 0.0, last[2] = {0.0, 0.0};
    cudaStream_t s = as_stream(stream);
    CHEB_CUDA(cudaMemcpyAsync(&v, out, 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(last, moments + n_terms - 2, 16, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    if (value) *value = v;
    // A level outside [-1, 1] makes T_k grow like cosh(k acosh|x~|), and the
    // penalty polynomial grows with it outside the interval, so |trace| says
    // that a bound fails but its sign does not say which.  The moments do: the
    // level's term dominates them, with one sign above +1 and alternating
    // signs (T_k(-y) = (-1)^k T_k(y)) below -1.
    const bool finite = v == v && v - v == 0.0 && last[0] - last[0] == 0.0 && last[1] - last[1] == 0.0;
    if (!finite) *verdict = 2;
    else if (fabs(v) < threshold) *verdict = 0;
    else *verdict = last[0] * last[1] < 0.0 ? -1 : 1;
    return CHEB_OK;
}

extern "C" int cheb_widen_bounds(double *bounds, int32_t verdict, double frac) {
    if (!bounds || !(frac >= 0) || verdict < -1 || verdict > 2 || !(bounds[1] > bounds[0]))
        return fail(CHEB_ERR_INVALID, "cheb_widen_bounds: bad arguments");
    const double w = frac * (bounds[1] - bounds[0]);
    if (verdict == -1 || verdict == 2) bounds[0] -= w;
    if (verdict == 1 || verdict == 2) bounds[1] += w;
    return CHEB_OK;
}

extern "C" int cheb_mlp_bracket(const float *out, double emin, double emax, double kT, double min_half_kT,
                                double max_half_kT, double *mu_hat, double *half) {
    if (!out || !mu_hat || !half || !(emax > emin) || !(kT > 0) || !(min_half_kT >= 0) ||
        !(max_half_kT >= min_half_kT))
        return fail(CHEB_ERR_INVALID, "cheb_mlp_bracket: bad arguments");
    // the network works in the scaled variable of Eq. 2: x~ = sigma (e - tau)
    const double sigma = 2.0 / (emax - emin), tau = 0.5 * (emin + emax);
    *mu_hat = (double)out[0] / sigma + tau;
    const double h = exp((double)out[1]) / sigma;
    *half = fmin(fmax(h, min_half_kT * kT), max_half_kT * kT);
    return CHEB_OK;
}

extern "C" int cheb_mu_nodes(double center, double half, int32_t n, double *nodes) {
    if (n < 1 || n > 64 || !nodes || !(half >= 0)) return fail(CHEB_ERR_INVALID, "cheb_mu_nodes: bad arguments");
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) nodes[i] = center + half * cos(pi * (i + 0.5) / n);
    return CHEB_OK;
}

extern "C" int cheb_lagrange_weights(const double *nodes, int32_t n, double x, double *weights) {
    if (n < 1 || n > 64 || !nodes || !weights) return fail(CHEB_ERR_INVALID, "cheb_lagrange_weights: bad arguments");
    for (int i = 0; i < n; ++i) {
        double v = 1.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            if (nodes[i] == nodes[j]) return fail(CHEB_ERR_INVALID, "cheb_lagrange_weights: repeated node");
            v *= (x - nodes[j]) / (nodes[i] - nodes[j]);
        }
        weights[i] = v;
    }
    return CHEB_OK;
}

extern "C" int cheb_bounds_spd(const cheb_bsr *S, int32_t k, const double *v0, double margin_frac, double *emin,
                               double *emax, void *ws, size_t ws_bytes, void *stream) {
    double th[2];
    CHEB_TRY(cheb_bounds(S, k, v0, margin_frac, emin, emax, th, ws, ws_bytes, stream));
    if (!(th[0] > 0)) return fail(CHEB_ERR_NOT_SPD, "cheb_bounds_spd: lowest Ritz value %g <= 0", th[0]);
    if (*emin < 0.5 * th[0]) *emin = 0.5 * th[0];
    return CHEB_OK;
}

extern "C" int cheb_series_value(const double *coeffs, const double *moments, int32_t n_terms, double *out,
                                 void *stream) {
    if (!coeffs || !moments || !out || n_terms < 1) return fail(CHEB_ERR_INVALID, "cheb_series_value: bad arguments");
    k_dot_terms<256><<<1, 256, 0, as_stream(stream)>>>(coeffs, moments, n_terms, out);
    return check_launch("k_dot_terms");
}
