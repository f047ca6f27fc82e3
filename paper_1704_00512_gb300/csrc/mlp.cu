// Learned mu proposal (not in the paper): a 35 -> 128 -> 128 -> 2 ReLU network
// in FP32 with hand-written forward, loss, backward and Adam kernels.
//
// Parameters are one flat vector: W1[128][35], b1[128], W2[128][128], b2[128],
// W3[2][128], b3[2] (row-major, y = W x + b).  Every reduction over the batch is
// a sequential loop in one thread (no atomics), so results are reproducible.
#include "common.cuh"

namespace cheb {

constexpr int MLP_IN = 35, MLP_H = 128, MLP_OUT = 2;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H,
              OFF_B2 = OFF_W2 + MLP_H * MLP_H, OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_OUT * MLP_H,
              MLP_NPARAMS = OFF_B3 + MLP_OUT;

// pre[s][o] = b[o] + sum_i W[o][i] * in(s, i); in = relu(x) when relu_in.
__global__ void k_dense(const float *__restrict__ W, const float *__restrict__ b, const float *__restrict__ x,
                        int ldx, int B, int nin, int nout, int relu_in, float *__restrict__ pre, int ldp) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * nout) return;
    const int s = idx / nout, o = idx % nout;
    float acc = b[o];
    const float *w = W + (size_t)o * nin;
    const float *xs = x + (size_t)s * ldx;
    for (int i = 0; i < nin; ++i) {
        float v = xs[i];
        if (relu_in) v = fmaxf(v, 0.f);
        acc = fmaf(w[i], v, acc);
    }
    pre[(size_t)s * ldp + o] = acc;
}

// Loss of the module docstring of the oracle: d = (xhat - xstar)/scale,
// w = exp(z)/scale, L = huber(d) + relu(|d| - w) + 0.01 w; mean over the batch.
__global__ void k_mlp_loss(const float *out, const float *xstar, const float *scale, int B, float *dout,
                           double *loss) {
    __shared__ double sh[8];
    double acc = 0.0;
    for (int s = threadIdx.x; s < B; s += blockDim.x) {
        const float sc = scale[s];
        const float d = (out[2 * s] - xstar[s]) / sc;
        const float w = expf(out[2 * s + 1]) / sc;
        const float ad = fabsf(d);
        const float hub = ad <= 1.f ? 0.5f * d * d : ad - 0.5f;
        const bool miss = ad > w;
        acc += (double)(hub + (miss ? ad - w : 0.f) + 0.01f * w);
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        const float dh = ad <= 1.f ? d : sgn;
        dout[2 * s] = (dh + (miss ? sgn : 0.f)) / sc / (float)B;
        dout[2 * s + 1] = ((miss ? -1.f : 0.f) + 0.01f) * w / (float)B;
    }
    double r = block_sum<256>(acc, sh);
    if (threadIdx.x == 0 && loss) *loss = r / B;
}

// dprev[s][i] = (sum_o dy[s][o] W[o][i]) * [pre[s][i] > 0]
__global__ void k_back_act(const float *__restrict__ W, const float *__restrict__ dy, int lddy, int nout,
                           const float *__restrict__ pre, int ldp, int B, int nin, float *__restrict__ dprev,
                           int ldd) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * nin) return;
    const int s = idx / nin, i = idx % nin;
    float acc = 0.f;
    for (int o = 0; o < nout; ++o) acc = fmaf(dy[(size_t)s * lddy + o], W[(size_t)o * nin + i], acc);
    dprev[(size_t)s * ldd + i] = pre[(size_t)s * ldp + i] > 0.f ? acc : 0.f;
}

// gW[o][i] = sum_s dy[s][o] in(s, i), gb[o] = sum_s dy[s][o]; one thread per parameter.
__global__ void k_wgrad(const float *__restrict__ dy, int lddy, const float *__restrict__ x, int ldx, int relu_in,
                        int B, int nin, int nout, float *__restrict__ gW, float *__restrict__ gb) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < nout * nin) {
        const int o = idx / nin, i = idx % nin;
        float acc = 0.f;
        for (int s = 0; s < B; ++s) {
            float v = x[(size_t)s * ldx + i];
            if (relu_in) v = fmaxf(v, 0.f);
            acc = fmaf(dy[(size_t)s * lddy + o], v, acc);
        }
        gW[idx] = acc;
    } else if (idx < nout * nin + nout) {
        const int o = idx - nout * nin;
        float acc = 0.f;
        for (int s = 0; s < B; ++s) acc += dy[(size_t)s * lddy + o];
        gb[o] = acc;
    }
}

__global__ void k_adam(float *theta, const float *g, float *m, float *v, int n, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// The 35 inputs from the moments of the scaled operator: Tr T_k / N for k < 32,
// emin/10, emax/10, N_e/N.
__global__ void k_features(const double *t, int64_t n_rows, double emin, double emax, double N_e, float *f) {
    const int i = threadIdx.x;
    if (i < 32) f[i] = (float)(t[i] / (double)n_rows);
    else if (i == 32) f[i] = (float)(emin / 10.0);
    else if (i == 33) f[i] = (float)(emax / 10.0);
    else if (i == 34) f[i] = (float)(N_e / (double)n_rows);
}

inline unsigned nb(int64_t n, int t = 128) { return (unsigned)((n + t - 1) / t); }

// Xavier-uniform initialisation: W ~ U(-a, a) with a = sqrt(6 / (fan_in +
// fan_out)) per layer, biases 0.  Uniforms from a counter-based generator:
// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", 2014) of (seed * 0xD1B54A32D192ED03) ^ i for parameter i, top 24
// bits + 1/2 scaled to (0, 1); the product a (2u - 1) is formed in FP64 and
// rounded once to FP32, so any IEEE host restatement gives the same bits.
__device__ __forceinline__ uint64_t mlp_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_mlp_init(float *theta, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NPARAMS) return;
    int fan = 0;  // fan_in + fan_out of the weight matrix holding i, 0 for a bias
    if (i < OFF_B1) fan = MLP_IN + MLP_H;
    else if (i >= OFF_W2 && i < OFF_B2) fan = MLP_H + MLP_H;
    else if (i >= OFF_W3 && i < OFF_B3) fan = MLP_H + MLP_OUT;
    if (fan == 0) {
        theta[i] = 0.f;
        return;
    }
    const uint64_t r = mlp_splitmix64((seed * 0xD1B54A32D192ED03ull) ^ (uint64_t)i);
    const double u = ((double)(r >> 40) + 0.5) * (1.0 / 16777216.0);
    const double lim = sqrt(6.0 / (double)fan);
    theta[i] = (float)(lim * (2.0 * u - 1.0));
}

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_mlp_param_count(void) { return MLP_NPARAMS; }

extern "C" int cheb_mlp_init(float *theta, uint64_t seed, void *stream) {
    if (!theta) return fail(CHEB_ERR_INVALID, "cheb_mlp_init: theta is NULL");
    k_mlp_init<<<(MLP_NPARAMS + 255) / 256, 256, 0, as_stream(stream)>>>(theta, seed);
    return check_launch("k_mlp_init");
}

extern "C" int cheb_mlp_forward(const float *theta, const float *X, int32_t batch, float *act, float *out,
                                void *stream) {
    if (!theta || !X || !act || !out || batch < 1) return fail(CHEB_ERR_INVALID, "cheb_mlp_forward: bad arguments");
    cudaStream_t s = as_stream(stream);
    float *a1 = act, *a2 = act + (size_t)batch * MLP_H;
    k_dense<<<nb((int64_t)batch * MLP_H), 128, 0, s>>>(theta + OFF_W1, theta + OFF_B1, X, MLP_IN, batch, MLP_IN,
                                                        MLP_H, 0, a1, MLP_H);
    k_dense<<<nb((int64_t)batch * MLP_H), 128, 0, s>>>(theta + OFF_W2, theta + OFF_B2, a1, MLP_H, batch, MLP_H,
                                                        MLP_H, 1, a2, MLP_H);
    k_dense<<<nb((int64_t)batch * MLP_OUT), 128, 0, s>>>(theta + OFF_W3, theta + OFF_B3, a2, MLP_H, batch, MLP_H,
                                                          MLP_OUT, 1, out, MLP_OUT);
    return check_launch("cheb_mlp_forward", 3);
}

extern "C" int cheb_mlp_loss(const float *out, const float *xstar, const float *scale, int32_t batch, float *dout,
                             double *loss, void *stream) {
    if (!out || !xstar || !scale || !dout || batch < 1) return fail(CHEB_ERR_INVALID, "cheb_mlp_loss: bad arguments");
    k_mlp_loss<<<1, 256, 0, as_stream(stream)>>>(out, xstar, scale, batch, dout, loss);
    return check_launch("k_mlp_loss");
}

extern "C" int cheb_mlp_backward(const float *theta, const float *X, int32_t batch, const float *act,
                                 const float *dout, float *grad, float *ws, void *stream) {
    if (!theta || !X || !act || !dout || !grad || !ws || batch < 1)
        return fail(CHEB_ERR_INVALID, "cheb_mlp_backward: bad arguments");
    cudaStream_t s = as_stream(stream);
    const float *a1 = act, *a2 = act + (size_t)batch * MLP_H;
    float *d2 = ws, *d1 = ws + (size_t)batch * MLP_H;
    k_wgrad<<<nb(MLP_OUT * MLP_H + MLP_OUT), 128, 0, s>>>(dout, MLP_OUT, a2, MLP_H, 1, batch, MLP_H, MLP_OUT,
                                                          grad + OFF_W3, grad + OFF_B3);
    k_back_act<<<nb((int64_t)batch * MLP_H), 128, 0, s>>>(theta + OFF_W3, dout, MLP_OUT, MLP_OUT, a2, MLP_H, batch,
                                                           MLP_H, d2, MLP_H);
    k_wgrad<<<nb(MLP_H * MLP_H + MLP_H), 128, 0, s>>>(d2, MLP_H, a1, MLP_H, 1, batch, MLP_H, MLP_H, grad + OFF_W2,
                                                      grad + OFF_B2);
    k_back_act<<<nb((int64_t)batch * MLP_H), 128, 0, s>>>(theta + OFF_W2, d2, MLP_H, MLP_H, a1, MLP_H, batch, MLP_H,
                                                           d1, MLP_H);
    k_wgrad<<<nb(MLP_H * MLP_IN + MLP_H), 128, 0, s>>>(d1, MLP_H, X, MLP_IN, 0, batch, MLP_IN, MLP_H, grad + OFF_W1,
                                                       grad + OFF_B1);
    return check_launch("cheb_mlp_backward", 5);
}

extern "C" int cheb_mlp_adam(float *theta, const float *grad, float *m, float *v, int32_t t, float lr, void *stream) {
    if (!theta || !grad || !m || !v || t < 1) return fail(CHEB_ERR_INVALID, "cheb_mlp_adam: bad arguments");
    const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
    k_adam<<<nb(MLP_NPARAMS, 256), 256, 0, as_stream(stream)>>>(theta, grad, m, v, MLP_NPARAMS, lr, c1, c2);
    return check_launch("k_adam");
}

extern "C" int cheb_mlp_features(const double *moments, int64_t n_rows, double emin, double emax, double N_e,
                                 float *features, void *stream) {
    if (!moments || !features || n_rows < 1) return fail(CHEB_ERR_INVALID, "cheb_mlp_features: bad arguments");
    k_features<<<1, 64, 0, as_stream(stream)>>>(moments, n_rows, emin, emax, N_e, features);
    return check_launch("k_features");
}
