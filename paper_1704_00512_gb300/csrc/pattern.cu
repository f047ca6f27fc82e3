// Distance-cutoff block patterns (Sec. "Sparsity and truncation": a fixed
// pattern, with a larger "buffer" pattern for the products' output).
//
// One warp per block row I sweeps all atoms J in ascending order (so the column
// list comes out sorted with no sort pass).  Atom tiles are staged in shared
// memory.  A float32 pre-test with a 0.01 bohr pad discards far pairs; every
// survivor is decided by the exact float64 test with explicit round-to-nearest
// operations (no fused multiply-add), so the decision is the same one a plain
// CPU loop makes: dx = x_J - x_I wrapped once by +-L when |dx| > L/2, then
// (dx*dx + dy*dy) + dz*dz <= r*r.
#include "common.cuh"

namespace cheb {

constexpr int PAT_WARPS = 8;
constexpr int PAT_TILE = 256;

__global__ void __launch_bounds__(PAT_WARPS * 32)
k_pattern(const double *__restrict__ xyz, int64_t n, double L, double r, float rpad2,
          int64_t *__restrict__ row_ptr, int32_t *__restrict__ col_idx) {
    __shared__ double sx[PAT_TILE * 3];
    __shared__ float sf[PAT_TILE * 3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t I = (int64_t)blockIdx.x * PAT_WARPS + warp;
    const bool valid = I < n;
    double xi[3] = {0.0, 0.0, 0.0};
    float fi[3] = {0.f, 0.f, 0.f};
    if (valid) {
        for (int a = 0; a < 3; ++a) {
            xi[a] = xyz[I * 3 + a];
            fi[a] = (float)xi[a];
        }
    }
    const double half = 0.5 * L;
    const double r2 = __dmul_rn(r, r);
    const float Lf = (float)L, halff = (float)half;
    const unsigned lt = (1u << lane) - 1u;
    int64_t cnt = 0;
    const int64_t base = (col_idx && valid) ? row_ptr[I] : 0;
    for (int64_t t0 = 0; t0 < n; t0 += PAT_TILE) {
        __syncthreads();
        const int64_t tn = min((int64_t)PAT_TILE, n - t0);
        for (int i = threadIdx.x; i < PAT_TILE * 3; i += PAT_WARPS * 32) {
            double v = i < tn * 3 ? xyz[t0 * 3 + i] : 0.0;
            sx[i] = v;
            sf[i] = (float)v;
        }
        __syncthreads();
        if (!valid) continue;
        for (int j0 = 0; j0 < tn; j0 += 32) {
            const int j = j0 + lane;
            bool pass = false;
            if (j < tn) {
                float d2f = 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float d = sf[j * 3 + a] - fi[a];
                    if (d > halff) d -= Lf;
                    else if (d < -halff) d += Lf;
                    d2f += d * d;
                }
                if (d2f <= rpad2) {
                    double d[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        double t = __dsub_rn(sx[j * 3 + a], xi[a]);
                        if (t > half) t = __dsub_rn(t, L);
                        else if (t < -half) t = __dadd_rn(t, L);
                        d[a] = t;
                    }
                    double dd = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                                          __dmul_rn(d[2], d[2]));
                    pass = dd <= r2;
                }
                pass = pass || (t0 + j == I);
            }
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            if (col_idx && pass) col_idx[base + cnt + __popc(m & lt)] = (int32_t)(t0 + j);
            cnt += __popc(m);
        }
    }
    if (valid && !col_idx && lane == 0) row_ptr[I + 1] = cnt;
}

// In-place inclusive scan of row_ptr[1..n] (counts) with row_ptr[0] = 0; one block.
__global__ void __launch_bounds__(1024) k_scan_rows(int64_t *row_ptr, int64_t n) {
    __shared__ int64_t tot[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t b = 1 + t * chunk, e = min(n + 1, b + chunk);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += row_ptr[i];
    tot[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t v = t >= o ? tot[t - o] : 0;
        __syncthreads();
        tot[t] += v;
        __syncthreads();
    }
    int64_t run = t > 0 ? tot[t - 1] : 0;
    for (int64_t i = b; i < e; ++i) {
        run += row_ptr[i];
        row_ptr[i] = run;
    }
    if (t == 0) row_ptr[0] = 0;
}

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_pattern_build(const double *xyz, int64_t n_atoms, double box_L, double r_cut,
                                  int64_t *row_ptr, int32_t *col_idx, int64_t *nnzb, void *stream) {
    if (!xyz || !row_ptr || n_atoms < 1 || !(box_L > 0) || !(r_cut >= 0))
        return fail(CHEB_ERR_INVALID, "cheb_pattern_build: bad arguments");
    if (n_atoms >= (int64_t)INT32_MAX) return fail(CHEB_ERR_INVALID, "cheb_pattern_build: too many atoms");
    cudaStream_t s = as_stream(stream);
    const float rp = (float)(r_cut + 0.01);
    const unsigned grid = (unsigned)((n_atoms + PAT_WARPS - 1) / PAT_WARPS);
    k_pattern<<<grid, PAT_WARPS * 32, 0, s>>>(xyz, n_atoms, box_L, r_cut, rp * rp, row_ptr, col_idx);
    CHEB_TRY(check_launch("k_pattern"));
    if (col_idx) return CHEB_OK;
    k_scan_rows<<<1, 1024, 0, s>>>(row_ptr, n_atoms);
    CHEB_TRY(check_launch("k_scan_rows"));
    if (nnzb) {
        CHEB_CUDA(cudaMemcpyAsync(nnzb, row_ptr + n_atoms, 8, cudaMemcpyDeviceToHost, s));
        CHEB_CUDA(cudaStreamSynchronize(s));
    }
    return CHEB_OK;
}
