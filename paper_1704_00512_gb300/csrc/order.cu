// Locality order of the atoms (not in the paper): the column kernel takes its
// panels from consecutive block columns, and panels of atoms that lie close
// together have small unions of rows, so fewer operator entries per step.  The
// order is that of a 3-D Hilbert curve through the periodic box (J. Skilling,
// "Programming the Hilbert curve", AIP Conf. Proc. 707, 381 (2004)): unlike
// Morton order it has no long jumps between consecutive cells.  A system is
// relabelled by building its patterns from the reordered atoms and moving
// values between the two labellings with a position map.
#include <cstdint>

#include "common.cuh"

namespace cheb {

constexpr int HILBERT_BITS = 10;  // cells per axis: 1024

// Hilbert index of integer cell coordinates (x, y, z) < 2^HILBERT_BITS:
// Skilling's transpose form (inverse undo, then Gray encoding), then the bits
// interleaved from the most significant one, axis 0 first.
__device__ __forceinline__ uint64_t hilbert_key(uint32_t x0, uint32_t x1, uint32_t x2) {
    uint32_t X[3] = {x0, x1, x2};
    const uint32_t M = 1u << (HILBERT_BITS - 1);
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
#pragma unroll
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    uint64_t key = 0;
    for (int b = HILBERT_BITS - 1; b >= 0; --b)
#pragma unroll
        for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

// Sort words (Hilbert key << 32 | atom) of n atoms, padded with ~0 to N = 2^m.
__global__ void k_order_keys(const double *xyz, int64_t n, int64_t N, double box, uint64_t *v) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (i >= n) {
        v[i] = ~0ull;
        return;
    }
    uint32_t q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double u = xyz[3 * i + d] / box;
        u -= floor(u);  // periodic: the cell of the image in [0, box)
        int64_t c = (int64_t)(u * (double)(1 << HILBERT_BITS));
        c = c < 0 ? 0 : (c > (1 << HILBERT_BITS) - 1 ? (1 << HILBERT_BITS) - 1 : c);
        q[d] = (uint32_t)c;
    }
    v[i] = (hilbert_key(q[0], q[1], q[2]) << 32) | (uint64_t)i;
}

// One compare-exchange stage (k, j) of Batcher's bitonic sort, ascending.
__global__ void k_bitonic(uint64_t *v, int64_t N, int64_t j, int64_t k) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t l = i ^ j;
    if (l <= i) return;
    const uint64_t a = v[i], b = v[l];
    const bool up = (i & k) == 0;
    if (up ? a > b : a < b) {
        v[i] = b;
        v[l] = a;
    }
}

__global__ void k_order_out(const uint64_t *v, int64_t n, int64_t *perm) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) perm[i] = (int64_t)(v[i] & 0xffffffffull);
}

static int64_t pow2_at_least(int64_t n) {
    int64_t N = 1;
    while (N < n) N <<= 1;
    return N;
}

}  // namespace cheb

using namespace cheb;

extern "C" size_t cheb_locality_order_ws(int64_t n_atoms) {
    return n_atoms < 1 ? 0 : (size_t)pow2_at_least(n_atoms) * sizeof(uint64_t);
}

extern "C" int cheb_locality_order(const double *xyz, int64_t n_atoms, double box, int64_t *perm, void *ws,
                                   size_t ws_bytes, void *stream) {
    if (!xyz || !perm || n_atoms < 1 || n_atoms > INT32_MAX || !(box > 0))
        return fail(CHEB_ERR_INVALID, "cheb_locality_order: bad arguments");
    const int64_t N = pow2_at_least(n_atoms);
    if (!ws || ws_bytes < (size_t)N * sizeof(uint64_t))
        return fail(CHEB_ERR_NOSPACE, "cheb_locality_order: workspace %zu < %zu", ws_bytes,
                    (size_t)N * sizeof(uint64_t));
    uint64_t *v = static_cast<uint64_t *>(ws);
    const cudaStream_t s = as_stream(stream);
    const unsigned g = (unsigned)((N + 255) / 256);
    k_order_keys<<<g, 256, 0, s>>>(xyz, n_atoms, N, box, v);
    CHEB_TRY(check_launch("k_order_keys"));
    int launches = 0;
    for (int64_t k = 2; k <= N; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            k_bitonic<<<g, 256, 0, s>>>(v, N, j, k);
            ++launches;
        }
    if (launches) CHEB_TRY(check_launch("k_bitonic", launches));
    k_order_out<<<(unsigned)((n_atoms + 255) / 256), 256, 0, s>>>(v, n_atoms, perm);
    return check_launch("k_order_out");
}

namespace cheb {

// map[p'] = position in the old labelling's pattern of block p' = (I', J') of
// the new one, i.e. of (perm[I'], perm[J']); -1 (and *bad set) if absent.
__global__ void k_position_map(const int64_t *rp_new, const int32_t *ci_new, int64_t nbr, int64_t nnz_new,
                               const int64_t *rp_old, const int32_t *ci_old, const int64_t *perm, int64_t *map,
                               int32_t *bad) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nnz_new) return;
    const int64_t I = perm[row_of(rp_new, nbr, p)];
    const int64_t J = perm[ci_new[p]];
    if (I < 0 || I >= nbr || J < 0 || J >= nbr) {  // not a permutation of the rows
        map[p] = -1;
        atomicExch(bad, 1);
        return;
    }
    const int64_t q = find_in_row(rp_old, ci_old, I, (int32_t)J);
    map[p] = q;
    if (q < 0) atomicExch(bad, 1);
}

// Indices outside [0, rows of the other side) are skipped (gather writes 0).
__global__ void k_gather_rows(const double *src, int64_t n_src, const int64_t *map, int64_t n, int32_t w,
                              double *dst) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * w) return;
    const int64_t i = e / w, c = e % w, m = map[i];
    dst[e] = (m >= 0 && m < n_src) ? src[m * w + c] : 0.0;
}

__global__ void k_scatter_rows(const double *src, const int64_t *map, int64_t n, int32_t w, double *dst,
                               int64_t n_dst) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * w) return;
    const int64_t i = e / w, c = e % w, m = map[i];
    if (m >= 0 && m < n_dst) dst[m * w + c] = src[e];
}

}  // namespace cheb

extern "C" int cheb_position_map(const cheb_bsr *P_new, const cheb_bsr *P_old, const int64_t *perm, int64_t *map,
                                 void *ws, size_t ws_bytes, void *stream) {
    if (!P_new || !P_old || !perm || !map || P_new->nbr < 1 || P_new->nbr != P_old->nbr ||
        P_new->nnzb != P_old->nnzb || !P_new->row_ptr || !P_old->row_ptr ||
        (P_new->nnzb > 0 && (!P_new->col_idx || !P_old->col_idx)))
        return fail(CHEB_ERR_INVALID, "cheb_position_map: bad arguments");
    if (!ws || ws_bytes < 4) return fail(CHEB_ERR_NOSPACE, "cheb_position_map: workspace");
    int32_t *bad = static_cast<int32_t *>(ws);
    const cudaStream_t s = as_stream(stream);
    CHEB_CUDA(cudaMemsetAsync(bad, 0, 4, s));
    if (P_new->nnzb > 0) {
        k_position_map<<<(unsigned)((P_new->nnzb + 255) / 256), 256, 0, s>>>(
            P_new->row_ptr, P_new->col_idx, P_new->nbr, P_new->nnzb, P_old->row_ptr, P_old->col_idx, perm, map, bad);
        CHEB_TRY(check_launch("k_position_map"));
    }
    int32_t h = 0;
    CHEB_CUDA(cudaMemcpyAsync(&h, bad, 4, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    if (h) return fail(CHEB_ERR_INVALID, "cheb_position_map: a block of the new pattern is not in the old one");
    return CHEB_OK;
}

extern "C" int cheb_gather_rows(const double *src, int64_t n_src, const int64_t *map, int64_t n, int32_t width,
                                double *dst, void *stream) {
    if (n < 0 || n_src < 0 || width < 1 || (n > 0 && (!src || !map || !dst)) || src == dst)
        return fail(CHEB_ERR_INVALID, "cheb_gather_rows: bad arguments");
    if (n == 0) return CHEB_OK;
    k_gather_rows<<<(unsigned)((n * width + 255) / 256), 256, 0, as_stream(stream)>>>(src, n_src, map, n, width,
                                                                                     dst);
    return check_launch("k_gather_rows");
}

extern "C" int cheb_scatter_rows(const double *src, const int64_t *map, int64_t n, int32_t width, double *dst,
                                 int64_t n_dst, void *stream) {
    if (n < 0 || n_dst < 0 || width < 1 || (n > 0 && (!src || !map || !dst)) || src == dst)
        return fail(CHEB_ERR_INVALID, "cheb_scatter_rows: bad arguments");
    if (n == 0) return CHEB_OK;
    k_scatter_rows<<<(unsigned)((n * width + 255) / 256), 256, 0, as_stream(stream)>>>(src, map, n, width, dst,
                                                                                      n_dst);
    return check_launch("k_scatter_rows");
}
