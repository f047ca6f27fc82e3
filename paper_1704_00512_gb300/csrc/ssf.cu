// Segment Storage Format import and export (Sec. "Storage format of the
// sparse matrices"): the nonzeros of the scalar matrix in one array, the
// pattern as segments of consecutive entries, keyg = (c_s, c_e; r_s, r_e) per
// segment (first and last column and row, dense coordinates, 1-based) and keyv
// = the 1-based position in the value array where the segment starts.
//
// Export writes the scalar pattern of a 4x4 block-CSR matrix (every entry of a
// present block) row by row; each maximal run of consecutive block columns of
// a block row gives one segment per scalar row.  Import reads segments that may
// span rows (the entries from (r_s, c_s) to (r_e, c_e) in row-major order): the
// block pattern is every block holding one of their entries plus every
// diagonal block, and the values are scattered into it (zero elsewhere).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "common.cuh"

namespace cheb {

// runs[I] = maximal runs of consecutive block columns in block row I
__global__ void k_ssf_runs(const int64_t *rp, const int32_t *ci, int64_t nbr, int64_t *runs) {
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= nbr) return;
    int64_t n = 0;
    for (int64_t p = rp[I]; p < rp[I + 1]; ++p) n += (p == rp[I] || ci[p] != ci[p - 1] + 1);
    runs[I] = n;
}

// off[i] = sum of v[0..i), off[n] = total (one thread block of 1024)
__global__ void __launch_bounds__(1024) k_ssf_scan(const int64_t *v, int64_t n, int64_t *off) {
    __shared__ int64_t part[1024];
    const int tid = threadIdx.x;
    const int64_t per = (n + 1023) / 1024, b = min(n, (int64_t)tid * per), e = min(n, b + per);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += v[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int64_t run = 0;
        for (int i = 0; i < 1024; ++i) {
            const int64_t t = part[i];
            part[i] = run;
            run += t;
        }
        off[n] = run;
    }
    __syncthreads();
    int64_t run = part[tid];
    for (int64_t i = b; i < e; ++i) {
        off[i] = run;
        run += v[i];
    }
}

// One thread per (block row, scalar row r): its segments, descriptors and values.
__global__ void k_ssf_export(const int64_t *rp, const int32_t *ci, const double *vals, int64_t nbr,
                             const int64_t *runs, const int64_t *run_off, int32_t *keyg, int64_t *keyv,
                             double *out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nbr * BS) return;
    const int64_t I = t / BS;
    const int r = (int)(t % BS);
    const int64_t nb = rp[I + 1] - rp[I];
    int64_t s = BS * run_off[I] + r * runs[I];  // segments: block rows, then scalar rows, then runs
    int64_t v = BS * BS * rp[I] + r * BS * nb;  // values in row-major order of the scalar matrix
    const int32_t row1 = (int32_t)(BS * I + r + 1);
    int64_t p = rp[I];
    while (p < rp[I + 1]) {
        int64_t q = p;
        while (q + 1 < rp[I + 1] && ci[q + 1] == ci[q] + 1) ++q;
        keyg[4 * s] = BS * ci[p] + 1;
        keyg[4 * s + 1] = BS * ci[q] + BS;
        keyg[4 * s + 2] = row1;
        keyg[4 * s + 3] = row1;
        keyv[s] = v + 1;
        for (int64_t b = p; b <= q; ++b)
            for (int c = 0; c < BS; ++c) out[v++] = vals[b * BB + r * BS + c];
        ++s;
        p = q + 1;
    }
}

// One warp per segment: entry j of segment s sits at linear position
// (r_s - 1) n + (c_s - 1) + j of the n x n matrix.
__global__ void k_ssf_import(const int64_t *rp, const int32_t *ci, int64_t n, int64_t nseg, const int32_t *keyg,
                             const int64_t *keyv, const double *vals, int64_t nvals, double *out, int32_t *status) {
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= nseg) return;
    const int64_t cs = keyg[4 * s] - 1, ce = keyg[4 * s + 1] - 1, rs = keyg[4 * s + 2] - 1, re = keyg[4 * s + 3] - 1;
    const int64_t start = rs * n + cs, end = re * n + ce, v0 = keyv[s] - 1;
    if (cs < 0 || ce >= n || rs < 0 || re >= n || end < start || v0 < 0 || v0 + (end - start) >= nvals) {
        if (lane == 0) atomicExch(status, 1);
        return;
    }
    for (int64_t j = lane; j <= end - start; j += 32) {
        const int64_t lin = start + j, r = lin / n, c = lin % n;
        const int64_t b = find_in_row(rp, ci, r / BS, (int32_t)(c / BS));
        if (b < 0) {
            atomicExch(status, 2);
            continue;
        }
        out[b * BB + (r % BS) * BS + (c % BS)] = vals[v0 + j];
    }
}

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_ssf_export_size(const cheb_bsr *A, int64_t *nseg, int64_t *nnz, void *stream) {
    if (!A || !A->row_ptr || !A->col_idx || A->nbr < 1 || !nseg || !nnz)
        return fail(CHEB_ERR_INVALID, "cheb_ssf_export_size: bad arguments");
    cudaStream_t s = as_stream(stream);
    int64_t *buf = nullptr;
    CHEB_CUDA(cudaMallocAsync(&buf, (2 * A->nbr + 1) * sizeof(int64_t), s));
    k_ssf_runs<<<(unsigned)((A->nbr + 255) / 256), 256, 0, s>>>(A->row_ptr, A->col_idx, A->nbr, buf);
    k_ssf_scan<<<1, 1024, 0, s>>>(buf, A->nbr, buf + A->nbr);
    int64_t total = 0;
    const int rc = check_launch("ssf runs", 2);
    if (rc == CHEB_OK) CHEB_CUDA(cudaMemcpyAsync(&total, buf + 2 * A->nbr, 8, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaFreeAsync(buf, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    CHEB_TRY(rc);
    *nseg = BS * total;
    *nnz = BS * BS * A->nnzb;
    return CHEB_OK;
}

extern "C" int cheb_ssf_export(const cheb_bsr *A, int64_t nseg, int32_t *keyg, int64_t *keyv, double *vals,
                               void *stream) {
    if (!A || !A->row_ptr || !A->col_idx || !A->vals || A->dtype != CHEB_F64 || A->nbr < 1 || !keyg || !keyv ||
        !vals)
        return fail(CHEB_ERR_INVALID, "cheb_ssf_export: bad arguments");
    int64_t want = 0, nnz = 0;
    CHEB_TRY(cheb_ssf_export_size(A, &want, &nnz, stream));
    if (nseg != want) return fail(CHEB_ERR_INVALID, "cheb_ssf_export: %lld segments, not %lld", (long long)want,
                                  (long long)nseg);
    cudaStream_t s = as_stream(stream);
    int64_t *buf = nullptr;
    CHEB_CUDA(cudaMallocAsync(&buf, (2 * A->nbr + 1) * sizeof(int64_t), s));
    k_ssf_runs<<<(unsigned)((A->nbr + 255) / 256), 256, 0, s>>>(A->row_ptr, A->col_idx, A->nbr, buf);
    k_ssf_scan<<<1, 1024, 0, s>>>(buf, A->nbr, buf + A->nbr);
    const int64_t nt = A->nbr * BS;
    k_ssf_export<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(A->row_ptr, A->col_idx, (const double *)A->vals,
                                                              A->nbr, buf, buf + A->nbr, keyg, keyv, vals);
    const int rc = check_launch("k_ssf_export", 3);
    CHEB_CUDA(cudaFreeAsync(buf, s));
    return rc;
}

extern "C" int cheb_ssf_import_pattern(int64_t n, int64_t nseg, const int32_t *keyg, int64_t *nnzb,
                                       int64_t *row_ptr, int32_t *col_idx, void *stream) {
    if (n < BS || n % BS || nseg < 0 || (nseg > 0 && !keyg) || !nnzb)
        return fail(CHEB_ERR_INVALID, "cheb_ssf_import_pattern: n must be a positive multiple of 4");
    const int64_t nbr = n / BS;
    std::vector<std::vector<int32_t>> cols(nbr);
    for (int64_t I = 0; I < nbr; ++I) cols[I].push_back((int32_t)I);  // every diagonal block
    for (int64_t s = 0; s < nseg; ++s) {
        const int64_t cs = keyg[4 * s] - 1, ce = keyg[4 * s + 1] - 1, rs = keyg[4 * s + 2] - 1,
                      re = keyg[4 * s + 3] - 1;
        if (cs < 0 || ce >= n || rs < 0 || re >= n || re < rs || (re == rs && ce < cs))
            return fail(CHEB_ERR_INVALID, "cheb_ssf_import_pattern: segment %lld out of range", (long long)s);
        for (int64_t r = rs; r <= re; ++r) {
            const int64_t c0 = r == rs ? cs : 0, c1 = r == re ? ce : n - 1;
            for (int64_t J = c0 / BS; J <= c1 / BS; ++J) cols[r / BS].push_back((int32_t)J);
        }
    }
    int64_t total = 0;
    for (auto &v : cols) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        total += (int64_t)v.size();
    }
    *nnzb = total;
    if (!row_ptr && !col_idx) return CHEB_OK;
    if (!row_ptr || !col_idx) return fail(CHEB_ERR_INVALID, "cheb_ssf_import_pattern: give both arrays or neither");
    std::vector<int64_t> rp(nbr + 1, 0);
    std::vector<int32_t> ci;
    ci.reserve(total);
    for (int64_t I = 0; I < nbr; ++I) {
        ci.insert(ci.end(), cols[I].begin(), cols[I].end());
        rp[I + 1] = (int64_t)ci.size();
    }
    cudaStream_t s = as_stream(stream);
    CHEB_CUDA(cudaMemcpyAsync(row_ptr, rp.data(), (nbr + 1) * 8, cudaMemcpyHostToDevice, s));
    CHEB_CUDA(cudaMemcpyAsync(col_idx, ci.data(), total * 4, cudaMemcpyHostToDevice, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    return CHEB_OK;
}

extern "C" int cheb_ssf_import_values(const cheb_bsr *A, int64_t nseg, const int32_t *keyg, const int64_t *keyv,
                                      const double *vals, int64_t nvals, void *stream) {
    if (!A || !A->row_ptr || !A->col_idx || !A->vals || A->dtype != CHEB_F64 || nseg < 0 ||
        (nseg > 0 && (!keyg || !keyv || !vals)))
        return fail(CHEB_ERR_INVALID, "cheb_ssf_import_values: bad arguments");
    cudaStream_t s = as_stream(stream);
    int32_t *status = nullptr;
    CHEB_CUDA(cudaMallocAsync(&status, 4, s));
    CHEB_CUDA(cudaMemsetAsync(status, 0, 4, s));
    CHEB_CUDA(cudaMemsetAsync(A->vals, 0, A->nnzb * BB * sizeof(double), s));
    if (nseg > 0) {
        const int64_t threads = nseg * 32;
        k_ssf_import<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(A->row_ptr, A->col_idx, A->nbr * BS, nseg,
                                                                      keyg, keyv, vals, nvals, (double *)A->vals,
                                                                      status);
    }
    int rc = check_launch("k_ssf_import");
    int32_t h = 0;
    if (rc == CHEB_OK) CHEB_CUDA(cudaMemcpyAsync(&h, status, 4, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaFreeAsync(status, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    CHEB_TRY(rc);
    if (h == 1) return fail(CHEB_ERR_INVALID, "cheb_ssf_import_values: a segment or its values are out of range");
    if (h == 2) return fail(CHEB_ERR_INVALID, "cheb_ssf_import_values: an entry lies outside the block pattern");
    return CHEB_OK;
}
