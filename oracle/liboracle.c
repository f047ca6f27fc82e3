/*
 * FP64 CPU oracle kernels -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct loops used by oracle/ref.py.  Nothing in the
 * product path links or calls this file; it shares no code with the CUDA
 * library.  Compiled with -ffp-contract=off so every product and sum rounds
 * separately, in the order written.
 *
 * Matrices are 4x4 block-CSR: row_ptr int64[nbr+1], col_idx int32 (sorted
 * ascending within a row), vals double[nnzb][4][4] row-major.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BS 4

/* Index of block (K, J) in row K of a block-CSR pattern, or -1.  Plain binary
 * search over the sorted column list. */
static int64_t find_block(const int64_t *rp, const int32_t *ci, int64_t K, int32_t J)
{
    int64_t lo = rp[K], hi = rp[K + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (ci[mid] == J) return mid;
        if (ci[mid] < J) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/*
 * Masked block product C = P_C(L R): for every block (I, J) of the output
 * pattern P_C,  C_IJ = sum over K with (I,K) in P_L and (K,J) in P_R of
 * L_IK R_KJ.  Entries of L R outside P_C are dropped (the truncation to a
 * fixed sparsity pattern, Sec. "Sparsity and truncation").  If colmask is
 * non-NULL only output blocks with colmask[J] != 0 are computed (others are
 * left untouched): by Eq. 3 a column of the recursion depends only on the same
 * column of the previous terms, so column subsets can be advanced alone.
 */
void oracle_masked_product(int64_t nbr,
                           const int64_t *Lrp, const int32_t *Lci, const double *Lv,
                           const int64_t *Rrp, const int32_t *Rci, const double *Rv,
                           const int64_t *Crp, const int32_t *Cci, double *Cv,
                           const unsigned char *colmask)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t I = 0; I < nbr; ++I) {
        for (int64_t c = Crp[I]; c < Crp[I + 1]; ++c) {
            int32_t J = Cci[c];
            if (colmask && !colmask[J]) continue;
            double acc[BS * BS];
            memset(acc, 0, sizeof(acc));
            for (int64_t a = Lrp[I]; a < Lrp[I + 1]; ++a) {
                int64_t K = Lci[a];
                int64_t b = find_block(Rrp, Rci, K, J);
                if (b < 0) continue;
                const double *l = Lv + a * BS * BS;
                const double *r = Rv + b * BS * BS;
                for (int i = 0; i < BS; ++i)
                    for (int j = 0; j < BS; ++j) {
                        double s = acc[i * BS + j];
                        for (int m = 0; m < BS; ++m) s += l[i * BS + m] * r[m * BS + j];
                        acc[i * BS + j] = s;
                    }
            }
            memcpy(Cv + c * BS * BS, acc, sizeof(acc));
        }
    }
}

/* y = A x for a 4x4 block-CSR A (x, y of length 4*nbr). */
void oracle_spmv(int64_t nbr, const int64_t *rp, const int32_t *ci, const double *v,
                 const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t I = 0; I < nbr; ++I) {
        double acc[BS] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t a = rp[I]; a < rp[I + 1]; ++a) {
            const double *blk = v + a * BS * BS;
            const double *xx = x + (int64_t)ci[a] * BS;
            for (int i = 0; i < BS; ++i)
                for (int m = 0; m < BS; ++m) acc[i] += blk[i * BS + m] * xx[m];
        }
        for (int i = 0; i < BS; ++i) y[I * BS + i] = acc[i];
    }
}

/*
 * Brute-force block pattern {(I, J): minimum-image distance <= r}: every pair
 * is tested, O(n^2).  dx = x_J - x_I wrapped once by +/-L, then
 * d2 = (dx*dx + dy*dy) + dz*dz compared with r*r (inclusive).  Pass 1
 * (col_idx == NULL) writes the per-row counts into row_ptr[1..n]; pass 2
 * fills col_idx using the row_ptr offsets.  Columns come out ascending.
 */
void oracle_pattern(int64_t n, const double *xyz, double L, double r,
                    int64_t *row_ptr, int32_t *col_idx)
{
    const double r2 = r * r, half = 0.5 * L;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t I = 0; I < n; ++I) {
        int64_t cnt = 0;
        int64_t base = col_idx ? row_ptr[I] : 0;
        for (int64_t J = 0; J < n; ++J) {
            double d[3];
            for (int ax = 0; ax < 3; ++ax) {
                double t = xyz[J * 3 + ax] - xyz[I * 3 + ax];
                if (t > half) t = t - L;
                else if (t < -half) t = t + L;
                d[ax] = t;
            }
            double dd = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (dd <= r2 || I == J) {
                if (col_idx) col_idx[base + cnt] = (int32_t)J;
                ++cnt;
            }
        }
        if (!col_idx) row_ptr[I + 1] = cnt;
    }
}

/*
 * Column-sampled Chebyshev expansion (Eq. 1 + Eq. 3).  Column J of T_{k+1}
 * needs only column J of T_k and T_{k-1} (Sec. "Expansion in Chebyshev
 * polynomials"), so a few block columns can be advanced alone, at the cost of
 * their own rows only.  For every sampled column J = cols[c]: its rows are
 * the blocks (I, J) of P_out, i.e. the column list of row J (P_out is
 * symmetric), in ascending I; T_0 = identity block at I = J, T_1 = Mt's block
 * (I, J) (zero when Mt has none), T_{k+1}(I,J) = 2 sum_K Mt(I,K) T_k(K,J) -
 * T_{k-1}(I,J) over K with (I,K) in Mt and (K,J) in P_out; acc_f(:,J) =
 * coeffs[f][0]/2 T_0 + sum_{k>=1} coeffs[f][k] T_k.
 * out: double[nf][total rows over the sampled columns][16], the columns one
 * after the other, each in its row order.  The operator's entries of each
 * row that fall in the column's row set are found once per column (binary
 * search); the recursion then runs on that restricted list.
 */
void oracle_column_expand(int64_t nbr, const int64_t *Lrp, const int32_t *Lci, const double *Lv,
                          const int64_t *Prp, const int32_t *Pci, int64_t ncols, const int32_t *cols,
                          int64_t nterms, int64_t nf, const double *coeffs, double *out)
{
    int64_t *base = (int64_t *)malloc((size_t)(ncols + 1) * sizeof(int64_t));
    base[0] = 0;
    for (int64_t c = 0; c < ncols; ++c) base[c + 1] = base[c] + (Prp[cols[c] + 1] - Prp[cols[c]]);
    const int64_t total = base[ncols];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < ncols; ++c) {
        const int32_t J = cols[c];
        const int32_t *rows = Pci + Prp[J];
        const int64_t n = Prp[J + 1] - Prp[J];
        /* restricted operator: for each local row i, (operator block a, local index of K) */
        int64_t *ptr = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
        int64_t cap = 0;
        for (int64_t i = 0; i < n; ++i) cap += Lrp[rows[i] + 1] - Lrp[rows[i]];
        int64_t *ea = (int64_t *)malloc((size_t)(cap + 1) * sizeof(int64_t));
        int64_t *ek = (int64_t *)malloc((size_t)(cap + 1) * sizeof(int64_t));
        int64_t m = 0;
        for (int64_t i = 0; i < n; ++i) {
            ptr[i] = m;
            for (int64_t a = Lrp[rows[i]]; a < Lrp[rows[i] + 1]; ++a) {
                int64_t lo = 0, hi = n - 1, kk = -1;
                while (lo <= hi) {
                    int64_t mid = lo + (hi - lo) / 2;
                    if (rows[mid] == Lci[a]) { kk = mid; break; }
                    if (rows[mid] < Lci[a]) lo = mid + 1; else hi = mid - 1;
                }
                if (kk >= 0) { ea[m] = a; ek[m] = kk; ++m; }
            }
        }
        ptr[n] = m;
        double *Tm = (double *)calloc((size_t)n * 16, sizeof(double));
        double *T = (double *)calloc((size_t)n * 16, sizeof(double));
        double *Tn = (double *)calloc((size_t)n * 16, sizeof(double));
        for (int64_t i = 0; i < n; ++i) {
            if (rows[i] == J)
                for (int d = 0; d < BS; ++d) Tm[i * 16 + d * BS + d] = 1.0;
            const int64_t a = find_block(Lrp, Lci, rows[i], J);
            if (a >= 0) memcpy(T + i * 16, Lv + a * 16, 16 * sizeof(double));
        }
        for (int64_t f = 0; f < nf; ++f) {
            double *acc = out + (f * total + base[c]) * 16;
            const double c0 = coeffs[f * nterms + 0], c1 = nterms > 1 ? coeffs[f * nterms + 1] : 0.0;
            for (int64_t e = 0; e < n * 16; ++e) acc[e] = 0.5 * c0 * Tm[e] + (nterms > 1 ? c1 * T[e] : 0.0);
        }
        for (int64_t k = 1; k + 1 < nterms; ++k) {
            for (int64_t i = 0; i < n; ++i) {
                double s[16];
                memset(s, 0, sizeof(s));
                for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
                    const double *l = Lv + ea[e] * 16;
                    const double *r = T + ek[e] * 16;
                    for (int ii = 0; ii < BS; ++ii)
                        for (int jj = 0; jj < BS; ++jj) {
                            double v = s[ii * BS + jj];
                            for (int mm = 0; mm < BS; ++mm) v += l[ii * BS + mm] * r[mm * BS + jj];
                            s[ii * BS + jj] = v;
                        }
                }
                for (int e = 0; e < 16; ++e) Tn[i * 16 + e] = 2.0 * s[e] - Tm[i * 16 + e];
            }
            for (int64_t f = 0; f < nf; ++f) {
                double *acc = out + (f * total + base[c]) * 16;
                const double ck = coeffs[f * nterms + k + 1];
                for (int64_t e = 0; e < n * 16; ++e) acc[e] += ck * Tn[e];
            }
            double *tmp = Tm;
            Tm = T;
            T = Tn;
            Tn = tmp;
        }
        free(Tm); free(T); free(Tn); free(ptr); free(ea); free(ek);
    }
    free(base);
}
