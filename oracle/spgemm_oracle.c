/*
 * CPU oracle for the sparse x sparse product C = A * B on CSR matrices.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file; the CUDA library never does, and this file
 * includes nothing from it.  It is deliberately plain and slow: one thread,
 * 64-bit indices (as in the paper's Section III), no blocking or reordering.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so every
 * product a*b is rounded on its own before it is added).
 *
 * oracle_spgemm  -- the row-major algorithm of Section IV-A (Gustavson): for
 *                   every row r of A and every a_rc in it, every b_cx of row c
 *                   of B is multiplied by a_rc and added into a dense
 *                   temporary vector at position x, which starts at zero.
 *                   The row is stored with the "Sort" strategy of Section
 *                   IV-B: the touched positions are kept in an index list,
 *                   sorted ascending (std::sort there, qsort here) and
 *                   appended in that order.  A char flag vector (the lookup
 *                   vector of the "Brute Force"-char variant) marks touched
 *                   positions, so an entry whose products cancel to 0.0 is
 *                   still stored: the structure of C is the union of the
 *                   structures of the scaled rows of B.
 *                   Capacity for C is the number of multiplications, the
 *                   never-underestimating nnz estimate of Section IV-B.
 * oracle_flops   -- the multiplication count of Section III:
 *                   sum over k of (nnz in column k of A) * (nnz in row k of B).
 * oracle_grad    -- gradients of loss = sum_{(i,x) in C} W_ix C_ix:
 *                   dA_ij = sum_x B_jx W_ix, dB_jx = sum_i A_ij W_ix.
 * oracle_transpose -- CSR -> CSC by counting sort (the storage-order
 *                   conversion of Section IV-A).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

/* Multiplication count per Section III (column counts of A times row counts of B). */
int64_t oracle_flops(int64_t m, int64_t k, const int64_t* A_rp, const int64_t* A_col,
                     const int64_t* B_rp) {
    int64_t* colcnt = (int64_t*)calloc((size_t)(k > 0 ? k : 1), sizeof(int64_t));
    if (!colcnt) return -1;
    for (int64_t p = 0; p < A_rp[m]; ++p) colcnt[A_col[p]] += 1;
    int64_t mults = 0;
    for (int64_t c = 0; c < k; ++c) mults += colcnt[c] * (B_rp[c + 1] - B_rp[c]);
    free(colcnt);
    return mults;
}

/*
 * C = A * B.  A is m x k, B is k x n.  Outputs:
 *   C_rp[m+1], C_col[cap], C_val[cap], C_abs[cap] (sum of |a*b| per entry),
 *   C_cnt[cap] (number of products in each entry), u[m] (multiplications of each row).
 * Returns nnz(C), or -1 if cap is too small, -2 on allocation failure.
 */
int64_t oracle_spgemm(int64_t m, int64_t k, int64_t n,
                      const int64_t* A_rp, const int64_t* A_col, const double* A_val,
                      const int64_t* B_rp, const int64_t* B_col, const double* B_val,
                      int64_t cap, int64_t* C_rp, int64_t* C_col, double* C_val,
                      double* C_abs, int64_t* C_cnt, int64_t* u) {
    (void)k;
    double* temp = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double* tabs = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int64_t* tcnt = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    char* flag = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t* list = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!temp || !tabs || !tcnt || !flag || !list) {
        free(temp); free(tabs); free(tcnt); free(flag); free(list);
        return -2;
    }
    int64_t nnz = 0;
    C_rp[0] = 0;
    for (int64_t r = 0; r < m; ++r) {
        int64_t len = 0, mults = 0;
        for (int64_t p = A_rp[r]; p < A_rp[r + 1]; ++p) {
            int64_t c = A_col[p];
            double a = A_val[p];
            for (int64_t q = B_rp[c]; q < B_rp[c + 1]; ++q) {
                int64_t x = B_col[q];
                double prod = a * B_val[q];
                if (!flag[x]) {
                    flag[x] = 1;
                    list[len++] = x;
                }
                temp[x] += prod;
                tabs[x] += fabs(prod);
                tcnt[x] += 1;
                ++mults;
            }
        }
        u[r] = mults;
        qsort(list, (size_t)len, sizeof(int64_t), cmp_i64);
        if (nnz + len > cap) {
            free(temp); free(tabs); free(tcnt); free(flag); free(list);
            return -1;
        }
        for (int64_t t = 0; t < len; ++t) {
            int64_t x = list[t];
            C_col[nnz] = x;
            C_val[nnz] = temp[x];
            C_abs[nnz] = tabs[x];
            C_cnt[nnz] = tcnt[x];
            ++nnz;
            temp[x] = 0.0;
            tabs[x] = 0.0;
            tcnt[x] = 0;
            flag[x] = 0;
        }
        C_rp[r + 1] = nnz;
    }
    free(temp); free(tabs); free(tcnt); free(flag); free(list);
    return nnz;
}

/*
 * Gradients of loss = sum over C's entries of W * C, with W given on C's
 * pattern (C_rp, C_col, W aligned with C).  dA is aligned with A's entries,
 * dB with B's entries.  Row i of W is scattered into a dense vector first.
 * Returns 0, or -2 on allocation failure, -3 if a product lands outside C.
 */
int oracle_grad(int64_t m, int64_t k, int64_t n,
                const int64_t* A_rp, const int64_t* A_col, const double* A_val,
                const int64_t* B_rp, const int64_t* B_col, const double* B_val,
                const int64_t* C_rp, const int64_t* C_col, const double* W,
                double* dA, double* dB) {
    (void)k;
    double* wrow = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    char* have = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!wrow || !have) { free(wrow); free(have); return -2; }
    for (int64_t q = 0; q < B_rp[k]; ++q) dB[q] = 0.0;
    int rc = 0;
    for (int64_t i = 0; i < m && rc == 0; ++i) {
        for (int64_t t = C_rp[i]; t < C_rp[i + 1]; ++t) { wrow[C_col[t]] = W[t]; have[C_col[t]] = 1; }
        for (int64_t p = A_rp[i]; p < A_rp[i + 1]; ++p) {
            int64_t j = A_col[p];
            double g = 0.0;
            for (int64_t q = B_rp[j]; q < B_rp[j + 1]; ++q) {
                int64_t x = B_col[q];
                if (!have[x]) { rc = -3; break; }
                double t1 = B_val[q] * wrow[x];
                g += t1;
                double t2 = A_val[p] * wrow[x];
                dB[q] += t2;
            }
            dA[p] = g;
        }
        for (int64_t t = C_rp[i]; t < C_rp[i + 1]; ++t) { wrow[C_col[t]] = 0.0; have[C_col[t]] = 0; }
    }
    free(wrow); free(have);
    return rc;
}

/* CSR (m x n) -> CSC: T_cp[n+1], T_row[nnz], T_val[nnz]; entries of a column keep row order. */
int oracle_transpose(int64_t m, int64_t n, const int64_t* rp, const int64_t* col, const double* val,
                     int64_t* T_cp, int64_t* T_row, double* T_val) {
    for (int64_t c = 0; c <= n; ++c) T_cp[c] = 0;
    for (int64_t p = 0; p < rp[m]; ++p) T_cp[col[p] + 1] += 1;
    for (int64_t c = 0; c < n; ++c) T_cp[c + 1] += T_cp[c];
    int64_t* next = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!next) return -2;
    for (int64_t c = 0; c < n; ++c) next[c] = T_cp[c];
    for (int64_t r = 0; r < m; ++r)
        for (int64_t p = rp[r]; p < rp[r + 1]; ++p) {
            int64_t d = next[col[p]]++;
            T_row[d] = r;
            T_val[d] = val[p];
        }
    free(next);
    return 0;
}
