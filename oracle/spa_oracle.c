/*
 * CPU oracle for the sparse product C = A.B and for the sum of k-slice
 * partial products.  TEST INFRASTRUCTURE ONLY: tests, the smoke check and the
 * benchmark's CPU-baseline leg may call it; the library never does.
 *
 * What it computes (the plain definition, no blocking, no reordering):
 *
 *   Structural pattern  P(C) = {(i,j) : exists k, (i,k) in P(A), (k,j) in P(B)}
 *   Value               C(i,j) = (+)_{k ascending} A(i,k) (x) B(k,j)
 *
 * over the semiring given by `vtype`:
 *   ORACLE_F64   (+,x) on IEEE binary64, every product rounded, then added to
 *                the running sum (compiled with -ffp-contract=off: no FMA);
 *   ORACLE_I64   (+,x) on int64 with two's-complement wraparound;
 *   ORACLE_BOOL  (or,and) -- pattern only, no values.
 *
 * The method is Gustavson's (Alg. 1, written column-wise in the paper; here
 * row-wise over CSR, the same algorithm on the transposed problem) with a
 * dense sparse accumulator (SPA, Sec. 3 "Background and Related Work"): one
 * value array of length n plus a stamp array that marks which columns the
 * current row already touched.  Each output row is emitted with its columns
 * sorted ascending (the paper keeps columns sorted, Sec. 5.2).
 *
 * Explicit zeros and cancellations stay in the pattern: the pattern is purely
 * structural (the paper counts explicit zeros as nonzeros, Sec. 5).
 *
 * oracle_sum_*: entrywise sum C = (+)_{s ascending} C_s of c matrices of the
 * same shape -- the result the paper's multiway merge with duplicate reduction
 * produces (Sec. 4.3); here written as the plain definition with a SPA, not
 * as a heap merge.
 *
 * Rows are independent, so an OpenMP loop over rows (per-thread SPA) changes
 * nothing in the result.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORACLE_F64 = 0, ORACLE_I64 = 1, ORACLE_BOOL = 2 };

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

static int threads_or_default(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_num_threads(int nthreads) { return threads_or_default(nthreads); }

/* flops(A,B) per row: the number of scalar multiplications,
 * flops_i = sum_{k in A(i,:)} nnz(B(k,:))  (Sec. 2 "Notation"). */
int64_t oracle_row_flops(int64_t m, const int64_t* rpA, const int64_t* ciA,
                         const int64_t* rpB, int64_t* flops) {
    int64_t total = 0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t f = 0;
        for (int64_t p = rpA[i]; p < rpA[i + 1]; ++p) {
            int64_t k = ciA[p];
            f += rpB[k + 1] - rpB[k];
        }
        flops[i] = f;
        total += f;
    }
    return total;
}

/* Row counts of C: |union over k in A(i,:) of cols(B(k,:))|.  Returns nnz(C)
 * or -1 when out of memory. */
int64_t oracle_spgemm_count(int64_t m, int64_t n, const int64_t* rpA, const int64_t* ciA,
                            const int64_t* rpB, const int64_t* ciB, int64_t* rowcnt,
                            int nthreads) {
    int nt = threads_or_default(nthreads);
    int failed = 0;
    int64_t total = 0;
#pragma omp parallel num_threads(nt) reduction(+ : total)
    {
        int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!stamp) {
#pragma omp atomic write
            failed = 1;
        } else {
            for (int64_t j = 0; j < n; ++j) stamp[j] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < m; ++i) {
                int64_t cnt = 0;
                for (int64_t p = rpA[i]; p < rpA[i + 1]; ++p) {
                    int64_t k = ciA[p];
                    for (int64_t q = rpB[k]; q < rpB[k + 1]; ++q) {
                        int64_t j = ciB[q];
                        if (stamp[j] != i) {
                            stamp[j] = i;
                            ++cnt;
                        }
                    }
                }
                rowcnt[i] = cnt;
                total += cnt;
            }
            free(stamp);
        }
    }
    return failed ? -1 : total;
}

/* Fill colC/valC given rpC (exclusive scan of the row counts).  Returns 0, or
 * -1 out of memory, or -2 when a row count disagrees with rpC. */
int oracle_spgemm_fill(int64_t m, int64_t n, const int64_t* rpA, const int64_t* ciA,
                       const void* vA, const int64_t* rpB, const int64_t* ciB, const void* vB,
                       int vtype, const int64_t* rpC, int64_t* ciC, void* vC, int nthreads) {
    int nt = threads_or_default(nthreads);
    int status = 0;
#pragma omp parallel num_threads(nt)
    {
        size_t nn = (size_t)(n > 0 ? n : 1);
        int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * nn);
        int64_t* list = (int64_t*)malloc(sizeof(int64_t) * nn);
        double* spa_d = NULL;
        uint64_t* spa_i = NULL;
        if (vtype == ORACLE_F64) spa_d = (double*)malloc(sizeof(double) * nn);
        if (vtype == ORACLE_I64) spa_i = (uint64_t*)malloc(sizeof(uint64_t) * nn);
        if (!stamp || !list || (vtype == ORACLE_F64 && !spa_d) || (vtype == ORACLE_I64 && !spa_i)) {
#pragma omp atomic write
            status = -1;
        } else {
            const double* aD = (const double*)vA;
            const double* bD = (const double*)vB;
            const uint64_t* aI = (const uint64_t*)vA;
            const uint64_t* bI = (const uint64_t*)vB;
            double* cD = (double*)vC;
            uint64_t* cI = (uint64_t*)vC;
            for (int64_t j = 0; j < n; ++j) stamp[j] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < m; ++i) {
                int64_t nz = 0;
                for (int64_t p = rpA[i]; p < rpA[i + 1]; ++p) {
                    int64_t k = ciA[p];
                    for (int64_t q = rpB[k]; q < rpB[k + 1]; ++q) {
                        int64_t j = ciB[q];
                        int first = stamp[j] != i;
                        if (first) {
                            stamp[j] = i;
                            list[nz++] = j;
                        }
                        if (vtype == ORACLE_F64) {
                            double prod = aD[p] * bD[q];
                            spa_d[j] = first ? prod : spa_d[j] + prod;
                        } else if (vtype == ORACLE_I64) {
                            uint64_t prod = aI[p] * bI[q];
                            spa_i[j] = first ? prod : spa_i[j] + prod;
                        }
                    }
                }
                if (nz != rpC[i + 1] - rpC[i]) {
#pragma omp atomic write
                    status = -2;
                    continue;
                }
                qsort(list, (size_t)nz, sizeof(int64_t), cmp_i64);
                int64_t base = rpC[i];
                for (int64_t t = 0; t < nz; ++t) {
                    int64_t j = list[t];
                    ciC[base + t] = j;
                    if (vtype == ORACLE_F64) cD[base + t] = spa_d[j];
                    else if (vtype == ORACLE_I64) cI[base + t] = spa_i[j];
                }
            }
        }
        free(stamp);
        free(list);
        free(spa_d);
        free(spa_i);
    }
    return status;
}

/* Entrywise sum of c same-shape CSR matrices, slices in ascending order.
 * rps/cis/vs are arrays of c pointers.  Count pass. */
int64_t oracle_sum_count(int c, int64_t m, int64_t n, const int64_t* const* rps,
                         const int64_t* const* cis, int64_t* rowcnt, int nthreads) {
    int nt = threads_or_default(nthreads);
    int failed = 0;
    int64_t total = 0;
#pragma omp parallel num_threads(nt) reduction(+ : total)
    {
        int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!stamp) {
#pragma omp atomic write
            failed = 1;
        } else {
            for (int64_t j = 0; j < n; ++j) stamp[j] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < m; ++i) {
                int64_t cnt = 0;
                for (int s = 0; s < c; ++s)
                    for (int64_t q = rps[s][i]; q < rps[s][i + 1]; ++q) {
                        int64_t j = cis[s][q];
                        if (stamp[j] != i) {
                            stamp[j] = i;
                            ++cnt;
                        }
                    }
                rowcnt[i] = cnt;
                total += cnt;
            }
            free(stamp);
        }
    }
    return failed ? -1 : total;
}

int oracle_sum_fill(int c, int64_t m, int64_t n, const int64_t* const* rps,
                    const int64_t* const* cis, const void* const* vs, int vtype,
                    const int64_t* rpC, int64_t* ciC, void* vC, int nthreads) {
    int nt = threads_or_default(nthreads);
    int status = 0;
#pragma omp parallel num_threads(nt)
    {
        size_t nn = (size_t)(n > 0 ? n : 1);
        int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * nn);
        int64_t* list = (int64_t*)malloc(sizeof(int64_t) * nn);
        double* spa_d = NULL;
        uint64_t* spa_i = NULL;
        if (vtype == ORACLE_F64) spa_d = (double*)malloc(sizeof(double) * nn);
        if (vtype == ORACLE_I64) spa_i = (uint64_t*)malloc(sizeof(uint64_t) * nn);
        if (!stamp || !list || (vtype == ORACLE_F64 && !spa_d) || (vtype == ORACLE_I64 && !spa_i)) {
#pragma omp atomic write
            status = -1;
        } else {
            double* cD = (double*)vC;
            uint64_t* cI = (uint64_t*)vC;
            for (int64_t j = 0; j < n; ++j) stamp[j] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < m; ++i) {
                int64_t nz = 0;
                for (int s = 0; s < c; ++s) {
                    const double* vd = (const double*)vs[s];
                    const uint64_t* vi = (const uint64_t*)vs[s];
                    for (int64_t q = rps[s][i]; q < rps[s][i + 1]; ++q) {
                        int64_t j = cis[s][q];
                        int first = stamp[j] != i;
                        if (first) {
                            stamp[j] = i;
                            list[nz++] = j;
                        }
                        if (vtype == ORACLE_F64) spa_d[j] = first ? vd[q] : spa_d[j] + vd[q];
                        else if (vtype == ORACLE_I64) spa_i[j] = first ? vi[q] : spa_i[j] + vi[q];
                    }
                }
                if (nz != rpC[i + 1] - rpC[i]) {
#pragma omp atomic write
                    status = -2;
                    continue;
                }
                qsort(list, (size_t)nz, sizeof(int64_t), cmp_i64);
                int64_t base = rpC[i];
                for (int64_t t = 0; t < nz; ++t) {
                    int64_t j = list[t];
                    ciC[base + t] = j;
                    if (vtype == ORACLE_F64) cD[base + t] = spa_d[j];
                    else if (vtype == ORACLE_I64) cI[base + t] = spa_i[j];
                }
            }
        }
        free(stamp);
        free(list);
        free(spa_d);
        free(spa_i);
    }
    return status;
}
