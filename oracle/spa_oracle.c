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
 *   ORACLE_BOOL  (or,and) -- pattern only, no values;
 *   ORACLE_MINPLUS_F64 / _I64    (min,+): C(i,j) = min over k of A(i,k)+B(k,j)
 *                (binary64 sums rounded; int64 sums wrap around);
 *   ORACLE_MINSEL_F64 / _I64     (min,select2nd): C(i,j) = min over k of B(k,j)
 *                (the operations MIS-2 aggregation is built from, Alg. 3).
 * A min reduction starts from its identity (+infinity, INT64_MAX) and keeps
 * the running value x unless the next term y satisfies y < x, so a NaN term
 * never becomes the minimum and the first of equal terms is kept.
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

enum {
    ORACLE_F64 = 0,
    ORACLE_I64 = 1,
    ORACLE_BOOL = 2,
    ORACLE_MINPLUS_F64 = 3,
    ORACLE_MINPLUS_I64 = 4,
    ORACLE_MINSEL_F64 = 5,
    ORACLE_MINSEL_I64 = 6
};

static int is_f64(int vt) {
    return vt == ORACLE_F64 || vt == ORACLE_MINPLUS_F64 || vt == ORACLE_MINSEL_F64;
}
static int is_i64(int vt) {
    return vt == ORACLE_I64 || vt == ORACLE_MINPLUS_I64 || vt == ORACLE_MINSEL_I64;
}
static int is_min(int vt) { return vt >= ORACLE_MINPLUS_F64; }

/* a (x) b of the semiring */
static double mul_d(int vt, double a, double b) {
    if (vt == ORACLE_MINPLUS_F64) return a + b;
    if (vt == ORACLE_MINSEL_F64) return b;
    return a * b;
}
static uint64_t mul_i(int vt, uint64_t a, uint64_t b) {
    if (vt == ORACLE_MINPLUS_I64) return a + b;
    if (vt == ORACLE_MINSEL_I64) return b;
    return a * b;
}
/* running (+) of the semiring; `first` starts from the identity */
static double add_d(int vt, int first, double x, double y) {
    if (is_min(vt)) {
        if (first) x = 1.0 / 0.0;
        return y < x ? y : x;
    }
    return first ? y : x + y;
}
static uint64_t add_i(int vt, int first, uint64_t x, uint64_t y) {
    if (is_min(vt)) {
        int64_t sx = first ? INT64_MAX : (int64_t)x, sy = (int64_t)y;
        return (uint64_t)(sy < sx ? sy : sx);
    }
    return first ? y : x + y;
}

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

static int thread_index(void) {
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

/* Per-thread SPA buffers (stamp, list of touched columns, value arrays),
 * allocated before a parallel region: an allocation failure is then reported
 * before any thread starts, instead of one thread skipping the work-sharing
 * loop that the others enter. */
typedef struct {
    int64_t* stamp;
    int64_t* list;
    double* spa_d;
    uint64_t* spa_i;
} spa_buf;

static void free_bufs(spa_buf* b, int nt) {
    if (!b) return;
    for (int t = 0; t < nt; ++t) {
        free(b[t].stamp);
        free(b[t].list);
        free(b[t].spa_d);
        free(b[t].spa_i);
    }
    free(b);
}

/* nt buffers over n columns; lists and value arrays only when `fill`. */
static spa_buf* alloc_bufs(int nt, int64_t n, int fill, int vtype) {
    size_t nn = (size_t)(n > 0 ? n : 1);
    spa_buf* b = (spa_buf*)calloc((size_t)nt, sizeof(spa_buf));
    if (!b) return NULL;
    for (int t = 0; t < nt; ++t) {
        b[t].stamp = (int64_t*)malloc(sizeof(int64_t) * nn);
        int ok = b[t].stamp != NULL;
        if (fill) {
            b[t].list = (int64_t*)malloc(sizeof(int64_t) * nn);
            ok = ok && b[t].list != NULL;
            if (is_f64(vtype)) ok = ok && (b[t].spa_d = (double*)malloc(sizeof(double) * nn));
            if (is_i64(vtype)) ok = ok && (b[t].spa_i = (uint64_t*)malloc(sizeof(uint64_t) * nn));
        }
        if (!ok) {
            free_bufs(b, nt);
            return NULL;
        }
    }
    return b;
}

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
    spa_buf* bufs = alloc_bufs(nt, n, 0, ORACLE_BOOL);
    if (!bufs) return -1;
    int64_t total = 0;
#pragma omp parallel num_threads(nt) reduction(+ : total)
    {
        int64_t* stamp = bufs[thread_index()].stamp;
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
    }
    free_bufs(bufs, nt);
    return total;
}

/* Fill colC/valC given rpC (exclusive scan of the row counts).  Returns 0, or
 * -1 out of memory, or -2 when a row count disagrees with rpC. */
int oracle_spgemm_fill(int64_t m, int64_t n, const int64_t* rpA, const int64_t* ciA,
                       const void* vA, const int64_t* rpB, const int64_t* ciB, const void* vB,
                       int vtype, const int64_t* rpC, int64_t* ciC, void* vC, int nthreads) {
    int nt = threads_or_default(nthreads);
    spa_buf* bufs = alloc_bufs(nt, n, 1, vtype);
    if (!bufs) return -1;
    int status = 0;
#pragma omp parallel num_threads(nt)
    {
        spa_buf* my = &bufs[thread_index()];
        int64_t* stamp = my->stamp;
        int64_t* list = my->list;
        double* spa_d = my->spa_d;
        uint64_t* spa_i = my->spa_i;
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
                    if (is_f64(vtype)) {
                        double prod = mul_d(vtype, aD[p], bD[q]);
                        spa_d[j] = add_d(vtype, first, spa_d[j], prod);
                    } else if (is_i64(vtype)) {
                        uint64_t prod = mul_i(vtype, aI[p], bI[q]);
                        spa_i[j] = add_i(vtype, first, spa_i[j], prod);
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
                if (is_f64(vtype)) cD[base + t] = spa_d[j];
                else if (is_i64(vtype)) cI[base + t] = spa_i[j];
            }
        }
    }
    free_bufs(bufs, nt);
    return status;
}

/* Entrywise sum of c same-shape CSR matrices, slices in ascending order.
 * rps/cis/vs are arrays of c pointers.  Count pass. */
int64_t oracle_sum_count(int c, int64_t m, int64_t n, const int64_t* const* rps,
                         const int64_t* const* cis, int64_t* rowcnt, int nthreads) {
    int nt = threads_or_default(nthreads);
    spa_buf* bufs = alloc_bufs(nt, n, 0, ORACLE_BOOL);
    if (!bufs) return -1;
    int64_t total = 0;
#pragma omp parallel num_threads(nt) reduction(+ : total)
    {
        int64_t* stamp = bufs[thread_index()].stamp;
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
    }
    free_bufs(bufs, nt);
    return total;
}

int oracle_sum_fill(int c, int64_t m, int64_t n, const int64_t* const* rps,
                    const int64_t* const* cis, const void* const* vs, int vtype,
                    const int64_t* rpC, int64_t* ciC, void* vC, int nthreads) {
    int nt = threads_or_default(nthreads);
    spa_buf* bufs = alloc_bufs(nt, n, 1, vtype);
    if (!bufs) return -1;
    int status = 0;
#pragma omp parallel num_threads(nt)
    {
        spa_buf* my = &bufs[thread_index()];
        int64_t* stamp = my->stamp;
        int64_t* list = my->list;
        double* spa_d = my->spa_d;
        uint64_t* spa_i = my->spa_i;
        double* cD = (double*)vC;
        uint64_t* cI = (uint64_t*)vC;
        for (int64_t j = 0; j < n; ++j) stamp[j] = -1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < m; ++i) {
            int64_t nz = 0;
            for (int s = 0; s < c; ++s) {
                /* pattern-only sums pass no value arrays (vs may be NULL) */
                const double* vd = vs ? (const double*)vs[s] : NULL;
                const uint64_t* vi = vs ? (const uint64_t*)vs[s] : NULL;
                for (int64_t q = rps[s][i]; q < rps[s][i + 1]; ++q) {
                    int64_t j = cis[s][q];
                    int first = stamp[j] != i;
                    if (first) {
                        stamp[j] = i;
                        list[nz++] = j;
                    }
                    if (is_f64(vtype)) spa_d[j] = add_d(vtype, first, spa_d[j], vd[q]);
                    else if (is_i64(vtype)) spa_i[j] = add_i(vtype, first, spa_i[j], vi[q]);
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
                if (is_f64(vtype)) cD[base + t] = spa_d[j];
                else if (is_i64(vtype)) cI[base + t] = spa_i[j];
            }
        }
    }
    free_bufs(bufs, nt);
    return status;
}
