/*
 * CPU oracle for the hash-based multi-phase SpGEMM C = A*B (arXiv 2512.12036).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library path may call this code:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code, header, table or helper with the CUDA kernels.
 *
 * Everything here is the plain definition of what the GPU phases compute,
 * written out slowly and obviously:
 *   - intermediate products per row (Algorithm 1),
 *   - row grouping by intermediate-product thresholds (Section III-B),
 *   - output structure: nnz of row i = |union of the column sets of the B rows
 *     selected by row i of A| (the allocation phase, Algorithms 2-4),
 *   - output values by Gustavson's row-wise product (Section III-A) with a dense
 *     accumulator held in fp64, columns in ascending order (the accumulation
 *     phase and its sort, Algorithm 5 and the column-index sorting step),
 *   - the per-entry error scale sum_k |a_ik||b_kj| used by the value tolerance,
 *   - the gradients of the product with respect to the stored values of A and
 *     B (the backward pass of the GNN aggregation, Eq. 3),
 *   - the Markov-clustering matrix steps (Algorithm 6): prune, top-k, inflate,
 *     normalise, applied to the rows of M^T.
 *
 * CSR convention: row r occupies [rpt[r], rpt[r+1]) of col/val; rows may be
 * unsorted and may repeat a column (repeats are summed, stored zeros count as
 * structure). Floating point is fp64 throughout unless a function says it
 * makes a decision in fp32 to match what the kernel decides in fp32.
 *
 * Parallelism: optional OpenMP over independent output rows (nthreads <= 0
 * means "all available"); results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int orc_threads(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int orc_max_threads(void) { return orc_threads(0); }

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Algorithm 1: for every row i, IP_i = sum over the stored entries (i,k) of A
 * of the length of row k of B. Returns the total; ip may be NULL. */
int64_t orc_ip_count(int32_t m, const int32_t* rptA, const int32_t* colA,
                     const int32_t* rptB, int64_t* ip) {
    int64_t total = 0;
    for (int32_t i = 0; i < m; ++i) {
        int64_t count = 0;
        for (int32_t j = rptA[i]; j < rptA[i + 1]; ++j) {
            int32_t k = colA[j];
            count += (int64_t)(rptB[k + 1] - rptB[k]);
        }
        if (ip) ip[i] = count;
        total += count;
    }
    return total;
}

/* Section III-B, row grouping: group g (0 <= g <= nthr) holds the rows whose key
 * satisfies thr[g-1] <= key < thr[g] (thr[-1] = -inf, thr[nthr] = +inf).
 * map lists the rows group after group, each group in ascending row order;
 * offsets (nthr+2 entries) gives where each group starts in map. */
void orc_group_rows(int32_t m, const int64_t* key, int32_t nthr, const int64_t* thr,
                    int32_t* map, int32_t* offsets) {
    int32_t ngroups = nthr + 1;
    int32_t pos = 0;
    for (int32_t g = 0; g < ngroups; ++g) {
        offsets[g] = pos;
        for (int32_t i = 0; i < m; ++i) {
            int32_t gi = 0;
            while (gi < nthr && key[i] >= thr[gi]) ++gi;
            if (gi == g) map[pos++] = i;
        }
    }
    offsets[ngroups] = pos;
}

/* Allocation phase result: nnz of every output row (or of rows[0..nr) when rows
 * is not NULL), i.e. the number of distinct columns among all B rows that row i
 * of A selects. A dense "seen" marker per column, stamped with the row id. */
int orc_symbolic(int32_t m, int32_t ncols, const int32_t* rptA, const int32_t* colA,
                 const int32_t* rptB, const int32_t* colB, const int32_t* rows, int32_t nr,
                 int32_t* nnz_row, int nthreads) {
    int32_t count = rows ? nr : m;
    int nt = orc_threads(nthreads);
    int bad = 0;
#pragma omp parallel num_threads(nt) reduction(| : bad)
    {
        int64_t* seen = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncols > 0 ? ncols : 1));
        for (int32_t c = 0; c < ncols; ++c) seen[c] = -1;
#pragma omp for schedule(dynamic, 64)
        for (int32_t r = 0; r < count; ++r) {
            int32_t i = rows ? rows[r] : r;
            int32_t nnz = 0;
            for (int32_t j = rptA[i]; j < rptA[i + 1]; ++j) {
                int32_t k = colA[j];
                for (int32_t t = rptB[k]; t < rptB[k + 1]; ++t) {
                    int32_t c = colB[t];
                    if (c < 0 || c >= ncols) { bad = 1; continue; }
                    if (seen[c] != (int64_t)r) { seen[c] = (int64_t)r; ++nnz; }
                }
            }
            nnz_row[r] = nnz;
        }
        free(seen);
    }
    return bad ? -1 : 0;
}

/* Accumulation phase result (Gustavson, Section III-A): for each output row,
 * c_ij = sum over stored (i,k) in A and stored (k,j) in B of a_ik * b_kj, in
 * fp64 with a dense accumulator, emitted in ascending column order at
 * out_ptr[r] (out_ptr from the row counts of orc_symbolic). bound (nullable)
 * receives sum |a_ik||b_kj| per entry. rows == NULL means all m rows. */
int orc_numeric(int32_t m, int32_t ncols, const int32_t* rptA, const int32_t* colA,
                const float* valA, const int32_t* rptB, const int32_t* colB, const float* valB,
                const int32_t* rows, int32_t nr, const int64_t* out_ptr, int32_t* colC,
                double* valC, double* bound, int nthreads) {
    int32_t count = rows ? nr : m;
    int nt = orc_threads(nthreads);
    int bad = 0;
#pragma omp parallel num_threads(nt) reduction(| : bad)
    {
        size_t nc = (size_t)(ncols > 0 ? ncols : 1);
        double* spa = (double*)calloc(nc, sizeof(double));
        double* mag = (double*)calloc(nc, sizeof(double));
        char* seen = (char*)calloc(nc, 1);
        int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * nc);
#pragma omp for schedule(dynamic, 64)
        for (int32_t r = 0; r < count; ++r) {
            int32_t i = rows ? rows[r] : r;
            int32_t nt_ = 0;
            for (int32_t j = rptA[i]; j < rptA[i + 1]; ++j) {
                int32_t k = colA[j];
                double a = (double)valA[j];
                for (int32_t t = rptB[k]; t < rptB[k + 1]; ++t) {
                    int32_t c = colB[t];
                    if (c < 0 || c >= ncols) { bad = 1; continue; }
                    double prod = a * (double)valB[t];
                    if (!seen[c]) { seen[c] = 1; touched[nt_++] = c; }
                    spa[c] += prod;
                    mag[c] += fabs(prod);
                }
            }
            qsort(touched, (size_t)nt_, sizeof(int32_t), cmp_i32);
            int64_t base = out_ptr[r];
            if (out_ptr[r + 1] - base != nt_) bad = 1;
            for (int32_t q = 0; q < nt_; ++q) {
                int32_t c = touched[q];
                if (q < out_ptr[r + 1] - base) {
                    colC[base + q] = c;
                    valC[base + q] = spa[c];
                    if (bound) bound[base + q] = mag[c];
                }
                spa[c] = 0.0;
                mag[c] = 0.0;
                seen[c] = 0;
            }
        }
        free(spa);
        free(mag);
        free(seen);
        free(touched);
    }
    return bad ? -1 : 0;
}

/* Backward of C = A*B with respect to the stored values (Eq. 3 read at the
 * value level): given dC on C's structure (rptC/colC sorted per row),
 *   dA[j] = sum over stored (k, t) of B row k of dC[i, colB[t]] * valB[t]   for entry j = (i,k),
 *   dB[t] = sum over stored entries j = (i,k) of A with k = row of t of valA[j] * dC[i, colB[t]].
 * Entries of C's structure that the product does not reach do not occur;
 * a product column absent from C's row is an error. Either output may be NULL. */
int orc_backward(int32_t m, int32_t ncols, const int32_t* rptA, const int32_t* colA,
                 const float* valA, int32_t brows, const int32_t* rptB, const int32_t* colB,
                 const float* valB, const int64_t* rptC, const int32_t* colC, const double* dC,
                 double* dA, double* dB) {
    double* g = (double*)calloc((size_t)(ncols > 0 ? ncols : 1), sizeof(double));
    char* inrow = (char*)calloc((size_t)(ncols > 0 ? ncols : 1), 1);
    int bad = 0;
    if (dB) {
        int64_t nb = rptB[brows] - rptB[0];
        for (int64_t t = 0; t < nb; ++t) dB[rptB[0] + t] = 0.0;
    }
    for (int32_t i = 0; i < m; ++i) {
        for (int64_t q = rptC[i]; q < rptC[i + 1]; ++q) { g[colC[q]] = dC[q]; inrow[colC[q]] = 1; }
        for (int32_t j = rptA[i]; j < rptA[i + 1]; ++j) {
            int32_t k = colA[j];
            double acc = 0.0;
            for (int32_t t = rptB[k]; t < rptB[k + 1]; ++t) {
                int32_t c = colB[t];
                if (!inrow[c]) { bad = 1; continue; }
                acc += g[c] * (double)valB[t];
                if (dB) dB[t] += (double)valA[j] * g[c];
            }
            if (dA) dA[j] = acc;
        }
        for (int64_t q = rptC[i]; q < rptC[i + 1]; ++q) { g[colC[q]] = 0.0; inrow[colC[q]] = 0; }
    }
    free(g);
    free(inrow);
    return bad ? -1 : 0;
}

/* One Markov-clustering step after the expansion (Algorithm 6), applied to
 * the rows of M^T (a column of M is a row of M^T):
 *   prune:     drop entries with value < theta;
 *   top-k:     keep the k largest of each row (ties: the smaller column wins);
 *   inflate:   v <- v^r;
 *   normalise: divide the row by its sum.
 * order 0 runs prune, top-k, inflate, normalise (the algorithm's order);
 * order 1 runs inflate first, then prune, top-k, normalise.
 * The keep/drop decisions compare the fp32 inputs (or the fp32-rounded
 * inflated value for order 1), matching a kernel that decides in fp32.
 * Input rows are sorted by column. out_ptr/out_col/out_val are sized by the
 * caller to the input nnz; returns the output nnz. */
static int cmp_topk(const void* a, const void* b) {
    const double* x = (const double*)a; /* (value, column) pairs */
    const double* y = (const double*)b;
    if (x[0] > y[0]) return -1;
    if (x[0] < y[0]) return 1;
    return (x[1] > y[1]) - (x[1] < y[1]);
}

int64_t orc_mcl_step(int32_t m, const int64_t* rpt, const int32_t* col, const float* val,
                     double theta, int32_t k, double r, int32_t order, int64_t* out_ptr,
                     int32_t* out_col, double* out_val) {
    int64_t pos = 0;
    double* buf = NULL;
    int32_t* keep = NULL;
    size_t cap = 0;
    out_ptr[0] = 0;
    for (int32_t i = 0; i < m; ++i) {
        int64_t s = rpt[i], e = rpt[i + 1];
        size_t n = (size_t)(e - s);
        if (n > cap) {
            cap = n;
            buf = (double*)realloc(buf, sizeof(double) * 2 * cap);
            keep = (int32_t*)realloc(keep, sizeof(int32_t) * cap);
        }
        size_t nk = 0;
        for (int64_t q = s; q < e; ++q) {
            float decide = val[q];
            if (order == 1) decide = (float)pow((double)val[q], r);
            if (decide < (float)theta) continue;
            buf[2 * nk] = (double)decide;
            buf[2 * nk + 1] = (double)col[q];
            ++nk;
        }
        qsort(buf, nk, 2 * sizeof(double), cmp_topk);
        if (k >= 0 && nk > (size_t)k) nk = (size_t)k;
        for (size_t q = 0; q < nk; ++q) keep[q] = (int32_t)buf[2 * q + 1];
        qsort(keep, nk, sizeof(int32_t), cmp_i32);
        double sum = 0.0;
        int64_t start = pos;
        for (size_t q = 0; q < nk; ++q) {
            /* value of the kept column from the fp32 input */
            int64_t src = -1;
            for (int64_t t = s; t < e; ++t)
                if (col[t] == keep[q]) { src = t; break; }
            double v = (double)val[src];
            double w = pow(v, r);
            out_col[pos] = keep[q];
            out_val[pos] = w;
            sum += w;
            ++pos;
        }
        for (int64_t q = start; q < pos; ++q) out_val[q] = sum > 0 ? out_val[q] / sum : 0.0;
        out_ptr[i + 1] = pos;
    }
    free(buf);
    free(keep);
    return pos;
}

/* Row normalisation of a CSR matrix (column normalisation of M when the
 * matrix is held as M^T): each stored value divided by its row's sum, fp64. */
void orc_row_normalise(int32_t m, const int64_t* rpt, const float* val, double* out) {
    for (int32_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t q = rpt[i]; q < rpt[i + 1]; ++q) s += (double)val[q];
        for (int64_t q = rpt[i]; q < rpt[i + 1]; ++q) out[q] = s > 0 ? (double)val[q] / s : 0.0;
    }
}
