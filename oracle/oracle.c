/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for Row-grouped CSR
 * (RgCSR) sparse matrix-vector multiplication (Oberhuber, Suzuki, Vacata).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA library; the only thing both sides see are the seeded input matrices.
 *
 * Conventions (all functions):
 *   - n rows, m columns, CSR row pointer int64[n+1], column index int32[nnz],
 *     values double[nnz] (or raw element bytes where a layout is copied).
 *   - every floating-point result is computed in double precision with plain
 *     left-to-right loops; no blocking, no reordering, no library kernels.
 *
 * Parity status: every function below is pinned by a test under tests/
 * against something other than itself (the paper's worked example counts,
 * dense matrix-vector products, closed forms, brute force on tiny inputs,
 * finite differences).  The HYB ELL-width default rule is a project choice
 * the paper leaves open; its layout for a given width is pinned.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Sec. 3.1 (Common CSR format): the sequential CSR SpMV.                   */
/* Ax[i] is overwritten with the sum over the row's entries, taken in the    */
/* stored order.  absy[i] (if non-NULL) receives sum |a_ij| |x_j|, the       */
/* scale of the elementwise error bound used by the parity tests.            */
/* ------------------------------------------------------------------------ */
void orc_csr_spmv(int64_t n, const int64_t *rowptr, const int32_t *col,
                  const double *val, const double *x, double *y, double *absy)
{
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0, a = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
            s += val[p] * x[col[p]];
            a += fabs(val[p]) * fabs(x[col[p]]);
        }
        y[i] = s;
        if (absy) absy[i] = a;
    }
}

/* Same definition applied to k right-hand sides at once: X is row-major
 * [m x k], Y is row-major [n x k].  Y[i,b] = sum_p val[p] X[col[p], b]. */
void orc_csr_spmm(int64_t n, int64_t k, const int64_t *rowptr,
                  const int32_t *col, const double *val, const double *X,
                  double *Y, double *absY)
{
    for (int64_t i = 0; i < n; i++) {
        for (int64_t b = 0; b < k; b++) {
            double s = 0.0, a = 0.0;
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
                double xv = X[(int64_t)col[p] * k + b];
                s += val[p] * xv;
                a += fabs(val[p]) * fabs(xv);
            }
            Y[i * k + b] = s;
            if (absY) absY[i * k + b] = a;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.4 (Row-grouped CSR format): layout builder.                        */
/* Rows are cut into groups of G consecutive rows; group g holds             */
/* R_g = min(G, n - g*G) rows (the last group is smaller, as the kernel's   */
/* "currentGroupSize" states).  Within a group the first entries of all     */
/* rows are stored first, then the second entries, and so on; rows shorter  */
/* than the group's longest row K_g are padded with artificial zeros.       */
/* groupPointers[g] is the offset of group g, rowLengths[i] the true length. */
/* Address of slot j of row i = g*G + t:  groupPointers[g] + j*R_g + t.      */
/* Returns n_stored = groupPointers[n_groups].                               */
/* ------------------------------------------------------------------------ */
int64_t orc_rgcsr_sizes(int64_t n, const int64_t *rowptr, int64_t G,
                        int32_t *row_lengths, int64_t *group_ptr)
{
    int64_t n_groups = (n + G - 1) / G;
    for (int64_t i = 0; i < n; i++)
        row_lengths[i] = (int32_t)(rowptr[i + 1] - rowptr[i]);
    group_ptr[0] = 0;
    for (int64_t g = 0; g < n_groups; g++) {
        int64_t first = g * G;
        int64_t rows = (n - first < G) ? (n - first) : G;
        int64_t kmax = 0;
        for (int64_t t = 0; t < rows; t++)
            if (row_lengths[first + t] > kmax) kmax = row_lengths[first + t];
        group_ptr[g + 1] = group_ptr[g] + rows * kmax;
    }
    return group_ptr[n_groups];
}

/* Fills the slabs.  Values are copied as raw elements of elem_size bytes so
 * the result can be compared bit for bit.  Padding ("artificial zeros" with
 * a "ghost index") holds all-zero value bits and column 0.  slot_to_csr[s]
 * is the CSR position stored at slot s, or -1 for padding. */
void orc_rgcsr_fill(int64_t n, const int64_t *rowptr, const int32_t *col,
                    const void *val, int64_t elem_size, int64_t G,
                    const int64_t *group_ptr, const int32_t *row_lengths,
                    void *values, int32_t *columns, int64_t *slot_to_csr)
{
    int64_t n_groups = (n + G - 1) / G;
    const unsigned char *src = (const unsigned char *)val;
    unsigned char *dst = (unsigned char *)values;
    for (int64_t g = 0; g < n_groups; g++) {
        int64_t first = g * G;
        int64_t rows = (n - first < G) ? (n - first) : G;
        int64_t kmax = rows ? (group_ptr[g + 1] - group_ptr[g]) / rows : 0;
        for (int64_t t = 0; t < rows; t++) {
            int64_t i = first + t;
            for (int64_t j = 0; j < kmax; j++) {
                int64_t s = group_ptr[g] + j * rows + t;
                if (j < row_lengths[i]) {
                    int64_t p = rowptr[i] + j;
                    memcpy(dst + s * elem_size, src + p * elem_size, (size_t)elem_size);
                    columns[s] = col[p];
                    if (slot_to_csr) slot_to_csr[s] = p;
                } else {
                    memset(dst + s * elem_size, 0, (size_t)elem_size);
                    columns[s] = 0;
                    if (slot_to_csr) slot_to_csr[s] = -1;
                }
            }
        }
    }
}

/* Sec. 3.4 kernel semantics on the CPU: one "thread" per row walks its
 * rowLengths[i] slots with stride R_g (currentGroupSize) and overwrites Ax.
 * Padding is never multiplied. */
void orc_rgcsr_spmv(int64_t n, int64_t G, const int64_t *group_ptr,
                    const int32_t *row_lengths, const double *values,
                    const int32_t *columns, const double *x, double *y)
{
    for (int64_t i = 0; i < n; i++) {
        int64_t g = i / G, t = i - g * G;
        int64_t rows = (n - g * G < G) ? (n - g * G) : G;
        int64_t ptr = group_ptr[g] + t;
        double s = 0.0;
        for (int32_t j = 0; j < row_lengths[i]; j++) {
            s += values[ptr] * x[columns[ptr]];
            ptr += rows;
        }
        y[i] = s;
    }
}

/* Sliced ELLPACK semantics (Sec. 3.4, last paragraphs): the same slabs but
 * without rowLengths; every row of group g runs over all K_g slots, where
 * K_g = (groupPointers[g+1] - groupPointers[g]) / R_g, multiplying padding. */
void orc_sliced_ell_spmv(int64_t n, int64_t G, const int64_t *group_ptr,
                         const double *values, const int32_t *columns,
                         const double *x, double *y)
{
    for (int64_t i = 0; i < n; i++) {
        int64_t g = i / G, t = i - g * G;
        int64_t rows = (n - g * G < G) ? (n - g * G) : G;
        int64_t kg = (group_ptr[g + 1] - group_ptr[g]) / rows;
        double s = 0.0;
        for (int64_t j = 0; j < kg; j++) {
            int64_t ptr = group_ptr[g] + j * rows + t;
            s += values[ptr] * x[columns[ptr]];
        }
        y[i] = s;
    }
}

/* Descending row-length ordering (Sec. 4.4.2, Table 7): perm[r] = original
 * row placed at position r; rows sorted by length, longest first, ties kept
 * in original order (a stable sort, written as a plain insertion of each
 * row after all earlier rows of greater or equal length, via counting). */
void orc_descending_order(int64_t n, const int64_t *rowptr, int64_t *perm)
{
    int64_t maxlen = 0;
    for (int64_t i = 0; i < n; i++)
        if (rowptr[i + 1] - rowptr[i] > maxlen) maxlen = rowptr[i + 1] - rowptr[i];
    int64_t *cnt = (int64_t *)calloc((size_t)(maxlen + 2), sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) cnt[maxlen - (rowptr[i + 1] - rowptr[i])]++;
    /* exclusive prefix over "length rank" (rank 0 = longest) */
    int64_t run = 0;
    for (int64_t r = 0; r <= maxlen; r++) { int64_t c = cnt[r]; cnt[r] = run; run += c; }
    for (int64_t i = 0; i < n; i++) {
        int64_t r = maxlen - (rowptr[i + 1] - rowptr[i]);
        perm[cnt[r]++] = i;
    }
    free(cnt);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3 (Hybrid ELLPACK and COO format).                                 */
/* ELL part: N x K1 slots, stored column-major (slot j of row i at j*n+i);  */
/* row i keeps its first min(len_i, K1) entries, the rest of the row's ELL  */
/* slots are padding (value bits 0, column -1: ELL keeps no row lengths).   */
/* COO part: every entry beyond the first K1 of its row, as (row, column,   */
/* value), ordered by row and then by the row's stored order.               */
/* ------------------------------------------------------------------------ */
int64_t orc_hyb_coo_count(int64_t n, const int64_t *rowptr, int64_t K1)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t len = rowptr[i + 1] - rowptr[i];
        if (len > K1) c += len - K1;
    }
    return c;
}

/* The paper states only that the choice of K1 matters (Sec. 3.3).  Project
 * rule: minimise the bytes one SpMV streams for the matrix,
 *   cost(K1) = n*K1*(sv+si) + 2*nnz_coo(K1)*(sv+2*si),
 * over K1 in [0, max row length]; ties go to the smaller K1.  Evaluated
 * here by direct summation for every candidate. */
int64_t orc_hyb_choose_k1(int64_t n, const int64_t *rowptr, int64_t sv, int64_t si)
{
    int64_t maxlen = 0;
    for (int64_t i = 0; i < n; i++)
        if (rowptr[i + 1] - rowptr[i] > maxlen) maxlen = rowptr[i + 1] - rowptr[i];
    int64_t best_k = 0;
    double best_cost = -1.0;
    for (int64_t k = 0; k <= maxlen; k++) {
        double cost = (double)n * (double)k * (double)(sv + si)
                    + 2.0 * (double)orc_hyb_coo_count(n, rowptr, k) * (double)(sv + 2 * si);
        if (best_cost < 0.0 || cost < best_cost) { best_cost = cost; best_k = k; }
    }
    return best_k;
}

void orc_hyb_fill(int64_t n, const int64_t *rowptr, const int32_t *col,
                  const void *val, int64_t elem_size, int64_t K1,
                  void *ell_val, int32_t *ell_col,
                  int32_t *coo_row, int32_t *coo_col, void *coo_val)
{
    const unsigned char *src = (const unsigned char *)val;
    unsigned char *ev = (unsigned char *)ell_val, *cv = (unsigned char *)coo_val;
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t len = rowptr[i + 1] - rowptr[i];
        for (int64_t j = 0; j < K1; j++) {
            int64_t s = j * n + i;
            if (j < len) {
                memcpy(ev + s * elem_size, src + (rowptr[i] + j) * elem_size, (size_t)elem_size);
                ell_col[s] = col[rowptr[i] + j];
            } else {
                memset(ev + s * elem_size, 0, (size_t)elem_size);
                ell_col[s] = -1;
            }
        }
        for (int64_t j = K1; j < len; j++) {
            int64_t p = rowptr[i] + j;
            coo_row[c] = (int32_t)i;
            coo_col[c] = col[p];
            memcpy(cv + c * elem_size, src + p * elem_size, (size_t)elem_size);
            c++;
        }
    }
}

/* HYB SpMV: the ELL step writes y, the COO step adds the overflow. */
void orc_hyb_spmv(int64_t n, int64_t K1, const double *ell_val,
                  const int32_t *ell_col, int64_t nnz_coo,
                  const int32_t *coo_row, const int32_t *coo_col,
                  const double *coo_val, const double *x, double *y)
{
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t j = 0; j < K1; j++) {
            int64_t sl = j * n + i;
            if (ell_col[sl] >= 0) s += ell_val[sl] * x[ell_col[sl]];
        }
        y[i] = s;
    }
    for (int64_t c = 0; c < nnz_coo; c++)
        y[coo_row[c]] += coo_val[c] * x[coo_col[c]];
}

/* ------------------------------------------------------------------------ */
/* Reduced-precision value storage (not in the paper; the paper only uses   */
/* single and double precision).  Per row i:                               */
/*   s_i = 2^ceil(log2(max_j |a_ij|)), s_i = 1 for an empty or zero row,    */
/*   q_ij = round-to-nearest-even of the exact quotient a_ij / s_i into     */
/*          bfloat16 (fmt 0) or IEEE binary16 (fmt 1), subnormals kept,     */
/*   y_i  = s_i * sum_j q_ij x_j.                                           */
/* The quotient is exact because s_i is a power of two.                     */
/* ------------------------------------------------------------------------ */
float orc_row_scale(double maxabs)
{
    if (!(maxabs > 0.0)) return 1.0f;
    int e;
    double m = frexp(maxabs, &e);         /* maxabs = m * 2^e, m in [0.5, 1) */
    /* ceil(log2(maxabs)) is e-1 when maxabs is a power of two, else e */
    int c = (m == 0.5) ? e - 1 : e;
    /* the scale is stored as a binary32 number: its exponent is kept in the
       normal range [-126, 127] so that it is finite, non-zero and exact */
    if (c < -126) c = -126;
    if (c > 127) c = 127;
    return (float)ldexp(1.0, c);
}

/* Round an exactly-known double to a binary format with `mant` explicit
 * mantissa bits and exponent range [emin, emax] (normal numbers), using
 * round-half-to-even on the exact value; returns the encoded bits for a
 * format with `ebits` exponent bits.  Values beyond the largest finite
 * number become infinity (cannot happen for |q| <= 1). */
static uint16_t orc_round_binary(double v, int ebits, int mant)
{
    int bias = (1 << (ebits - 1)) - 1;
    int emin = 1 - bias;                        /* smallest normal exponent */
    uint16_t sign = (v < 0.0 || (v == 0.0 && signbit(v))) ? 1u : 0u;
    double a = fabs(v);
    if (a == 0.0) return (uint16_t)(sign << 15);
    int e;
    frexp(a, &e);                               /* a in [2^(e-1), 2^e) */
    int ex = e - 1;                             /* a = 1.f * 2^ex */
    if (ex < emin) ex = emin;                   /* subnormal: fixed quantum */
    /* quantum of the target format at this exponent */
    double scaled = ldexp(a, mant - ex);        /* exact: power-of-two scale */
    double r = nearbyint(scaled);               /* default mode: half to even */
    /* rounding may carry into the next binade */
    double back = ldexp(r, ex - mant);
    int e2;
    frexp(back, &e2);
    int ex2 = e2 - 1;
    uint32_t bits;
    if (back == 0.0) {
        bits = 0;
    } else if (ex2 < emin) {                    /* subnormal result */
        bits = (uint32_t)r;                     /* mantissa field, exponent 0 */
    } else {
        if (ex2 > bias) return (uint16_t)((sign << 15) | (((1u << ebits) - 1u) << mant));
        double frac = ldexp(back, mant - ex2) - ldexp(1.0, mant);  /* integer */
        bits = ((uint32_t)(ex2 + bias) << mant) | (uint32_t)frac;
    }
    return (uint16_t)((sign << 15) | bits);
}

uint16_t orc_round_bf16(double v) { return orc_round_binary(v, 8, 7); }
uint16_t orc_round_f16(double v) { return orc_round_binary(v, 5, 10); }

static double orc_decode_binary(uint16_t h, int ebits, int mant)
{
    int bias = (1 << (ebits - 1)) - 1;
    int sign = (h >> 15) & 1;
    int ex = (h >> mant) & ((1 << ebits) - 1);
    int fr = h & ((1 << mant) - 1);
    double v;
    if (ex == 0) v = ldexp((double)fr, 1 - bias - mant);
    else if (ex == (1 << ebits) - 1) v = fr ? NAN : INFINITY;
    else v = ldexp((double)(fr + (1 << mant)), ex - bias - mant);
    return sign ? -v : v;
}

double orc_decode_bf16(uint16_t h) { return orc_decode_binary(h, 8, 7); }
double orc_decode_f16(uint16_t h) { return orc_decode_binary(h, 5, 10); }

/* Quantises every stored CSR entry (CSR order).  fmt 0 = bf16, 1 = fp16. */
void orc_quantize_rows(int64_t n, const int64_t *rowptr, const double *val,
                       int fmt, uint16_t *q, float *scale)
{
    for (int64_t i = 0; i < n; i++) {
        double mx = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (fabs(val[p]) > mx) mx = fabs(val[p]);
        float s = orc_row_scale(mx);
        scale[i] = s;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
            double quot = val[p] / (double)s;
            q[p] = fmt == 0 ? orc_round_bf16(quot) : orc_round_f16(quot);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Transposition (for dx = A^T g): CSR of A^T by counting sort over columns. */
/* t_rowptr int64[m+1]; t_col[q] = original row; perm[q] = original CSR      */
/* position, so the transposed value is val[perm[q]].  Entries of each      */
/* transposed row are in increasing original row (stable).                   */
/* ------------------------------------------------------------------------ */
void orc_csr_transpose(int64_t n, int64_t m, const int64_t *rowptr,
                       const int32_t *col, int64_t *t_rowptr, int32_t *t_col,
                       int64_t *perm)
{
    for (int64_t c = 0; c <= m; c++) t_rowptr[c] = 0;
    for (int64_t p = 0; p < rowptr[n]; p++) t_rowptr[col[p] + 1]++;
    for (int64_t c = 0; c < m; c++) t_rowptr[c + 1] += t_rowptr[c];
    int64_t *next = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    for (int64_t c = 0; c <= m; c++) next[c] = t_rowptr[c];
    for (int64_t i = 0; i < n; i++)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
            int64_t q = next[col[p]]++;
            t_col[q] = (int32_t)i;
            perm[q] = p;
        }
    free(next);
}

/* ------------------------------------------------------------------------ */
/* Gradients of Y = A X (X row-major [m x k]) for an upstream gradient Gy  */
/* ([n x k]):  dX = A^T Gy (via orc_csr_transpose + orc_csr_spmm) and       */
/* dval[p] = sum_b Gy[row_p, b] * X[col_p, b] for every stored entry p.    */
/* ------------------------------------------------------------------------ */
void orc_spmm_grad_values(int64_t n, int64_t k, const int64_t *rowptr,
                          const int32_t *col, const double *Gy,
                          const double *X, double *dval)
{
    for (int64_t i = 0; i < n; i++)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
            double s = 0.0;
            for (int64_t b = 0; b < k; b++)
                s += Gy[i * k + b] * X[(int64_t)col[p] * k + b];
            dval[p] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* Damped Jacobi (a repeated-SpMV workload, not in the paper):              */
/*   x_{s+1} = x_s + omega * dinv .* (b - A x_s),  x_0 = 0,                 */
/* with dinv a fixed vector (the inverse diagonal, not differentiated).     */
/* orc_jacobi_grad returns loss = ||x_T||^2 and its gradients with respect  */
/* to b and to every stored value, by the adjoint recursion                 */
/*   lam_T = 2 x_T,  w = omega*dinv.*lam_{s+1},                             */
/*   lam_s = lam_{s+1} - A^T w,  db += w,  dval_p -= w[row_p] x_s[col_p].   */
/* ------------------------------------------------------------------------ */
void orc_jacobi(int64_t n, const int64_t *rowptr, const int32_t *col,
                const double *val, const double *dinv, const double *b,
                double omega, int64_t steps, double *x_out)
{
    double *x = (double *)calloc((size_t)n, sizeof(double));
    double *ax = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t s = 0; s < steps; s++) {
        orc_csr_spmv(n, rowptr, col, val, x, ax, NULL);
        for (int64_t i = 0; i < n; i++) x[i] = x[i] + omega * dinv[i] * (b[i] - ax[i]);
    }
    memcpy(x_out, x, (size_t)n * sizeof(double));
    free(x); free(ax);
}

double orc_jacobi_grad(int64_t n, const int64_t *rowptr, const int32_t *col,
                       const double *val, const double *dinv, const double *b,
                       double omega, int64_t steps, double *db, double *dval)
{
    int64_t nnz = rowptr[n];
    double *xs = (double *)calloc((size_t)(n * (steps + 1)), sizeof(double));
    double *ax = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t s = 0; s < steps; s++) {
        double *xc = xs + s * n, *xn = xs + (s + 1) * n;
        orc_csr_spmv(n, rowptr, col, val, xc, ax, NULL);
        for (int64_t i = 0; i < n; i++) xn[i] = xc[i] + omega * dinv[i] * (b[i] - ax[i]);
    }
    double loss = 0.0;
    double *lam = (double *)malloc((size_t)n * sizeof(double));
    double *w = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; i++) {
        double xi = xs[steps * n + i];
        loss += xi * xi;
        lam[i] = 2.0 * xi;
        db[i] = 0.0;
    }
    for (int64_t p = 0; p < nnz; p++) dval[p] = 0.0;
    for (int64_t s = steps - 1; s >= 0; s--) {
        const double *xc = xs + s * n;
        for (int64_t i = 0; i < n; i++) { w[i] = omega * dinv[i] * lam[i]; db[i] += w[i]; }
        for (int64_t i = 0; i < n; i++)
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
                dval[p] -= w[i] * xc[col[p]];
                lam[col[p]] -= val[p] * w[i];
            }
    }
    free(xs); free(ax); free(lam); free(w);
    return loss;
}

/* ------------------------------------------------------------------------ */
/* Elementwise error bounds for the Jacobi gradients of orc_jacobi_grad    */
/* when they are computed in a floating-point format of unit roundoff u    */
/* (2^-24 for float), first order in u.  This is the tolerance of a        */
/* reduced-precision implementation, not a result of the method; it        */
/* follows the standard model fl(a op b) = (a op b)(1 + e), |e| <= u, and   */
/* gamma_m = m u / (1 - m u) (any m-term sum or product chain).           */
/*                                                                          */
/* Rounding model covered (any order of the sums, fused or not):            */
/*   forward:  y = fl(A x) (sum of at most La terms, La = longest row of A) */
/*             x' = fl(x + fl(fl(w_r d_r) fl(b_r - y)))  with omega, dinv  */
/*             and b first rounded to the format (w_r, d_r, b_r);           */
/*   adjoint:  lam_T = 2 x_T (exact);  w = fl(fl(w_r d_r) lam),             */
/*             g = fl(A^T w) (at most Lt terms, Lt = longest row of A^T),   */
/*             lam' = fl(lam - g);                                          */
/*   db   = the sum over the T steps of w (any order);                      */
/*   dval = the sum over the T steps of fl(fl(-w_r d_r) lam) * x (any       */
/*          order).                                                         */
/* With x_s, lam_s the exact iterates, J = I - omega D A (D = diag(dinv)),  */
/* a_s = |x_s| + E_s and l_s = |lam_s| + M_s:                               */
/*   E_0 = 0,  E_{s+1} = |J| E_s + g(La+7) omega |D| (|b| + |A| a_s)        */
/*                        + u a_s                                           */
/*   M_T = 2 E_T,  M_s = |J|^T M_{s+1} + g(Lt+6) |A|^T (omega |D| l_{s+1})  */
/*                        + u l_{s+1}                                       */
/*   |db~ - db| <= sum_s [omega |D| M_{s+1} + g4 omega |D| l_{s+1}]         */
/*                 + g(T-1) sum_s (1+g4) omega |D| l_{s+1}                  */
/*   |dval~_p - dval_p| <= sum_s omega|d_i| [M_{s+1,i} a_{s,j}              */
/*                 + |lam_{s+1,i}| E_{s,j} + g5 l_{s+1,i} a_{s,j}]          */
/*                 + g(T-1) sum_s (1+g5) omega |d_i| l_{s+1,i} a_{s,j}      */
/* for entry p in row i, column j.  Derivation: the computed step differs  */
/* from the exact step applied to the computed iterate by at most the      */
/* rounding terms above, and that difference propagates through J (or J^T  */
/* in the adjoint); second-order terms are absorbed by the gamma constants */
/* (gamma_a + gamma_b + gamma_a gamma_b <= gamma_{a+b}).  u = 0 gives 0.    */
/* ------------------------------------------------------------------------ */
static double orc_gamma(double m, double u)
{
    return m * u / (1.0 - m * u);
}

/* y = |A| v (or |A|^T v when transposed is non-zero), entries of |A| are |val|. */
static void orc_abs_matvec(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                           const double *v, double *y, int transposed)
{
    if (!transposed) {
        for (int64_t i = 0; i < n; i++) {
            double s = 0.0;
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) s += fabs(val[p]) * v[col[p]];
            y[i] = s;
        }
    } else {
        for (int64_t i = 0; i < n; i++) y[i] = 0.0;
        for (int64_t i = 0; i < n; i++)
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) y[col[p]] += fabs(val[p]) * v[i];
    }
}

/* y = |J| v or |J|^T v for J = I - omega D A (square A). */
static void orc_abs_jacobi_matvec(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                                  const double *dinv, double omega, const double *v, double *y,
                                  int transposed)
{
    for (int64_t i = 0; i < n; i++) y[i] = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double diag = 1.0;                  /* J_ii = 1 - omega d_i a_ii (duplicates summed) */
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (col[p] == i) diag -= omega * dinv[i] * val[p];
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
            if (col[p] == i) continue;
            double jij = fabs(omega * dinv[i] * val[p]);
            if (!transposed) y[i] += jij * v[col[p]];
            else y[col[p]] += jij * v[i];
        }
        y[i] += fabs(diag) * v[i];
    }
}

void orc_jacobi_grad_bound(int64_t n, const int64_t *rowptr, const int32_t *col,
                           const double *val, const double *dinv, const double *b,
                           double omega, int64_t steps, double u,
                           double *db_bound, double *dval_bound)
{
    int64_t nnz = rowptr[n];
    int64_t La = 0, Lt = 0;
    int64_t *ccount = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        if (rowptr[i + 1] - rowptr[i] > La) La = rowptr[i + 1] - rowptr[i];
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) ccount[col[p]]++;
    }
    for (int64_t j = 0; j < n; j++) if (ccount[j] > Lt) Lt = ccount[j];
    free(ccount);
    const double gf = orc_gamma((double)(La + 7), u), gb = orc_gamma((double)(Lt + 6), u);
    const double g4 = orc_gamma(4.0, u), g5 = orc_gamma(5.0, u);
    const double gT = orc_gamma((double)(steps > 1 ? steps - 1 : 0), u);
    /* exact iterates x_s and their bounds E_s, s = 0..T */
    double *xs = (double *)calloc((size_t)(n * (steps + 1)), sizeof(double));
    double *Es = (double *)calloc((size_t)(n * (steps + 1)), sizeof(double));
    double *t1 = (double *)malloc((size_t)n * sizeof(double));
    double *t2 = (double *)malloc((size_t)n * sizeof(double));
    double *a = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t s = 0; s < steps; s++) {
        double *xc = xs + s * n, *xn = xs + (s + 1) * n, *Ec = Es + s * n, *En = Es + (s + 1) * n;
        orc_csr_spmv(n, rowptr, col, val, xc, t1, NULL);
        for (int64_t i = 0; i < n; i++) xn[i] = xc[i] + omega * dinv[i] * (b[i] - t1[i]);
        for (int64_t i = 0; i < n; i++) a[i] = fabs(xc[i]) + Ec[i];
        orc_abs_matvec(n, rowptr, col, val, a, t1, 0);                        /* |A| a_s */
        orc_abs_jacobi_matvec(n, rowptr, col, val, dinv, omega, Ec, t2, 0);    /* |J| E_s */
        for (int64_t i = 0; i < n; i++)
            En[i] = t2[i] + gf * omega * fabs(dinv[i]) * (fabs(b[i]) + t1[i]) + u * a[i];
    }
    /* adjoint: exact lam_s and its bound M_s, accumulated into the bounds */
    double *lam = (double *)malloc((size_t)n * sizeof(double));
    double *M = (double *)malloc((size_t)n * sizeof(double));
    double *l = (double *)malloc((size_t)n * sizeof(double));
    double *wl = (double *)malloc((size_t)n * sizeof(double));
    double *dval_sum = (double *)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
    double *db_sum = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int64_t i = 0; i < n; i++) {
        lam[i] = 2.0 * xs[steps * n + i];
        M[i] = 2.0 * Es[steps * n + i];
        db_bound[i] = 0.0;
    }
    for (int64_t p = 0; p < nnz; p++) dval_bound[p] = 0.0;
    for (int64_t s = steps - 1; s >= 0; s--) {
        const double *xc = xs + s * n, *Ec = Es + s * n;
        /* here lam = lam_{s+1}, M = M_{s+1} */
        for (int64_t i = 0; i < n; i++) {
            l[i] = fabs(lam[i]) + M[i];
            wl[i] = omega * fabs(dinv[i]) * l[i];
            db_bound[i] += omega * fabs(dinv[i]) * M[i] + g4 * wl[i];
            db_sum[i] += (1.0 + g4) * wl[i];
        }
        for (int64_t i = 0; i < n; i++)
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
                const int64_t j = col[p];
                const double aj = fabs(xc[j]) + Ec[j], od = omega * fabs(dinv[i]);
                dval_bound[p] += od * (M[i] * aj + fabs(lam[i]) * Ec[j]) + g5 * od * l[i] * aj;
                dval_sum[p] += (1.0 + g5) * od * l[i] * aj;
            }
        /* lam_s = lam_{s+1} - A^T (omega D lam_{s+1}) */
        for (int64_t i = 0; i < n; i++) t1[i] = omega * dinv[i] * lam[i];
        for (int64_t i = 0; i < n; i++)
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) lam[col[p]] -= val[p] * t1[i];
        /* M_s = |J|^T M_{s+1} + gamma(Lt+6) |A|^T (omega |D| l_{s+1}) + u l_{s+1} */
        orc_abs_jacobi_matvec(n, rowptr, col, val, dinv, omega, M, t2, 1);
        orc_abs_matvec(n, rowptr, col, val, wl, t1, 1);
        for (int64_t i = 0; i < n; i++) M[i] = t2[i] + gb * t1[i] + u * l[i];
    }
    for (int64_t i = 0; i < n; i++) db_bound[i] += gT * db_sum[i];
    for (int64_t p = 0; p < nnz; p++) dval_bound[p] += gT * dval_sum[p];
    free(xs); free(Es); free(t1); free(t2); free(a);
    free(lam); free(M); free(l); free(wl); free(dval_sum); free(db_sum);
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradients in double precision (Krylov context of Sec. 1: CG    */
/* needs SpMV, SAXPY and SDOT).  Textbook CG from x_0 = 0, stopping when    */
/* ||r||_2 <= tol * ||b||_2 or after maxit iterations.  Returns iterations. */
/* ------------------------------------------------------------------------ */
int64_t orc_cg(int64_t n, const int64_t *rowptr, const int32_t *col,
               const double *val, const double *b, double tol, int64_t maxit,
               double *x)
{
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *d = (double *)malloc((size_t)n * sizeof(double));
    double *q = (double *)malloc((size_t)n * sizeof(double));
    double bb = 0.0, rr = 0.0;
    for (int64_t i = 0; i < n; i++) { x[i] = 0.0; r[i] = b[i]; d[i] = b[i]; bb += b[i] * b[i]; }
    rr = bb;
    int64_t it = 0;
    while (it < maxit && sqrt(rr) > tol * sqrt(bb)) {
        orc_csr_spmv(n, rowptr, col, val, d, q, NULL);
        double dq = 0.0;
        for (int64_t i = 0; i < n; i++) dq += d[i] * q[i];
        double alpha = rr / dq;
        double rr_new = 0.0;
        for (int64_t i = 0; i < n; i++) {
            x[i] += alpha * d[i];
            r[i] -= alpha * q[i];
            rr_new += r[i] * r[i];
        }
        double beta = rr_new / rr;
        for (int64_t i = 0; i < n; i++) d[i] = r[i] + beta * d[i];
        rr = rr_new;
        it++;
    }
    free(r); free(d); free(q);
    return it;
}
