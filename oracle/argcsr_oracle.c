/*
 * ARG-CSR reference oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, sequential C that states what the Adaptive Row-grouped CSR
 * method computes (Heller & Oberhuber, "Adaptive Row-grouped CSR format for
 * storing of sparse matrices on GPU").  It exists so the CUDA library can be
 * checked against something written independently from the paper; only the
 * test suite, the smoke check and the bench's CPU-baseline leg may load it.
 * It shares no code, header or constant with the CUDA library.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off (no FMA contraction,
 * so every product and sum is one IEEE-754 double operation in source order).
 *
 * Functions and the passage each follows:
 *   oracle_csr_spmv_f64      Section 2 (CSR format): y_i = sum over the row's
 *                            stored entries of values[k] * x[columns[k]].
 *   oracle_csr_abs_spmv_f64  the same sum over |values[k] * x[columns[k]]|;
 *                            the per-row scale of the floating-point
 *                            tolerance (not in the paper).
 *   oracle_group_rows        Section 3, conversion step 1 (grouping).
 *   oracle_greedy_chunk_size Section 3, conversion step 2 and the worked
 *                            example of Fig. 3 (greedy thread assignment).
 *   oracle_argcsr_structure  Section 3, steps 1-3 plus the group layout of
 *                            Listing 1 (firstRow, size, offset, chunkSize).
 *   oracle_argcsr_structure_mode  the same, optionally without the adaptive
 *                            step: every row keeps the one thread the greedy
 *                            starts with (Section 3 step 2's starting state;
 *                            Sliced ELLPACK / Row-grouped CSR of Section 2
 *                            when every group holds G rows).
 *   oracle_argcsr_fill       Section 3, last step (chunk-wise copy) with the
 *                            interleaved layout of Section 3 / Fig. 3 and the
 *                            column -1 padding of Section 4.
 *   oracle_argcsr_spmv_f64   Section 4, the SpMV kernel's semantics executed
 *                            sequentially (diagnostic; same summation shape).
 *
 * Readings where the paper is silent or ambiguous (each one is exercised by
 * the pins in the test suite):
 *   A1  a row is added to the open group first; the group is closed when its
 *       nonzero count exceeds desiredChunkSize * G (strictly), or before a row
 *       would become its (G+1)-th row.  This is the only reading under which
 *       the Fig. 3 example (15 nonzeros, 12 threads, D = 1) is one group.
 *   A2  after the greedy fixes chunkSize C, every row keeps only
 *       max(1, ceil(len / C)) threads; leftover threads stay free (Fig. 3:
 *       the last row gets four threads and one of the twelve is left over).
 *   A3  greedy ties go to the lowest row index (C does not depend on it).
 *   A4  an empty row gets one all-padding chunk; a group without nonzeros
 *       has chunkSize 0 and no slots.
 *   A5  threadsMapping is the group-local INCLUSIVE prefix sum of the
 *       thread counts: the kernel of Section 4 reads it as the end of a row's
 *       chunk range and the previous entry (0 for the first row) as its begin.
 *   A6  a row's entries are cut into contiguous runs of C in CSR order; the
 *       k-th run goes to the row's k-th chunk; chunk indices of a row are
 *       consecutive, rows in order; padding trails each chunk.
 *   A7  padding slots hold column -1 and value +0.0.
 *   A8  every group owns exactly G chunks, i.e. C * G slots.
 *   A10 slot offsets are int32 as in Listing 1: more than 2^31 - 1 slots is
 *       an overflow error.
 *   A13 optional vector width V (not in the paper): C is rounded up to a
 *       multiple of V and element j of chunk c sits at
 *       offset + (j / V) * G * V + c * V + j % V.  V = 1 is the paper's layout.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK         0
#define ORACLE_EINVAL    -1
#define ORACLE_ENOMEM    -2
#define ORACLE_EOVERFLOW -4

#define ORACLE_MAX_G 1024

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

/* -------------------------------------------------------------------------
 * CSR (Section 2)
 * ---------------------------------------------------------------------- */

static int check_csr(int32_t n_rows, int32_t n_cols, const int32_t *rowPointers,
                     const int32_t *columns)
{
    if (n_rows < 0 || n_cols < 0) return ORACLE_EINVAL;
    if (rowPointers[0] != 0) return ORACLE_EINVAL;
    for (int32_t i = 0; i < n_rows; i++)
        if (rowPointers[i + 1] < rowPointers[i]) return ORACLE_EINVAL;
    if (columns) {
        for (int64_t k = 0; k < rowPointers[n_rows]; k++)
            if (columns[k] < 0 || columns[k] >= n_cols) return ORACLE_EINVAL;
    }
    return ORACLE_OK;
}

int oracle_csr_spmv_f64(int32_t n_rows, int32_t n_cols, const int32_t *rowPointers,
                        const int32_t *columns, const double *values,
                        const double *x, double *y)
{
    int st = check_csr(n_rows, n_cols, rowPointers, columns);
    if (st) return st;
    for (int32_t i = 0; i < n_rows; i++) {
        double sum = 0.0;
        for (int32_t k = rowPointers[i]; k < rowPointers[i + 1]; k++)
            sum += values[k] * x[columns[k]];
        y[i] = sum;
    }
    return ORACLE_OK;
}

int oracle_csr_abs_spmv_f64(int32_t n_rows, int32_t n_cols, const int32_t *rowPointers,
                            const int32_t *columns, const double *values,
                            const double *x, double *y)
{
    int st = check_csr(n_rows, n_cols, rowPointers, columns);
    if (st) return st;
    for (int32_t i = 0; i < n_rows; i++) {
        double sum = 0.0;
        for (int32_t k = rowPointers[i]; k < rowPointers[i + 1]; k++) {
            double p = values[k] * x[columns[k]];
            sum += p < 0 ? -p : p;
        }
        y[i] = sum;
    }
    return ORACLE_OK;
}

/* -------------------------------------------------------------------------
 * Conversion, step 1 (Section 3): read the matrix row by row, counting the
 * nonzeros of the open group; close it once the count exceeds
 * desiredChunkSize * G, or when one more row would exceed G rows (A1).
 * Writes firstRow/size when the arrays are given; returns the group count.
 * ---------------------------------------------------------------------- */
int64_t oracle_group_rows(int32_t n_rows, const int32_t *rowPointers, int32_t G,
                          int32_t desiredChunkSize, int32_t *firstRow, int32_t *size)
{
    const int64_t limit = (int64_t)desiredChunkSize * G;
    int64_t groups = 0;
    int32_t start = 0, rows = 0;
    int64_t count = 0;
    for (int32_t r = 0; r < n_rows; r++) {
        if (rows == G) {                       /* one more row would exceed G */
            if (firstRow) { firstRow[groups] = start; size[groups] = rows; }
            groups++;
            start = r; rows = 0; count = 0;
        }
        count += rowPointers[r + 1] - rowPointers[r];
        rows++;
        if (count > limit) {                   /* nonzeros exceed D * G */
            if (firstRow) { firstRow[groups] = start; size[groups] = rows; }
            groups++;
            start = r + 1; rows = 0; count = 0;
        }
    }
    if (rows > 0) {
        if (firstRow) { firstRow[groups] = start; size[groups] = rows; }
        groups++;
    }
    return groups;
}

/* -------------------------------------------------------------------------
 * Conversion, step 2 (Section 3, Fig. 3): one thread per row, then while
 * threads are left, give one more thread to the row whose chunk filling
 * ceil(len / threads) is greatest (lowest row on ties, A3).  The chunk size
 * is the greatest filling once all G threads are placed.  Returns -1 if the
 * group has more rows than threads.
 * ---------------------------------------------------------------------- */
int64_t oracle_greedy_chunk_size(int32_t size, const int64_t *len, int32_t G)
{
    int64_t t[ORACLE_MAX_G];
    if (size < 0 || size > G || G > ORACLE_MAX_G) return -1;
    for (int32_t i = 0; i < size; i++) t[i] = 1;
    for (int32_t left = G - size; left > 0 && size > 0; left--) {
        int32_t best = 0;
        int64_t bestFill = ceil_div(len[0], t[0]);
        for (int32_t i = 1; i < size; i++) {
            int64_t f = ceil_div(len[i], t[i]);
            if (f > bestFill) { bestFill = f; best = i; }
        }
        t[best] += 1;
    }
    int64_t chunk = 0;
    for (int32_t i = 0; i < size; i++) {
        int64_t f = ceil_div(len[i], t[i]);
        if (f > chunk) chunk = f;
    }
    return chunk;
}

/* -------------------------------------------------------------------------
 * Conversion, steps 1-3 (Section 3) and the group descriptor of Listing 1.
 *
 * groupInfo (if given) receives n_groups records {firstRow, size, offset,
 * chunkSize}; threadsMapping (if given) receives, per row, the group-local
 * inclusive prefix of its thread count (A2, A5).  offset is the running sum
 * of chunkSize * G over the preceding groups (A8).  *n_groups_out and
 * *n_slots_out always receive the totals, also when the status is
 * ORACLE_EOVERFLOW (more than 2^31 - 1 slots, A10).
 * ---------------------------------------------------------------------- */
int oracle_argcsr_structure_mode(int32_t n_rows, const int32_t *rowPointers, int32_t G,
                                 int32_t desiredChunkSize, int32_t V, int32_t one_thread_per_row,
                                 int32_t *groupInfo, int32_t *threadsMapping,
                                 int64_t *n_groups_out, int64_t *n_slots_out)
{
    *n_groups_out = 0;
    *n_slots_out = 0;
    if (n_rows < 0 || G < 1 || G > ORACLE_MAX_G || desiredChunkSize < 1) return ORACLE_EINVAL;
    if (V != 1 && V != 2 && V != 4) return ORACLE_EINVAL;
    if (one_thread_per_row != 0 && one_thread_per_row != 1) return ORACLE_EINVAL;
    int st = check_csr(n_rows, 0, rowPointers, NULL);
    if (st) return st;

    int64_t n_groups = oracle_group_rows(n_rows, rowPointers, G, desiredChunkSize, NULL, NULL);
    int32_t *firstRow = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_groups + 1));
    int32_t *size = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_groups + 1));
    if (!firstRow || !size) { free(firstRow); free(size); return ORACLE_ENOMEM; }
    oracle_group_rows(n_rows, rowPointers, G, desiredChunkSize, firstRow, size);

    int64_t len[ORACLE_MAX_G];
    int64_t offset = 0;
    for (int64_t g = 0; g < n_groups; g++) {
        for (int32_t i = 0; i < size[g]; i++) {
            int32_t r = firstRow[g] + i;
            len[i] = rowPointers[r + 1] - rowPointers[r];
        }
        /* the greedy with G threads; without the adaptive step it has no
         * spare thread to place (a budget of one thread per row), so C is
         * the longest row: the starting state of step 2 */
        int64_t chunk = oracle_greedy_chunk_size(size[g], len, one_thread_per_row ? size[g] : G);
        if (chunk > 0) chunk = ceil_div(chunk, V) * V;          /* A13 */
        int64_t prefix = 0;
        for (int32_t i = 0; i < size[g]; i++) {
            int64_t threads = chunk == 0 ? 1 : ceil_div(len[i], chunk);
            if (threads < 1) threads = 1;                        /* A2, A4 */
            prefix += threads;                                   /* A5 */
            if (threadsMapping) threadsMapping[firstRow[g] + i] = (int32_t)prefix;
        }
        if (groupInfo) {
            groupInfo[4 * g + 0] = firstRow[g];
            groupInfo[4 * g + 1] = size[g];
            groupInfo[4 * g + 2] = offset <= INT32_MAX ? (int32_t)offset : -1;
            groupInfo[4 * g + 3] = chunk <= INT32_MAX ? (int32_t)chunk : -1;
        }
        offset += chunk * G;
    }
    free(firstRow);
    free(size);
    *n_groups_out = n_groups;
    *n_slots_out = offset;
    return offset > INT32_MAX ? ORACLE_EOVERFLOW : ORACLE_OK;
}

int oracle_argcsr_structure(int32_t n_rows, const int32_t *rowPointers, int32_t G,
                            int32_t desiredChunkSize, int32_t V,
                            int32_t *groupInfo, int32_t *threadsMapping,
                            int64_t *n_groups_out, int64_t *n_slots_out)
{
    return oracle_argcsr_structure_mode(n_rows, rowPointers, G, desiredChunkSize, V, 0, groupInfo,
                                        threadsMapping, n_groups_out, n_slots_out);
}

/* -------------------------------------------------------------------------
 * Conversion, last step (Section 3): copy the CSR data chunk-wise into the
 * interleaved arrays.  Element j of chunk c of group g sits at
 * offset_g + j * G + c (V = 1): the chunks are stored like the rows of a
 * column-major ELLPACK slice.  Unused slots hold (-1, +0.0) (A7).
 * Values are copied as raw elements of elem_size bytes (a permutation).
 * ---------------------------------------------------------------------- */
int oracle_argcsr_fill(int32_t n_rows, int32_t n_cols, const int32_t *rowPointers,
                       const int32_t *columns, const void *values, int32_t elem_size,
                       int32_t G, int32_t V, const int32_t *groupInfo, int64_t n_groups,
                       const int32_t *threadsMapping, int32_t *out_columns,
                       void *out_values, int64_t n_slots)
{
    int st = check_csr(n_rows, n_cols, rowPointers, columns);
    if (st) return st;
    const char *src = (const char *)values;
    char *dst = (char *)out_values;
    for (int64_t s = 0; s < n_slots; s++) out_columns[s] = -1;
    memset(dst, 0, (size_t)(n_slots * elem_size));

    for (int64_t g = 0; g < n_groups; g++) {
        const int32_t firstRow = groupInfo[4 * g + 0];
        const int32_t size = groupInfo[4 * g + 1];
        const int64_t offset = groupInfo[4 * g + 2];
        const int64_t chunk = groupInfo[4 * g + 3];
        int64_t c = 0;                                   /* chunk (thread) index */
        for (int32_t i = 0; i < size; i++) {
            const int32_t r = firstRow + i;
            const int64_t len = rowPointers[r + 1] - rowPointers[r];
            const int64_t begin = i == 0 ? 0 : threadsMapping[r - 1];
            const int64_t threads = threadsMapping[r] - begin;
            for (int64_t k = 0; k < threads; k++, c++) {
                for (int64_t j = 0; j < chunk; j++) {
                    const int64_t e = k * chunk + j;     /* element of the row (A6) */
                    if (e >= len) break;                 /* padding trails */
                    const int64_t slot = offset + (j / V) * G * V + c * V + (j % V);
                    if (slot < 0 || slot >= n_slots) return ORACLE_EINVAL;
                    const int64_t src_k = rowPointers[r] + e;
                    out_columns[slot] = columns[src_k];
                    memcpy(dst + slot * elem_size, src + src_k * elem_size, (size_t)elem_size);
                }
            }
        }
        if (c > G) return ORACLE_EINVAL;
    }
    return ORACLE_OK;
}

/* -------------------------------------------------------------------------
 * SpMV on ARG-CSR with the semantics of the Section 4 kernel, executed one
 * group and one chunk at a time: each chunk's partial sum runs over its
 * slots until the first column -1; each row then adds the partial sums of
 * its chunk range [threadsMapping[r-1], threadsMapping[r]) in order.
 * ---------------------------------------------------------------------- */
int oracle_argcsr_spmv_f64(int64_t n_groups, const int32_t *groupInfo,
                           const int32_t *threadsMapping, const int32_t *columns,
                           const double *values, int64_t n_slots, int32_t n_cols,
                           int32_t G, int32_t V, const double *x, double *y)
{
    double partial[ORACLE_MAX_G];
    if (G < 1 || G > ORACLE_MAX_G) return ORACLE_EINVAL;
    /* every index is checked, so a malformed encoding is an error, not a crash */
    for (int64_t g = 0; g < n_groups; g++) {
        const int32_t firstRow = groupInfo[4 * g + 0];
        const int32_t size = groupInfo[4 * g + 1];
        const int64_t offset = groupInfo[4 * g + 2];
        const int64_t chunk = groupInfo[4 * g + 3];
        for (int32_t c = 0; c < G; c++) {
            double sum = 0.0;
            for (int64_t j = 0; j < chunk; j++) {
                const int64_t slot = offset + (j / V) * G * V + (int64_t)c * V + (j % V);
                if (slot < 0 || slot >= n_slots) return ORACLE_EINVAL;
                const int32_t col = columns[slot];
                if (col == -1) break;
                if (col < 0 || col >= n_cols) return ORACLE_EINVAL;
                sum += values[slot] * x[col];
            }
            partial[c] = sum;
        }
        for (int32_t i = 0; i < size; i++) {
            const int32_t r = firstRow + i;
            const int32_t begin = i == 0 ? 0 : threadsMapping[r - 1];
            const int32_t end = threadsMapping[r];
            if (begin < 0 || end > G) return ORACLE_EINVAL;
            double sum = 0.0;
            for (int32_t k = begin; k < end; k++) sum += partial[k];
            y[r] = sum;
        }
    }
    return ORACLE_OK;
}
