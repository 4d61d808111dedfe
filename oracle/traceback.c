/*
 * CPU oracle for the traceback of one optimal local alignment.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU
 * baseline leg of the benchmark may build, load or call this file.  It
 * shares no code, header or table with the CUDA path.
 *
 * The matrices are those of Section 2.2 (Smith-Waterman local alignment) in
 * the affine-gap form used in the experiments of Section 4.1, as in
 * gotoh.c:
 *
 *   H(i,0) = H(0,j) = 0,  E(i,0) = F(0,j) = -inf
 *   E(i,j) = max(E(i,j-1) - e, H(i,j-1) - o)     gap along the target
 *   F(i,j) = max(F(i-1,j) - e, H(i-1,j) - o)     gap along the query
 *   H(i,j) = max(0, H(i-1,j-1) + S(q_i,t_j), E(i,j), F(i,j))
 *
 * Section 2.2 fixes the optimal score; several alignments can reach it and
 * the paper does not say which one a tool reports.  This library reports
 * the one fixed by the following rules:
 *
 *   End cell: the first cell (i, j) in row-major order (smallest i, then
 *   smallest j) whose H equals the maximum.
 *   State H at (i, j): stop if H(i,j) = 0 (or i = 0 or j = 0).  Otherwise
 *     take the diagonal step if H(i,j) = H(i-1,j-1) + S(q_i,t_j): emit M and
 *     go to state H at (i-1, j-1); else, if H(i,j) = E(i,j), go to state E
 *     at (i, j); else go to state F at (i, j).
 *   State E at (i, j): emit D (t_j opposite a gap); go to state H at
 *     (i, j-1) if E(i,j) = H(i,j-1) - o (the gap opens there), else stay in
 *     state E at (i, j-1).
 *   State F at (i, j): emit I (q_i opposite a gap); go to state H at
 *     (i-1, j) if F(i,j) = H(i-1,j) - o, else stay in state F at (i-1, j).
 *
 * The alignment covers q[q_begin, q_end) and t[t_begin, t_end) (0-based,
 * half-open) and its ops are listed from its start to its end:
 * 0 = M (q_i aligned with t_j), 1 = I (q_i opposite a gap), 2 = D (t_j
 * opposite a gap).  A score of 0 gives the empty alignment with all four
 * coordinates 0.
 *
 * The forward loop is the recurrence row by row in int64, keeping one row
 * of H and F; for every cell it records the comparisons the rules above
 * read (one byte per cell, so memory is (m+1)(n+1) bytes).  The traceback
 * then applies the rules literally.
 */
#include <stdint.h>
#include <stdlib.h>

#define NEG_INF (INT64_MIN / 4)

/* per-cell record */
#define R_ZERO 1   /* H(i,j) = 0 */
#define R_DIAG 2   /* H(i,j) = H(i-1,j-1) + S(q_i,t_j) */
#define R_HE 4     /* H(i,j) = E(i,j) */
#define R_EOPEN 8  /* E(i,j) = H(i,j-1) - o */
#define R_FOPEN 16 /* F(i,j) = H(i-1,j) - o */
#define R_HF 32    /* H(i,j) = F(i,j) */

static int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }

/* Returns the score (>= 0), or -1 if scratch memory cannot be allocated.
 * coords receives q_begin, q_end, t_begin, t_end; ops needs room for m + n
 * entries; *ops_len receives the number written. */
int64_t swo_align(const uint8_t *q, int64_t m, const uint8_t *t, int64_t n,
                  const int32_t *S, int32_t A, int64_t o, int64_t e,
                  int64_t *coords, uint8_t *ops, int64_t *ops_len)
{
    coords[0] = coords[1] = coords[2] = coords[3] = 0;
    *ops_len = 0;
    if (m <= 0 || n <= 0) return 0;
    const int64_t W = n + 1;
    uint8_t *rec = (uint8_t *)calloc((size_t)(m + 1) * (size_t)W, 1);
    int64_t *Hrow = (int64_t *)malloc(sizeof(int64_t) * (size_t)W);
    int64_t *Frow = (int64_t *)malloc(sizeof(int64_t) * (size_t)W);
    uint8_t *rev = (uint8_t *)malloc((size_t)(m + n));
    if (!rec || !Hrow || !Frow || !rev) {
        free(rec); free(Hrow); free(Frow); free(rev);
        return -1;
    }
    for (int64_t j = 0; j <= n; ++j) { Hrow[j] = 0; Frow[j] = NEG_INF; }

    int64_t best = 0, bi = 0, bj = 0;
    for (int64_t i = 1; i <= m; ++i) {
        const int32_t *Srow = S + (size_t)q[i - 1] * (size_t)A;
        int64_t Hdiag = 0, Hleft = 0, E = NEG_INF;
        for (int64_t j = 1; j <= n; ++j) {
            const int64_t Hup = Hrow[j];
            E = max2(E - e, Hleft - o);
            const int64_t F = max2(Frow[j] - e, Hup - o);
            const int64_t D = Hdiag + (int64_t)Srow[t[j - 1]];
            const int64_t H = max2(max2(D, E), max2(F, 0));
            uint8_t r = 0;
            if (H == 0) r |= R_ZERO;
            if (H == D) r |= R_DIAG;
            if (H == E) r |= R_HE;
            if (H == F) r |= R_HF;
            if (E == Hleft - o) r |= R_EOPEN;
            if (F == Hup - o) r |= R_FOPEN;
            rec[i * W + j] = r;
            if (H > best) { best = H; bi = i; bj = j; }   /* strict: first in row-major order */
            Hdiag = Hup;
            Hleft = H;
            Hrow[j] = H;
            Frow[j] = F;
        }
    }

    int64_t k = 0;
    if (best > 0) {
        int64_t i = bi, j = bj;
        int state = 0;                  /* 0 = H, 1 = E, 2 = F */
        /* The guards marked "not reached" hold for the rules above (a gap
         * always opens at j = 1 or i = 1, and every step consumes a residue);
         * they only keep a wrong rule from walking off the arrays. */
        for (;;) {
            if (k >= m + n) break;          /* not reached */
            if (state == 0) {
                if (i == 0 || j == 0) break;
                const uint8_t r = rec[i * W + j];
                if (r & R_ZERO) break;
                if (r & R_DIAG) { rev[k++] = 0; --i; --j; }
                else if (r & R_HE) state = 1;
                else if (r & R_HF) state = 2;
                else break;       /* not reached: a positive H equals one of the three */
            } else if (state == 1) {
                if (j == 0) break;          /* not reached */
                const uint8_t r = rec[i * W + j];
                rev[k++] = 2;
                if (r & R_EOPEN) state = 0;
                --j;
            } else {
                if (i == 0) break;          /* not reached */
                const uint8_t r = rec[i * W + j];
                rev[k++] = 1;
                if (r & R_FOPEN) state = 0;
                --i;
            }
        }
        coords[0] = i;
        coords[1] = bi;
        coords[2] = j;
        coords[3] = bj;
        for (int64_t x = 0; x < k; ++x) ops[x] = rev[k - 1 - x];
    }
    *ops_len = k;
    free(rec);
    free(Hrow);
    free(Frow);
    free(rev);
    return best;
}
