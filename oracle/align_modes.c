/*
 * CPU oracle for the traceback of one optimal global, semi-global or
 * overlap alignment.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU
 * baseline leg of the benchmark may build, load or call this file.  It
 * shares no code, header or table with the CUDA path.
 *
 * The matrices are those of modes.c (the non-local modes that SW# offers
 * besides local alignment, Section 2.3; the paper leaves other alignment
 * operations to future work, Section 5): the Gotoh recurrences of Section
 * 2.2 without the zero floor of H,
 *
 *   E(i,j) = max(E(i,j-1) - e, H(i,j-1) - o)     gap along the target
 *   F(i,j) = max(F(i-1,j) - e, H(i-1,j) - o)     gap along the query
 *   H(i,j) = max(H(i-1,j-1) + S(q_i,t_j), E(i,j), F(i,j))
 *   E(i,0) = F(0,j) = -inf,  H(0,0) = 0, g(k) = o + (k-1)*min(o, e)
 *   global (mode 1):      H(i,0) = -g(i),  H(0,j) = -g(j)
 *   semi-global (mode 2): H(i,0) = -g(i),  H(0,j) = 0
 *   overlap (mode 3):     H(i,0) = H(0,j) = 0
 *
 * The paper does not say which of several optimal alignments a tool
 * reports.  This library takes the local traceback's rules (traceback.c)
 * with the mode's end cell and boundary:
 *
 *   End cell: global (m, n); semi-global the first cell (m, j), j = 0..n,
 *   in row-major order whose H is the maximum of the last row; overlap the
 *   first cell in row-major order among the last column (i, n), i = 0..m,
 *   and the last row (m, j), j = 0..n, whose H is the maximum of them.
 *   State H at (i, j), i > 0 and j > 0: take the diagonal step if
 *     H(i,j) = H(i-1,j-1) + S(q_i,t_j) (emit M); else, if H(i,j) = E(i,j),
 *     go to state E; else go to state F (no stop at H = 0: there is no
 *     zero floor).
 *   State E / F: as in the local traceback (emit D / I; back to state H
 *     where the gap opens, E(i,j) = H(i,j-1) - o / F(i,j) = H(i-1,j) - o).
 *   Boundary, state H at (i, j) with i = 0 or j = 0: stop at (0, 0).  At
 *     (0, j), j > 0: global emits j D (the first row's leading gap) and
 *     stops at (0, 0); semi-global and overlap stop (free prefix of the
 *     target).  At (i, 0), i > 0: global and semi-global emit i I (the
 *     first column's leading gap) and stop at (0, 0); overlap stops.
 *
 * The alignment covers q[q_begin, q_end) and t[t_begin, t_end) with
 * (q_end, t_end) the end cell and (q_begin, t_begin) where the walk stops;
 * ops run from its start to its end: 0 = M, 1 = I (q_i opposite a gap), 2 =
 * D (t_j opposite a gap).  The score is H at the end cell (the mode's score
 * of modes.c).
 *
 * The forward loop is the recurrence row by row in int64 (one row of H and
 * F, and H of the last column of every row); it records the comparisons the
 * rules read, one byte per cell.  The walk applies the rules literally.
 */
#include <stdint.h>
#include <stdlib.h>

#define NEG_INF (INT64_MIN / 4)

/* per-cell record */
#define R_DIAG 2   /* H(i,j) = H(i-1,j-1) + S(q_i,t_j) */
#define R_HE 4     /* H(i,j) = E(i,j) */
#define R_EOPEN 8  /* E(i,j) = H(i,j-1) - o */
#define R_FOPEN 16 /* F(i,j) = H(i-1,j) - o */
#define R_HF 32    /* H(i,j) = F(i,j) */

static int64_t amax2(int64_t a, int64_t b) { return a > b ? a : b; }

/* leading gap of k residues on the first row or column */
static int64_t lead(int64_t k, int64_t o, int64_t e) { return k <= 0 ? 0 : o + (k - 1) * (e < o ? e : o); }

/* Returns 0, -1 if scratch memory cannot be allocated, -2 for an unknown
 * mode.  *score_out receives the score; coords q_begin, q_end, t_begin,
 * t_end; ops needs room for m + n entries; *ops_len the number written. */
int swo_align_mode(const uint8_t *q, int64_t m, const uint8_t *t, int64_t n,
                   const int32_t *S, int32_t A, int64_t o, int64_t e, int32_t mode,
                   int64_t *score_out, int64_t *coords, uint8_t *ops, int64_t *ops_len)
{
    coords[0] = coords[1] = coords[2] = coords[3] = 0;
    *ops_len = 0;
    *score_out = 0;
    if (mode < 1 || mode > 3) return -2;
    if (m < 0) m = 0;
    if (n < 0) n = 0;
    const int64_t W = n + 1;
    uint8_t *rec = (uint8_t *)calloc((size_t)(m + 1) * (size_t)W, 1);
    int64_t *Hrow = (int64_t *)malloc(sizeof(int64_t) * (size_t)W);
    int64_t *Frow = (int64_t *)malloc(sizeof(int64_t) * (size_t)W);
    int64_t *Hlast = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));   /* H(i, n) */
    uint8_t *rev = (uint8_t *)malloc((size_t)(m + n + 1));
    if (!rec || !Hrow || !Frow || !Hlast || !rev) {
        free(rec); free(Hrow); free(Frow); free(Hlast); free(rev);
        return -1;
    }
    for (int64_t j = 0; j <= n; ++j) {
        Hrow[j] = (mode == 1) ? -lead(j, o, e) : 0;
        Frow[j] = NEG_INF;
    }
    Hlast[0] = Hrow[n];
    for (int64_t i = 1; i <= m; ++i) {
        const int32_t *Srow = S + (size_t)q[i - 1] * (size_t)A;
        const int64_t Hcol0 = (mode == 3) ? 0 : -lead(i, o, e);
        int64_t Hdiag = Hrow[0], Hleft = Hcol0, E = NEG_INF;
        Hrow[0] = Hcol0;
        for (int64_t j = 1; j <= n; ++j) {
            const int64_t Hup = Hrow[j];
            E = amax2(E - e, Hleft - o);
            const int64_t F = amax2(Frow[j] - e, Hup - o);
            const int64_t D = Hdiag + (int64_t)Srow[t[j - 1]];
            const int64_t H = amax2(D, amax2(E, F));
            uint8_t r = 0;
            if (H == D) r |= R_DIAG;
            if (H == E) r |= R_HE;
            if (H == F) r |= R_HF;
            if (E == Hleft - o) r |= R_EOPEN;
            if (F == Hup - o) r |= R_FOPEN;
            rec[i * W + j] = r;
            Hdiag = Hup;
            Hleft = H;
            Hrow[j] = H;
            Frow[j] = F;
        }
        Hlast[i] = Hrow[n];
    }

    /* end cell: candidates in row-major order, strict > keeps the first */
    int64_t best, bi = m, bj = n;
    if (mode == 1) {
        best = Hrow[n];
    } else {
        best = NEG_INF;
        if (mode == 3)
            for (int64_t i = 0; i < m; ++i)
                if (Hlast[i] > best) { best = Hlast[i]; bi = i; bj = n; }
        for (int64_t j = 0; j <= n; ++j)
            if (Hrow[j] > best) { best = Hrow[j]; bi = m; bj = j; }
    }

    int64_t i = bi, j = bj, k = 0;
    int state = 0;                      /* 0 = H, 1 = E, 2 = F */
    /* The guards marked "not reached" hold for the rules above (a gap opens
     * at j = 1 or i = 1 at the latest, and every step consumes a residue);
     * they only keep a wrong rule from walking off the arrays. */
    for (;;) {
        if (k > m + n) break;           /* not reached */
        if (state == 0) {
            if (i == 0 && j == 0) break;
            if (i == 0) {
                if (mode == 1) while (j > 0) { rev[k++] = 2; --j; }
                break;
            }
            if (j == 0) {
                if (mode != 3) while (i > 0) { rev[k++] = 1; --i; }
                break;
            }
            const uint8_t r = rec[i * W + j];
            if (r & R_DIAG) { rev[k++] = 0; --i; --j; }
            else if (r & R_HE) state = 1;
            else if (r & R_HF) state = 2;
            else break;                 /* not reached: H equals one of the three */
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
    *ops_len = k;
    *score_out = best;
    free(rec);
    free(Hrow);
    free(Frow);
    free(Hlast);
    free(rev);
    return 0;
}
