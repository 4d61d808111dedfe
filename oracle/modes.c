/*
 * CPU oracle for the alignment modes other than local: global, semi-global
 * and overlap scores with affine gaps.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU
 * baseline leg of the benchmark may build, load or call this file.  It
 * shares no code, header or table with the CUDA path.
 *
 * The paper scores local alignments (Section 2.2) and names other alignment
 * operations as future work (Section 5); SW#, the tool it measures, offers
 * global and semi-global modes besides local (Section 2.3).  The modes here
 * are the textbook variants of the same Gotoh recurrences (gap of length k
 * costs o + (k-1)e; when o < e the recurrences price a run as adjacent
 * gaps, o each), without the zero floor of H, differing only in the first
 * row and column and in where the score is read:
 *
 *   E(i,j) = max(E(i,j-1) - e, H(i,j-1) - o)
 *   F(i,j) = max(F(i-1,j) - e, H(i-1,j) - o)
 *   H(i,j) = max(H(i-1,j-1) + S(q_i,t_j), E(i,j), F(i,j))
 *   E(i,0) = F(0,j) = -inf,  H(0,0) = 0, and for i, j >= 1:
 *
 *   global (mode 1):      H(i,0) = -g(i),  H(0,j) = -g(j);  score = H(m,n)
 *   semi-global (mode 2): the whole query against any part of the target:
 *                         H(i,0) = -g(i),  H(0,j) = 0;
 *                         score = max over 0 <= j <= n of H(m,j)
 *   overlap (mode 3):     end gaps free on both sequences:
 *                         H(i,0) = H(0,j) = 0;
 *                         score = max(max_j H(m,j), max_i H(i,n))
 *
 * where g(k) = o + (k-1)*min(o, e) is the first row's and column's own
 * recurrence from H(0,0) = 0 (o + (k-1)e whenever o >= e).
 *
 * With m = 0 or n = 0 the same definitions apply to the empty matrix:
 * global scores -g of the other sequence's length (0 if both are empty),
 * semi-global scores -g(m) when only the target is empty, overlap scores 0.
 * The loop below is the definition row by row in int64 with one row of H
 * and F.
 */
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

#define NEG_INF (INT64_MIN / 4)

static int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }

/* Cost of a leading gap of k residues on the first row or column: what the
 * recurrence for F (or E) gives from H(0,0) = 0 with F(0,0) = -inf, i.e.
 * o + (k-1)*min(o, e) (a run continues for e, or closes and reopens for o,
 * whichever is cheaper, as everywhere else in the matrix). */
static int64_t gap_cost(int64_t k, int64_t o, int64_t e) { return k <= 0 ? 0 : o + (k - 1) * (e < o ? e : o); }

/* Score of one pair in the given mode (1 global, 2 semi-global, 3 overlap).
 * Returns INT64_MIN if scratch memory cannot be allocated or the mode is
 * unknown. */
int64_t swo_score_mode(const uint8_t *q, int64_t m, const uint8_t *t, int64_t n,
                       const int32_t *S, int32_t A, int64_t o, int64_t e, int32_t mode)
{
    if (mode < 1 || mode > 3) return INT64_MIN;
    int64_t *Hrow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *Frow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!Hrow || !Frow) { free(Hrow); free(Frow); return INT64_MIN; }
    /* row 0 */
    for (int64_t j = 0; j <= n; ++j) {
        Hrow[j] = (mode == 1) ? -gap_cost(j, o, e) : 0;
        Frow[j] = NEG_INF;
    }
    int64_t best_row = Hrow[n];       /* overlap: max over the last column, H(0,n) so far */
    for (int64_t i = 1; i <= m; ++i) {
        const int32_t *Srow = S + (size_t)q[i - 1] * (size_t)A;
        const int64_t Hcol0 = (mode == 3) ? 0 : -gap_cost(i, o, e);    /* H(i,0) */
        int64_t Hdiag = Hrow[0];      /* H(i-1, 0) */
        int64_t Hleft = Hcol0;        /* H(i, j-1) */
        int64_t E = NEG_INF;          /* E(i, 0) */
        Hrow[0] = Hcol0;
        for (int64_t j = 1; j <= n; ++j) {
            const int64_t Hup = Hrow[j];                   /* H(i-1, j) */
            E = max2(E - e, Hleft - o);                    /* E(i, j)   */
            const int64_t F = max2(Frow[j] - e, Hup - o);  /* F(i, j)   */
            int64_t H = Hdiag + (int64_t)Srow[t[j - 1]];
            H = max2(H, E);
            H = max2(H, F);
            Hdiag = Hup;
            Hleft = H;
            Hrow[j] = H;
            Frow[j] = F;
        }
        best_row = max2(best_row, Hrow[n]);          /* H(i, n) */
    }
    int64_t score;
    if (mode == 1) {
        score = Hrow[n];                             /* H(m, n) */
    } else {
        int64_t last = Hrow[0];                      /* max over j of H(m, j) */
        for (int64_t j = 1; j <= n; ++j) last = max2(last, Hrow[j]);
        score = (mode == 2) ? last : max2(last, best_row);
    }
    free(Hrow);
    free(Frow);
    return score;
}

struct mode_job {
    const uint8_t *qres; const int64_t *qoff; const int64_t *qidx;
    const uint8_t *tres; const int64_t *toff; const int64_t *tidx;
    int64_t npairs;
    const int32_t *S; int32_t A; int64_t o, e; int32_t mode;
    int64_t *out;
    int64_t next;
    pthread_mutex_t lock;
};

static void *mode_worker(void *arg)
{
    struct mode_job *job = (struct mode_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t k = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (k >= job->npairs) break;
        int64_t qi = job->qidx[k], ti = job->tidx[k];
        job->out[k] = swo_score_mode(job->qres + job->qoff[qi], job->qoff[qi + 1] - job->qoff[qi],
                                     job->tres + job->toff[ti], job->toff[ti + 1] - job->toff[ti],
                                     job->S, job->A, job->o, job->e, job->mode);
    }
    return NULL;
}

/* Scores of npairs (query qidx[k], target tidx[k]) pairs in one mode, over
 * nthreads POSIX threads. */
int swo_score_pairs_mode(const uint8_t *qres, const int64_t *qoff, const int64_t *qidx,
                         const uint8_t *tres, const int64_t *toff, const int64_t *tidx,
                         int64_t npairs, const int32_t *S, int32_t A, int64_t o, int64_t e,
                         int32_t mode, int nthreads, int64_t *out)
{
    struct mode_job job = {qres, qoff, qidx, tres, toff, tidx, npairs, S, A, o, e, mode, out, 0,
                           PTHREAD_MUTEX_INITIALIZER};
    if (nthreads < 1) nthreads = 1;
    if (nthreads == 1) { mode_worker(&job); return 0; }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return -1;
    int started = 0;
    for (int i = 0; i < nthreads; ++i) {
        if (pthread_create(&th[i], NULL, mode_worker, &job) != 0) break;
        ++started;
    }
    if (started == 0) mode_worker(&job);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    free(th);
    return 0;
}
