/*
 * CPU oracle for Smith-Waterman local alignment scoring with affine gaps.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU
 * baseline leg of the benchmark may build, load or call this file.  It
 * shares no code, header or table with the CUDA path.
 *
 * What it computes (Section 2.2, "Smith-Waterman Algorithm": the optimal
 * local alignment score of two sequences by dynamic programming, in the
 * affine-gap form of Gotoh with gap-open / gap-extend penalties as in the
 * experiments of Section 4.1).  For query q[1..m], target t[1..n] and an
 * integer substitution matrix S (row = query residue, column = target
 * residue):
 *
 *   H(i,0) = H(0,j) = 0,  E(i,0) = F(0,j) = -inf
 *   E(i,j) = max(E(i,j-1) - e, H(i,j-1) - o)     gap along the target
 *   F(i,j) = max(F(i-1,j) - e, H(i-1,j) - o)     gap along the query
 *   H(i,j) = max(0, H(i-1,j-1) + S(q_i,t_j), E(i,j), F(i,j))
 *   score  = max over all i,j of H(i,j)           (0 when m = 0 or n = 0)
 *
 * A gap of length k therefore costs o + (k-1)*e.
 *
 * The loop below is that definition row by row, in int64, with one row of
 * H and F kept (O(n) memory).  It is deliberately scalar and unvectorised.
 * The only parallelism is over independent (query, target) pairs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

#define NEG_INF (INT64_MIN / 4)

static int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }

/* Score of one pair.  Returns -1 if scratch memory cannot be allocated. */
int64_t swo_score(const uint8_t *q, int64_t m, const uint8_t *t, int64_t n,
                  const int32_t *S, int32_t A, int64_t o, int64_t e)
{
    if (m <= 0 || n <= 0) return 0;
    /* Hrow[j] = H(i-1, j) before row i is processed, H(i, j) after.
     * Frow[j] = F(i-1, j) likewise. */
    int64_t *Hrow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *Frow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!Hrow || !Frow) { free(Hrow); free(Frow); return -1; }
    for (int64_t j = 0; j <= n; ++j) { Hrow[j] = 0; Frow[j] = NEG_INF; }
    int64_t best = 0;
    for (int64_t i = 1; i <= m; ++i) {
        const int32_t *Srow = S + (size_t)q[i - 1] * (size_t)A;
        int64_t Hdiag = 0;        /* H(i-1, j-1); H(i-1, 0) = 0 */
        int64_t Hleft = 0;        /* H(i, j-1);   H(i, 0)   = 0 */
        int64_t E = NEG_INF;      /* E(i, j-1);   E(i, 0)   = -inf */
        for (int64_t j = 1; j <= n; ++j) {
            int64_t Hup = Hrow[j];                         /* H(i-1, j) */
            E = max2(E - e, Hleft - o);                    /* E(i, j)   */
            int64_t F = max2(Frow[j] - e, Hup - o);        /* F(i, j)   */
            int64_t H = Hdiag + (int64_t)Srow[t[j - 1]];
            H = max2(H, E);
            H = max2(H, F);
            H = max2(H, 0);
            Hdiag = Hup;
            Hleft = H;
            Hrow[j] = H;
            Frow[j] = F;
            if (H > best) best = H;
        }
    }
    free(Hrow);
    free(Frow);
    return best;
}

struct pair_job {
    const uint8_t *qres; const int64_t *qoff; const int64_t *qidx;
    const uint8_t *tres; const int64_t *toff; const int64_t *tidx;
    int64_t npairs;
    const int32_t *S; int32_t A; int64_t o, e;
    int64_t *out;
    int64_t next;              /* shared work counter */
    pthread_mutex_t lock;
};

static void *pair_worker(void *arg)
{
    struct pair_job *job = (struct pair_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t k = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (k >= job->npairs) break;
        int64_t qi = job->qidx[k], ti = job->tidx[k];
        const uint8_t *q = job->qres + job->qoff[qi];
        const uint8_t *t = job->tres + job->toff[ti];
        int64_t m = job->qoff[qi + 1] - job->qoff[qi];
        int64_t n = job->toff[ti + 1] - job->toff[ti];
        job->out[k] = swo_score(q, m, t, n, job->S, job->A, job->o, job->e);
    }
    return NULL;
}

/* Scores of npairs (query qidx[k], target tidx[k]) pairs, spread over
 * nthreads POSIX threads (one pair at a time per thread). */
int swo_score_pairs(const uint8_t *qres, const int64_t *qoff, const int64_t *qidx,
                    const uint8_t *tres, const int64_t *toff, const int64_t *tidx,
                    int64_t npairs, const int32_t *S, int32_t A, int64_t o, int64_t e,
                    int nthreads, int64_t *out)
{
    struct pair_job job = {qres, qoff, qidx, tres, toff, tidx, npairs, S, A, o, e, out, 0,
                           PTHREAD_MUTEX_INITIALIZER};
    if (nthreads < 1) nthreads = 1;
    if (nthreads == 1) { pair_worker(&job); return 0; }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return -1;
    int started = 0;
    for (int i = 0; i < nthreads; ++i) {
        if (pthread_create(&th[i], NULL, pair_worker, &job) != 0) break;
        ++started;
    }
    if (started == 0) pair_worker(&job);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    free(th);
    return 0;
}
