/*
 * Smith-Waterman / Gotoh score oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct CPU implementation of what the GPU path computes:
 * the best local-alignment score with affine gaps, one query against each database
 * sequence.  Only tests/, the smoke check and the benchmark's CPU-baseline leg may load
 * this library.  It shares no code, header or table with the CUDA path.
 *
 * Follows the paper's Section 2 literally, in int64:
 *   H[i][j] = max{0, H[i-1][j-1] + SM(S1[i], S2[j]), E[i][j], F[i][j]}     (Eq. sw2)
 *   E[i][j] = max{H[i][j-1] - Goe, E[i][j-1] - Ge}                        (Eq. sw3)
 *   F[i][j] = max{H[i-1][j] - Goe, F[i-1][j] - Ge}                        (Eq. sw4)
 * for 1 <= i <= m, 1 <= j <= n, with H, E, F initialised to 0 where i = 0 or j = 0;
 * the score is the maximum entry of H (0 when m = 0 or n = 0).  Goe is the cost of the
 * first position of a gap and Ge that of each further position, so a gap of length k
 * costs Goe + (k - 1) * Ge.  SM is row-major with the query letter as the row:
 * SM(a, b) = sm[a * alphabet + b].
 *
 * Two rows of each matrix are kept (row i-1 and row i); nothing else is reordered.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }

/* Score of query s1[0..m) against subject s2[0..n).  Returns -1 if scratch cannot be
 * allocated (never a valid score, scores are >= 0). */
int64_t oracle_sw_score(const uint8_t *s1, int64_t m, const uint8_t *s2, int64_t n,
                        const int8_t *sm, int32_t alphabet, int64_t goe, int64_t ge)
{
    if (m <= 0 || n <= 0) return 0;
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * 6 * (size_t)(n + 1));
    if (!buf) return -1;
    int64_t *Hp = buf, *Ep = buf + (n + 1), *Fp = buf + 2 * (n + 1);
    int64_t *Hc = buf + 3 * (n + 1), *Ec = buf + 4 * (n + 1), *Fc = buf + 5 * (n + 1);
    for (int64_t j = 0; j <= n; ++j) { Hp[j] = 0; Ep[j] = 0; Fp[j] = 0; }   /* row i = 0 */
    int64_t best = 0;
    for (int64_t i = 1; i <= m; ++i) {
        Hc[0] = 0; Ec[0] = 0; Fc[0] = 0;                                     /* column j = 0 */
        const int8_t *row = sm + (size_t)s1[i - 1] * (size_t)alphabet;
        for (int64_t j = 1; j <= n; ++j) {
            Ec[j] = max2(Hc[j - 1] - goe, Ec[j - 1] - ge);                   /* Eq. sw3 */
            Fc[j] = max2(Hp[j] - goe, Fp[j] - ge);                           /* Eq. sw4 */
            int64_t h = max2(0, Hp[j - 1] + (int64_t)row[s2[j - 1]]);        /* Eq. sw2 */
            h = max2(h, Ec[j]);
            h = max2(h, Fc[j]);
            Hc[j] = h;
            best = max2(best, h);
        }
        int64_t *t;
        t = Hp; Hp = Hc; Hc = t;
        t = Ep; Ep = Ec; Ec = t;
        t = Fp; Fp = Fc; Fc = t;
    }
    free(buf);
    return best;
}

/* One query against every sequence of a database given as concatenated residues with
 * offsets[0..num_seqs] (sequence k = residues[offsets[k] .. offsets[k+1])).  Scores land in
 * original order.  Database sequences are independent, so they are spread over up to
 * `threads` OpenMP threads (<= 0: the OpenMP default).  Returns the thread count used. */
int32_t oracle_sw_search(const uint8_t *query, int64_t m, const uint8_t *residues,
                         const int64_t *offsets, int64_t num_seqs, const int8_t *sm,
                         int32_t alphabet, int64_t goe, int64_t ge, int64_t *scores,
                         int32_t threads)
{
    int32_t used = 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
    {
#pragma omp single
        used = (int32_t)omp_get_num_threads();
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < num_seqs; ++k)
            scores[k] = oracle_sw_score(query, m, residues + offsets[k],
                                        offsets[k + 1] - offsets[k], sm, alphabet, goe, ge);
    }
#else
    (void)threads;
    for (int64_t k = 0; k < num_seqs; ++k)
        scores[k] = oracle_sw_score(query, m, residues + offsets[k],
                                    offsets[k + 1] - offsets[k], sm, alphabet, goe, ge);
#endif
    return used;
}

/* Same, for a list of (query, subject) pairs: pair p aligns query qsel[p] (queries given by
 * qres/qoff like the database) against database sequence dsel[p]. */
int32_t oracle_sw_pairs(const uint8_t *qres, const int64_t *qoff, const uint8_t *residues,
                        const int64_t *offsets, const int64_t *qsel, const int64_t *dsel,
                        int64_t num_pairs, const int8_t *sm, int32_t alphabet, int64_t goe,
                        int64_t ge, int64_t *scores, int32_t threads)
{
    int32_t used = 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
    {
#pragma omp single
        used = (int32_t)omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
        for (int64_t p = 0; p < num_pairs; ++p) {
            int64_t q = qsel[p], d = dsel[p];
            scores[p] = oracle_sw_score(qres + qoff[q], qoff[q + 1] - qoff[q],
                                        residues + offsets[d], offsets[d + 1] - offsets[d],
                                        sm, alphabet, goe, ge);
        }
    }
#else
    (void)threads;
    for (int64_t p = 0; p < num_pairs; ++p) {
        int64_t q = qsel[p], d = dsel[p];
        scores[p] = oracle_sw_score(qres + qoff[q], qoff[q + 1] - qoff[q],
                                    residues + offsets[d], offsets[d + 1] - offsets[d],
                                    sm, alphabet, goe, ge);
    }
#endif
    return used;
}
