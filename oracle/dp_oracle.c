/*
 * dp_oracle.c -- plain single-threaded CPU oracle for the two dynamic programs
 * of Matsumae & Miyazaki, "Solving Dynamic Programming Problem by Pipeline
 * Implementation on GPU".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA path.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg load it; the library never does.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * Functions:
 *   dp_oracle_mcm  -- matrix-chain multiplication table (Section IV-A; the
 *                     paper takes the problem from Cormen et al., whose
 *                     textbook recurrence is written out here).
 *   dp_oracle_sdp  -- simplified DP problem, Definition 1 / Eq. (1), filled by
 *                     the sequential algorithm of Fig. 1.
 *   dp_oracle_interval -- the triangular-table DP of Section IV with a more
 *                     general combining function f of Eq. (2): the MCM
 *                     weight plus a per-cell weight w[i][j] (the paper
 *                     presents MCM as one instance of the general technique).
 *
 * Readings where the paper is silent:
 *   - indices are 0-based: chain A_0..A_{n-1}, A_i is p[i] x p[i+1];
 *   - f(l, r) of Eq. (2) is l + r + p[i]*p[k+1]*p[j+1] (the textbook cost);
 *   - ties between equal-cost splits go to the smallest k;
 *   - on and below the diagonal m = 0 and s = -1;
 *   - S-DP values are uint32; "+" wraps modulo 2^32.
 */
#include <stdint.h>

/* Status codes (local to the oracle). */
#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_EOVERFLOW 4

/*
 * Matrix-chain table.  m and s are n*n row-major arrays (leading dimension n).
 * For i < j:
 *     m[i][j] = min over i <= k < j of  m[i][k] + m[k+1][j] + p[i]*p[k+1]*p[j+1]
 *     s[i][j] = the smallest k attaining that minimum.
 * Cells are filled diagonal by diagonal (d = j - i = 1 .. n-1), which is the
 * computation order of the paper's Fig. 5; k runs upward and only a strictly
 * smaller candidate replaces the current best, so ties keep the smaller k.
 * Every candidate is formed in int64; ORACLE_EOVERFLOW if one does not fit.
 */
int dp_oracle_mcm(const int32_t *p, int32_t n, int64_t *m, int16_t *s)
{
    if (n < 1 || n > 32767) return ORACLE_EINVAL;
    for (int32_t t = 0; t <= n; ++t)
        if (p[t] < 1) return ORACLE_EINVAL;
    for (int64_t t = 0; t < (int64_t)n * n; ++t) {
        m[t] = 0;
        s[t] = -1;
    }
    for (int32_t d = 1; d < n; ++d) {
        for (int32_t i = 0; i + d < n; ++i) {
            const int32_t j = i + d;
            int64_t best = 0;
            int32_t best_k = -1;
            for (int32_t k = i; k < j; ++k) {
                /* p[i]*p[k+1]*p[j+1]: three factors below 2^31 each; guard the
                   product against int64 overflow before forming it. */
                const int64_t a = p[i], b = p[k + 1], c = p[j + 1];
                if (a * b > INT64_MAX / c) return ORACLE_EOVERFLOW;
                const int64_t w = a * b * c;
                const int64_t left = m[(int64_t)i * n + k];
                const int64_t right = m[(int64_t)(k + 1) * n + j];
                if (left > INT64_MAX - right || left + right > INT64_MAX - w)
                    return ORACLE_EOVERFLOW;
                const int64_t cand = left + right + w;
                if (best_k < 0 || cand < best) {
                    best = cand;
                    best_k = k;
                }
            }
            m[(int64_t)i * n + j] = best;
            s[(int64_t)i * n + j] = (int16_t)best_k;
        }
    }
    return ORACLE_OK;
}

/*
 * Interval DP with a user weight.  For i < j:
 *     m[i][j] = min over i <= k < j of
 *                 m[i][k] + m[k+1][j] + p[i]*p[k+1]*p[j+1] + w[i][j]
 *     s[i][j] = the smallest k attaining that minimum,
 * i.e. Eq. (2) with f(l, r) = l + r + p[i]*p[k+1]*p[j+1] + w[i][j].  With w = 0
 * this is dp_oracle_mcm; with p = 0 it is the split form of Knuth's optimal
 * binary search tree and of optimal merging.  p[0..n] >= 0; w is n*n
 * row-major and only its entries with i < j are read (each >= 0).  Same fill
 * order, tie rule and overflow checks as dp_oracle_mcm.
 */
int dp_oracle_interval(const int32_t *p, const int64_t *w, int32_t n, int64_t *m, int16_t *s)
{
    if (n < 1 || n > 32767) return ORACLE_EINVAL;
    for (int32_t t = 0; t <= n; ++t)
        if (p[t] < 0) return ORACLE_EINVAL;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j)
            if (w[(int64_t)i * n + j] < 0) return ORACLE_EINVAL;
    for (int64_t t = 0; t < (int64_t)n * n; ++t) {
        m[t] = 0;
        s[t] = -1;
    }
    for (int32_t d = 1; d < n; ++d) {
        for (int32_t i = 0; i + d < n; ++i) {
            const int32_t j = i + d;
            const int64_t wij = w[(int64_t)i * n + j];
            int64_t best = 0;
            int32_t best_k = -1;
            for (int32_t k = i; k < j; ++k) {
                const int64_t a = p[i], b = p[k + 1], c = p[j + 1];
                if (c != 0 && a * b > INT64_MAX / c) return ORACLE_EOVERFLOW;
                const int64_t r1 = a * b * c;
                const int64_t left = m[(int64_t)i * n + k];
                const int64_t right = m[(int64_t)(k + 1) * n + j];
                if (left > INT64_MAX - right || left + right > INT64_MAX - r1 ||
                    left + right + r1 > INT64_MAX - wij)
                    return ORACLE_EOVERFLOW;
                const int64_t cand = left + right + r1 + wij;
                if (best_k < 0 || cand < best) {
                    best = cand;
                    best_k = k;
                }
            }
            m[(int64_t)i * n + j] = best;
            s[(int64_t)i * n + j] = (int16_t)best_k;
        }
    }
    return ORACLE_OK;
}

/*
 * Simplified DP problem (Definition 1):  ST[i] = (x)_{1<=j<=k} ST[i - a_j]
 * for i = a_1 .. n-1, with a_1 > a_2 > ... > a_k > 0 and ST[0 .. a_1-1] preset.
 * The fill follows the sequential algorithm of Fig. 1: ST[i] starts as
 * ST[i - a_1] and is then combined with ST[i - a_j] for j = 2 .. k in order.
 * op 0: (x) = min over uint32.  op 1: (x) = + modulo 2^32.
 * st holds n values; st[0 .. a[0]-1] are read as the preset.
 */
int dp_oracle_sdp(uint32_t *st, int64_t n, const int32_t *a, int32_t k, int32_t op)
{
    if (k < 1 || (op != 0 && op != 1) || n < 0) return ORACLE_EINVAL;
    for (int32_t j = 0; j < k; ++j) {
        if (a[j] < 1) return ORACLE_EINVAL;
        if (j > 0 && a[j] >= a[j - 1]) return ORACLE_EINVAL;
    }
    const int64_t a1 = a[0];
    for (int64_t i = a1; i < n; ++i) {
        uint32_t v = st[i - a1];
        for (int32_t j = 1; j < k; ++j) {
            const uint32_t x = st[i - a[j]];
            if (op == 0)
                v = x < v ? x : v;
            else
                v = v + x; /* unsigned arithmetic wraps modulo 2^32 */
        }
        st[i] = v;
    }
    return ORACLE_OK;
}
