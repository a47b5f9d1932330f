/*
 * oracle.c -- plain, slow, obviously-correct CPU reference for exact
 * Levenshtein distance and the pieces of the breadth-first (Landau-Vishkin)
 * method built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library, and neither includes the
 * other.
 *
 * Conventions follow the paper, not the GPU code:
 *   - strings A[1..n], B[1..m] are passed 0-based (A[x] here is the paper's
 *     A[x+1]);
 *   - a DP cell is (x, y): x characters of A and y characters of B consumed;
 *   - a diagonal is i = x - y (Sec. 3.1, Appendix A);
 *   - f_t[i] is the largest row x on diagonal i reachable with t edits.
 * Every quantity is int64; "minus infinity" (no cell on that diagonal yet) is
 * ORC_NEG.
 *
 * Readings of the paper taken where it is silent (each is listed in the
 * design notes):
 *   - Algorithm 1 has no bound check; a candidate row past the end of
 *     diagonal i is clamped to its last cell, row min(n, m + i).  This is
 *     exact: neighbouring DP cells differ by at most one edit.
 *   - a predecessor f_{t-1}[j] counts only if |j| <= t-1 and the diagonal has
 *     a cell (-m <= j <= n); otherwise it is minus infinity.
 *   - the loop keeps running while the target diagonal n - m lies outside
 *     [-t, t].
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC -o liboracle.so oracle.c
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NEG (INT64_MIN / 4)

/* ------------------------------------------------------------------ */
/* (o1) The DP recurrence of Sec. 1 (and Sec. 2, "String Edit Distance"):
 *   G[i][j] = max(i, j)                      if i = 0 or j = 0
 *   G[i][j] = G[i-1][j-1]                    if A[i] = B[j]
 *   G[i][j] = 1 + min(G[i-1][j], G[i-1][j-1], G[i][j-1])   otherwise
 * kept as two rows of length m + 1.                                   */
int64_t orc_dp(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m)
{
    int64_t *prev = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    int64_t *cur = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return -1;
    }
    for (int64_t j = 0; j <= m; j++)
        prev[j] = j; /* row i = 0: G[0][j] = max(0, j) */
    for (int64_t i = 1; i <= n; i++) {
        cur[0] = i; /* G[i][0] = max(i, 0) */
        for (int64_t j = 1; j <= m; j++) {
            if (A[i - 1] == B[j - 1]) {
                cur[j] = prev[j - 1];
            } else {
                int64_t best = prev[j];
                if (prev[j - 1] < best)
                    best = prev[j - 1];
                if (cur[j - 1] < best)
                    best = cur[j - 1];
                cur[j] = 1 + best;
            }
        }
        int64_t *tmp = prev;
        prev = cur;
        cur = tmp;
    }
    int64_t r = prev[m];
    free(prev);
    free(cur);
    return r;
}

/* Full DP table, (n+1) x (m+1) row-major, for tiny inputs only: the
 * frontier definition max{x : G[x][x-i] <= t} is checked against it.  */
int orc_dp_table(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                 int64_t *G)
{
    const int64_t w = m + 1;
    for (int64_t i = 0; i <= n; i++) {
        for (int64_t j = 0; j <= m; j++) {
            int64_t v;
            if (i == 0 || j == 0) {
                v = i > j ? i : j;
            } else if (A[i - 1] == B[j - 1]) {
                v = G[(i - 1) * w + (j - 1)];
            } else {
                int64_t best = G[(i - 1) * w + j];
                if (G[(i - 1) * w + (j - 1)] < best)
                    best = G[(i - 1) * w + (j - 1)];
                if (G[i * w + (j - 1)] < best)
                    best = G[i * w + (j - 1)];
                v = 1 + best;
            }
            G[i * w + j] = v;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* LCP(A, B, x, y) of Sec. 2: the length of the longest common prefix of
 * A[x..n) and B[y..m) (0-based here), found one character at a time.   */
int64_t orc_lcp(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                int64_t x, int64_t y)
{
    int64_t l = 0;
    if (x < 0 || y < 0)
        return 0;
    while (x + l < n && y + l < m && A[x + l] == B[y + l])
        l++;
    return l;
}

/* ------------------------------------------------------------------ */
/* Frontier storage: f[i] for i in [-cap, cap], grown by doubling.       */
typedef struct {
    int64_t cap;
    int64_t *prev; /* f_{t-1}, index i + cap */
    int64_t *cur;  /* f_t */
} orc_front;

static int front_init(orc_front *F, int64_t cap)
{
    F->cap = cap;
    F->prev = (int64_t *)malloc((size_t)(2 * cap + 1) * sizeof(int64_t));
    F->cur = (int64_t *)malloc((size_t)(2 * cap + 1) * sizeof(int64_t));
    if (!F->prev || !F->cur)
        return -1;
    for (int64_t k = 0; k < 2 * cap + 1; k++)
        F->prev[k] = F->cur[k] = ORC_NEG;
    return 0;
}

static void front_free(orc_front *F)
{
    free(F->prev);
    free(F->cur);
    F->prev = F->cur = NULL;
}

static int front_grow(orc_front *F, int64_t need)
{
    if (need <= F->cap)
        return 0;
    int64_t nc = F->cap;
    while (nc < need)
        nc *= 2;
    orc_front G;
    if (front_init(&G, nc) != 0) {
        front_free(&G);
        return -1;
    }
    for (int64_t i = -F->cap; i <= F->cap; i++) {
        G.prev[i + nc] = F->prev[i + F->cap];
        G.cur[i + nc] = F->cur[i + F->cap];
    }
    front_free(F);
    *F = G;
    return 0;
}

#define FP(F, i) ((F)->prev[(i) + (F)->cap])
#define FC(F, i) ((F)->cur[(i) + (F)->cap])

/* One diagonal of one round of Algorithm 1: f_t[i] from f_{t-1}.
 * The three predecessors are the moves <dx,dy> in {<0,1>,<1,0>,<1,1>};
 * the predecessor's diagonal is j = i - dx + dy; each candidate row is
 * slid by LCP and the largest is kept.                                 */
static int64_t lv_cell(const uint8_t *A, int64_t n, const uint8_t *B,
                       int64_t m, const orc_front *F, int64_t t, int64_t i)
{
    static const int DX[3] = {0, 1, 1};
    static const int DY[3] = {1, 0, 1};
    if (i < -m || i > n)
        return ORC_NEG; /* diagonal i has no cell of the (n+1)x(m+1) grid */
    const int64_t last_row = n < m + i ? n : m + i;
    int64_t best = ORC_NEG;
    for (int e = 0; e < 3; e++) {
        int64_t j = i - DX[e] + DY[e];
        if (j < -(t - 1) || j > t - 1)
            continue;
        int64_t fj = FP(F, j);
        if (fj == ORC_NEG)
            continue;
        int64_t x = fj + DX[e];
        if (x > last_row)
            x = last_row; /* reading: clamp to the diagonal's last cell */
        int64_t y = x - i;
        x += orc_lcp(A, n, B, m, x, y);
        if (x > best)
            best = x;
    }
    return best;
}

static int64_t iabs64(int64_t v) { return v < 0 ? -v : v; }

/* (o2)/(o3) Algorithm 1 (Sec. 3.1, Appendix A).
 *   f_0[0] = LCP(A, B, 0, 0); t = 0;
 *   while f_t[n - m] != n: t++; for every i in [-t, t]: f_t[i] = max over
 *   the three predecessors of (their row + dx, slid by LCP).
 * nthreads > 1 runs the loop over diagonals of a round in parallel
 * (OpenMP), as the paper's parallel-for does.
 * max_rounds < 0: no limit.  Returns k, or -1 if max_rounds was reached
 * first, or -2 on allocation failure.
 * stats (optional, 2 entries): [0] rounds run, [1] diagonal-extensions
 * (cells (t, i) evaluated, including f_0[0]).                          */
int64_t orc_lv(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
               int64_t max_rounds, int nthreads, int64_t *stats)
{
    orc_front F;
    if (front_init(&F, 64) != 0) {
        front_free(&F);
        return -2;
    }
    FP(&F, 0) = orc_lcp(A, n, B, m, 0, 0);
    int64_t t = 0;
    int64_t ext = 1;
    const int64_t target = n - m;
    int64_t result = -1;
    for (;;) {
        if (iabs64(target) <= t && FP(&F, target) == n) {
            result = t;
            break;
        }
        if (max_rounds >= 0 && t >= max_rounds)
            break;
        t++;
        if (front_grow(&F, t + 1) != 0) {
            front_free(&F);
            return -2;
        }
        const int64_t lo = -t, hi = t;
        if (nthreads > 1 && hi - lo + 1 >= 256) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 64)
#endif
            for (int64_t i = lo; i <= hi; i++)
                FC(&F, i) = lv_cell(A, n, B, m, &F, t, i);
        } else {
            for (int64_t i = lo; i <= hi; i++)
                FC(&F, i) = lv_cell(A, n, B, m, &F, t, i);
        }
        {
            int64_t vlo = lo < -m ? -m : lo;
            int64_t vhi = hi > n ? n : hi;
            if (vhi >= vlo)
                ext += vhi - vlo + 1;
        }
        int64_t *tmp = F.prev;
        F.prev = F.cur;
        F.cur = tmp;
    }
    if (stats) {
        stats[0] = t;
        stats[1] = ext;
    }
    front_free(&F);
    return result;
}

/* Runs Algorithm 1 for rounds 0..t_max (or until it stops) and writes
 * out[t * (2*t_max+1) + (i + t_max)] = f_t[i] for i in [-t_max, t_max];
 * entries never computed (|i| > t, or rounds after the stop) hold ORC_NEG.
 * Returns k if the loop stopped within t_max rounds, else -1.          */
int64_t orc_lv_frontiers(const uint8_t *A, int64_t n, const uint8_t *B,
                         int64_t m, int64_t t_max, int64_t *out)
{
    const int64_t w = 2 * t_max + 1;
    for (int64_t k = 0; k < (t_max + 1) * w; k++)
        out[k] = ORC_NEG;
    orc_front F;
    if (front_init(&F, t_max + 2) != 0) {
        front_free(&F);
        return -2;
    }
    FP(&F, 0) = orc_lcp(A, n, B, m, 0, 0);
    out[0 * w + t_max] = FP(&F, 0);
    int64_t t = 0;
    const int64_t target = n - m;
    for (;;) {
        if (iabs64(target) <= t && FP(&F, target) == n)
            break;
        if (t >= t_max) {
            front_free(&F);
            return -1;
        }
        t++;
        for (int64_t i = -t; i <= t; i++)
            FC(&F, i) = lv_cell(A, n, B, m, &F, t, i);
        for (int64_t i = -t; i <= t; i++)
            out[t * w + (i + t_max)] = FC(&F, i);
        int64_t *tmp = F.prev;
        F.prev = F.cur;
        F.cur = tmp;
    }
    front_free(&F);
    return t;
}

/* ------------------------------------------------------------------ */
/* Many pairs at once (concatenated strings + offsets), for exhaustive and
 * batched checks.  method: 0 = DP, 1 = Algorithm 1.  Pairs run in
 * parallel over nthreads host threads; each pair is the sequential code. */
int orc_many(int method, int64_t npairs, const uint8_t *Acat,
             const int64_t *aoff, const uint8_t *Bcat, const int64_t *boff,
             int nthreads, int64_t *out)
{
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 1)
#endif
    for (int64_t p = 0; p < npairs; p++) {
        const uint8_t *A = Acat + aoff[p];
        const uint8_t *B = Bcat + boff[p];
        int64_t n = aoff[p + 1] - aoff[p];
        int64_t m = boff[p + 1] - boff[p];
        out[p] = method == 0 ? orc_dp(A, n, B, m)
                             : orc_lv(A, n, B, m, -1, 1, NULL);
    }
    (void)nthreads;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Polynomial string hash of Sec. 2 ("Hash Functions") and the prefix table
 * of Sec. 3.2: T[x] = h(X[1..x]) = sum_{j<x} c(X[j]) * p^(x-1-j) mod q,
 * with q = 2^61 - 1 and character code c(v) = v + 1 (reading: the paper
 * leaves q and the character code open).  Written as Horner's rule with
 * exact 128-bit products; T has len + 1 entries, T[0] = 0.             */
#define ORC_Q ((((uint64_t)1) << 61) - 1)

static uint64_t mulmod_q(uint64_t a, uint64_t b)
{
    unsigned __int128 p = (unsigned __int128)a * b;
    return (uint64_t)(p % ORC_Q);
}

int orc_prefix_hash(const uint8_t *X, int64_t len, uint64_t base,
                    uint64_t *T)
{
    T[0] = 0;
    for (int64_t x = 0; x < len; x++) {
        uint64_t v = mulmod_q(T[x], base) + (uint64_t)X[x] + 1;
        T[x + 1] = v % ORC_Q;
    }
    return 0;
}

/* h(X[l..l+len)) from the prefix table, by the inverse of concatenation:
 * h(S2) = h([S1,S2]) - p^|S2| * h(S1) (Sec. 2).  pw = p^len mod q.     */
uint64_t orc_range_hash(const uint64_t *T, int64_t l, int64_t len,
                        uint64_t pw)
{
    uint64_t a = T[l + len] % ORC_Q;
    uint64_t b = mulmod_q(T[l], pw);
    return (a + ORC_Q - b) % ORC_Q;
}

uint64_t orc_powmod(uint64_t base, int64_t e)
{
    uint64_t r = 1, b = base % ORC_Q;
    while (e > 0) {
        if (e & 1)
            r = mulmod_q(r, b);
        b = mulmod_q(b, b);
        e >>= 1;
    }
    return r;
}

/* Blocked prefix-hash table of Sec. 3.3 (Alg. 2, Build): the prefix hashes
 * of whole blocks only, TB[j] = h(X[0..j*b)) for j = 0 .. floor(len/b).
 * Built the paper's way: every block hashed on its own, then a scan that
 * concatenates them (Sec. 2: h(S1 S2) = h(S1) * p^|S2| + h(S2), |S2| = b). */
int orc_prefix_hash_blocked(const uint8_t *X, int64_t len, int64_t b,
                            uint64_t base, uint64_t *TB)
{
    const int64_t w = len / b;
    const uint64_t pb = orc_powmod(base, b);
    TB[0] = 0;
    for (int64_t j = 1; j <= w; j++) {
        uint64_t hb = 0; /* h(X[(j-1)b .. jb)) */
        for (int64_t i = (j - 1) * b; i < j * b; i++)
            hb = (mulmod_q(hb, base) + (uint64_t)X[i] + 1) % ORC_Q;
        TB[j] = (mulmod_q(TB[j - 1], pb) + hb) % ORC_Q;
    }
    return 0;
}

/* GetHash of Alg. 2: h(X[0..i)) from the blocked table, the prefix of the
 * last whole block at or before i (r = floor(i/b); the printed formula
 * for r is garbled) extended by the i - r*b < b characters after it. */
uint64_t orc_get_hash_blocked(const uint8_t *X, const uint64_t *TB, int64_t b,
                              uint64_t base, int64_t i)
{
    const int64_t r = i / b;
    uint64_t h = TB[r] % ORC_Q;
    for (int64_t j = r * b; j < i; j++)
        h = (mulmod_q(h, base) + (uint64_t)X[j] + 1) % ORC_Q;
    return h;
}

/* A prefix-hash table as the LCP search sees it: full (b = 1: T[i] is
 * h(X[0..i)) itself) or blocked (GetHash). */
struct orc_htab {
    const uint64_t *T;
    const uint8_t *X;
    int64_t b;
};

static uint64_t htab_prefix(const struct orc_htab *t, uint64_t base, int64_t i)
{
    return t->b == 1 ? t->T[i] % ORC_Q : orc_get_hash_blocked(t->X, t->T, t->b, base, i);
}

/* h(X[l..l+len)) = h(X[0..l+len)) - p^len * h(X[0..l)) (Sec. 2). */
static uint64_t htab_range(const struct orc_htab *t, uint64_t base, int64_t l,
                           int64_t len)
{
    const uint64_t a = htab_prefix(t, base, l + len);
    const uint64_t c = mulmod_q(htab_prefix(t, base, l), orc_powmod(base, len));
    return (a + ORC_Q - c) % ORC_Q;
}

/* LCP by hashes, Sec. 3.2 and Alg. 2's LongestPrefix: compare chunks of
 * length 1, 2, 4, ... until the first unequal one, then binary-search the
 * length inside the last bracket.  Returns the largest l <= min(n-x, m-y)
 * whose length-l hashes agree (reading of the garbled search; no
 * confirmation here: the oracle reports what the hashes say).            */
static int64_t htab_lcp(const struct orc_htab *ta, int64_t n,
                        const struct orc_htab *tb, int64_t m, uint64_t base,
                        int64_t x, int64_t y)
{
    int64_t lim = (n - x) < (m - y) ? (n - x) : (m - y);
    if (lim <= 0)
        return 0;
#define ORC_EQ(L) (htab_range(ta, base, x, (L)) == htab_range(tb, base, y, (L)))
    if (!ORC_EQ(1))
        return 0;
    int64_t good = 1; /* longest length known equal */
    int64_t bad = -1; /* shortest length known unequal, -1 = none yet */
    for (int64_t len = 2;; len *= 2) {
        if (len >= lim) {
            if (ORC_EQ(lim))
                return lim;
            bad = lim;
            break;
        }
        if (ORC_EQ(len)) {
            good = len;
        } else {
            bad = len;
            break;
        }
    }
    /* invariant: length good is equal, length bad is not */
    while (bad - good > 1) {
        int64_t mid = good + (bad - good) / 2;
        if (ORC_EQ(mid))
            good = mid;
        else
            bad = mid;
    }
#undef ORC_EQ
    return good;
}

int64_t orc_hash_lcp(const uint64_t *TA, int64_t n, const uint64_t *TB,
                     int64_t m, uint64_t base, int64_t x, int64_t y)
{
    const struct orc_htab ta = {TA, 0, 1}, tb = {TB, 0, 1};
    return htab_lcp(&ta, n, &tb, m, base, x, y);
}

/* The same search with blocked tables (Alg. 2): every hash from GetHash. */
int64_t orc_hash_lcp_blocked(const uint8_t *A, int64_t n, const uint64_t *TA,
                             const uint8_t *B, int64_t m, const uint64_t *TB,
                             int64_t b, uint64_t base, int64_t x, int64_t y)
{
    const struct orc_htab ta = {TA, A, b}, tb = {TB, B, b};
    return htab_lcp(&ta, n, &tb, m, base, x, y);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
