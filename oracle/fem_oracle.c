/*
 * fem_oracle.c -- plain serial CPU oracle for counting non-overlapped
 * occurrences of serial episodes with inter-event constraints.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link
 * or call this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm use it.  It shares no code, header or table
 * with the CUDA library and is deliberately slow and obvious.
 *
 * Definitions followed (paper section "Temporal Data Mining"):
 *   - Definition 1: an event stream is a time-ordered sequence of (type, time)
 *     pairs, t_i <= t_{i+1} (ties allowed).
 *   - Definition 2: a serial episode is an ordered tuple of event types.
 *   - The unnumbered constraint equation: an occurrence picks one event per
 *     node, with t_low^k < t_{k+1} - t_k <= t_high^k on every edge k.
 *   - Frequency = size of the largest set of non-overlapped occurrences.
 *
 * Readings of points the paper leaves open:
 *   R1  Two occurrences are non-overlapped when one ends strictly before the
 *       other starts (Algorithm 1's test "prev_e < s_i", strict in time).
 *   R2  Algorithm 1 starts with prev_e = 0; we start with prev_e = -infinity so
 *       that an occurrence starting at t = 0 is not wrongly rejected.
 *   R3  The commented serial algorithm completes at node |alpha|-1; we
 *       complete at the LAST node, then count++, clear every list and leave
 *       the node loop for this event.
 *   R5  Lower bounds satisfy 0 <= lo < hi, so the times inside one occurrence
 *       strictly increase.
 *
 * Three independent counters are provided so that each can check the others:
 *   O1 orc_count_fsm    -- the serial state machine of section "Episode
 *                          Counting Algorithm" (lists s[1..N], reset on
 *                          completion), with readings R1-R3.
 *   O2 orc_count_dp     -- the problem decomposition of section "Problem
 *                          decomposition": for every end event the latest
 *                          possible start (dynamic programme over nodes), then
 *                          Algorithm 1 (greedy interval scheduling by end).
 *   O3 orc_count_brute  -- enumerate every occurrence (index tuples), then an
 *                          exhaustive include/exclude search for the largest
 *                          pairwise non-overlapped subset (memoised).
 * and orc_greedy_sorted, Algorithm 1 on its own, so that it can be pinned
 * against the exhaustive interval search.
 *
 * Mutants: compiling with -DORC_MUTANT=k plants one deliberate mistake in O1
 * or O2 (see the #if blocks).  The tests build each mutant and check that the
 * pins catch it; a normal build has ORC_MUTANT undefined.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

#define ORC_NEG_INF INT64_MIN

/* ------------------------------------------------------------------------ */
/* A growable list of timestamps with a moving front (entries before `front`
 * are deleted).  This is the per-node list s[i] of the serial algorithm.     */
typedef struct {
    int64_t *t;
    int64_t len;
    int64_t cap;
    int64_t front;
} orc_list;

static int list_push(orc_list *l, int64_t v) {
    if (l->len == l->cap) {
        int64_t nc = l->cap ? 2 * l->cap : 16;
        int64_t *nt = (int64_t *)realloc(l->t, (size_t)nc * sizeof(int64_t));
        if (!nt) return -1;
        l->t = nt;
        l->cap = nc;
    }
    l->t[l->len++] = v;
    return 0;
}

static void list_clear(orc_list *l) {
    l->len = 0;
    l->front = 0;
}

/* ------------------------------------------------------------------------ */
/* O1: the serial finite-state-machine counter ("Episode Counting
 * Algorithm").  For every event (E, t), nodes are visited from the last to
 * the first.  A match at node i > 1 first deletes the entries of s[i-1] that
 * can no longer satisfy the upper bound, then looks (newest first) for an
 * entry t_prev with lo < t - t_prev <= hi; at the last node that completes an
 * occurrence (count++, all lists cleared), otherwise t is appended to s[i].
 * A match at node 1 appends t, provided t is after the end of the last
 * counted occurrence (R1).  Returns the count, or UINT64_MAX on allocation
 * failure. */
uint64_t orc_count_fsm(const uint16_t *ev_type, const int32_t *ev_time, int64_t n,
                       int N, const uint16_t *E, const int32_t *lo, const int32_t *hi) {
    if (N < 1) return 0;
    orc_list *s = (orc_list *)calloc((size_t)N, sizeof(orc_list));
    if (!s) return UINT64_MAX;
    uint64_t count = 0;
    int64_t prev_end = ORC_NEG_INF; /* R2 */
    int oom = 0;

    for (int64_t j = 0; j < n && !oom; ++j) {
        const int64_t t = ev_time[j];
        const uint16_t ty = ev_type[j];
        for (int i = N - 1; i >= 0; --i) {
            if (ty != E[i]) continue;
            int has_pred;
            if (i == 0) {
#if ORC_MUTANT == 1
                has_pred = (t >= prev_end); /* mutant: tie at the overlap boundary admitted */
#else
                has_pred = (t > prev_end);  /* R1 */
#endif
            } else {
                orc_list *p = &s[i - 1];
                const int64_t l = lo[i - 1], h = hi[i - 1];
                /* delete entries older than t - hi: they can never match again */
#if ORC_MUTANT == 7
                while (p->front < p->len && p->t[p->front] < t - l) p->front++; /* mutant: prunes by lo */
#else
                while (p->front < p->len && p->t[p->front] < t - h) p->front++;
#endif
                has_pred = 0;
#if ORC_MUTANT == 6
                const int64_t kstop = p->len - 1; /* mutant: only the newest entry is examined */
#else
                const int64_t kstop = p->front;
#endif
                for (int64_t k = p->len - 1; k >= kstop && k >= p->front; --k) {
                    const int64_t d = t - p->t[k];
#if ORC_MUTANT == 2
                    if (l <= d && d <= h) { has_pred = 1; break; } /* mutant: closed lower bound */
#elif ORC_MUTANT == 3
                    if (l < d && d < h) { has_pred = 1; break; }   /* mutant: open upper bound */
#else
                    if (l < d && d <= h) { has_pred = 1; break; }
#endif
                }
            }
            if (!has_pred) continue;
#if ORC_MUTANT == 5
            const int last = (N > 1) ? N - 2 : 0; /* mutant: garbled completion node */
#else
            const int last = N - 1;               /* R3 */
#endif
            if (i == last) {
                count++;
                prev_end = t;
#if ORC_MUTANT != 4
                for (int q = 0; q < N; ++q) list_clear(&s[q]); /* mutant 4: no reset */
#endif
                break;
            }
            if (list_push(&s[i], t)) { oom = 1; break; }
        }
    }
    for (int q = 0; q < N; ++q) free(s[q].t);
    free(s);
    return oom ? UINT64_MAX : count;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 on its own: occurrences (s_i, e_i) sorted by end time; select an
 * occurrence when its start is after the end of the last selected one. */
uint64_t orc_greedy_sorted(const int64_t *s, const int64_t *e, int64_t m) {
    uint64_t count = 0;
    int64_t prev_e = ORC_NEG_INF; /* R2 */
    for (int64_t i = 0; i < m; ++i) {
        if (prev_e < s[i]) {
            prev_e = e[i];
            count++;
        }
    }
    return count;
}

/* ------------------------------------------------------------------------ */
/* O2: problem decomposition.  L[k][j] = latest start time over all partial
 * occurrences of nodes 1..k+1 that end at event j (ORC_NEG_INF if none):
 *   L[0][j] = t_j                                        when type_j = E_1
 *   L[k][j] = max { L[k-1][i] : type_i = E_k, lo_k < t_j - t_i <= hi_k }.
 * Every end event j with L[N-1][j] defined stands for the occurrence
 * (L[N-1][j], t_j); these are already sorted by end (stream order) and
 * Algorithm 1 picks from them.  Using only the latest start per end loses
 * nothing: a start after prev_e exists iff the latest one is after prev_e. */
uint64_t orc_count_dp(const uint16_t *ev_type, const int32_t *ev_time, int64_t n,
                      int N, const uint16_t *E, const int32_t *lo, const int32_t *hi) {
    if (N < 1 || n <= 0) return 0;
    int64_t *L = (int64_t *)malloc((size_t)N * (size_t)n * sizeof(int64_t));
    if (!L) return UINT64_MAX;
    for (int64_t q = 0; q < (int64_t)N * n; ++q) L[q] = ORC_NEG_INF;

    for (int64_t j = 0; j < n; ++j) {
        const int64_t t = ev_time[j];
        for (int k = 0; k < N; ++k) {
            if (ev_type[j] != E[k]) continue;
            if (k == 0) {
                L[j] = t;
                continue;
            }
            const int64_t l = lo[k - 1], h = hi[k - 1];
            int64_t best = ORC_NEG_INF;
            for (int64_t i = j - 1; i >= 0 && t - ev_time[i] <= h; --i) {
                if (ev_type[i] != E[k - 1]) continue;
                const int64_t d = t - ev_time[i];
                const int64_t li = L[(int64_t)(k - 1) * n + i];
                if (li != ORC_NEG_INF && l < d && d <= h && li > best) best = li;
            }
            L[(int64_t)k * n + j] = best;
        }
    }

    uint64_t count = 0;
#if ORC_MUTANT == 8
    int64_t prev_e = 0; /* mutant: Algorithm 1's literal prev_e = 0 */
#else
    int64_t prev_e = ORC_NEG_INF; /* R2 */
#endif
    const int64_t *Ls = L + (int64_t)(N - 1) * n;
    for (int64_t j = 0; j < n; ++j) {
        if (Ls[j] == ORC_NEG_INF) continue;
#if ORC_MUTANT == 9
        if (prev_e <= Ls[j]) { /* mutant: non-strict overlap test */
#else
        if (prev_e < Ls[j]) {
#endif
            prev_e = ev_time[j];
            count++;
        }
    }
    free(L);
    return count;
}

/* ------------------------------------------------------------------------ */
/* O3: brute force for tiny inputs.  Every index tuple j_1 < ... < j_N with the
 * right types and all edge constraints is an occurrence with start t_{j_1}
 * and end t_{j_N}.  The largest pairwise non-overlapped subset is found by an
 * exhaustive include/exclude search over occurrences sorted by start; the
 * search state is (next occurrence, largest end included so far), memoised. */
typedef struct {
    int64_t s, e;
} orc_occ;

typedef struct {
    orc_occ *o;
    int64_t m, cap;
    int overflow;
} orc_occ_list;

static void enum_occ(const uint16_t *ev_type, const int32_t *ev_time, int64_t n, int N,
                     const uint16_t *E, const int32_t *lo, const int32_t *hi, int k,
                     int64_t prev_idx, int64_t start, orc_occ_list *out) {
    if (out->overflow) return;
    for (int64_t j = prev_idx + 1; j < n; ++j) {
        if (ev_type[j] != E[k]) continue;
        if (k > 0) {
            const int64_t d = (int64_t)ev_time[j] - ev_time[prev_idx];
            if (!(lo[k - 1] < d && d <= hi[k - 1])) continue;
        }
        const int64_t st = (k == 0) ? ev_time[j] : start;
        if (k == N - 1) {
            if (out->m == out->cap) { out->overflow = 1; return; }
            out->o[out->m].s = st;
            out->o[out->m].e = ev_time[j];
            out->m++;
        } else {
            enum_occ(ev_type, ev_time, n, N, E, lo, hi, k + 1, j, st, out);
        }
    }
}

static int occ_by_start(const void *a, const void *b) {
    const orc_occ *x = (const orc_occ *)a, *y = (const orc_occ *)b;
    if (x->s != y->s) return x->s < y->s ? -1 : 1;
    if (x->e != y->e) return x->e < y->e ? -1 : 1;
    return 0;
}

/* best[i][c]: largest subset of occurrences i..m-1 that can be added when the
 * largest end already included is ends[c] (c = m means nothing included). */
static int64_t brute_best(const orc_occ *o, int64_t m, int64_t i, int64_t c,
                          int64_t *memo) {
    if (i == m) return 0;
    int64_t *slot = &memo[i * (m + 1) + c];
    if (*slot >= 0) return *slot;
    const int64_t maxend = (c == m) ? ORC_NEG_INF : o[c].e;
    int64_t best = brute_best(o, m, i + 1, c, memo); /* exclude occurrence i */
    /* include occurrence i: with starts sorted, it is disjoint from every
     * included one iff it starts after the largest included end */
    if (o[i].s > maxend) {
        const int64_t nc = (c == m || o[i].e > o[c].e) ? i : c;
        const int64_t inc = 1 + brute_best(o, m, i + 1, nc, memo);
        if (inc > best) best = inc;
    }
    *slot = best;
    return best;
}

/* Returns the count, or UINT64_MAX when more than max_occ occurrences exist
 * or allocation fails (the caller must keep the input tiny). */
uint64_t orc_count_brute(const uint16_t *ev_type, const int32_t *ev_time, int64_t n, int N,
                         const uint16_t *E, const int32_t *lo, const int32_t *hi,
                         int64_t max_occ) {
    if (N < 1 || n <= 0) return 0;
    orc_occ_list L = {0};
    L.cap = max_occ;
    L.o = (orc_occ *)malloc((size_t)(max_occ > 0 ? max_occ : 1) * sizeof(orc_occ));
    if (!L.o) return UINT64_MAX;
    enum_occ(ev_type, ev_time, n, N, E, lo, hi, 0, -1, 0, &L);
    if (L.overflow) { free(L.o); return UINT64_MAX; }
    qsort(L.o, (size_t)L.m, sizeof(orc_occ), occ_by_start);
    int64_t *memo = (int64_t *)malloc((size_t)(L.m + 1) * (size_t)(L.m + 1) * sizeof(int64_t));
    if (!memo) { free(L.o); return UINT64_MAX; }
    for (int64_t q = 0; q < (L.m + 1) * (L.m + 1); ++q) memo[q] = -1;
    const int64_t best = brute_best(L.o, L.m, 0, L.m, memo);
    free(memo);
    free(L.o);
    return (uint64_t)best;
}

/* Largest pairwise non-overlapped subset of arbitrary closed intervals
 * [s_i, e_i] (s_i <= e_i), by the same exhaustive search; used to pin
 * Algorithm 1 against the textbook optimum.  The input need not be sorted. */
uint64_t orc_intervals_brute(const int64_t *s, const int64_t *e, int64_t m) {
    orc_occ *o = (orc_occ *)malloc((size_t)(m > 0 ? m : 1) * sizeof(orc_occ));
    if (!o) return UINT64_MAX;
    for (int64_t i = 0; i < m; ++i) { o[i].s = s[i]; o[i].e = e[i]; }
    qsort(o, (size_t)m, sizeof(orc_occ), occ_by_start);
    int64_t *memo = (int64_t *)malloc((size_t)(m + 1) * (size_t)(m + 1) * sizeof(int64_t));
    if (!memo) { free(o); return UINT64_MAX; }
    for (int64_t q = 0; q < (m + 1) * (m + 1); ++q) memo[q] = -1;
    const int64_t best = brute_best(o, m, 0, m, memo);
    free(memo);
    free(o);
    return (uint64_t)best;
}

/* ------------------------------------------------------------------------ */
/* Many candidates at once with O1, one candidate per task on a plain pthread
 * pool (each thread takes every n_threads-th candidate).  Candidates are in
 * CSR form: candidate c has nodes offs[c] .. offs[c+1]-1 and edges
 * offs[c]-c .. offs[c+1]-c-2.  counts[c] receives the count. */
typedef struct {
    const uint16_t *ev_type;
    const int32_t *ev_time;
    int64_t n;
    int64_t n_cand;
    const int64_t *offs;
    const uint16_t *types;
    const int32_t *lo, *hi;
    uint64_t *counts;
    int n_threads, tid;
    int method;
} orc_job;

static void *orc_worker(void *arg) {
    orc_job *J = (orc_job *)arg;
    for (int64_t c = J->tid; c < J->n_cand; c += J->n_threads) {
        const int64_t o = J->offs[c];
        const int N = (int)(J->offs[c + 1] - o);
        const int64_t eo = o - c;
        if (J->method == 1)
            J->counts[c] = orc_count_dp(J->ev_type, J->ev_time, J->n, N, J->types + o,
                                        J->lo + eo, J->hi + eo);
        else
            J->counts[c] = orc_count_fsm(J->ev_type, J->ev_time, J->n, N, J->types + o,
                                         J->lo + eo, J->hi + eo);
    }
    return NULL;
}

/* method 0 = O1 (FSM), 1 = O2 (DP + Algorithm 1).  Returns the number of
 * threads used. */
int orc_count_many(const uint16_t *ev_type, const int32_t *ev_time, int64_t n, int64_t n_cand,
                   const int64_t *offs, const uint16_t *types, const int32_t *lo,
                   const int32_t *hi, uint64_t *counts, int n_threads, int method) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 1024) n_threads = 1024;
    orc_job *jobs = (orc_job *)calloc((size_t)n_threads, sizeof(orc_job));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    for (int i = 0; i < n_threads; ++i) {
        orc_job J = {ev_type, ev_time, n, n_cand, offs, types, lo, hi, counts, n_threads, i, method};
        jobs[i] = J;
    }
    int started = 0;
    for (int i = 1; i < n_threads; ++i) {
        if (pthread_create(&th[i], NULL, orc_worker, &jobs[i]) != 0) break;
        started = i;
    }
    if (started < n_threads - 1) {
        /* could not start every thread: redo the whole job on this thread */
        for (int i = 1; i <= started; ++i) pthread_join(th[i], NULL);
        jobs[0].n_threads = 1;
        orc_worker(&jobs[0]);
        free(jobs); free(th);
        return 1;
    }
    orc_worker(&jobs[0]);
    for (int i = 1; i < n_threads; ++i) pthread_join(th[i], NULL);
    free(jobs);
    free(th);
    return n_threads;
}

/* The oracle's build-time identity, so tests can tell a mutant from the real
 * oracle. */
int orc_mutant_id(void) { return ORC_MUTANT; }
