/*
 * fsp_oracle.c -- plain, slow CPU oracle for the two-machine (Johnson /
 * Lageweg-Lenstra-Rinnooy Kan) lower bound of the permutation flow-shop and
 * for the depth-first branch-and-bound built on it.
 *
 * Source: Melab, Chakroun, Mezmaz, Tuyttens, "A GPU-accelerated
 * Branch-and-Bound Algorithm for the Flow-Shop Scheduling Problem"
 * (arXiv:1208.3933): Section II-B (problem, forward branching), Section II-C
 * (the bound of Lageweg et al. built on Johnson's rule), Section II-D
 * (the six tables PTM, LM, JM, RM, QM, MM and Table I) and the figure
 * "Pseudo-code implementing the LB function".
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library, and the CUDA library never calls it.
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *   - the pair set is every couple (M_k, M_l) with k < l (Section II-D);
 *   - the lag of job j on couple (k,l) is the sum of its processing times on
 *     the machines strictly between k and l (Section II-D, garbled there);
 *   - Johnson's rule with lags: set 1 = {p_jk <= p_jl} in ascending
 *     p_jk + lag_j, then set 2 = {p_jk > p_jl} in descending p_jl + lag_j,
 *     ties broken by job index (Johnson 1954; the paper fixes no tie-break);
 *   - the release time of machine k is max(C(sigma,k), min over unscheduled j
 *     of sum_{h<k} p_jh) and the latency of machine l is min over unscheduled
 *     j of sum_{h>l} p_jh, both minima over the empty set being 0 (the RM and
 *     QM rows of the pseudo-code; the paper computes these minima on the CPU);
 *     fo_lb_ex also offers the tighter per-job reading of RM, the minimum over
 *     unscheduled j of the earliest start of j on machine k after the prefix;
 *   - LB starts at 0 (the pseudo-code's maxInteger start cannot be meant);
 *   - the couple loop, the filtered Johnson scan and the two-machine update
 *     follow the LB pseudo-code of Section II-D in its order.
 *
 * All arithmetic is in int64_t; results are returned as int32_t.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FO_OK 0
#define FO_EINVAL (-1)
#define FO_ENOMEM (-2)
#define FO_EBADNODE (-4)
#define FO_ENOTFOUND (-6)

/* Release-time readings of RM (see fo_lb_ex). */
#define FO_RELEASE_HEADS 0 /* max(C(sigma,k), min_U sum_{h<k} p_jh) */
#define FO_RELEASE_EST 1   /* min_U earliest start of j on k after the prefix */

/* Number of machine couples (k,l), k<l: m(m-1)/2 (Section II-D). */
int fo_num_pairs(int m) { return m * (m - 1) / 2; }

/* One job of one couple, as Johnson's rule sees it. */
typedef struct {
    int set;      /* 1 or 2 */
    int64_t key;  /* set 1: p_jk+lag ascending; set 2: -(p_jl+lag) so ascending */
    int job;
} fo_jitem;

static int fo_jcmp(const void *a, const void *b) {
    const fo_jitem *x = (const fo_jitem *)a, *y = (const fo_jitem *)b;
    if (x->set != y->set) return x->set < y->set ? -1 : 1;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->job != y->job) return x->job < y->job ? -1 : 1;
    return 0;
}

/*
 * Builds the tables of Section II-D for an n x m instance p (row-major
 * [n][m]):
 *   mm [P][2]  the couples (k,l), k<l, in lexicographic order (MM);
 *   lag[P][n]  lag of job j on couple c (LM, stored couple-major);
 *   jm [P][n]  Johnson's order with lags of couple c (JM, couple-major).
 * Computed once per instance, as the paper does.
 */
int fo_tables(int n, int m, const int32_t *p, int32_t *mm, int32_t *lag, int32_t *jm) {
    if (n < 1 || m < 2 || !p || !mm || !lag || !jm) return FO_EINVAL;
    fo_jitem *items = (fo_jitem *)malloc(sizeof(fo_jitem) * (size_t)n);
    if (!items) return FO_ENOMEM;
    int c = 0;
    for (int k = 0; k < m; ++k) {
        for (int l = k + 1; l < m; ++l, ++c) {
            mm[2 * c] = k;
            mm[2 * c + 1] = l;
            for (int j = 0; j < n; ++j) {
                int64_t lg = 0;
                for (int h = k + 1; h < l; ++h) lg += p[j * m + h];
                lag[(size_t)c * n + j] = (int32_t)lg;
                int64_t a = (int64_t)p[j * m + k] + lg; /* time on the first machine */
                int64_t b = (int64_t)p[j * m + l] + lg; /* time on the second machine */
                items[j].job = j;
                if (p[j * m + k] <= p[j * m + l]) {
                    items[j].set = 1;
                    items[j].key = a;
                } else {
                    items[j].set = 2;
                    items[j].key = -b;
                }
            }
            qsort(items, (size_t)n, sizeof(fo_jitem), fo_jcmp);
            for (int i = 0; i < n; ++i) jm[(size_t)c * n + i] = items[i].job;
        }
    }
    free(items);
    return FO_OK;
}

/*
 * Lower bound of one node: prefix row[0..d) of scheduled jobs; the
 * unscheduled set U is every other job.  Returns FO_EBADNODE (and leaves
 * *lb untouched) if d is outside [0,n], a prefix job is outside [0,n) or
 * appears twice.  pair_out, if not NULL, receives the value of every couple
 * (timeOnM2 once the pseudo-code has added the latency of M2).
 */
int fo_lb_ex(int n, int m, const int32_t *p, const int32_t *mm, const int32_t *lag,
             const int32_t *jm, const int16_t *row, int32_t d, int release,
             int64_t *pair_out, int32_t *lb_out) {
    if (d < 0 || d > n) return FO_EBADNODE;
    char *sched = (char *)calloc((size_t)n, 1);
    int64_t *C = (int64_t *)calloc((size_t)m, sizeof(int64_t));
    int64_t *R = (int64_t *)calloc((size_t)m, sizeof(int64_t));
    int64_t *Q = (int64_t *)calloc((size_t)m, sizeof(int64_t));
    if (!sched || !C || !R || !Q) {
        free(sched); free(C); free(R); free(Q);
        return FO_ENOMEM;
    }
    int rc = FO_OK;
    /* Completion times C(sigma,k) of the prefix by the flow-shop recurrence
       (Section II-B: same order on every machine, each machine one job at a
       time, each job through M_1..M_m in order). */
    for (int i = 0; i < d; ++i) {
        int j = row[i];
        if (j < 0 || j >= n || sched[j]) { rc = FO_EBADNODE; break; }
        sched[j] = 1;
        int64_t prev = 0; /* completion of job j on machine k-1 */
        for (int k = 0; k < m; ++k) {
            int64_t start = C[k] > prev ? C[k] : prev;
            C[k] = start + p[j * m + k];
            prev = C[k];
        }
    }
    if (rc == FO_OK) {
        /* RM: release of machine k = max(C(sigma,k), min_{j in U} sum_{h<k} p_jh).
           QM: latency of machine l = min_{j in U} sum_{h>l} p_jh.  Empty U: 0. */
        int nu = n - d;
        if (release == FO_RELEASE_EST && nu > 0) {
            /* RM read as the earliest starting time of each unscheduled job j
               on each machine k after the prefix (Section II-D names RM "the
               matrix of the earliest starting times of jobs", indexed by
               machine and job, and the pseudo-code takes its minimum over j
               when it starts a couple): est_j0 = C(sigma,0),
               est_jk = max(C(sigma,k), est_j,k-1 + p_j,k-1);
               release of machine k = min over U of est_jk. */
            for (int k = 0; k < m; ++k) R[k] = -1;
            for (int j = 0; j < n; ++j) {
                if (sched[j]) continue;
                int64_t est = C[0];
                for (int k = 0; k < m; ++k) {
                    if (k > 0) {
                        int64_t ready = est + p[j * m + k - 1];
                        est = C[k] > ready ? C[k] : ready;
                    }
                    if (R[k] < 0 || est < R[k]) R[k] = est;
                }
            }
        }
        for (int k = 0; k < m; ++k) {
            int64_t mh = 0, mq = 0;
            int first = 1;
            for (int j = 0; j < n; ++j) {
                if (sched[j]) continue;
                int64_t head = 0, tail = 0;
                for (int h = 0; h < k; ++h) head += p[j * m + h];
                for (int h = k + 1; h < m; ++h) tail += p[j * m + h];
                if (first || head < mh) mh = head;
                if (first || tail < mq) mq = tail;
                first = 0;
            }
            if (nu == 0) { mh = 0; mq = 0; }
            if (release != FO_RELEASE_EST || nu == 0) R[k] = C[k] > mh ? C[k] : mh;
            Q[k] = mq;
        }
        /* The couple loop of the LB pseudo-code (Section II-D). */
        int64_t LB = 0;
        int P = fo_num_pairs(m);
        for (int c = 0; c < P; ++c) {
            int M1 = mm[2 * c], M2 = mm[2 * c + 1];
            int64_t t1 = R[M1]; /* timeOnM1 at the couple's start */
            int64_t t2 = R[M2]; /* timeOnM2 at the couple's start */
            for (int i = 0; i < n; ++i) {
                int job = jm[(size_t)c * n + i];
                if (sched[job]) continue; /* only unscheduled jobs */
                t1 = t1 + p[job * m + M1];
                int64_t lg = lag[(size_t)c * n + job];
                if (t2 > t1 + lg)
                    t2 += p[job * m + M2];
                else
                    t2 = t1 + lg + p[job * m + M2];
            }
            t2 += Q[M2];           /* latency of M2 */
            if (pair_out) pair_out[c] = t2;
            if (t2 > LB) LB = t2;  /* max over couples */
        }
        *lb_out = (int32_t)LB;
    }
    free(sched); free(C); free(R); free(Q);
    return rc;
}

/* fo_lb_ex with the release times of the default reading. */
int fo_lb(int n, int m, const int32_t *p, const int32_t *mm, const int32_t *lag,
          const int32_t *jm, const int16_t *row, int32_t d, int64_t *pair_out,
          int32_t *lb_out) {
    return fo_lb_ex(n, m, p, mm, lag, jm, row, d, FO_RELEASE_HEADS, pair_out, lb_out);
}

/* Bounds a pool of N nodes stored as int16 rows [N][n] plus depths [N];
   invalid rows get -1.  Returns the number of invalid rows, or a negative
   error code. */
int64_t fo_lb_pool_ex(int n, int m, const int32_t *p, const int32_t *mm, const int32_t *lag,
                      const int32_t *jm, const int16_t *rows, const int32_t *depths,
                      int64_t N, int release, int32_t *out) {
    int64_t bad = 0;
    for (int64_t x = 0; x < N; ++x) {
        int32_t v = -1;
        int rc = fo_lb_ex(n, m, p, mm, lag, jm, rows + (size_t)x * n, depths[x], release, NULL, &v);
        if (rc == FO_ENOMEM) return FO_ENOMEM;
        if (rc != FO_OK) { v = -1; ++bad; }
        out[x] = v;
    }
    return bad;
}

int64_t fo_lb_pool(int n, int m, const int32_t *p, const int32_t *mm, const int32_t *lag,
                   const int32_t *jm, const int16_t *rows, const int32_t *depths,
                   int64_t N, int32_t *out) {
    return fo_lb_pool_ex(n, m, p, mm, lag, jm, rows, depths, N, FO_RELEASE_HEADS, out);
}

/*
 * Depth-first branch-and-bound (Section II-A operators, Section II-B forward
 * branching: a child appends one unscheduled job to the prefix).
 *   - UB starts at ub0 + 1; there is no incumbent;
 *   - the root is bounded; every child is bounded when generated;
 *   - a popped node with LB >= UB is eliminated;
 *   - a popped leaf (d = n, so LB = its makespan) becomes the incumbent;
 *   - the children of a popped inner node are bounded together, sorted by
 *     (LB, job) ascending and pushed so that the smallest is popped first;
 *     children with LB >= UB are dropped at once.
 * *nodes counts LB evaluations (root included).  Returns FO_ENOTFOUND when no
 * schedule has makespan <= ub0.  `release` picks the reading of RM used by
 * every bound (FO_RELEASE_HEADS or FO_RELEASE_EST, see fo_lb_ex): both give
 * valid bounds, so both searches reach the same optimum; the per-job reading
 * is at least as tight and prunes at least as early.
 * fo_bnb_ex searches only the subtree of the node whose prefix is
 * root[0..root_d) (every schedule that starts with it); root_d = 0 is the
 * whole tree.  The subtrees of all prefixes of one length cover every
 * schedule, so the smallest of their optima is the optimum.
 */
typedef struct {
    int32_t lb;
    int32_t d;
    int16_t *row;
} fo_node;

typedef struct {
    int32_t lb;
    int32_t job;
} fo_child;

static int fo_ccmp(const void *a, const void *b) {
    const fo_child *x = (const fo_child *)a, *y = (const fo_child *)b;
    if (x->lb != y->lb) return x->lb < y->lb ? -1 : 1;
    if (x->job != y->job) return x->job < y->job ? -1 : 1;
    return 0;
}

int fo_bnb_ex(int n, int m, const int32_t *p, int32_t ub0, int release, const int16_t *root,
              int32_t root_d, int16_t *best_perm, int32_t *best_makespan, int64_t *nodes) {
    if (n < 1 || m < 2 || !p) return FO_EINVAL;
    if (release != FO_RELEASE_HEADS && release != FO_RELEASE_EST) return FO_EINVAL;
    if (root_d < 0 || root_d > n || (root_d > 0 && !root)) return FO_EINVAL;
    int P = fo_num_pairs(m);
    int32_t *mm = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)P);
    int32_t *lag = (int32_t *)malloc(sizeof(int32_t) * (size_t)P * n);
    int32_t *jm = (int32_t *)malloc(sizeof(int32_t) * (size_t)P * n);
    /* at most n children per level are alive on the stack, plus the root */
    size_t cap = (size_t)n * (size_t)n + 2;
    fo_node *stack = (fo_node *)malloc(sizeof(fo_node) * cap);
    int16_t *rows = (int16_t *)malloc(sizeof(int16_t) * cap * (size_t)n);
    fo_child *kids = (fo_child *)malloc(sizeof(fo_child) * (size_t)n);
    int16_t *tmp = (int16_t *)malloc(sizeof(int16_t) * (size_t)n);
    char *used = (char *)malloc((size_t)n);
    int rc = FO_OK;
    if (!mm || !lag || !jm || !stack || !rows || !kids || !tmp || !used) { rc = FO_ENOMEM; goto done; }
    rc = fo_tables(n, m, p, mm, lag, jm);
    if (rc != FO_OK) goto done;
    for (size_t s = 0; s < cap; ++s) stack[s].row = rows + s * (size_t)n;

    int64_t UB = (int64_t)ub0 + 1;
    int found = 0;
    int64_t count = 0;
    size_t top = 0;
    int32_t lb = 0;
    /* the search starts at the node of the given prefix (the whole tree for
       root_d = 0); a bad prefix is refused */
    for (int i = 0; i < root_d; ++i) tmp[i] = root[i];
    if (fo_lb_ex(n, m, p, mm, lag, jm, tmp, root_d, release, NULL, &lb) != FO_OK) { rc = FO_EBADNODE; goto done; }
    ++count;
    memcpy(stack[0].row, tmp, sizeof(int16_t) * (size_t)root_d);
    stack[0].lb = lb;
    stack[0].d = root_d;
    top = 1;
    while (top > 0) {
        fo_node *nd = &stack[--top];
        if (nd->lb >= UB) continue;
        if (nd->d == n) {
            UB = nd->lb;
            found = 1;
            if (best_perm) memcpy(best_perm, nd->row, sizeof(int16_t) * (size_t)n);
            continue;
        }
        int d = nd->d;
        memcpy(tmp, nd->row, sizeof(int16_t) * (size_t)d);
        memset(used, 0, (size_t)n);
        for (int i = 0; i < d; ++i) used[tmp[i]] = 1;
        int nk = 0;
        for (int j = 0; j < n; ++j) {
            if (used[j]) continue;
            tmp[d] = (int16_t)j;
            int32_t v = 0;
            fo_lb_ex(n, m, p, mm, lag, jm, tmp, d + 1, release, NULL, &v);
            ++count;
            kids[nk].lb = v;
            kids[nk].job = j;
            ++nk;
        }
        qsort(kids, (size_t)nk, sizeof(fo_child), fo_ccmp);
        /* nd's slot is reused by its children; its prefix is in tmp[0..d) */
        for (int t = nk - 1; t >= 0; --t) {
            if (kids[t].lb >= UB) continue;
            fo_node *c = &stack[top++];
            memcpy(c->row, tmp, sizeof(int16_t) * (size_t)d);
            c->row[d] = (int16_t)kids[t].job;
            c->d = d + 1;
            c->lb = kids[t].lb;
        }
    }
    if (nodes) *nodes = count;
    if (found) {
        if (best_makespan) *best_makespan = (int32_t)UB;
    } else {
        rc = FO_ENOTFOUND;
    }
done:
    free(mm); free(lag); free(jm); free(stack); free(rows); free(kids); free(tmp); free(used);
    return rc;
}

/* fo_bnb_ex with the release times of the default reading. */
int fo_bnb(int n, int m, const int32_t *p, int32_t ub0, int16_t *best_perm,
           int32_t *best_makespan, int64_t *nodes) {
    return fo_bnb_ex(n, m, p, ub0, FO_RELEASE_HEADS, NULL, 0, best_perm, best_makespan, nodes);
}
