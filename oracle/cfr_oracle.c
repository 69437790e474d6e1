/*
 * cfr_oracle.c - TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct FP64 implementation of counterfactual regret
 * minimization written as the textbook recursive tree walk (Zinkevich et al.,
 * which Section 2.3 takes as the definition of CFR).  It is the yardstick the
 * CUDA path is compared against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.  It
 * shares no source, header, table or helper with the CUDA path.
 *
 * What it computes, per iteration T with strategy sigma^T (Section 2.3):
 *   walk(v, ...) returns the node payoffs (u_1(v), u_2(v)) of Eq. 1:
 *     terminal:  u(v, .)
 *     otherwise: sum_a sigma(h, a) * walk(child_a, ...), summed in action order.
 *   It carries the counterfactual reaches pi-check(v, 1), pi-check(v, 2) by the recursion of
 *   Eq. 2 and the own reaches pi-hat(v, 1), pi-hat(v, 2) by the recursion of Eq. 4 (read as the
 *   product of the player's own factors; the printed Eq. 4 recurses on pi-check, a garble).
 *   At a node d of player p in infoset h the instantaneous regret of Eq. 7 collects
 *     inst(h, a) += pi-check(d, p) * (u_p(child_a) - u_p(d))
 *   which, summed over the nodes of h, is pi~(h) * (u~(sigma|h->a, h) - u~(sigma, h))
 *   by Eq. 3 and Eq. 6.  The own reach of the infoset is recorded.
 * End of the iteration:
 *   regrets   R += inst (vanilla; R = T * rbar of Eq. 8)     or R = max(R + inst, 0) (CFR+)
 *   averages  S += w_T * pi_p(h) * sigma^T  (numerator of Eq. 10; w_T = 1, or T for linear averaging)
 *   strategy  sigma^{T+1} = regret matching of R (Eq. 9); chance keeps sigma_0.
 * Readings taken where the paper is silent or ambiguous:
 *   - CFR+ (named in Section 1 only): regret-matching+ clipping, linear averaging w_T = T, no delay.
 *   - Eq. 5 sums the own reach over the nodes of h; under perfect recall every node of h has the
 *     same own reach, so the common factor |h| cancels in Eq. 10 and S stores one node's own reach.
 *   - Eq. 9's "sum of positive regrets = 0" branch is an exact test of the FP64 sum.
 *   - Alternating updates: player 1's pass and update first, then player 2's pass under the new
 *     sigma_1.
 * Variants beyond the paper (its Section 5 calls such reweightings direct in the matrix form):
 *   - Linear CFR: iteration T's instantaneous regret and average-strategy contribution are both
 *     weighted by T:  R += T * inst,  S += T * pi_p(h) * sigma^T.
 *   - Discounted CFR(alpha, beta, gamma) (Brown and Sandholm, 2019), read as: after iteration T's
 *     regret is added, the accumulated regret is scaled by T^alpha / (T^alpha + 1) where it is
 *     positive and by T^beta / (T^beta + 1) elsewhere; iteration T's average-strategy contribution
 *     is weighted by T^gamma:
 *       x = R + inst;  R = x * (x > 0 ? T^a/(T^a+1) : T^b/(T^b+1));  S += T^gamma * pi_p(h) * sigma^T.
 * Best response / exploitability (used in Appendix A for sanity testing; Section 2.2 defines
 * Nash and epsilon-Nash): a best response for player i against a fixed profile picks, at each of
 * i's infosets, argmax_a sum_{d in h} pi_-i(d) V(child_a(d)), where V is the value below with i
 * best responding.  NashConv = sum_i (BR_i - u_i(profile)); exploitability = NashConv / 2.
 * Ties pick the lowest action index.
 *
 * Multi-threaded passes (orc_iterate_mt; OpenMP, used to time the oracle on all host cores): the
 * subtrees below the root's outcomes are walked by separate threads with the same walk.  A node
 * then does not add its Eq. 7 terms into the shared sums; it stores them per edge (and its
 * counterfactual and own reach per node), and afterwards each infoset adds its nodes' stored terms
 * in the order the one-thread walk would have added them (depth-first post-order), so every sum
 * sees the same additions in the same order and the results are bit for bit those of orc_iterate.
 * The end-of-iteration update is independent per infoset and runs in parallel as it is.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n;
    int32_t H;
    int64_t Q;
    int32_t root;
    int64_t *cstart;   /* children of v: child[cstart[v] .. cstart[v+1]) in action order */
    int32_t *child;
    int32_t *infoset;
    int8_t *player;
    int32_t *nact;
    int64_t *qbase;    /* H + 1 */
    int64_t *hstart;   /* nodes of infoset h: hnode[hstart[h] .. hstart[h+1]) */
    int32_t *hnode;
    double *util;      /* n x 2 */
    double *sigma0;    /* Q, chance slots only */
    double *sigma, *R, *S, *inst, *own, *cfsum;   /* cfsum: pi~(h) of Eq. 3 in the last pass */
    int64_t T;
    int record;
    double *rec;       /* n x 6: u1, u2, pi-check 1, pi-check 2, pi-hat 1, pi-hat 2 of the last pass */
    int64_t recall_violations;
    uint8_t *own_seen;
    /* multi-threaded passes: per-edge Eq. 7 terms and per-node reaches of the last pass, and each
     * infoset's nodes in depth-first post-order */
    int mt;
    double *contrib, *cfnode, *ownnode;
    int32_t *hpost;
    /* best-response scratch */
    double *preach, *V;
    int32_t *astar;
    const double *prof;
    int br_player;
} orc;

static void orc_free_all(orc *o) {
    if (!o) return;
    free(o->cstart); free(o->child); free(o->infoset); free(o->player); free(o->nact); free(o->qbase);
    free(o->hstart); free(o->hnode); free(o->util); free(o->sigma0); free(o->sigma); free(o->R); free(o->S);
    free(o->inst); free(o->own); free(o->cfsum); free(o->rec); free(o->own_seen); free(o->preach); free(o->V); free(o->astar);
    free(o->contrib); free(o->cfnode); free(o->ownnode); free(o->hpost);
    free(o);
}

void orc_destroy(orc *o) { orc_free_all(o); }

static void regret_match(orc *o, int32_t h) {
    int64_t qb = o->qbase[h];
    int32_t na = o->nact[h];
    double pos = 0.0;
    for (int32_t a = 0; a < na; ++a) pos += o->R[qb + a] > 0.0 ? o->R[qb + a] : 0.0;
    for (int32_t a = 0; a < na; ++a)
        o->sigma[qb + a] = pos > 0.0 ? (o->R[qb + a] > 0.0 ? o->R[qb + a] : 0.0) / pos : 1.0 / na;
}

/* Returns NULL if the arrays do not describe a tree whose nodes' children biject onto actions. */
orc *orc_create(int64_t n, const int32_t *parent, const int32_t *action, const int32_t *infoset, int32_t H,
                const int8_t *player, const int32_t *nact, const double *chance_prob, const double *utility) {
    orc *o = calloc(1, sizeof(orc));
    if (!o || n < 1 || H < 0) { free(o); return NULL; }
    o->n = n; o->H = H; o->root = -1;
    o->infoset = malloc(sizeof(int32_t) * n); o->util = malloc(sizeof(double) * 2 * n);
    o->player = malloc(H + 1); o->nact = malloc(sizeof(int32_t) * (H + 1));
    o->qbase = malloc(sizeof(int64_t) * (H + 1)); o->cstart = calloc(n + 1, sizeof(int64_t));
    if (!o->infoset || !o->util || !o->player || !o->nact || !o->qbase || !o->cstart) goto bad;
    memcpy(o->infoset, infoset, sizeof(int32_t) * n);
    memcpy(o->util, utility, sizeof(double) * 2 * n);
    memcpy(o->player, player, H);
    memcpy(o->nact, nact, sizeof(int32_t) * H);
    o->qbase[0] = 0;
    for (int32_t h = 0; h < H; ++h) o->qbase[h + 1] = o->qbase[h] + nact[h];
    o->Q = o->qbase[H];
    /* children in action order */
    for (int64_t v = 0; v < n; ++v) {
        if (parent[v] < 0) { if (o->root >= 0) goto bad; o->root = (int32_t)v; continue; }
        if (parent[v] >= n || infoset[parent[v]] < 0) goto bad;
        o->cstart[parent[v] + 1]++;
    }
    if (o->root < 0) goto bad;
    for (int64_t v = 0; v < n; ++v) {
        int32_t h = infoset[v];
        int64_t want = h >= 0 ? (h < H ? nact[h] : -1) : 0;
        if (o->cstart[v + 1] != want) goto bad;
    }
    for (int64_t v = 0; v < n; ++v) o->cstart[v + 1] += o->cstart[v];
    o->child = malloc(sizeof(int32_t) * (o->cstart[n] > 0 ? o->cstart[n] : 1));
    if (!o->child) goto bad;
    for (int64_t i = 0; i < o->cstart[n]; ++i) o->child[i] = -1;
    for (int64_t v = 0; v < n; ++v) {
        if (parent[v] < 0) continue;
        int32_t d = parent[v], a = action[v];
        if (a < 0 || a >= nact[infoset[d]] || o->child[o->cstart[d] + a] != -1) goto bad;
        o->child[o->cstart[d] + a] = (int32_t)v;
    }
    /* nodes per infoset */
    o->hstart = calloc(H + 1, sizeof(int64_t));
    if (!o->hstart) goto bad;
    for (int64_t v = 0; v < n; ++v) if (infoset[v] >= 0) o->hstart[infoset[v] + 1]++;
    for (int32_t h = 0; h < H; ++h) o->hstart[h + 1] += o->hstart[h];
    o->hnode = malloc(sizeof(int32_t) * (o->hstart[H] > 0 ? o->hstart[H] : 1));
    int64_t *fill = malloc(sizeof(int64_t) * (H + 1));
    if (!o->hnode || !fill) { free(fill); goto bad; }
    memcpy(fill, o->hstart, sizeof(int64_t) * (H + 1));
    for (int64_t v = 0; v < n; ++v) if (infoset[v] >= 0) o->hnode[fill[infoset[v]]++] = (int32_t)v;
    free(fill);
    /* strategy state */
    int64_t Q = o->Q > 0 ? o->Q : 1;
    o->sigma0 = calloc(Q, sizeof(double)); o->sigma = calloc(Q, sizeof(double));
    o->R = calloc(Q, sizeof(double)); o->S = calloc(Q, sizeof(double)); o->inst = calloc(Q, sizeof(double));
    o->own = calloc(H + 1, sizeof(double)); o->own_seen = calloc(H + 1, 1); o->cfsum = calloc(H + 1, sizeof(double));
    if (!o->sigma0 || !o->sigma || !o->R || !o->S || !o->inst || !o->own || !o->own_seen || !o->cfsum) goto bad;
    int64_t c = 0;
    for (int32_t h = 0; h < H; ++h) {
        if (player[h] == 0)
            for (int32_t a = 0; a < nact[h]; ++a) o->sigma0[o->qbase[h] + a] = chance_prob[c++];
    }
    for (int32_t h = 0; h < H; ++h) {
        if (player[h] == 0) memcpy(o->sigma + o->qbase[h], o->sigma0 + o->qbase[h], sizeof(double) * nact[h]);
        else regret_match(o, h);                      /* R = 0: uniform sigma^1 */
    }
    return o;
bad:
    orc_free_all(o);
    return NULL;
}

int64_t orc_num_q(const orc *o) { return o->Q; }
int32_t orc_root(const orc *o) { return o->root; }

void orc_set_record(orc *o, int32_t on) {
    o->record = on;
    if (on && !o->rec) o->rec = calloc((size_t)o->n * 6, sizeof(double));
}

/* One recursive pass; players whose bit is set in `mask` collect regrets and own reach.
 * cf1, cf2: counterfactual reaches pi-check(v, 1), pi-check(v, 2) of Eq. 2, formed by its
 * recursion (the parent's value times sigma of the edge unless that player acted there);
 * own1, own2: own reaches pi-hat(v, 1), pi-hat(v, 2) of Eq. 4 (the parent's value times sigma of
 * the edge when that player acted there). */
static void walk(orc *o, int32_t v, double cf1, double cf2, double own1, double own2, int mask, double out[2]);

/* The walk below child a of v (player p of v acting with probability s on that edge). */
static void walk_child(orc *o, int32_t v, int32_t a, int p, double s, double cf1, double cf2, double own1,
                       double own2, int mask, double out[2]) {
    int32_t c = o->child[o->cstart[v] + a];
    if (p == 0) walk(o, c, cf1 * s, cf2 * s, own1, own2, mask, out);
    else if (p == 1) walk(o, c, cf1, cf2 * s, own1 * s, own2, mask, out);
    else walk(o, c, cf1 * s, cf2, own1, own2 * s, mask, out);
}

static void walk(orc *o, int32_t v, double cf1, double cf2, double own1, double own2, int mask, double out[2]) {
    if (o->record) {
        double *r = o->rec + (size_t)v * 6;
        r[2] = cf1; r[3] = cf2; r[4] = own1; r[5] = own2;
    }
    int32_t h = o->infoset[v];
    if (h < 0) {
        out[0] = o->util[2 * (size_t)v]; out[1] = o->util[2 * (size_t)v + 1];
    } else {
        int p = o->player[h];
        int32_t na = o->nact[h];
        int64_t qb = o->qbase[h];
        double ua[2 * na];
        double u[2] = {0.0, 0.0};
        if (o->mt && v == o->root) {
            /* multi-threaded pass: the subtrees below the root's outcomes on separate threads */
#pragma omp parallel for schedule(dynamic, 1)
            for (int32_t a = 0; a < na; ++a)
                walk_child(o, v, a, p, o->sigma[qb + a], cf1, cf2, own1, own2, mask, ua + 2 * a);
        } else {
            for (int32_t a = 0; a < na; ++a)
                walk_child(o, v, a, p, o->sigma[qb + a], cf1, cf2, own1, own2, mask, ua + 2 * a);
        }
        for (int32_t a = 0; a < na; ++a) {
            double s = o->sigma[qb + a];
            u[0] += s * ua[2 * a];
            u[1] += s * ua[2 * a + 1];
        }
        if (p > 0 && (mask & (1 << p))) {
            double cf = p == 1 ? cf1 : cf2;
            double mine = p == 1 ? own1 : own2;
            if (o->mt) {
                /* stored per edge and node; summed per infoset after the pass (reduce_infosets) */
                for (int32_t a = 0; a < na; ++a) o->contrib[o->cstart[v] + a] = cf * (ua[2 * a + p - 1] - u[p - 1]);
                o->cfnode[v] = cf;
                o->ownnode[v] = mine;
            } else {
                for (int32_t a = 0; a < na; ++a) o->inst[qb + a] += cf * (ua[2 * a + p - 1] - u[p - 1]);
                o->cfsum[h] += cf;
                if (o->own_seen[h] && fabs(o->own[h] - mine) > 1e-12 * (fabs(mine) + 1e-300)) o->recall_violations++;
                o->own[h] = mine;
                o->own_seen[h] = 1;
            }
        }
        out[0] = u[0]; out[1] = u[1];
    }
    if (o->record) {
        double *r = o->rec + (size_t)v * 6;
        r[0] = out[0]; r[1] = out[1];
    }
}

static void reduce_infosets(orc *o, int mask);

static void pass(orc *o, int mask, double root_value[2]) {
#pragma omp parallel for schedule(static) if (o->mt)
    for (int32_t h = 0; h < o->H; ++h) {
        if (o->player[h] > 0 && (mask & (1 << o->player[h]))) {
            for (int32_t a = 0; a < o->nact[h]; ++a) o->inst[o->qbase[h] + a] = 0.0;
            o->own[h] = 0.0;
            o->cfsum[h] = 0.0;
            o->own_seen[h] = 0;
        }
    }
    walk(o, o->root, 1.0, 1.0, 1.0, 1.0, mask, root_value);
    if (o->mt) reduce_infosets(o, mask);
}

/* Depth-first post-order number of every node below v (children in action order): the order in
 * which the one-thread walk finishes nodes, and so adds their Eq. 7 terms. */
static void number_post(const orc *o, int32_t v, int64_t *pos, int64_t *next) {
    int32_t h = o->infoset[v];
    if (h >= 0)
        for (int32_t a = 0; a < o->nact[h]; ++a) number_post(o, o->child[o->cstart[v] + a], pos, next);
    pos[v] = (*next)++;
}

static const int64_t *g_sort_pos;
static int by_post(const void *x, const void *y) {
    int64_t a = g_sort_pos[*(const int32_t *)x], b = g_sort_pos[*(const int32_t *)y];
    return a < b ? -1 : a > b;
}

/* Work arrays of the multi-threaded passes; 0 on success. */
static int mt_prepare(orc *o) {
    if (o->hpost) return 0;
    o->contrib = malloc(sizeof(double) * (o->cstart[o->n] > 0 ? o->cstart[o->n] : 1));
    o->cfnode = malloc(sizeof(double) * o->n);
    o->ownnode = malloc(sizeof(double) * o->n);
    int64_t *pos = malloc(sizeof(int64_t) * o->n);
    int32_t *hp = malloc(sizeof(int32_t) * (o->hstart[o->H] > 0 ? o->hstart[o->H] : 1));
    if (!o->contrib || !o->cfnode || !o->ownnode || !pos || !hp) { free(pos); free(hp); return -1; }
    int64_t next = 0;
    number_post(o, o->root, pos, &next);
    memcpy(hp, o->hnode, sizeof(int32_t) * o->hstart[o->H]);
    g_sort_pos = pos;
    for (int32_t h = 0; h < o->H; ++h)
        qsort(hp + o->hstart[h], (size_t)(o->hstart[h + 1] - o->hstart[h]), sizeof(int32_t), by_post);
    free(pos);
    o->hpost = hp;
    return 0;
}

/* After a multi-threaded pass: each collecting infoset adds its nodes' stored terms, counterfactual
 * reaches and own reaches in post-order, as the one-thread walk does. */
static void reduce_infosets(orc *o, int mask) {
    int64_t viol = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : viol)
    for (int32_t h = 0; h < o->H; ++h) {
        int p = o->player[h];
        if (p == 0 || !(mask & (1 << p))) continue;
        int64_t qb = o->qbase[h];
        int32_t na = o->nact[h];
        for (int64_t i = o->hstart[h]; i < o->hstart[h + 1]; ++i) {
            int32_t v = o->hpost[i];
            for (int32_t a = 0; a < na; ++a) o->inst[qb + a] += o->contrib[o->cstart[v] + a];
            o->cfsum[h] += o->cfnode[v];
            double mine = o->ownnode[v];
            if (o->own_seen[h] && fabs(o->own[h] - mine) > 1e-12 * (fabs(mine) + 1e-300)) viol++;
            o->own[h] = mine;
            o->own_seen[h] = 1;
        }
    }
    o->recall_violations += viol;
}

/* variant: 0 vanilla, 1 CFR+, 2 linear CFR, 3 discounted CFR with dcfr = {alpha, beta, gamma}. */
static void update(orc *o, int mask, int variant, int avg, const double *dcfr, int64_t T) {
    const double t = (double)T;
    double w = avg == 1 ? t : 1.0;
    double fpos = 1.0, fneg = 1.0;
    if (variant == 2) w = t;
    if (variant == 3) {
        const double ta = pow(t, dcfr[0]), tb = pow(t, dcfr[1]);
        fpos = ta / (ta + 1.0);
        fneg = tb / (tb + 1.0);
        w = pow(t, dcfr[2]);
    }
    /* independent per infoset; in parallel in a multi-threaded pass */
#pragma omp parallel for schedule(static) if (o->mt)
    for (int32_t h = 0; h < o->H; ++h) {
        int p = o->player[h];
        if (p == 0 || !(mask & (1 << p))) continue;
        int64_t qb = o->qbase[h];
        for (int32_t a = 0; a < o->nact[h]; ++a) {
            const double in = o->inst[qb + a];
            if (variant == 2) {
                o->R[qb + a] = o->R[qb + a] + t * in;
            } else if (variant == 3) {
                const double x = o->R[qb + a] + in;
                o->R[qb + a] = x * (x > 0.0 ? fpos : fneg);
            } else {
                double r = o->R[qb + a] + in;
                o->R[qb + a] = variant == 1 ? (r > 0.0 ? r : 0.0) : r;
            }
            o->S[qb + a] += w * o->own[h] * o->sigma[qb + a];
        }
        regret_match(o, h);
    }
}

/* variant: 0 vanilla CFR, 1 CFR+, 2 linear CFR, 3 discounted CFR (dcfr = {alpha, beta, gamma}, may be
 * NULL otherwise);  avg: 0 uniform weights, 1 linear (w_T = T), ignored by variants 2 and 3;
 * alternating: 0/1. */
void orc_iterate(orc *o, int32_t iters, int32_t variant, int32_t avg, int32_t alternating, const double *dcfr,
                 double *root_value) {
    double rv[2] = {0.0, 0.0};
    for (int32_t it = 0; it < iters; ++it) {
        int64_t T = o->T + 1;
        if (!alternating) {
            pass(o, 6, rv);
            update(o, 6, variant, avg, dcfr, T);
        } else {
            pass(o, 2, rv);
            update(o, 2, variant, avg, dcfr, T);
            pass(o, 4, rv);
            update(o, 4, variant, avg, dcfr, T);
        }
        o->T = T;
    }
    if (root_value) { root_value[0] = rv[0]; root_value[1] = rv[1]; }
}

/* orc_iterate with each pass on `threads` host threads (<= 0: all of them), bit-identical to it.
 * Returns the thread count used, or -1 if the work arrays could not be allocated. */
int32_t orc_iterate_mt(orc *o, int32_t iters, int32_t variant, int32_t avg, int32_t alternating, const double *dcfr,
                       double *root_value, int32_t threads) {
    if (mt_prepare(o) != 0) return -1;
    int32_t used = 1;
#ifdef _OPENMP
    used = threads > 0 ? threads : omp_get_max_threads();
    const int before = omp_get_max_threads();
    omp_set_num_threads(used);
#else
    (void)threads;
#endif
    o->mt = 1;
    orc_iterate(o, iters, variant, avg, alternating, dcfr, root_value);
    o->mt = 0;
#ifdef _OPENMP
    omp_set_num_threads(before);
#endif
    return used;
}

/* Host threads a multi-threaded pass uses by default (1 without OpenMP). */
int32_t orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* pi~(h) of Eq. 3 (sum of the counterfactual reaches of h's nodes) from the last pass. */
void orc_get_cf_reach_sum(const orc *o, double *out) { memcpy(out, o->cfsum, sizeof(double) * o->H); }

void orc_get_state(const orc *o, double *R, double *S, double *inst, double *sigma, double *own, int64_t *T) {
    if (R) memcpy(R, o->R, sizeof(double) * o->Q);
    if (S) memcpy(S, o->S, sizeof(double) * o->Q);
    if (inst) memcpy(inst, o->inst, sizeof(double) * o->Q);
    if (sigma) memcpy(sigma, o->sigma, sizeof(double) * o->Q);
    if (own) memcpy(own, o->own, sizeof(double) * o->H);
    if (T) *T = o->T;
}

/* Sets cumulative regrets, strategy sums and the iteration count; sigma := regret matching of R. */
void orc_set_state(orc *o, const double *R, const double *S, int64_t T) {
    memcpy(o->R, R, sizeof(double) * o->Q);
    memcpy(o->S, S, sizeof(double) * o->Q);
    o->T = T;
    for (int32_t h = 0; h < o->H; ++h) if (o->player[h] > 0) regret_match(o, h);
}

/* Per node of the last pass: u1, u2, pi-check 1, pi-check 2, pi-hat 1, pi-hat 2
 * (needs orc_set_record(o, 1) before the pass). */
int32_t orc_get_nodes(const orc *o, double *out) {
    if (!o->rec) return -1;
    memcpy(out, o->rec, sizeof(double) * 6 * (size_t)o->n);
    return 0;
}

int64_t orc_recall_violations(const orc *o) { return o->recall_violations; }

/* Average strategy (Eq. 10 normalised): S / sum_a S per player infoset, uniform if the sum is 0. */
void orc_average_strategy(const orc *o, double *out) {
    for (int32_t h = 0; h < o->H; ++h) {
        int64_t qb = o->qbase[h];
        int32_t na = o->nact[h];
        if (o->player[h] == 0) { memcpy(out + qb, o->sigma0 + qb, sizeof(double) * na); continue; }
        double s = 0.0;
        for (int32_t a = 0; a < na; ++a) s += o->S[qb + a];
        for (int32_t a = 0; a < na; ++a) out[qb + a] = s > 0.0 ? o->S[qb + a] / s : 1.0 / na;
    }
}

/* ---- best response ------------------------------------------------------------------------- */

static double prob(const orc *o, int32_t v, int32_t a) {
    int32_t h = o->infoset[v];
    int64_t q = o->qbase[h] + a;
    return o->player[h] == 0 ? o->sigma0[q] : o->prof[q];
}

static void opp_reach(orc *o, int32_t v, double r) {
    o->preach[v] = r;
    int32_t h = o->infoset[v];
    if (h < 0) return;
    for (int32_t a = 0; a < o->nact[h]; ++a)
        opp_reach(o, o->child[o->cstart[v] + a], o->player[h] == o->br_player ? r : r * prob(o, v, a));
}

static double br_value(orc *o, int32_t v);

static void choose(orc *o, int32_t h) {
    int32_t na = o->nact[h];
    double *acc = calloc(na, sizeof(double));
    for (int64_t i = o->hstart[h]; i < o->hstart[h + 1]; ++i) {
        int32_t d = o->hnode[i];
        for (int32_t a = 0; a < na; ++a) acc[a] += o->preach[d] * br_value(o, o->child[o->cstart[d] + a]);
    }
    int32_t best = 0;
    for (int32_t a = 1; a < na; ++a) if (acc[a] > acc[best]) best = a;
    o->astar[h] = best;
    free(acc);
}

static double br_value(orc *o, int32_t v) {
    if (!isnan(o->V[v])) return o->V[v];
    int32_t h = o->infoset[v];
    double val = 0.0;
    if (h < 0) {
        val = o->util[2 * (size_t)v + o->br_player - 1];
    } else if (o->player[h] == o->br_player) {
        if (o->astar[h] < 0) choose(o, h);
        val = br_value(o, o->child[o->cstart[v] + o->astar[h]]);
    } else {
        for (int32_t a = 0; a < o->nact[h]; ++a) val += prob(o, v, a) * br_value(o, o->child[o->cstart[v] + a]);
    }
    o->V[v] = val;
    return val;
}

/* Value to `player` (1 or 2) of a best response against profile `prof` (Q entries; chance slots ignored).
 * If `choice` is non-NULL it receives the chosen action per infoset of `player` (-1 elsewhere). */
double orc_best_response(orc *o, int32_t player, const double *prof, int32_t *choice) {
    if (!o->preach) {
        o->preach = malloc(sizeof(double) * o->n); o->V = malloc(sizeof(double) * o->n);
        o->astar = malloc(sizeof(int32_t) * (o->H + 1));
    }
    o->prof = prof; o->br_player = player;
    for (int64_t v = 0; v < o->n; ++v) o->V[v] = NAN;
    for (int32_t h = 0; h < o->H; ++h) o->astar[h] = -1;
    opp_reach(o, o->root, 1.0);
    double val = br_value(o, o->root);
    if (choice) {
        for (int32_t h = 0; h < o->H; ++h) {
            if (o->player[h] == player && o->astar[h] < 0) choose(o, h);   /* unreached infosets too */
            choice[h] = o->player[h] == player ? o->astar[h] : -1;
        }
    }
    return val;
}

static double ev(const orc *o, int32_t v, int32_t player) {
    int32_t h = o->infoset[v];
    if (h < 0) return o->util[2 * (size_t)v + player - 1];
    double val = 0.0;
    for (int32_t a = 0; a < o->nact[h]; ++a) val += prob(o, v, a) * ev(o, o->child[o->cstart[v] + a], player);
    return val;
}

/* Expected payoff of `player` under profile `prof` (the expected payoff of Section 2.2). */
double orc_expected_value(orc *o, int32_t player, const double *prof) {
    o->prof = prof;
    return ev(o, o->root, player);
}

/* NashConv = sum_i (BR_i - u_i(prof)); exploitability = NashConv / 2. */
void orc_exploitability(orc *o, const double *prof, double *nash_conv, double *expl) {
    double nc = 0.0;
    for (int32_t i = 1; i <= 2; ++i) {
        double br = orc_best_response(o, i, prof, NULL);
        nc += br - orc_expected_value(o, i, prof);
    }
    if (nash_conv) *nash_conv = nc;
    if (expl) *expl = nc / 2.0;
}
