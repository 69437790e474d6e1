/*
 * gamegen.c - seeded synthetic two-player game trees ("public tree x private deal").
 *
 * This module only BUILDS INPUTS: it writes the finite extensive-form game
 * <T, H, f_h, A, f_a, I, f_i, sigma_0, u> of the Definition in Section 2.1 as
 * flat arrays (parent, action, infoset, infoset player, infoset action count,
 * chance probabilities, utilities).  It contains none of the CFR arithmetic and
 * is shared by the CUDA path's tests/benchmarks and by the CPU oracle's tests.
 *
 * Construction.  The game root is a chance node that deals one of K outcomes
 * (k -> private bucket b1(k) of player 1, b2(k) of player 2).  Below every deal
 * hangs a copy of one seeded PUBLIC tree.  A public node is a player-1 node, a
 * player-2 node, a public chance node or a terminal.  A decision node of the
 * game is the pair (deal k, public node p); its infoset is keyed by
 * (acting player, that player's own bucket, p).  Every node of an infoset thus
 * shares the public node, so it has the same action count, the same player,
 * the same depth, and the acting player's own history is identical across it
 * (perfect recall).
 *
 * Every random draw comes from splitmix64 applied to (seed, salt, key), where a
 * public node's key hashes its action path.  Generation therefore does not
 * depend on traversal order, and raising p_cont only adds subtrees (the size
 * is monotone in p_cont for a fixed seed, which the size fit relies on).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* splitmix64 finaliser (Steele, Lea, Flood 2014). */
static inline uint64_t mix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
static inline uint64_t draw(uint64_t seed, uint64_t salt, uint64_t a, uint64_t b) {
    return mix64(mix64(mix64(seed ^ (salt * 0xD1B54A32D192ED03ull)) ^ a) ^ (b + 0x632BE59BD9B4E019ull));
}
static inline double unit01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

enum { SALT_NA = 1, SALT_KIND = 2, SALT_CHANCE = 3, SALT_CPROB = 4, SALT_POT = 5, SALT_UTIL = 6,
       SALT_UTIL2 = 7, SALT_DEAL = 8 };

enum { DEAL_BUCKET_PAIRS = 0, DEAL_HOLDEM_169 = 1 };
enum { PAY_UNIFORM = 0, PAY_FOLD_SHOWDOWN = 1 };

typedef struct {
    uint64_t seed;
    int32_t deal_kind;    /* DEAL_BUCKET_PAIRS: ordered pairs of distinct buckets out of num_buckets;
                             DEAL_HOLDEM_169: player 1 holds each of the 1326 two-card combos of a
                             52-card deck, player 2 a seeded disjoint combo; buckets = 169 classes */
    int32_t num_buckets;  /* DEAL_BUCKET_PAIRS only */
    int32_t depth;        /* maximum leaf depth, the root (deal) at depth 0 */
    int32_t amin, amax;   /* action count of a public decision node, uniform in [amin, amax] */
    double p_cont;        /* probability that a child of a public decision node above the last
                             level is itself a decision node */
    double p_chance;      /* probability that a non-root public decision node is a chance node */
    int32_t payoff_kind;  /* PAY_UNIFORM: u1 ~ U[-umax, umax] per (deal, public terminal);
                             PAY_FOLD_SHOWDOWN: +-pot, pot in {1,2,4,8} per public terminal */
    double umax;
    int32_t general_sum;  /* 1: u2 drawn independently instead of u2 = -u1 */
    int32_t first_actor;  /* player to act at the public root: 1 or 2 */
} gg_params;

typedef struct {
    gg_params prm;
    /* deals */
    int32_t K;
    int32_t *b1, *b2;          /* private buckets per deal */
    int32_t *s1, *s2;          /* showdown strength per deal */
    int32_t nb1, nb2;          /* number of bucket ids in use */
    int32_t *rank1, *rank2;    /* bucket -> dense rank among present buckets, -1 if absent */
    int32_t npres1, npres2;
    /* public tree in BFS order; index 0 is the public root (game depth 1) */
    int64_t P;
    int32_t *ppar, *pact, *pactor, *pna, *pdepth, *pinf; /* pactor: -1 terminal, 0 chance, 1, 2 */
    uint64_t *pkey;            /* hash of the action path: keys every draw of the node */
    int32_t *pfold;            /* terminal: folding player (1/2) or 0 for showdown */
    int32_t *ppot;             /* terminal pot */
    int64_t *pcprob_off;       /* chance public node: offset into chance_prob */
    /* totals */
    int64_t num_nodes, num_infosets, num_chance_q, num_public_terminals, num_public_decisions;
} gg_plan;

static int class169(int c1, int c2) {
    int r1 = c1 / 4, r2 = c2 / 4, su1 = c1 % 4, su2 = c2 % 4;
    if (r1 < r2) { int t = r1; r1 = r2; r2 = t; }
    if (r1 == r2) return r1;                          /* 13 pairs: 0..12 */
    int idx = r1 * (r1 - 1) / 2 + r2;                 /* 78 unordered rank pairs: 0..77 */
    return 13 + 2 * idx + (su1 == su2 ? 1 : 0);       /* suited / offsuit: 13..168 */
}

void gg_free_plan(gg_plan *p) {
    if (!p) return;
    free(p->b1); free(p->b2); free(p->s1); free(p->s2); free(p->rank1); free(p->rank2);
    free(p->ppar); free(p->pact); free(p->pactor); free(p->pna); free(p->pdepth); free(p->pinf);
    free(p->pfold); free(p->ppot); free(p->pkey); free(p->pcprob_off);
    free(p);
}

static int build_deals(gg_plan *p) {
    const gg_params *q = &p->prm;
    if (q->deal_kind == DEAL_BUCKET_PAIRS) {
        int nb = q->num_buckets;
        if (nb < 2) return -1;
        p->K = nb * (nb - 1);
        p->nb1 = p->nb2 = nb;
    } else if (q->deal_kind == DEAL_HOLDEM_169) {
        p->K = 1326;
        p->nb1 = p->nb2 = 169;
    } else {
        return -1;
    }
    p->b1 = malloc(sizeof(int32_t) * p->K); p->b2 = malloc(sizeof(int32_t) * p->K);
    p->s1 = malloc(sizeof(int32_t) * p->K); p->s2 = malloc(sizeof(int32_t) * p->K);
    if (!p->b1 || !p->b2 || !p->s1 || !p->s2) return -1;
    int k = 0;
    if (q->deal_kind == DEAL_BUCKET_PAIRS) {
        for (int i = 0; i < q->num_buckets; ++i)
            for (int j = 0; j < q->num_buckets; ++j)
                if (i != j) { p->b1[k] = i; p->b2[k] = j; p->s1[k] = i; p->s2[k] = j; ++k; }
    } else {
        for (int c1 = 0; c1 < 52; ++c1)
            for (int c2 = c1 + 1; c2 < 52; ++c2) {
                int d1, d2;
                for (uint64_t att = 0;; ++att) {      /* uniform disjoint combo by rejection */
                    uint64_t r = draw(q->seed, SALT_DEAL, (uint64_t)k, att);
                    d1 = (int)(r % 52); d2 = (int)((r >> 32) % 52);
                    if (d1 == d2 || d1 == c1 || d1 == c2 || d2 == c1 || d2 == c2) continue;
                    break;
                }
                p->b1[k] = class169(c1, c2); p->b2[k] = class169(d1, d2);
                p->s1[k] = p->b1[k]; p->s2[k] = p->b2[k];
                ++k;
            }
    }
    p->rank1 = malloc(sizeof(int32_t) * p->nb1); p->rank2 = malloc(sizeof(int32_t) * p->nb2);
    if (!p->rank1 || !p->rank2) return -1;
    for (int b = 0; b < p->nb1; ++b) p->rank1[b] = -1;
    for (int b = 0; b < p->nb2; ++b) p->rank2[b] = -1;
    for (k = 0; k < p->K; ++k) { p->rank1[p->b1[k]] = 0; p->rank2[p->b2[k]] = 0; }
    p->npres1 = p->npres2 = 0;
    for (int b = 0; b < p->nb1; ++b) if (p->rank1[b] == 0) p->rank1[b] = p->npres1++;
    for (int b = 0; b < p->nb2; ++b) if (p->rank2[b] == 0) p->rank2[b] = p->npres2++;
    return 0;
}

static int build_public(gg_plan *p) {
    const gg_params *q = &p->prm;
    int64_t cap = 1024, n = 1;
    int32_t *par = malloc(sizeof(int32_t) * cap), *act = malloc(sizeof(int32_t) * cap);
    int32_t *actor = malloc(sizeof(int32_t) * cap), *na = malloc(sizeof(int32_t) * cap);
    int32_t *dep = malloc(sizeof(int32_t) * cap), *tomove = malloc(sizeof(int32_t) * cap);
    uint64_t *key = malloc(sizeof(uint64_t) * cap);
    if (!par || !act || !actor || !na || !dep || !tomove || !key) return -1;
    key[0] = mix64(q->seed ^ 0x5DEECE66Dull);
    par[0] = -1; act[0] = -1; dep[0] = 1; tomove[0] = q->first_actor == 2 ? 2 : 1;
    actor[0] = q->depth >= 2 ? tomove[0] : -1;
    /* BFS: nodes are appended in order, so index order is breadth-first. */
    for (int64_t i = 0; i < n; ++i) {
        na[i] = 0;
        if (actor[i] < 0) continue;
        int span = q->amax - q->amin + 1;
        na[i] = q->amin + (int)(draw(q->seed, SALT_NA, key[i], 0) % (uint64_t)(span > 0 ? span : 1));
        int next_move = actor[i] == 0 ? tomove[i] : 3 - actor[i];
        for (int a = 0; a < na[i]; ++a) {
            if (n == cap) {
                cap *= 2;
                par = realloc(par, sizeof(int32_t) * cap); act = realloc(act, sizeof(int32_t) * cap);
                actor = realloc(actor, sizeof(int32_t) * cap); na = realloc(na, sizeof(int32_t) * cap);
                dep = realloc(dep, sizeof(int32_t) * cap); tomove = realloc(tomove, sizeof(int32_t) * cap);
                key = realloc(key, sizeof(uint64_t) * cap);
                if (!par || !act || !actor || !na || !dep || !tomove || !key) return -1;
            }
            int64_t c = n++;
            par[c] = (int32_t)i; act[c] = a; dep[c] = dep[i] + 1; tomove[c] = next_move;
            key[c] = mix64(key[i] ^ ((uint64_t)(a + 1) * 0x9E3779B97F4A7C15ull));
            int decision = dep[c] < q->depth &&
                           unit01(draw(q->seed, SALT_KIND, key[c], 0)) < q->p_cont;
            if (!decision) actor[c] = -1;
            else if (unit01(draw(q->seed, SALT_CHANCE, key[c], 0)) < q->p_chance) actor[c] = 0;
            else actor[c] = next_move;
        }
        if (n > ((int64_t)1 << 31) - 2) return -1;
    }
    free(tomove);
    p->pkey = key;
    p->P = n; p->ppar = par; p->pact = act; p->pactor = actor; p->pna = na; p->pdepth = dep;
    p->pinf = malloc(sizeof(int32_t) * n); p->pfold = malloc(sizeof(int32_t) * n);
    p->ppot = malloc(sizeof(int32_t) * n); p->pcprob_off = malloc(sizeof(int64_t) * n);
    if (!p->pinf || !p->pfold || !p->ppot || !p->pcprob_off) return -1;
    /* infoset ids: 0 = deal chance; then public BFS order, bucket-rank minor */
    int64_t hid = 1, coff = p->K;
    p->num_public_terminals = 0; p->num_public_decisions = 0;
    for (int64_t i = 0; i < n; ++i) {
        p->pinf[i] = -1; p->pfold[i] = 0; p->ppot[i] = 0; p->pcprob_off[i] = -1;
        if (actor[i] < 0) {
            p->num_public_terminals++;
            static const int pots[4] = {1, 2, 4, 8};
            p->ppot[i] = pots[draw(q->seed, SALT_POT, key[i], 0) % 4];
            int pa = par[i] >= 0 ? actor[par[i]] : 0;
            p->pfold[i] = (dep[i] < q->depth && pa > 0) ? pa : 0;
            continue;
        }
        p->num_public_decisions++;
        p->pinf[i] = (int32_t)hid;
        if (actor[i] == 0) { hid += 1; p->pcprob_off[i] = coff; coff += na[i]; }
        else hid += actor[i] == 1 ? p->npres1 : p->npres2;
    }
    p->num_infosets = hid;
    p->num_chance_q = coff;
    return 0;
}

/* Builds deals and the public tree; returns NULL on bad parameters or if the game has >= 2^31 nodes. */
gg_plan *gg_make_plan(const gg_params *prm) {
    gg_plan *p = calloc(1, sizeof(gg_plan));
    if (!p) return NULL;
    p->prm = *prm;
    if (prm->depth < 1 || prm->amin < 1 || prm->amax < prm->amin || prm->amax > 64) { gg_free_plan(p); return NULL; }
    if (build_deals(p) != 0 || build_public(p) != 0) { gg_free_plan(p); return NULL; }
    p->num_nodes = 1 + (int64_t)p->K * p->P;
    if (p->num_nodes >= ((int64_t)1 << 31) || p->num_infosets >= ((int64_t)1 << 31)) { gg_free_plan(p); return NULL; }
    return p;
}

void gg_plan_counts(const gg_plan *p, int64_t *out /* 7 */) {
    out[0] = p->num_nodes; out[1] = p->num_infosets; out[2] = p->num_chance_q; out[3] = p->K;
    out[4] = p->P; out[5] = p->num_public_decisions; out[6] = p->num_public_terminals;
}

/* Writes the game.  Arrays are caller-allocated: parent/action/infoset [num_nodes],
 * infoset_player/infoset_num_actions [num_infosets], chance_prob [num_chance_q],
 * utility [num_nodes * 2] (row-major, players 1 and 2; zero at decision nodes). */
void gg_fill(const gg_plan *p, int32_t *parent, int32_t *action, int32_t *infoset,
             int8_t *infoset_player, int32_t *infoset_num_actions, double *chance_prob, double *utility) {
    const gg_params *q = &p->prm;
    const int64_t P = p->P;
    /* infoset tables */
    infoset_player[0] = 0; infoset_num_actions[0] = p->K;
    for (int64_t i = 0; i < P; ++i) {
        int a = p->pactor[i];
        if (a < 0) continue;
        int64_t h = p->pinf[i];
        if (a == 0) { infoset_player[h] = 0; infoset_num_actions[h] = p->pna[i]; continue; }
        int np = a == 1 ? p->npres1 : p->npres2;
        for (int r = 0; r < np; ++r) { infoset_player[h + r] = (int8_t)a; infoset_num_actions[h + r] = p->pna[i]; }
    }
    /* chance probabilities: uniform deal, then seeded positive weights per public chance node */
    for (int k = 0; k < p->K; ++k) chance_prob[k] = 1.0 / p->K;
    for (int64_t i = 0; i < P; ++i) {
        if (p->pactor[i] != 0) continue;
        int64_t o = p->pcprob_off[i];
        double s = 0;
        for (int a = 0; a < p->pna[i]; ++a) {
            chance_prob[o + a] = 0.25 + unit01(draw(q->seed, SALT_CPROB, p->pkey[i], (uint64_t)a));
            s += chance_prob[o + a];
        }
        for (int a = 0; a < p->pna[i]; ++a) chance_prob[o + a] /= s;
    }
    parent[0] = -1; action[0] = -1; infoset[0] = 0; utility[0] = 0; utility[1] = 0;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < p->K; ++k) {
        int64_t base = 1 + (int64_t)k * P;
        for (int64_t i = 0; i < P; ++i) {
            int64_t id = base + i;
            parent[id] = i == 0 ? 0 : (int32_t)(base + p->ppar[i]);
            action[id] = i == 0 ? k : p->pact[i];
            int a = p->pactor[i];
            double u1 = 0, u2 = 0;
            if (a < 0) {
                infoset[id] = -1;
                if (q->payoff_kind == PAY_UNIFORM) {
                    u1 = q->umax * (2.0 * unit01(draw(q->seed, SALT_UTIL, (uint64_t)k, p->pkey[i])) - 1.0);
                } else {
                    double pot = p->ppot[i];
                    if (p->pfold[i] == 1) u1 = -pot;
                    else if (p->pfold[i] == 2) u1 = pot;
                    else u1 = p->s1[k] > p->s2[k] ? pot : (p->s1[k] < p->s2[k] ? -pot : 0.0);
                }
                u2 = q->general_sum ? q->umax * (2.0 * unit01(draw(q->seed, SALT_UTIL2, (uint64_t)k, p->pkey[i])) - 1.0)
                                    : -u1;
            } else if (a == 0) {
                infoset[id] = p->pinf[i];
            } else {
                int r = a == 1 ? p->rank1[p->b1[k]] : p->rank2[p->b2[k]];
                infoset[id] = p->pinf[i] + r;
            }
            utility[2 * id] = u1; utility[2 * id + 1] = u2;
        }
    }
}
