// Validation of a game description (Definition in Section 2.1) and construction of the
// level-ordered layout described in layout.hpp.  Host code only; no CUDA calls.
#include "layout.hpp"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <limits>

namespace cfrgb {
namespace {

cfr_status fail(std::string *err, cfr_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (err) *err = buf;
    return st;
}

}  // namespace

cfr_status build_layout(const cfr_game_desc *g, Layout *out, std::string *err, bool infoset_lists, bool forest) {
    if (!g) return fail(err, CFR_ERR_INVALID, "game description is NULL");
    const int64_t n = g->num_nodes;
    if (n < 1) return fail(err, CFR_ERR_INVALID, "num_nodes must be >= 1 (got %lld)", (long long)n);
    if (n >= (int64_t)std::numeric_limits<int32_t>::max())
        return fail(err, CFR_ERR_UNSUPPORTED, "num_nodes must be < 2^31 - 1 (got %lld)", (long long)n);
    if (!g->parent || !g->action || !g->infoset || !g->utility)
        return fail(err, CFR_ERR_INVALID, "parent, action, infoset and utility must be non-NULL");
    const int32_t H = g->num_infosets;
    if (H < 0) return fail(err, CFR_ERR_INVALID, "num_infosets must be >= 0");
    if (H > 0 && (!g->infoset_player || !g->infoset_num_actions))
        return fail(err, CFR_ERR_INVALID, "infoset_player and infoset_num_actions must be non-NULL");

    // ---- infoset tables ------------------------------------------------------------------
    std::vector<int64_t> qbase_user((size_t)H + 1, 0), coff((size_t)H, -1);
    int64_t nchance = 0;
    int32_t max_actions = 0;
    for (int32_t h = 0; h < H; ++h) {
        const int p = g->infoset_player[h];
        const int32_t na = g->infoset_num_actions[h];
        if (p < 0 || p > 2) return fail(err, CFR_ERR_INVALID, "infoset %d: player %d not in {0,1,2}", h, p);
        if (na < 1) return fail(err, CFR_ERR_INVALID, "infoset %d: %d actions (need >= 1)", h, na);
        if (na > max_actions) max_actions = na;
        qbase_user[h + 1] = qbase_user[h] + na;
        if (p == 0) { coff[h] = nchance; nchance += na; }
    }
    const int64_t Q = qbase_user[H];
    if (Q >= (int64_t)std::numeric_limits<int32_t>::max())
        return fail(err, CFR_ERR_UNSUPPORTED, "too many infoset-action pairs (%lld)", (long long)Q);
    if (g->num_chance_prob != nchance)
        return fail(err, CFR_ERR_INVALID, "num_chance_prob is %lld but chance infosets have %lld actions",
                    (long long)g->num_chance_prob, (long long)nchance);
    if (nchance > 0 && !g->chance_prob) return fail(err, CFR_ERR_INVALID, "chance_prob is NULL");
    for (int32_t h = 0; h < H; ++h) {
        if (g->infoset_player[h] != 0) continue;
        double s = 0.0;
        for (int32_t a = 0; a < g->infoset_num_actions[h]; ++a) {
            const double pr = g->chance_prob[coff[h] + a];
            if (!(pr >= 0.0) || !std::isfinite(pr))
                return fail(err, CFR_ERR_INVALID, "chance infoset %d action %d: probability %g", h, a, pr);
            s += pr;
        }
        if (std::fabs(s - 1.0) > 1e-9)
            return fail(err, CFR_ERR_INVALID, "chance infoset %d: probabilities sum to %.17g, not 1", h, s);
    }

    // ---- nodes: one root (a forest: any number), ids in range, children a bijection onto actions ----
    std::vector<int32_t> roots;
    for (int64_t v = 0; v < n; ++v) {
        const int32_t par = g->parent[v];
        if (par == -1) {
            if (!roots.empty() && !forest)
                return fail(err, CFR_ERR_INVALID, "two roots: nodes %d and %lld", roots[0], (long long)v);
            roots.push_back((int32_t)v);
        } else if (par < 0 || par >= n) {
            return fail(err, CFR_ERR_INVALID, "node %lld: parent %d out of range", (long long)v, par);
        }
        const int32_t hv = g->infoset[v];
        if (hv < -1 || hv >= H) return fail(err, CFR_ERR_INVALID, "node %lld: infoset %d out of range", (long long)v, hv);
    }
    if (roots.empty()) return fail(err, CFR_ERR_INVALID, "no root (no node with parent -1)");
    std::vector<int32_t> cstart((size_t)n + 1, 0);
    for (int64_t v = 0; v < n; ++v) {
        if (g->parent[v] == -1) continue;
        const int32_t par = g->parent[v];
        if (g->infoset[par] < 0)
            return fail(err, CFR_ERR_INVALID, "node %lld: parent %d is a terminal (infoset -1)", (long long)v, par);
        cstart[(size_t)par + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) {
        const int32_t hv = g->infoset[v];
        const int32_t want = hv >= 0 ? g->infoset_num_actions[hv] : 0;
        if (cstart[(size_t)v + 1] != want)
            return fail(err, CFR_ERR_INVALID, "node %lld has %d children but its infoset %d has %d actions",
                        (long long)v, cstart[(size_t)v + 1], hv, want);
    }
    for (int64_t v = 0; v < n; ++v) cstart[(size_t)v + 1] += cstart[(size_t)v];
    std::vector<int32_t> child((size_t)n, -1);
    for (int64_t v = 0; v < n; ++v) {
        if (g->parent[v] == -1) continue;
        const int32_t par = g->parent[v];
        const int32_t a = g->action[v];
        if (a < 0 || a >= g->infoset_num_actions[g->infoset[par]])
            return fail(err, CFR_ERR_INVALID, "node %lld: action %d out of range for its parent", (long long)v, a);
        int32_t &slot = child[(size_t)cstart[par] + a];
        if (slot != -1)
            return fail(err, CFR_ERR_INVALID, "nodes %d and %lld: same action %d under parent %d", slot, (long long)v, a, par);
        slot = (int32_t)v;
    }
    bool zero_sum = true;
    for (int64_t v = 0; v < n; ++v) {
        if (g->infoset[v] >= 0) continue;
        const double u1 = g->utility[2 * v], u2 = g->utility[2 * v + 1];
        if (!std::isfinite(u1) || !std::isfinite(u2))
            return fail(err, CFR_ERR_INVALID, "terminal %lld: non-finite utility", (long long)v);
        if (std::fabs(u1 + u2) > 1e-12 * std::fmax(1.0, std::fmax(std::fabs(u1), std::fabs(u2)))) zero_sum = false;
    }

    // ---- breadth-first pass: connectivity, perfect recall, level-ordered ids -----------------
    Layout tmp;
    Layout &Lo = out ? *out : tmp;
    Lo = Layout();
    Lo.N = n; Lo.H = H; Lo.Q = Q; Lo.max_actions = max_actions;
    std::vector<int32_t> order((size_t)n);
    std::vector<int32_t> seq1((size_t)n, -1), seq2((size_t)n, -1);   // last own (h, a) slot of players 1, 2
    std::vector<int64_t> rep((size_t)H, -2);                         // own history shared by the infoset
    std::vector<int32_t> hmap((size_t)H, -1), hlvl((size_t)H, -1);
    const bool build = out != nullptr;
    if (build) {
        int64_t ndec = 0;
        for (int64_t v = 0; v < n; ++v) ndec += g->infoset[v] >= 0;
        Lo.dfirst.reserve((size_t)ndec + 1); Lo.tfirst.reserve((size_t)ndec + 1); Lo.dinfo.reserve((size_t)ndec);
        Lo.kmask.reserve((size_t)ndec); Lo.dnode_user.reserve((size_t)ndec);
        Lo.tnode_user.reserve((size_t)(n - ndec)); Lo.util.reserve((size_t)(n - ndec));
    }
    int64_t head = 0, tail = 0;
    int64_t nd_proc = 0, dq = 0, tq = 0;     // decision nodes processed; decision/terminal nodes enqueued
    int32_t Hp = 0;                          // player infosets take internal ids [0, Hp), chance ones [Hp, H)
    for (int32_t h = 0; h < H; ++h) Hp += g->infoset_player[h] > 0;
    int32_t nh = 0, nhc = 0, depth = 0;
    for (int32_t r : roots) {                // depth 0: the roots in id order
        order[(size_t)tail++] = r;
        if (g->infoset[r] >= 0) {
            ++dq;
            if (build) Lo.dnode_user.push_back(r);
        } else {
            ++tq;
            if (build) { Lo.tnode_user.push_back(r); Lo.util.push_back(g->utility[2 * (size_t)r]); }
        }
    }
    bool single_level = true;
    while (head < tail) {
        const int64_t end = tail;
        bool level_has_decision = false;
        for (int64_t i = head; i < end; ++i) {
            const int32_t v = order[(size_t)i];
            const int32_t hu = g->infoset[v];
            if (hu < 0) continue;
            if (!level_has_decision) {
                level_has_decision = true;
                if (build) {
                    Lo.dlevel.push_back((int32_t)nd_proc);
                    Lo.hlevel.push_back(nh);
                    Lo.wlevel.push_back((int32_t)Lo.wide.size());
                }
            }
            const int p = g->infoset_player[hu];
            if (p > 0) {
                const int64_t s = p == 1 ? seq1[v] : seq2[v];
                if (rep[hu] == -2) rep[hu] = s;
                else if (rep[hu] != s)
                    return fail(err, CFR_ERR_INVALID,
                                "imperfect recall: infoset %d holds nodes with different own histories of player %d "
                                "(e.g. node %d)", hu, p, v);
            }
            if (hmap[hu] < 0) { hmap[hu] = p > 0 ? nh++ : Hp + nhc++; hlvl[hu] = depth; }
            else if (hlvl[hu] != depth) single_level = false;
            const int32_t na = g->infoset_num_actions[hu];
            if (build && na > 32) Lo.wide.push_back((int32_t)nd_proc);
            uint32_t mask = 0;
            size_t woff = 0;
            if (build && na > 32) {
                woff = Lo.wbits.size();
                Lo.wbits.resize(woff + (size_t)(na + 31) / 32, 0u);
            }
            if (build) {
                Lo.dfirst.push_back((int32_t)dq);
                Lo.tfirst.push_back((int32_t)tq);
                Lo.dinfo.push_back(hmap[hu]);
            }
            for (int32_t a = 0; a < na; ++a) {
                const int32_t c = child[(size_t)cstart[v] + a];
                order[(size_t)tail++] = c;
                const int32_t q = (int32_t)(qbase_user[hu] + a);
                seq1[c] = p == 1 ? q : seq1[v];
                seq2[c] = p == 2 ? q : seq2[v];
                if (g->infoset[c] >= 0) {
                    if (build) Lo.dnode_user.push_back(c);
                    ++dq;
                } else {
                    if (na > 32) { if (build) Lo.wbits[woff + (size_t)a / 32] |= 1u << (a % 32); }
                    else mask |= 1u << a;
                    if (build) { Lo.tnode_user.push_back(c); Lo.util.push_back(g->utility[2 * (size_t)c]); }
                    ++tq;
                }
            }
            if (build) {
                if (na > 32 && woff > (size_t)std::numeric_limits<uint32_t>::max())
                    return fail(err, CFR_ERR_UNSUPPORTED, "too many wide nodes");
                Lo.kmask.push_back(na > 32 ? (uint32_t)woff : mask);
            }
            ++nd_proc;
        }
        head = end;
        if (tail > head) ++depth;
    }
    if (tail != n)
        return fail(err, CFR_ERR_INVALID, "only %lld of %lld nodes are reachable from the root (cycle or forest)",
                    (long long)tail, (long long)n);
    if (!zero_sum)
        return fail(err, CFR_ERR_UNSUPPORTED, "utilities are not zero-sum (u1 + u2 != 0 at some terminal)");
    if (!build) return CFR_OK;

    Lo.Nd = dq; Lo.Nt = tq;
    Lo.L = (int32_t)Lo.dlevel.size();
    Lo.max_depth = depth;
    Lo.single_level = single_level;
    Lo.dlevel.push_back((int32_t)Lo.Nd);
    Lo.hlevel.push_back(nh);
    Lo.wlevel.push_back((int32_t)Lo.wide.size());
    Lo.dfirst.push_back((int32_t)Lo.Nd);
    Lo.tfirst.push_back((int32_t)Lo.Nt);
    Lo.Hp = Hp;
    // infosets without nodes follow the others of their kind
    for (int32_t h = 0; h < H; ++h)
        if (hmap[h] < 0) hmap[h] = g->infoset_player[h] > 0 ? nh++ : Hp + nhc++;
    Lo.h_int2user.assign((size_t)H, 0);
    for (int32_t h = 0; h < H; ++h) Lo.h_int2user[(size_t)hmap[h]] = h;
    Lo.qbase.assign((size_t)H + 1, 0);
    Lo.iplayer.assign((size_t)H, 0);
    for (int32_t hi = 0; hi < H; ++hi) {
        const int32_t hu = Lo.h_int2user[(size_t)hi];
        Lo.qbase[(size_t)hi + 1] = Lo.qbase[(size_t)hi] + g->infoset_num_actions[hu];
        Lo.iplayer[(size_t)hi] = g->infoset_player[hu];
    }
    Lo.q_int2user.assign((size_t)Q, 0);
    std::vector<int32_t> q_user2int((size_t)Q, 0);
    Lo.sigma0.assign((size_t)Q, 0.0);
    for (int32_t hi = 0; hi < H; ++hi) {
        const int32_t hu = Lo.h_int2user[(size_t)hi];
        for (int32_t a = 0; a < g->infoset_num_actions[hu]; ++a) {
            const int32_t qi = Lo.qbase[(size_t)hi] + a;
            const int32_t qu = (int32_t)(qbase_user[hu] + a);
            Lo.q_int2user[(size_t)qi] = qu;
            q_user2int[(size_t)qu] = qi;
            if (g->infoset_player[hu] == 0) Lo.sigma0[(size_t)qi] = g->chance_prob[coff[hu] + a];
        }
    }
    std::vector<int32_t> q2h_user((size_t)Q, 0);
    for (int32_t h = 0; h < H; ++h)
        for (int64_t q = qbase_user[h]; q < qbase_user[(size_t)h + 1]; ++q) q2h_user[(size_t)q] = h;
    Lo.pseq.assign((size_t)H, -1);
    Lo.pseq_h.assign((size_t)H, -1);
    for (int32_t hi = 0; hi < H; ++hi) {
        const int32_t hu = Lo.h_int2user[(size_t)hi];
        if (Lo.iplayer[(size_t)hi] > 0 && rep[hu] >= 0) {
            Lo.pseq[(size_t)hi] = q_user2int[(size_t)rep[hu]];
            Lo.pseq_h[(size_t)hi] = hmap[(size_t)q2h_user[(size_t)rep[hu]]];
        }
    }
    // Per decision node, its infoset's first slot, a wide flag and the acting player in one word, so
    // the iteration kernels need no dependent lookup through the infoset tables.
    if (Q >= ((int64_t)1 << 29))
        return fail(err, CFR_ERR_UNSUPPORTED, "too many infoset-action pairs (%lld; at most 2^29)", (long long)Q);
    Lo.qp.resize((size_t)Lo.Nd);
    for (int64_t j = 0; j < Lo.Nd; ++j) {
        const int32_t hi = Lo.dinfo[(size_t)j];
        const uint32_t wide = Lo.qbase[(size_t)hi + 1] - Lo.qbase[(size_t)hi] > 32 ? 1u : 0u;
        Lo.qp[(size_t)j] = (uint32_t)Lo.qbase[(size_t)hi] | (wide << 29) | ((uint32_t)Lo.iplayer[(size_t)hi] << 30);
    }
    if (!infoset_lists) return CFR_OK;

    // ---- nodes of each infoset in depth-first (lexicographic path) order ---------------------
    // The order in which a recursive walk reaches them; a deterministic reduction over this list
    // adds the instantaneous regrets of an infoset's nodes in the same order as such a walk.
    std::vector<int32_t> dec_of_user((size_t)n, -1);
    for (int64_t j = 0; j < Lo.Nd; ++j) dec_of_user[(size_t)Lo.dnode_user[(size_t)j]] = (int32_t)j;
    Lo.hnode_start.assign((size_t)H + 1, 0);
    for (int64_t j = 0; j < Lo.Nd; ++j) Lo.hnode_start[(size_t)Lo.dinfo[(size_t)j] + 1]++;
    for (int32_t h = 0; h < H; ++h) Lo.hnode_start[(size_t)h + 1] += Lo.hnode_start[(size_t)h];
    Lo.hnode.assign((size_t)Lo.Nd, 0);
    std::vector<int32_t> fillp(Lo.hnode_start.begin(), Lo.hnode_start.end() - 1);
    std::vector<std::pair<int32_t, int32_t>> stack;       // (node, next action)
    for (int32_t r : roots) {
        if (g->infoset[r] < 0) continue;
        stack.emplace_back(r, 0);
        const int32_t j0 = dec_of_user[(size_t)r];
        Lo.hnode[(size_t)fillp[(size_t)Lo.dinfo[(size_t)j0]]++] = j0;
        while (!stack.empty()) {
            auto &top = stack.back();
            const int32_t v = top.first;
            const int32_t na = g->infoset_num_actions[g->infoset[v]];
            if (top.second == na) { stack.pop_back(); continue; }
            const int32_t c = child[(size_t)cstart[v] + top.second++];
            if (g->infoset[c] < 0) continue;
            const int32_t jc = dec_of_user[(size_t)c];
            Lo.hnode[(size_t)fillp[(size_t)Lo.dinfo[(size_t)jc]]++] = jc;
            stack.emplace_back(c, 0);
        }
    }
    return CFR_OK;
}

}  // namespace cfrgb
