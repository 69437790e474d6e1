// Validation of a game description (Definition in Section 2.1) and construction of the
// level-ordered layout described in layout.hpp.  Host code only; no CUDA calls.
#include "layout.hpp"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <functional>
#include <memory>
#include <limits>
#include <mutex>
#include <thread>

namespace cfrgb {
namespace {

int host_threads() {
    static const int n = (int)std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    return n;
}

int64_t nchunks(int64_t n) { return std::max<int64_t>(1, std::min<int64_t>(host_threads(), n / 65536)); }

// f(chunk, begin, end) over nchunks(n) contiguous ranges of [0, n), in parallel.
template <typename F>
void parallel_ranges(int64_t n, F f) {
    const int64_t T = nchunks(n);
    if (T == 1) { f((int64_t)0, (int64_t)0, n); return; }
    std::vector<std::thread> th;
    th.reserve((size_t)T - 1);
    for (int64_t c = 1; c < T; ++c) th.emplace_back([&f, c, n, T] { f(c, n * c / T, n * (c + 1) / T); });
    f((int64_t)0, (int64_t)0, n / T);
    for (auto &t : th) t.join();
}

// x[i] += x[i - 1] for i = 1 .. n in place (a running sum over x[1 .. n] starting from x[0]), in
// parallel: each range's total, the totals' running sum as the ranges' offsets, then each range's own
// running sum from its offset.  The ranges are parallel_ranges' (the same split in both passes).
void running_sum(std::vector<int32_t> &x, int64_t n) {
    const int64_t T = nchunks(n);
    std::vector<int64_t> off((size_t)T + 1, 0);
    parallel_ranges(n, [&](int64_t c, int64_t b, int64_t e) {
        int64_t t = 0;
        for (int64_t i = b + 1; i <= e; ++i) t += x[(size_t)i];
        off[(size_t)c + 1] = t;
    });
    off[0] = x[0];
    for (int64_t c = 0; c < T; ++c) off[(size_t)c + 1] += off[(size_t)c];
    parallel_ranges(n, [&](int64_t c, int64_t b, int64_t e) {
        int64_t t = off[(size_t)c];
        for (int64_t i = b + 1; i <= e; ++i) {
            t += x[(size_t)i];
            x[(size_t)i] = (int32_t)t;
        }
    });
}

// The first failure of a parallel pass: the lowest node index wins.
struct FirstError {
    std::mutex mu;
    int64_t at = std::numeric_limits<int64_t>::max();
    cfr_status st = CFR_OK;
    std::string msg;
    void set(int64_t v, cfr_status s, const std::string &m) {
        std::lock_guard<std::mutex> lk(mu);
        if (v < at) { at = v; st = s; msg = m; }
    }
    cfr_status report(std::string *err) const {
        if (st != CFR_OK && err) *err = msg;
        return st;
    }
};

std::string fmt(const char *f, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, f);
    std::vsnprintf(buf, sizeof buf, f, ap);
    va_end(ap);
    return buf;
}


// Runs the given tasks on their own threads (the large zero-filled allocations of a build, whose page
// faults would otherwise be taken one array after another).
void run_concurrently(std::initializer_list<std::function<void()>> tasks) {
    std::vector<std::thread> th;
    for (const auto &t : tasks) th.emplace_back(t);
    for (auto &t : th) t.join();
}

cfr_status fail(std::string *err, cfr_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (err) *err = buf;
    return st;
}

// The decision nodes of each infoset in depth-first (lexicographic path) order: the order in which a
// recursive walk reaches them; a deterministic reduction over this list adds the instantaneous regrets
// of an infoset's nodes in the same order as such a walk.
void build_infoset_lists(const cfr_game_desc *g, const std::vector<int32_t> &roots, const std::vector<int32_t> &cstart,
                         const std::vector<int32_t> &child, Layout &Lo) {
    const int64_t n = g->num_nodes;
    const int32_t H = g->num_infosets;
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
}

// The infoset and slot tables of a layout whose decision nodes are placed (dinfo still holds caller
// infoset ids): internal infoset ids (hmap; infosets without nodes follow the others of their kind),
// slot maps, sigma_0, the parent sequences for the own reaches, and the packed per-node word qp.
cfr_status finish_tables(const cfr_game_desc *g, Layout &Lo, std::vector<int32_t> &hmap, const std::vector<int64_t> &rep,
                         const std::vector<int64_t> &qbase_user, const std::vector<int64_t> &coff, int32_t nh, int32_t nhc,
                         std::string *err) {
    const int32_t H = g->num_infosets;
    const int64_t Q = qbase_user[(size_t)H];
    const int32_t Hp = Lo.Hp;
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
    std::vector<int32_t> q_user2int, q2h_user;
    run_concurrently({[&] { Lo.q_int2user.assign((size_t)Q, 0); }, [&] { q_user2int.assign((size_t)Q, 0); },
                      [&] { Lo.sigma0.assign((size_t)Q, 0.0); }, [&] { q2h_user.assign((size_t)Q, 0); }});
    parallel_ranges(H, [&](int64_t, int64_t b, int64_t e) {
        for (int64_t hi = b; hi < e; ++hi) {
            const int32_t hu = Lo.h_int2user[(size_t)hi];
            for (int32_t a = 0; a < g->infoset_num_actions[hu]; ++a) {
                const int32_t qi = Lo.qbase[(size_t)hi] + a;
                const int32_t qu = (int32_t)(qbase_user[hu] + a);
                Lo.q_int2user[(size_t)qi] = qu;
                q_user2int[(size_t)qu] = qi;
                q2h_user[(size_t)qu] = hu;
                if (g->infoset_player[hu] == 0) Lo.sigma0[(size_t)qi] = g->chance_prob[coff[hu] + a];
            }
        }
    });
    Lo.pseq.assign((size_t)H, -1);
    Lo.pseq_h.assign((size_t)H, -1);
    parallel_ranges(H, [&](int64_t, int64_t b, int64_t e) {
        for (int64_t hi = b; hi < e; ++hi) {
            const int32_t hu = Lo.h_int2user[(size_t)hi];
            if (Lo.iplayer[(size_t)hi] > 0 && rep[hu] >= 0) {
                Lo.pseq[(size_t)hi] = q_user2int[(size_t)rep[hu]];
                Lo.pseq_h[(size_t)hi] = hmap[(size_t)q2h_user[(size_t)rep[hu]]];
            }
        }
    });
    // Per decision node, its infoset's first slot, a wide flag and the acting player in one word, so
    // the iteration kernels need no dependent lookup through the infoset tables.
    if (Q >= ((int64_t)1 << 29))
        return fail(err, CFR_ERR_UNSUPPORTED, "too many infoset-action pairs (%lld; at most 2^29)", (long long)Q);
    Lo.qp.resize((size_t)Lo.Nd);
    parallel_ranges(Lo.Nd, [&](int64_t, int64_t b, int64_t e) {
        for (int64_t j = b; j < e; ++j) {
            const int32_t hi = Lo.dinfo[(size_t)j] = hmap[(size_t)Lo.dinfo[(size_t)j]];
            const uint32_t wide = Lo.qbase[(size_t)hi + 1] - Lo.qbase[(size_t)hi] > 32 ? 1u : 0u;
            Lo.qp[(size_t)j] = (uint32_t)Lo.qbase[(size_t)hi] | (wide << 29) | ((uint32_t)Lo.iplayer[(size_t)hi] << 30);
        }
    });
    return CFR_OK;
}

// The description's sizes, pointers and infoset tables: qbase_user (caller slot bases), coff (each chance
// infoset's first entry in chance_prob), the largest action count; chance distributions sum to 1.
cfr_status validate_infosets(const cfr_game_desc *g, std::vector<int64_t> &qbase_user, std::vector<int64_t> &coff,
                             int32_t *max_actions_out, std::string *err) {
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

    qbase_user.assign((size_t)H + 1, 0);
    coff.assign((size_t)H, -1);
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

    *max_actions_out = max_actions;
    return CFR_OK;
}

}  // namespace

cfr_status build_layout_serial(const cfr_game_desc *g, Layout *out, std::string *err, bool infoset_lists, bool forest) {
    std::vector<int64_t> qbase_user, coff;
    int32_t max_actions = 0;
    {
        const cfr_status st = validate_infosets(g, qbase_user, coff, &max_actions, err);
        if (st != CFR_OK) return st;
    }
    const int64_t n = g->num_nodes;
    const int32_t H = g->num_infosets;
    const int64_t Q = qbase_user[(size_t)H];

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
                Lo.dinfo.push_back(hu);            // caller id; finish_tables maps it
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
    const cfr_status ft = finish_tables(g, Lo, hmap, rep, qbase_user, coff, nh, nhc, err);
    if (ft != CFR_OK) return ft;
    if (!infoset_lists) return CFR_OK;

    build_infoset_lists(g, roots, cstart, child, Lo);
    return CFR_OK;
}

}  // namespace cfrgb

// ---- the same layout built by several host threads (large trees) ---------------------------------
// Validation passes run over node ranges in parallel, each range reporting its lowest failing node, so
// the error reported is the serial builder's.  The breadth-first numbering is built depth by depth:
// per range of the depth's nodes the children, decision children, terminal children, decision nodes,
// wide nodes and mask words are counted, the counts are turned into offsets, and every range then
// writes its nodes' entries at those offsets - the serial builder's order exactly.  Perfect recall is
// checked with a compare-and-swap per infoset; infoset ids follow first appearance, found as the
// smallest decision id of each infoset.
namespace cfrgb {

cfr_status build_layout_parallel(const cfr_game_desc *g, Layout *out, std::string *err, bool infoset_lists, bool forest) {
    std::vector<int64_t> qbase_user, coff;
    int32_t max_actions = 0;
    {
        const cfr_status st = validate_infosets(g, qbase_user, coff, &max_actions, err);
        if (st != CFR_OK) return st;
    }
    const int64_t n = g->num_nodes;
    const int32_t H = g->num_infosets;
    const int64_t Q = qbase_user[(size_t)H];
    const int32_t *par = g->parent, *act = g->action, *inf = g->infoset, *nact = g->infoset_num_actions;

    // ---- nodes: roots, ids in range ----------------------------------------------------------
    std::vector<int32_t> roots;
    {
        FirstError fe;
        const int64_t T = nchunks(n);
        std::vector<std::vector<int32_t>> rts((size_t)T);
        parallel_ranges(n, [&](int64_t c, int64_t b, int64_t e) {
            for (int64_t v = b; v < e; ++v) {
                const int32_t p = par[v];
                if (p == -1) rts[(size_t)c].push_back((int32_t)v);
                else if (p < 0 || p >= n) { fe.set(v, CFR_ERR_INVALID, fmt("node %lld: parent %d out of range", (long long)v, p)); return; }
                const int32_t hv = inf[v];
                if (hv < -1 || hv >= H) { fe.set(v, CFR_ERR_INVALID, fmt("node %lld: infoset %d out of range", (long long)v, hv)); return; }
            }
        });
        for (auto &r : rts) roots.insert(roots.end(), r.begin(), r.end());
        // the serial pass reports a second root before any later range error
        if (!forest && roots.size() > 1 && (int64_t)roots[1] < fe.at)
            return fail(err, CFR_ERR_INVALID, "two roots: nodes %d and %lld", roots[0], (long long)roots[1]);
        if (fe.st != CFR_OK) return fe.report(err);
    }
    if (roots.empty()) return fail(err, CFR_ERR_INVALID, "no root (no node with parent -1)");

    // ---- children: counts, a bijection onto actions ------------------------------------------
    // seq1 / seq2: each node's last own slot of player 1 / 2 (-1: none yet), kept by breadth-first position
    // (the node order[i] at i), so that the numbering pass reads and writes them in order.  order, seq1 and
    // seq2 are written before they are read (the roots' entries when they are placed), so they are left
    // uninitialised: their pages are first touched by the parallel numbering pass.
    std::vector<int32_t> cstart, child;
    std::unique_ptr<int32_t[]> order(new int32_t[(size_t)std::max<int64_t>(n, 1)]);
    std::unique_ptr<int32_t[]> seq1(new int32_t[(size_t)std::max<int64_t>(n, 1)]);
    std::unique_ptr<int32_t[]> seq2(new int32_t[(size_t)std::max<int64_t>(n, 1)]);
    run_concurrently({[&] { cstart.assign((size_t)n + 1, 0); }, [&] { child.assign((size_t)n, -1); }});
    {
        FirstError fe;
        parallel_ranges(n, [&](int64_t, int64_t b, int64_t e) {
            for (int64_t v = b; v < e; ++v) {
                const int32_t p = par[v];
                if (p == -1) continue;
                if (inf[p] < 0) { fe.set(v, CFR_ERR_INVALID, fmt("node %lld: parent %d is a terminal (infoset -1)", (long long)v, p)); return; }
                __atomic_fetch_add(&cstart[(size_t)p + 1], 1, __ATOMIC_RELAXED);
            }
        });
        if (fe.st != CFR_OK) return fe.report(err);
        parallel_ranges(n, [&](int64_t, int64_t b, int64_t e) {
            for (int64_t v = b; v < e; ++v) {
                const int32_t hv = inf[v];
                const int32_t want = hv >= 0 ? nact[hv] : 0;
                if (cstart[(size_t)v + 1] != want) {
                    fe.set(v, CFR_ERR_INVALID, fmt("node %lld has %d children but its infoset %d has %d actions",
                                                   (long long)v, cstart[(size_t)v + 1], hv, want));
                    return;
                }
            }
        });
        if (fe.st != CFR_OK) return fe.report(err);
    }
    running_sum(cstart, n);
    {
        FirstError fe;
        parallel_ranges(n, [&](int64_t, int64_t b, int64_t e) {
            for (int64_t v = b; v < e; ++v) {
                const int32_t p = par[v];
                if (p == -1) continue;
                const int32_t a = act[v];
                if (a < 0 || a >= nact[inf[p]]) {
                    fe.set(v, CFR_ERR_INVALID, fmt("node %lld: action %d out of range for its parent", (long long)v, a));
                    return;
                }
                int32_t expect = -1;
                if (!__atomic_compare_exchange_n(&child[(size_t)cstart[p] + a], &expect, (int32_t)v, false, __ATOMIC_RELAXED,
                                                 __ATOMIC_RELAXED)) {
                    const int32_t lo = std::min(expect, (int32_t)v), hi = std::max(expect, (int32_t)v);
                    fe.set(hi, CFR_ERR_INVALID, fmt("nodes %d and %d: same action %d under parent %d", lo, hi, a, p));
                    return;
                }
            }
        });
        if (fe.st != CFR_OK) return fe.report(err);
    }
    {
        FirstError fe;
        std::atomic<bool> zero_sum{true};
        parallel_ranges(n, [&](int64_t, int64_t b, int64_t e) {
            bool zs = true;
            for (int64_t v = b; v < e; ++v) {
                if (inf[v] >= 0) continue;
                const double u1 = g->utility[2 * v], u2 = g->utility[2 * v + 1];
                if (!std::isfinite(u1) || !std::isfinite(u2)) {
                    fe.set(v, CFR_ERR_INVALID, fmt("terminal %lld: non-finite utility", (long long)v));
                    return;
                }
                if (std::fabs(u1 + u2) > 1e-12 * std::fmax(1.0, std::fmax(std::fabs(u1), std::fabs(u2)))) zs = false;
            }
            if (!zs) zero_sum = false;
        });
        if (fe.st != CFR_OK) return fe.report(err);
        if (!zero_sum) {
            // the serial builder reports unreachable nodes first; the breadth-first pass below finds them
        }
        // ---- breadth-first numbering, depth by depth ---------------------------------------------
        Layout tmp;
        Layout &Lo = out ? *out : tmp;
        Lo = Layout();
        Lo.N = n; Lo.H = H; Lo.Q = Q; Lo.max_actions = max_actions;
        int32_t Hp = 0;
        for (int32_t h = 0; h < H; ++h) Hp += g->infoset_player[h] > 0;
        Lo.Hp = Hp;
        int64_t ndec = 0;
        {
            std::atomic<int64_t> nd{0};
            parallel_ranges(n, [&](int64_t, int64_t b, int64_t e) {
                int64_t k = 0;
                for (int64_t v = b; v < e; ++v) k += inf[v] >= 0;
                nd += k;
            });
            ndec = nd;
        }
        std::vector<int64_t> rep;
        run_concurrently({[&] { rep.assign((size_t)H, -2); }, [&] { Lo.dfirst.assign((size_t)ndec + 1, 0); },
                          [&] { Lo.tfirst.assign((size_t)ndec + 1, 0); }, [&] { Lo.dinfo.assign((size_t)ndec, 0); },
                          [&] { Lo.kmask.assign((size_t)ndec, 0); }, [&] { Lo.dnode_user.assign((size_t)ndec, 0); },
                          [&] { Lo.tnode_user.assign((size_t)(n - ndec), 0); },
                          [&] { Lo.util.assign((size_t)(n - ndec), 0.0); }});
        int64_t tail = 0, dq = 0, tq = 0, nd_proc = 0;
        for (int32_t r : roots) {
            seq1[(size_t)tail] = seq2[(size_t)tail] = -1;
            order[(size_t)tail++] = r;
            if (inf[r] >= 0) Lo.dnode_user[(size_t)dq++] = r;
            else { Lo.tnode_user[(size_t)tq] = r; Lo.util[(size_t)tq++] = g->utility[2 * (size_t)r]; }
        }
        std::vector<int32_t> dlevel_all;      // decision-node offset at the start of every depth
        std::vector<int32_t> wide_all;
        std::vector<uint32_t> wbits;
        FirstError recall;
        int64_t head = 0;
        int32_t depth = 0;
        while (head < tail) {
            const int64_t lo = head, hi = tail, cnt = hi - lo;
            const int64_t T = nchunks(cnt);
            // per range: children, decision children, terminal children, decision nodes, wide nodes, mask words
            std::vector<int64_t> k_ch((size_t)T + 1, 0), k_dc((size_t)T + 1, 0), k_tc((size_t)T + 1, 0),
                k_dn((size_t)T + 1, 0), k_wn((size_t)T + 1, 0), k_ww((size_t)T + 1, 0);
            parallel_ranges(cnt, [&](int64_t c, int64_t b, int64_t e) {
                int64_t ch = 0, dc = 0, dn = 0, wn = 0, ww = 0;
                for (int64_t i = lo + b; i < lo + e; ++i) {
                    const int32_t v = order[(size_t)i];
                    const int32_t hu = inf[v];
                    if (hu < 0) continue;
                    const int32_t na = nact[hu];
                    ++dn;
                    ch += na;
                    for (int32_t a = 0; a < na; ++a) dc += inf[child[(size_t)cstart[v] + a]] >= 0;
                    if (na > 32) { ++wn; ww += (na + 31) / 32; }
                }
                k_ch[(size_t)c + 1] = ch; k_dc[(size_t)c + 1] = dc; k_tc[(size_t)c + 1] = ch - dc;
                k_dn[(size_t)c + 1] = dn; k_wn[(size_t)c + 1] = wn; k_ww[(size_t)c + 1] = ww;
            });
            for (int64_t c = 0; c < T; ++c) {
                k_ch[(size_t)c + 1] += k_ch[(size_t)c]; k_dc[(size_t)c + 1] += k_dc[(size_t)c];
                k_tc[(size_t)c + 1] += k_tc[(size_t)c]; k_dn[(size_t)c + 1] += k_dn[(size_t)c];
                k_wn[(size_t)c + 1] += k_wn[(size_t)c]; k_ww[(size_t)c + 1] += k_ww[(size_t)c];
            }
            const int64_t level_dn = k_dn[(size_t)T];
            if (level_dn > 0) {
                Lo.dlevel.push_back((int32_t)nd_proc);
                Lo.wlevel.push_back((int32_t)wide_all.size());
            }
            dlevel_all.push_back((int32_t)nd_proc);
            const size_t wbase = wbits.size(), wnbase = wide_all.size();
            wbits.resize(wbase + (size_t)k_ww[(size_t)T], 0u);
            wide_all.resize(wnbase + (size_t)k_wn[(size_t)T], 0);
            const int64_t child_base = tail, dq_base = dq, tq_base = tq, nd_base = nd_proc;
            parallel_ranges(cnt, [&](int64_t c, int64_t b, int64_t e) {
                int64_t ch = k_ch[(size_t)c], dc = k_dc[(size_t)c], tc = k_tc[(size_t)c], dn = k_dn[(size_t)c],
                        wn = k_wn[(size_t)c], ww = k_ww[(size_t)c];
                for (int64_t i = lo + b; i < lo + e; ++i) {
                    const int32_t v = order[(size_t)i];
                    const int32_t hu = inf[v];
                    if (hu < 0) continue;
                    const int p = g->infoset_player[hu];
                    const int32_t s1v = seq1[(size_t)i], s2v = seq2[(size_t)i];
                    if (p > 0) {
                        const int64_t sq = p == 1 ? s1v : s2v;
                        int64_t expect = -2;
                        if (!__atomic_compare_exchange_n(&rep[(size_t)hu], &expect, sq, false, __ATOMIC_RELAXED, __ATOMIC_RELAXED) &&
                            expect != sq)
                            recall.set(nd_base + dn, CFR_ERR_INVALID,
                                       fmt("imperfect recall: infoset %d holds nodes with different own histories of "
                                           "player %d (e.g. node %d)", hu, p, v));
                    }
                    const int32_t na = nact[hu];
                    const int64_t j = nd_base + dn;
                    Lo.dfirst[(size_t)j] = (int32_t)(dq_base + dc);
                    Lo.tfirst[(size_t)j] = (int32_t)(tq_base + tc);
                    Lo.dinfo[(size_t)j] = hu;
                    uint32_t mask = 0;
                    const size_t woff = wbase + (size_t)ww;
                    for (int32_t a = 0; a < na; ++a) {
                        const int32_t cv = child[(size_t)cstart[v] + a];
                        const int64_t pos = child_base + ch++;
                        order[(size_t)pos] = cv;
                        const int32_t q = (int32_t)(qbase_user[(size_t)hu] + a);
                        seq1[(size_t)pos] = p == 1 ? q : s1v;
                        seq2[(size_t)pos] = p == 2 ? q : s2v;
                        if (inf[cv] >= 0) {
                            Lo.dnode_user[(size_t)(dq_base + dc++)] = cv;
                        } else {
                            if (na > 32) wbits[woff + (size_t)a / 32] |= 1u << (a % 32);
                            else mask |= 1u << a;
                            Lo.tnode_user[(size_t)(tq_base + tc)] = cv;
                            Lo.util[(size_t)(tq_base + tc++)] = g->utility[2 * (size_t)cv];
                        }
                    }
                    if (na > 32) {
                        wide_all[wnbase + (size_t)wn++] = (int32_t)j;
                        Lo.kmask[(size_t)j] = (uint32_t)woff;
                        ww += (na + 31) / 32;
                    } else {
                        Lo.kmask[(size_t)j] = mask;
                    }
                    ++dn;
                }
            });
            if (recall.st != CFR_OK) return recall.report(err);
            if (wbits.size() > (size_t)std::numeric_limits<uint32_t>::max())
                return fail(err, CFR_ERR_UNSUPPORTED, "too many wide nodes");
            tail += k_ch[(size_t)T];
            dq += k_dc[(size_t)T];
            tq += k_tc[(size_t)T];
            nd_proc += level_dn;
            head = hi;
            if (tail > head) ++depth;
        }
        if (tail != n)
            return fail(err, CFR_ERR_INVALID, "only %lld of %lld nodes are reachable from the root (cycle or forest)",
                        (long long)tail, (long long)n);
        if (!zero_sum)
            return fail(err, CFR_ERR_UNSUPPORTED, "utilities are not zero-sum (u1 + u2 != 0 at some terminal)");
        if (!out) return CFR_OK;
        Lo.wide = std::move(wide_all);
        Lo.wbits = std::move(wbits);
        Lo.Nd = dq; Lo.Nt = tq;
        Lo.L = (int32_t)Lo.dlevel.size();
        Lo.max_depth = depth;
        Lo.dlevel.push_back((int32_t)Lo.Nd);
        Lo.wlevel.push_back((int32_t)Lo.wide.size());
        Lo.dfirst[(size_t)Lo.Nd] = (int32_t)Lo.Nd;
        Lo.tfirst[(size_t)Lo.Nd] = (int32_t)Lo.Nt;
        // internal infoset ids in order of first appearance (the smallest decision id of each infoset),
        // player infosets first; the depth of first appearance decides single_level
        std::vector<int32_t> first((size_t)H, std::numeric_limits<int32_t>::max());
        parallel_ranges(Lo.Nd, [&](int64_t, int64_t b, int64_t e) {
            for (int64_t j = b; j < e; ++j) {
                int32_t *f = &first[(size_t)Lo.dinfo[(size_t)j]];
                int32_t cur = __atomic_load_n(f, __ATOMIC_RELAXED);
                while ((int32_t)j < cur &&
                       !__atomic_compare_exchange_n(f, &cur, (int32_t)j, true, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
                }
            }
        });
        std::vector<int32_t> hmap((size_t)H, -1);
        int32_t nh = 0, nhc = 0;
        {
            // per range of decision ids: the player and chance infosets first seen there, counted, then
            // numbered from the range's offsets
            const int64_t T = nchunks(Lo.Nd);
            std::vector<int64_t> kp((size_t)T + 1, 0), kc((size_t)T + 1, 0);
            parallel_ranges(Lo.Nd, [&](int64_t c, int64_t b, int64_t e) {
                int64_t a = 0, z = 0;
                for (int64_t j = b; j < e; ++j) {
                    const int32_t hu = Lo.dinfo[(size_t)j];
                    if (first[(size_t)hu] != j) continue;
                    if (g->infoset_player[hu] > 0) ++a; else ++z;
                }
                kp[(size_t)c + 1] = a;
                kc[(size_t)c + 1] = z;
            });
            for (int64_t c = 0; c < T; ++c) { kp[(size_t)c + 1] += kp[(size_t)c]; kc[(size_t)c + 1] += kc[(size_t)c]; }
            parallel_ranges(Lo.Nd, [&](int64_t c, int64_t b, int64_t e) {
                int64_t a = kp[(size_t)c], z = kc[(size_t)c];
                for (int64_t j = b; j < e; ++j) {
                    const int32_t hu = Lo.dinfo[(size_t)j];
                    if (first[(size_t)hu] != j) continue;
                    hmap[(size_t)hu] = g->infoset_player[hu] > 0 ? (int32_t)a++ : (int32_t)(Hp + z++);
                }
            });
            nh = (int32_t)kp[(size_t)T];
            nhc = (int32_t)kc[(size_t)T];
            // player infosets first seen before each decision depth: their first decision ids, in id order
            // (ascending, as the numbering follows first appearance), counted below each depth's start
            std::vector<int32_t> pos((size_t)nh, 0);
            parallel_ranges(H, [&](int64_t, int64_t b, int64_t e) {
                for (int64_t h = b; h < e; ++h)
                    if (g->infoset_player[h] > 0 && hmap[(size_t)h] >= 0) pos[(size_t)hmap[(size_t)h]] = first[(size_t)h];
            });
            for (int32_t l = 0; l < Lo.L; ++l)
                Lo.hlevel.push_back((int32_t)(std::lower_bound(pos.begin(), pos.end(), Lo.dlevel[(size_t)l]) - pos.begin()));
            Lo.hlevel.push_back(nh);
        }
        // single_level: every node of an infoset at the depth of its first node
        std::atomic<bool> single{true};
        parallel_ranges(Lo.Nd, [&](int64_t, int64_t b, int64_t e) {
            bool ok = true;
            for (int64_t j = b; j < e && ok; ++j) {
                const int32_t f = first[(size_t)Lo.dinfo[(size_t)j]];
                const auto lj = std::upper_bound(dlevel_all.begin(), dlevel_all.end(), (int32_t)j);
                const auto lf = std::upper_bound(dlevel_all.begin(), dlevel_all.end(), f);
                if (lj != lf) ok = false;
            }
            if (!ok) single = false;
        });
        Lo.single_level = single;
        const cfr_status ft = finish_tables(g, Lo, hmap, rep, qbase_user, coff, nh, nhc, err);
        if (ft != CFR_OK) return ft;
        if (infoset_lists) build_infoset_lists(g, roots, cstart, child, Lo);
    }
    return CFR_OK;
}

cfr_status build_layout(const cfr_game_desc *g, Layout *out, std::string *err, bool infoset_lists, bool forest) {
    const bool big = g && g->num_nodes >= kParallelLayoutNodes && host_threads() > 1;
    return big ? build_layout_parallel(g, out, err, infoset_lists, forest)
               : build_layout_serial(g, out, err, infoset_lists, forest);
}

}  // namespace cfrgb
