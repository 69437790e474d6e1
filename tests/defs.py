"""Brute-force evaluations of the paper's definitions, for TINY games only (test helper).

Everything here goes through explicit root-to-terminal PATH PRODUCTS and enumeration, a route
independent of the oracle's recursive tree walk:

* reach of a node (Section 2.2), counterfactual reach pi-check (Eq. 2), own reach pi-hat (Eq. 4,
  read as the product of the acting player's own factors), infoset reaches (Eq. 3, Eq. 5);
* node payoff u-check (Eq. 1) as sum over the terminals below a node of (conditional path
  product) x utility;
* counterfactual utility (Eq. 6) and instantaneous regret (Eq. 7) with the overridden profile
  sigma|h->a evaluated by the same path products;
* average strategy (Eq. 10) with the paper's weights pi-bar = sum over the infoset's nodes;
* overall regret (Section 2.3) and best responses by enumerating pure strategies;
* the game value from the sequence-form linear program (Koller, Megiddo, von Stengel).
"""
from __future__ import annotations

import itertools

import numpy as np


class Tree:
    def __init__(self, g):
        self.g = g
        self.n = g.num_nodes
        self.parent = [int(x) for x in g.parent]
        self.action = [int(x) for x in g.action]
        self.infoset = [int(x) for x in g.infoset]
        self.player = [int(x) for x in g.infoset_player]
        self.nact = [int(x) for x in g.infoset_num_actions]
        self.H = len(self.player)
        self.qbase = [0]
        for k in self.nact:
            self.qbase.append(self.qbase[-1] + k)
        self.Q = self.qbase[-1]
        self.util = np.asarray(g.utility, dtype=float)
        self.root = self.parent.index(-1)
        self.sigma0 = np.zeros(self.Q)
        c = 0
        for h in range(self.H):
            if self.player[h] == 0:
                for a in range(self.nact[h]):
                    self.sigma0[self.qbase[h] + a] = g.chance_prob[c]
                    c += 1
        # path of each node: list of (ancestor node, action taken there), root first
        self.path = []
        for v in range(self.n):
            p, u = [], v
            while self.parent[u] >= 0:
                p.append((self.parent[u], self.action[u]))
                u = self.parent[u]
            self.path.append(p[::-1])
        self.depth = [len(p) for p in self.path]
        self.terminals = [v for v in range(self.n) if self.infoset[v] < 0]
        self.nodes_of = [[] for _ in range(self.H)]
        for v in range(self.n):
            if self.infoset[v] >= 0:
                self.nodes_of[self.infoset[v]].append(v)
        # terminals below each node (inclusive)
        self.below = [[] for _ in range(self.n)]
        for t in self.terminals:
            self.below[t].append(t)
            for (d, _a) in self.path[t]:
                self.below[d].append(t)

    # ----- probabilities of single edges -----
    def q(self, d, a):
        return self.qbase[self.infoset[d]] + a

    def edge_prob(self, prof, d, a):
        h = self.infoset[d]
        return self.sigma0[self.q(d, a)] if self.player[h] == 0 else prof[self.q(d, a)]

    def actor(self, d):
        return self.player[self.infoset[d]]

    # ----- reaches by path products -----
    def reach(self, prof, v):
        """pi(sigma, v): product of every edge probability on the root->v path (Section 2.2)."""
        return float(np.prod([self.edge_prob(prof, d, a) for (d, a) in self.path[v]])) if self.path[v] else 1.0

    def reach_split(self, prof, v):
        """(r_chance, r_1, r_2): the path product split by acting player."""
        r = [1.0, 1.0, 1.0]
        for (d, a) in self.path[v]:
            r[self.actor(d)] *= self.edge_prob(prof, d, a)
        return r

    def cf_reach(self, prof, v, i):
        """pi-check(sigma, v, i), Eq. 2: the path product skipping player i's own factors."""
        r = 1.0
        for (d, a) in self.path[v]:
            if self.actor(d) != i:
                r *= self.edge_prob(prof, d, a)
        return r

    def own_reach(self, prof, v, i):
        """pi-hat(sigma, v, i), Eq. 4: the path product of player i's own factors only."""
        r = 1.0
        for (d, a) in self.path[v]:
            if self.actor(d) == i:
                r *= self.edge_prob(prof, d, a)
        return r

    # ----- payoffs -----
    def node_value(self, prof, v, i):
        """u-check(sigma, v, i), Eq. 1, as sum over terminals t below v of P(t | v) u(t, i)."""
        tot = 0.0
        k = self.depth[v]
        for t in self.below[v]:
            pr = 1.0
            for (d, a) in self.path[t][k:]:
                pr *= self.edge_prob(prof, d, a)
            tot += pr * self.util[t, i - 1]
        return tot

    def expected_payoff(self, prof, i):
        """u-hat(sigma, i) = sum_t pi(sigma, t) u(t, i)  (Section 2.2)."""
        return sum(self.reach(prof, t) * self.util[t, i - 1] for t in self.terminals)

    def override(self, prof, h, a):
        """sigma|h->a (Section 2.3)."""
        p = np.array(prof, dtype=float)
        for b in range(self.nact[h]):
            p[self.qbase[h] + b] = 1.0 if b == a else 0.0
        return p

    def inst_regret(self, prof):
        """r-tilde(sigma, (h, a)), Eq. 7, for every player infoset-action; chance slots 0.

        Computed as pi~(h) * (u~(sigma|h->a, h) - u~(sigma, h)) with u~ from Eq. 6; when
        pi~(h) = 0 the regret is 0.
        """
        out = np.zeros(self.Q)
        for h in range(self.H):
            p = self.player[h]
            if p == 0:
                continue
            nodes = self.nodes_of[h]
            pit = sum(self.cf_reach(prof, d, p) for d in nodes)                        # Eq. 3
            if pit == 0.0:
                continue
            ut = sum(self.cf_reach(prof, d, p) * self.node_value(prof, d, p) for d in nodes) / pit  # Eq. 6
            for a in range(self.nact[h]):
                pa = self.override(prof, h, a)
                uta = sum(self.cf_reach(pa, d, p) * self.node_value(pa, d, p) for d in nodes) / pit
                out[self.qbase[h] + a] = pit * (uta - ut)
        return out

    def player_reach(self, prof, h):
        """pi-bar(sigma, h), Eq. 5: sum over the nodes of h of the own reach."""
        p = self.player[h]
        return sum(self.own_reach(prof, d, p) for d in self.nodes_of[h])

    def average_strategy(self, history):
        """sigma-bar^(T), Eq. 10, from the list of profiles sigma^(1..T)."""
        out = np.zeros(self.Q)
        for h in range(self.H):
            qb, na = self.qbase[h], self.nact[h]
            if self.player[h] == 0:
                out[qb:qb + na] = self.sigma0[qb:qb + na]
                continue
            num = np.zeros(na)
            den = 0.0
            for prof in history:
                w = self.player_reach(prof, h)
                num += w * np.asarray(prof[qb:qb + na])
                den += w
            out[qb:qb + na] = num / den if den > 0 else 1.0 / na
        return out

    # ----- pure strategies -----
    def pure_strategies(self, i, limit=200000):
        hs = [h for h in range(self.H) if self.player[h] == i]
        count = int(np.prod([self.nact[h] for h in hs])) if hs else 1
        if count > limit:
            raise ValueError("too many pure strategies")
        for choice in itertools.product(*[range(self.nact[h]) for h in hs]):
            yield {h: a for h, a in zip(hs, choice)}

    def with_pure(self, prof, pure):
        p = np.array(prof, dtype=float)
        for h, a in pure.items():
            p[self.qbase[h]:self.qbase[h] + self.nact[h]] = 0.0
            p[self.qbase[h] + a] = 1.0
        return p

    def best_response_value(self, prof, i):
        """max over pure strategies of player i of u-hat(sigma'_i + sigma_-i, i)."""
        return max(self.expected_payoff(self.with_pure(prof, s), i) for s in self.pure_strategies(i))

    def overall_regret(self, history, i):
        """r^(T)(i) of Section 2.3 by enumeration over player i's pure strategies."""
        T = len(history)
        realised = sum(self.expected_payoff(p, i) for p in history)
        best = max(sum(self.expected_payoff(self.with_pure(p, s), i) for p in history)
                   for s in self.pure_strategies(i))
        return (best - realised) / T

    # ----- sequence form -----
    def parent_sequence(self, v, i):
        """Index into the sequence list of player i of the last own (infoset, action) above v."""
        last = 0
        for (d, a) in self.path[v]:
            if self.actor(d) == i:
                last = 1 + self.q(d, a)
        return last

    def sequence_form(self, i):
        """(E, e) with E x = e for player i; sequences: 0 = empty, 1 + q for (h, a)."""
        nseq = 1 + self.Q
        rows = [np.eye(1, nseq, 0)[0]]
        for h in range(self.H):
            if self.player[h] != i or not self.nodes_of[h]:
                continue
            r = np.zeros(nseq)
            r[self.parent_sequence(self.nodes_of[h][0], i)] -= 1.0
            for a in range(self.nact[h]):
                r[1 + self.qbase[h] + a] += 1.0
            rows.append(r)
        E = np.array(rows)
        e = np.zeros(len(rows))
        e[0] = 1.0
        return E, e

    def payoff_matrix(self):
        nseq = 1 + self.Q
        A = np.zeros((nseq, nseq))
        for t in self.terminals:
            pc = 1.0
            for (d, a) in self.path[t]:
                if self.actor(d) == 0:
                    pc *= self.sigma0[self.q(d, a)]
            A[self.parent_sequence(t, 1), self.parent_sequence(t, 2)] += pc * self.util[t, 0]
        return A

    def lp_solve(self, i):
        """Equilibrium realisation plan of player i and the game value for player 1 (zero-sum)."""
        from scipy.optimize import linprog

        A = self.payoff_matrix() if i == 1 else -self.payoff_matrix().T
        E, e = self.sequence_form(i)
        F, f = self.sequence_form(3 - i)
        nx, nv = E.shape[1], F.shape[0]
        c = np.concatenate([np.zeros(nx), -f])
        A_ub = np.hstack([-A.T, F.T])
        b_ub = np.zeros(A_ub.shape[0])
        A_eq = np.hstack([E, np.zeros((E.shape[0], nv))])
        bounds = [(0, None)] * nx + [(None, None)] * nv
        res = linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=A_eq, b_eq=e, bounds=bounds, method="highs")
        assert res.status == 0, res.message
        value = -res.fun
        return res.x[:nx], (value if i == 1 else -value)

    def behavioural(self, x, i, prof=None):
        """Behaviour strategy of player i from realisation plan x (uniform where unreachable)."""
        out = np.array(self.sigma0 if prof is None else prof, dtype=float)
        for h in range(self.H):
            if self.player[h] != i:
                continue
            qb, na = self.qbase[h], self.nact[h]
            if not self.nodes_of[h]:
                out[qb:qb + na] = 1.0 / na
                continue
            par = x[self.parent_sequence(self.nodes_of[h][0], i)]
            out[qb:qb + na] = x[1 + qb:1 + qb + na] / par if par > 1e-12 else 1.0 / na
        return out


def uniform_profile(tr: Tree) -> np.ndarray:
    p = np.array(tr.sigma0)
    for h in range(tr.H):
        if tr.player[h] != 0:
            p[tr.qbase[h]:tr.qbase[h] + tr.nact[h]] = 1.0 / tr.nact[h]
    return p


def random_profile(tr: Tree, rng, zero_frac: float = 0.0) -> np.ndarray:
    """Random player strategies (some actions optionally zero), chance slots sigma_0."""
    p = np.array(tr.sigma0)
    for h in range(tr.H):
        if tr.player[h] == 0:
            continue
        w = rng.random(tr.nact[h]) + 0.05
        if zero_frac > 0:
            w[rng.random(tr.nact[h]) < zero_frac] = 0.0
            if w.sum() == 0:
                w[rng.integers(tr.nact[h])] = 1.0
        p[tr.qbase[h]:tr.qbase[h] + tr.nact[h]] = w / w.sum()
    return p
