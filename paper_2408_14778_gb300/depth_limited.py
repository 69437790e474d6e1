"""Depth-limited CFR+ with a learned leaf-value network (no counterpart in the paper).

A game of the "public tree x private deal" form - a root chance node deals one of K private states
pairs (x1(k), x2(k)), and below every deal hangs a copy of one public tree, node (k, i) having caller id
1 + k P + i - is cut at a public depth: every public decision node there becomes a leaf of the
depth-limited game.  A leaf (k, c) stands for the subgame below public node c; its player-1 utility is
the network's estimate of that subgame's value for the deal pair (x1(k), x2(k)) when the players reach c
with ranges r1, r2 (their own reach probabilities of each private state, Eq. 4, normalised), and the
subgame below is played in equilibrium.

Network (BF16 tensor-core kernels, cfr_mlp_*): input [64-dim public-node embedding, r1 zero-padded to
169, r2 zero-padded to 169]; output [V1 over the 13 x 13 = 169 private-state pairs (x1 major), V2 = -V1
over the same pairs], values divided by the game's payoff bound.  Leaves read V1.

Between iterations the leaves are refreshed on the device: cfr_gather_ranges writes the ranges at every
cut node into the network's input, cfr_mlp_forward evaluates it, and cfr_set_leaf_values writes the
leaves' utilities - no host round trip.

Training samples come from full-depth GPU CFR+: for a cut node c and random ranges, the subgame below c
under a chance root dealing k with probability proportional to pi_c(k) r1(x1(k)) r2(x2(k)) is solved,
many subgames at once as one tree, and the value of each deal's node under the average strategy is read
back (cfr_set_state with R = S makes sigma the average strategy; one iteration then evaluates it).

This module is host-side preparation (index arrays) and orchestration of the library's calls; every
CFR, range and network computation runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import (CFR_AVERAGE_STRATEGY, CFR_FP32, CFR_PLUS, cfr_average_strategy, cfr_exploitability, cfr_gather_ranges, cfr_get_nodes,
               cfr_get_state, cfr_iterate, cfr_load_tree, cfr_mlp_adam, cfr_mlp_backward, cfr_mlp_create,
               cfr_mlp_forward, cfr_mlp_set_params, cfr_set_leaf_values, cfr_set_leaves, cfr_set_range_program,
               cfr_set_state)

EMBED = 64
RANGE = 169


@dataclass
class GameArrays:
    """The fields of a game description this module reads (any object with these attributes works)."""
    parent: np.ndarray
    action: np.ndarray
    infoset: np.ndarray
    infoset_player: np.ndarray
    infoset_num_actions: np.ndarray
    chance_prob: np.ndarray
    utility: np.ndarray


def _game(parent, action, infoset, player, nact, cprob, util, like):
    """A game description of the caller's class (a dataclass taking the seven arrays)."""
    return type(like)(parent.astype(np.int32), action.astype(np.int32), infoset.astype(np.int32),
                      player.astype(np.int8), nact.astype(np.int32), cprob.astype(np.float64),
                      util.astype(np.float64), {}) if hasattr(like, "meta") else \
        GameArrays(parent, action, infoset, player, nact, cprob, util)


class PublicView:
    """The public structure of a deal-major game: K deals, P public nodes (BFS order), per public node
    its parent, incoming action, actor (-1 terminal, 0 chance, 1, 2) and depth; per deal its private
    states x1, x2 and probability."""

    def __init__(self, g):
        self.g = g
        N = int(g.num_nodes if hasattr(g, "num_nodes") else g.parent.shape[0])
        if g.parent[0] != -1 or g.infoset[0] != 0 or g.infoset_player[0] != 0:
            raise ValueError("the root must be the chance deal (infoset 0)")
        K = int(g.infoset_num_actions[0])
        if (N - 1) % K:
            raise ValueError("not a deal-major game")
        P = (N - 1) // K
        self.K, self.P = K, P
        ids = 1 + np.arange(K)[:, None] * P + np.arange(P)[None, :]
        par = g.parent[ids].astype(np.int64)
        if not (np.all(par[:, 0] == 0) and np.all((par[:, 1:] - 1) % P == (par[0, 1:] - 1)[None, :] % P)):
            raise ValueError("the deals' public trees differ")
        self.ppar = np.concatenate([[-1], par[0, 1:] - 1]).astype(np.int64)
        self.pact = g.action[1:1 + P].astype(np.int64)
        h0 = g.infoset[1:1 + P]
        self.actor = np.where(h0 < 0, -1, g.infoset_player[np.maximum(h0, 0)]).astype(np.int64)
        depth = np.zeros(P, np.int64)
        for i in range(1, P):
            depth[i] = depth[self.ppar[i]] + 1
        self.depth = depth
        self.deal_prob = np.asarray(g.chance_prob[:K], dtype=np.float64)
        # private state of each deal: the offset of its infoset among the deals' at a node of that player
        self.x = {}
        for p in (1, 2):
            nodes = np.nonzero(self.actor == p)[0]
            if nodes.size == 0:
                self.x[p] = np.zeros(K, np.int64)
                continue
            h = g.infoset[ids[:, nodes[0]]].astype(np.int64)
            self.x[p] = h - h.min()
        self.nx = {p: int(self.x[p].max()) + 1 for p in (1, 2)}
        if self.nx[1] > 13 or self.nx[2] > 13:
            raise ValueError("the value network's output holds at most 13 x 13 private-state pairs")
        self.qstart = np.concatenate([[0], np.cumsum(g.infoset_num_actions.astype(np.int64))])

    def node(self, k, i):
        return 1 + np.asarray(k, np.int64) * self.P + np.asarray(i, np.int64)

    def descendants(self, c: int) -> np.ndarray:
        """Public nodes of the subtree of c, BFS order (c first)."""
        inside = np.zeros(self.P, bool)
        inside[c] = True
        for i in range(c + 1, self.P):
            if self.ppar[i] >= 0 and inside[self.ppar[i]]:
                inside[i] = True
        return np.nonzero(inside)[0]

    def path(self, c: int) -> list:
        """(public node, action taken toward c) from the public root down to c's parent."""
        out = []
        i = c
        while self.ppar[i] >= 0:
            out.append((int(self.ppar[i]), int(self.pact[i])))
            i = int(self.ppar[i])
        return out[::-1]


@dataclass
class Cut:
    """The depth-limited game of a PublicView cut at public depth d (its decision nodes become leaves)."""
    game: object
    view: PublicView
    depth: int
    cut_nodes: np.ndarray     # public ids of the cut public nodes (one network row each)
    top_public: np.ndarray    # public ids kept, BFS order
    leaf_nodes: np.ndarray    # caller ids of the leaves in the depth-limited game
    leaf_src: np.ndarray      # per leaf: index of its value in the network output [rows][338]
    slot_to_full: np.ndarray  # depth-limited caller slot -> the full game's caller slot
    embed: np.ndarray         # [rows][64]
    seg_dst: np.ndarray
    seg_entries: np.ndarray
    entry_prod: np.ndarray
    slots: np.ndarray


def cut_game(g, depth: int, seed: int = 0) -> Cut:
    """The depth-limited game with the public decision nodes at public depth `depth` as leaves, the
    leaves' value indices, the range program and the public-node embeddings (seeded N(0, 1/64))."""
    v = PublicView(g)
    keep = np.nonzero(v.depth <= depth)[0]
    cut = keep[(v.depth[keep] == depth) & (v.actor[keep] >= 0)]
    Pt = keep.size
    loc = np.full(v.P, -1, np.int64)
    loc[keep] = np.arange(Pt)
    K = v.K
    full_ids = v.node(np.repeat(np.arange(K), Pt), np.tile(keep, K))
    N = 1 + K * Pt
    parent = np.empty(N, np.int64)
    action = np.empty(N, np.int64)
    infoset = np.full(N, -1, np.int64)
    parent[0], action[0], infoset[0] = -1, -1, 0
    kk = np.repeat(np.arange(K), Pt)
    jj = np.tile(np.arange(Pt), K)
    pp = v.ppar[keep][jj]
    parent[1:] = np.where(pp < 0, 0, 1 + kk * Pt + loc[np.maximum(pp, 0)])
    action[1:] = np.where(pp < 0, kk, v.pact[keep][jj])
    is_cut = np.isin(keep, cut)[jj]
    h_full = g.infoset[full_ids].astype(np.int64)
    h_keep = np.where(is_cut, -1, h_full)
    used = np.unique(np.concatenate([[0], h_keep[h_keep >= 0]]))
    hmap = np.full(g.infoset_player.shape[0], -1, np.int64)
    hmap[used] = np.arange(used.size)
    infoset[1:] = np.where(h_keep >= 0, hmap[np.maximum(h_keep, 0)], -1)
    util = np.zeros((N, 2))
    util[1:] = np.where(is_cut[:, None], 0.0, g.utility[full_ids])
    player = g.infoset_player[used]
    nact = g.infoset_num_actions[used]
    # chance probabilities of the kept chance infosets, in order
    cq = np.concatenate([[0], np.cumsum(np.where(g.infoset_player == 0, g.infoset_num_actions, 0))])
    cprob = np.concatenate([g.chance_prob[cq[h]:cq[h + 1]] for h in used if g.infoset_player[h] == 0])
    top = _game(parent, action, infoset, player, nact, cprob, util, g)
    # slots of the depth-limited game -> slots of the full game
    qs_new = np.concatenate([[0], np.cumsum(nact.astype(np.int64))])
    slot_to_full = np.concatenate([v.qstart[h] + np.arange(g.infoset_num_actions[h]) for h in used]).astype(np.int64)
    assert slot_to_full.size == qs_new[-1]
    # leaves and their value indices: row of the cut node, column x1 * 13 + x2
    rows = np.full(v.P, -1, np.int64)
    rows[cut] = np.arange(cut.size)
    lk = np.repeat(np.arange(K), cut.size)
    lc = np.tile(cut, K)
    leaf_nodes = 1 + lk * Pt + loc[lc]
    leaf_src = rows[lc] * (2 * RANGE) + v.x[1][lk] * 13 + v.x[2][lk]
    # range program: per cut node and player, per private state, the current strategy's product along
    # the public path over that player's own decisions (the infoset of any deal with that private state)
    in_w = EMBED + 2 * RANGE
    seg_dst, seg_entries, entry_prod, slots = [], [0], [0], []
    first_deal = {p: np.array([np.nonzero(v.x[p] == s)[0][0] for s in range(v.nx[p])]) for p in (1, 2)}
    for r, c in enumerate(cut):
        steps = v.path(int(c))
        for p in (1, 2):
            seg_dst.append(r * in_w + EMBED + (p - 1) * RANGE)
            for s in range(v.nx[p]):
                k = first_deal[p][s]
                for (q, a) in steps:
                    if v.actor[q] != p:
                        continue
                    h = infoset[1 + k * Pt + loc[q]]
                    slots.append(qs_new[h] + a)
                entry_prod.append(len(slots))
            seg_entries.append(len(entry_prod) - 1)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xE3B]))
    embed = rng.normal(0.0, 1.0 / 8.0, size=(cut.size, EMBED))
    return Cut(top, v, depth, cut, keep, leaf_nodes.astype(np.int32), leaf_src.astype(np.int64), slot_to_full, embed,
               np.array(seg_dst, np.int64), np.array(seg_entries, np.int64), np.array(entry_prod, np.int64),
               np.array(slots, np.int32))


def subgame(view: PublicView, c: int, r1: np.ndarray, r2: np.ndarray, desc=None, return_slots: bool = False):
    """The subgame below public node c when the players arrive with ranges r1, r2: a chance root deals
    k with probability proportional to pi_c(k) r1(x1(k)) r2(x2(k)), then deal k's copy of c's subtree.
    Node (k, d) of the subtree has id 1 + k D + (index of d among c's descendants)."""
    g = view.g
    d = view.descendants(c) if desc is None else desc
    D = d.size
    K = view.K
    loc = np.full(view.P, -1, np.int64)
    loc[d] = np.arange(D)
    w = view.deal_prob * r1[view.x[1]] * r2[view.x[2]]
    w = w / w.sum()
    full = view.node(np.repeat(np.arange(K), D), np.tile(d, K))
    N = 1 + K * D
    kk = np.repeat(np.arange(K), D)
    jj = np.tile(np.arange(D), K)
    pp = view.ppar[d][jj]
    parent = np.empty(N, np.int64)
    action = np.empty(N, np.int64)
    parent[0], action[0] = -1, -1
    root_child = jj == 0
    parent[1:] = np.where(root_child, 0, 1 + kk * D + loc[np.maximum(pp, 0)])
    action[1:] = np.where(root_child, kk, view.pact[d][jj])
    h_full = g.infoset[full].astype(np.int64)
    used = np.unique(h_full[h_full >= 0])
    hmap = np.full(g.infoset_player.shape[0], -1, np.int64)
    hmap[used] = 1 + np.arange(used.size)
    infoset = np.concatenate([[0], np.where(h_full >= 0, hmap[np.maximum(h_full, 0)], -1)])
    player = np.concatenate([[0], g.infoset_player[used]])
    nact = np.concatenate([[K], g.infoset_num_actions[used]])
    cq = np.concatenate([[0], np.cumsum(np.where(g.infoset_player == 0, g.infoset_num_actions, 0))])
    inner = [g.chance_prob[cq[h]:cq[h + 1]] for h in used if g.infoset_player[h] == 0]
    cprob = np.concatenate([w] + inner)
    util = np.zeros((N, 2))
    util[1:] = g.utility[full]
    sub = _game(parent, action, infoset, player, nact, cprob, util, g)
    if not return_slots:
        return sub
    # slots of the subgame's player infosets (ids 1..) -> the full game's slots; the root deal has none
    slot_to_full = np.concatenate([np.full(K, -1, np.int64)] +
                                  [view.qstart[h] + np.arange(g.infoset_num_actions[h]) for h in used])
    return sub, slot_to_full


def _with_root(games, like):
    """The games under one uniform chance root; returns the tree and each game's node offset."""
    n = len(games)
    sizes = np.array([gm.parent.shape[0] for gm in games], np.int64)
    off = 1 + np.concatenate([[0], np.cumsum(sizes)[:-1]])
    hs = np.array([gm.infoset_player.shape[0] for gm in games], np.int64)
    hoff = 1 + np.concatenate([[0], np.cumsum(hs)[:-1]])
    parent = np.concatenate([[-1]] + [np.where(gm.parent < 0, 0, gm.parent.astype(np.int64) + o)
                                      for gm, o in zip(games, off)])
    action = np.concatenate([[-1]] + [np.where(gm.parent < 0, i, gm.action) for i, gm in enumerate(games)])
    infoset = np.concatenate([[0]] + [np.where(gm.infoset < 0, -1, gm.infoset.astype(np.int64) + h)
                                      for gm, h in zip(games, hoff)])
    player = np.concatenate([[0]] + [gm.infoset_player for gm in games])
    nact = np.concatenate([[n]] + [gm.infoset_num_actions for gm in games])
    cprob = np.concatenate([np.full(n, 1.0 / n)] + [gm.chance_prob for gm in games])
    util = np.concatenate([np.zeros((1, 2))] + [gm.utility for gm in games])
    return _game(parent, action, infoset, player, nact, cprob, util, like), off


def random_ranges(rng: np.random.Generator, n: int, count: int) -> np.ndarray:
    """Random positive ranges over n private states, normalised: Dirichlet draws of mixed concentration
    (flat, peaked and near uniform), so that training sees the range shapes a solve produces."""
    alpha = rng.choice([0.3, 1.0, 5.0], size=count)
    return np.stack([rng.dirichlet(np.full(n, a)) for a in alpha])


def generate_samples(cut: Cut, per_node: int, iterations: int = 300, seed: int = 0, chunk_nodes: int = 20_000_000,
                     device=None):
    """Training samples (x [S][402], y [S][338], both FP32) for the cut's leaves: for every cut node,
    per_node random range pairs; each sample's subgame solved by full-depth CFR+ on the GPU (all of a
    chunk's subgames as one tree) and its deals' values read under the average strategy."""
    v = cut.view
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xDA7A]))
    umax = float(np.max(np.abs(v.g.utility))) or 1.0
    jobs = []
    for r, c in enumerate(cut.cut_nodes):
        r1 = random_ranges(rng, v.nx[1], per_node)
        r2 = random_ranges(rng, v.nx[2], per_node)
        jobs += [(r, int(c), r1[i], r2[i]) for i in range(per_node)]
    desc = {int(c): v.descendants(int(c)) for c in cut.cut_nodes}
    X = np.zeros((len(jobs), EMBED + 2 * RANGE), np.float32)
    Y = np.zeros((len(jobs), 2 * RANGE), np.float32)
    i0 = 0
    while i0 < len(jobs):
        subs, i1, n = [], i0, 0
        while i1 < len(jobs) and (n == 0 or n + 1 + v.K * desc[jobs[i1][1]].size <= chunk_nodes):
            r, c, r1, r2 = jobs[i1]
            subs.append(subgame(v, c, r1, r2, desc[c]))
            n += subs[-1].parent.shape[0]
            i1 += 1
        tree, off = _with_root(subs, v.g)
        s = cfr_load_tree(tree, variant=CFR_PLUS, precision=CFR_FP32, fuse_levels=0, device=device)
        cfr_iterate(s, iterations)
        st = cfr_get_state(s)
        cfr_set_state(s, st["strat_sum"], st["strat_sum"], st["iteration"])   # sigma := the average strategy
        cfr_iterate(s, 1)
        u1 = cfr_get_nodes(s, values_only=True)["u1"]
        s.close()
        for j in range(i0, i1):
            r, c, r1, r2 = jobs[j]
            D = desc[c].size
            vals = u1[off[j - i0] + 1 + np.arange(v.K) * D] / umax
            V = np.zeros((13, 13))
            V[v.x[1], v.x[2]] = vals
            X[j, :EMBED] = cut.embed[r]
            X[j, EMBED:EMBED + v.nx[1]] = r1
            X[j, EMBED + RANGE:EMBED + RANGE + v.nx[2]] = r2
            Y[j, :RANGE] = V.ravel()
            Y[j, RANGE:] = -V.ravel()
        i0 = i1
    return X, Y


def make_network(hidden=(1024, 1024, 1024), seed: int = 0, device=None):
    """The leaf network, He-initialised (seeded)."""
    dims = [EMBED + 2 * RANGE, *hidden, 2 * RANGE]
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x11E7]))
    flat = []
    for l in range(len(dims) - 1):
        flat.append(rng.normal(0.0, np.sqrt(2.0 / dims[l]), size=dims[l + 1] * dims[l]))
        flat.append(np.zeros(dims[l + 1]))
    net = cfr_mlp_create(dims, device=device)
    cfr_mlp_set_params(net, np.concatenate(flat).astype(np.float32))
    return net


def train(net, X, Y, steps: int = 2000, batch: int = 1024, lr: float = 1e-3, seed: int = 0, device=None):
    """Adam on minibatches drawn from (X, Y) (moved to the GPU once); the learning rate decays
    linearly to a tenth.  Returns the loss history (every 100 steps) of the full training set."""
    import torch

    dev = f"cuda:{device if device is not None else torch.cuda.current_device()}"
    Xd, Yd = torch.tensor(X, device=dev), torch.tensor(Y, device=dev)
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    n = Xd.shape[0]
    for step in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=g).to(dev)
        cfr_mlp_backward(net, Xd[idx], Yd[idx])
        cfr_mlp_adam(net, lr * (1.0 - 0.9 * step / max(steps, 1)))
        if step % 100 == 0 or step == steps - 1:
            hist.append(float(cfr_mlp_backward(net, Xd, Yd).item()))
    return hist


class DepthLimitedSolver:
    """CFR+ on the depth-limited game, its leaves refreshed from the network every `refresh` iterations
    (device-side: ranges -> network -> leaf utilities).  ranges: CFR_AVERAGE_STRATEGY (default; the
    leaves then settle as the average strategy converges) or CFR_CURRENT_STRATEGY."""

    def __init__(self, cut: Cut, net, refresh: int = 1, device=None, fuse_levels: int = -1,
                 ranges: int = CFR_AVERAGE_STRATEGY):
        import torch

        self.cut, self.net, self.refresh, self.ranges = cut, net, int(refresh), int(ranges)
        self.s = cfr_load_tree(cut.game, variant=CFR_PLUS, precision=CFR_FP32, device=device, fuse_levels=fuse_levels)
        dev = f"cuda:{device if device is not None else torch.cuda.current_device()}"
        rows = cut.cut_nodes.size
        self.x = torch.zeros((rows, EMBED + 2 * RANGE), dtype=torch.float32, device=dev)
        self.x[:, :EMBED] = torch.tensor(cut.embed, dtype=torch.float32, device=dev)
        self.y = torch.zeros((rows, 2 * RANGE), dtype=torch.float32, device=dev)
        self.umax = float(np.max(np.abs(cut.view.g.utility))) or 1.0
        cfr_set_range_program(self.s, cut.seg_dst, cut.seg_entries, cut.entry_prod, cut.slots)
        cfr_set_leaves(self.s, cut.leaf_nodes, cut.leaf_src)
        self.iteration = 0
        self._refresh()

    def _refresh(self):
        if self.cut.cut_nodes.size == 0:
            return
        cfr_gather_ranges(self.s, self.x, self.ranges)
        cfr_mlp_forward(self.net, self.x, out=self.y)
        cfr_set_leaf_values(self.s, self.y, self.umax)

    def iterate(self, n: int):
        done = 0
        while done < n:
            k = min(self.refresh - self.iteration % self.refresh, n - done)
            cfr_iterate(self.s, k)
            self.iteration += k
            done += k
            if self.iteration % self.refresh == 0:
                self._refresh()

    def exploitability(self) -> float:
        """Exploitability (NashConv / 2) in the depth-limited game with the leaves' current values."""
        return cfr_exploitability(self.s)[0] / 2.0

    def average_strategy(self) -> np.ndarray:
        return cfr_average_strategy(self.s)

    def close(self):
        self.s.close()


def blueprint_leaf_values(cut: Cut, strat_sum: np.ndarray, device=None):
    """The leaves' values in the network's output layout ([rows][338], FP32 CUDA tensor, divided by the
    payoff bound) when the full game is played by the average strategy of strat_sum (a full-game solve's
    strategy sums): each cut node's deal values under that play.  With these fixed leaves the
    depth-limited game's solution should reproduce the full solve above the cut - the check of the cut,
    the leaf indices and the combination, and the bound on what a perfect network could give."""
    import torch

    v = cut.view
    g = v.g
    s = cfr_load_tree(g, variant=CFR_PLUS, precision=CFR_FP32, fuse_levels=0, device=device)
    S = np.asarray(strat_sum, dtype=np.float64)
    cfr_set_state(s, S, S, 1)                  # sigma := the average strategy
    cfr_iterate(s, 1)
    u1 = cfr_get_nodes(s, values_only=True)["u1"]
    s.close()
    umax = float(np.max(np.abs(g.utility))) or 1.0
    rows = cut.cut_nodes.size
    y = np.zeros(rows * 2 * RANGE, np.float32)
    Pt = cut.top_public.size
    k = (cut.leaf_nodes.astype(np.int64) - 1) // Pt
    j = (cut.leaf_nodes.astype(np.int64) - 1) % Pt
    y[cut.leaf_src] = u1[v.node(k, cut.top_public[j])] / umax
    dev = f"cuda:{device if device is not None else torch.cuda.current_device()}"
    return torch.tensor(y.reshape(rows, 2 * RANGE), device=dev)


def solve_with_fixed_leaves(cut: Cut, y, iterations: int, device=None):
    """CFR+ on the depth-limited game with the leaves set once from y (the network output layout);
    returns the average strategy (depth-limited caller slots)."""
    s = cfr_load_tree(cut.game, variant=CFR_PLUS, precision=CFR_FP32, device=device)
    cfr_set_leaves(s, cut.leaf_nodes, cut.leaf_src)
    umax = float(np.max(np.abs(cut.view.g.utility))) or 1.0
    cfr_set_leaf_values(s, y, umax)
    cfr_iterate(s, iterations)
    avg = cfr_average_strategy(s)
    s.close()
    return avg


def combined_strategy(cut: Cut, top_avg: np.ndarray, below_avg: np.ndarray) -> np.ndarray:
    """A full-game strategy (caller slots of the full game): the depth-limited game's average strategy
    above the cut, below_avg (for instance a full-depth solve's) everywhere else."""
    out = np.array(below_avg, dtype=np.float64, copy=True)
    out[cut.slot_to_full] = top_avg
    return out


def full_game_exploitability(game, strategy: np.ndarray, device=None) -> float:
    """Exploitability (NashConv / 2) of a full-game strategy, by the library's best response."""
    s = cfr_load_tree(game, variant=CFR_PLUS, precision=CFR_FP32, device=device)
    q = np.asarray(strategy, dtype=np.float64)
    cfr_set_state(s, np.zeros_like(q), q, 1)
    nc = cfr_exploitability(s)[0]
    s.close()
    return nc / 2.0
