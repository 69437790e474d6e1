"""Seeded synthetic game inputs shared by the CUDA path's tests/bench and the oracle's tests.

This package builds inputs only: finite extensive-form games in the array form of the
Definition in Section 2.1 (parent function, action partition, information partition,
player partition, chance probabilities, utilities).  It performs none of the CFR
arithmetic.  The heavy lifting (trees up to ~1e8 nodes) is in ``gamegen.c``.

Families
--------
``public_private``   a seeded public tree hung below a root chance deal of private
                     buckets; infoset = (acting player, own bucket, public node).
``matrix_game``      a normal-form game written as a one-level tree (player 2 does not
                     observe player 1's action).
``config``           the three named workload shapes used throughout the repository:
                     ``bucket3_depth6`` (~1e3 nodes, vanilla CFR in FP64),
                     ``rank13_depth10`` (~2e6 nodes, 156-way deal, fold/showdown payoffs),
                     ``holdem169_depth12`` (~1e8 nodes, 1326-way deal bucketed to 169).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgamegen.so")

DEAL_BUCKET_PAIRS = 0
DEAL_HOLDEM_169 = 1
PAY_UNIFORM = 0
PAY_FOLD_SHOWDOWN = 1


def build(force: bool = False) -> str:
    """Compile gamegen.c into libgamegen.so next to it (gcc, OpenMP)."""
    src = os.path.join(_HERE, "gamegen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", src, "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("deal_kind", ctypes.c_int32),
        ("num_buckets", ctypes.c_int32),
        ("depth", ctypes.c_int32),
        ("amin", ctypes.c_int32),
        ("amax", ctypes.c_int32),
        ("p_cont", ctypes.c_double),
        ("p_chance", ctypes.c_double),
        ("payoff_kind", ctypes.c_int32),
        ("umax", ctypes.c_double),
        ("general_sum", ctypes.c_int32),
        ("first_actor", ctypes.c_int32),
    ]


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(_SO):
            build()
        lib = ctypes.CDLL(_SO)
        lib.gg_make_plan.restype = ctypes.c_void_p
        lib.gg_make_plan.argtypes = [ctypes.POINTER(_Params)]
        lib.gg_free_plan.argtypes = [ctypes.c_void_p]
        lib.gg_plan_counts.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
        lib.gg_fill.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 7
        _lib_handle = lib
    return _lib_handle


@dataclass
class GameDesc:
    """A finite extensive-form game as flat arrays (node order is arbitrary)."""

    parent: np.ndarray               # int32 [N]; -1 at the root
    action: np.ndarray               # int32 [N]; index in [0, |A(f_h(parent))|); -1 at the root
    infoset: np.ndarray              # int32 [N]; -1 at terminals
    infoset_player: np.ndarray       # int8  [H]; 0 = chance, 1, 2
    infoset_num_actions: np.ndarray  # int32 [H]
    chance_prob: np.ndarray          # float64, chance infosets in id order, actions in order
    utility: np.ndarray              # float64 [N, 2]; read at terminals only
    meta: dict = field(default_factory=dict)

    @property
    def num_nodes(self) -> int:
        return int(self.parent.shape[0])

    @property
    def num_infosets(self) -> int:
        return int(self.infoset_player.shape[0])

    @property
    def num_q(self) -> int:
        return int(self.infoset_num_actions.sum())


def _counts(plan) -> np.ndarray:
    out = (ctypes.c_int64 * 7)()
    _lib().gg_plan_counts(plan, out)
    return np.array(out[:], dtype=np.int64)


def _params(seed, deal_kind, num_buckets, depth, amin, amax, p_cont, p_chance, payoff_kind, umax,
            general_sum, first_actor) -> _Params:
    return _Params(int(seed) & 0xFFFFFFFFFFFFFFFF, deal_kind, num_buckets, depth, amin, amax, float(p_cont),
                   float(p_chance), payoff_kind, float(umax), int(bool(general_sum)), first_actor)


def public_size(**kw) -> int:
    """Number of game nodes the parameters produce, without writing the game."""
    prm = _params(**kw)
    plan = _lib().gg_make_plan(ctypes.byref(prm))
    if not plan:
        raise ValueError("invalid generator parameters")
    try:
        return int(_counts(plan)[0])
    finally:
        _lib().gg_free_plan(plan)


def public_private(seed: int = 0, deal_kind: int = DEAL_BUCKET_PAIRS, num_buckets: int = 3, depth: int = 6,
                   amin: int = 2, amax: int = 3, p_cont: float = 1.0, p_chance: float = 0.0,
                   payoff_kind: int = PAY_UNIFORM, umax: float = 2.0, general_sum: bool = False,
                   first_actor: int = 1) -> GameDesc:
    prm = _params(seed, deal_kind, num_buckets, depth, amin, amax, p_cont, p_chance, payoff_kind, umax,
                  general_sum, first_actor)
    lib = _lib()
    plan = lib.gg_make_plan(ctypes.byref(prm))
    if not plan:
        raise ValueError("invalid generator parameters")
    try:
        n, h, cq, k, pub, pdec, pterm = (int(x) for x in _counts(plan))
        parent = np.empty(n, np.int32)
        action = np.empty(n, np.int32)
        infoset = np.empty(n, np.int32)
        player = np.empty(h, np.int8)
        nact = np.empty(h, np.int32)
        cprob = np.empty(cq, np.float64)
        util = np.empty((n, 2), np.float64)
        lib.gg_fill(plan, *(a.ctypes.data for a in (parent, action, infoset, player, nact, cprob, util)))
    finally:
        lib.gg_free_plan(plan)
    meta = dict(seed=seed, deals=k, public_nodes=pub, public_decisions=pdec, public_terminals=pterm,
                depth=depth, amin=amin, amax=amax, p_cont=p_cont, p_chance=p_chance)
    return GameDesc(parent, action, infoset, player, nact, cprob, util, meta)


def fit_p_cont(target_nodes: int, tol: float = 0.1, **kw) -> float:
    """Bisection on the continuation probability so the game lands within +-tol of target_nodes."""
    lo, hi = 0.0, 1.0
    best, best_err = 0.5, float("inf")
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        n = public_size(p_cont=mid, **kw)
        err = abs(n - target_nodes) / target_nodes
        if err < best_err:
            best, best_err = mid, err
        if err <= tol * 0.25:
            break
        if n < target_nodes:
            lo = mid
        else:
            hi = mid
    if best_err > tol:
        raise ValueError(f"could not reach {target_nodes} nodes within {tol:.0%} (best {best_err:.1%})")
    return best


# Named workload shapes.  Sizes are realised counts of the seeded generator; callers report them.
CONFIGS = {
    # 6 ordered deals of 2 distinct buckets out of 3; depth 6 (deal + 5 decision levels); |A| in {2,3};
    # no early termination; u1 ~ U[-2, 2].
    "bucket3_depth6": dict(deal_kind=DEAL_BUCKET_PAIRS, num_buckets=3, depth=6, amin=2, amax=3,
                           payoff_kind=PAY_UNIFORM, umax=2.0, p_cont=1.0),
    # 156 ordered deals of 2 distinct ranks out of 13; depth 10; |A| in {3,4}; early cuts are folds,
    # last-level leaves showdowns; pot in {1,2,4,8}; ~2e6 nodes.
    "rank13_depth10": dict(deal_kind=DEAL_BUCKET_PAIRS, num_buckets=13, depth=10, amin=3, amax=4,
                           payoff_kind=PAY_FOLD_SHOWDOWN, umax=8.0, target_nodes=2_000_000),
    # 1326-way deal of 2-card combos bucketed to 169 classes; depth 12; |A| in {4,5}; u1 ~ U[-100, 100];
    # ~1e8 nodes.
    "holdem169_depth12": dict(deal_kind=DEAL_HOLDEM_169, depth=12, amin=4, amax=5,
                              payoff_kind=PAY_UNIFORM, umax=100.0, target_nodes=100_000_000),
}


def config(name: str, seed: int = 0, target_nodes: int | None = None, **override) -> GameDesc:
    """Build a named workload; ``target_nodes`` rescales the public tree (same family, other size),
    an explicit ``p_cont`` fixes the continuation probability instead of fitting a size."""
    kw = dict(CONFIGS[name])
    explicit_p = "p_cont" in override
    kw.update(override)
    tgt = target_nodes if target_nodes is not None else (None if explicit_p else kw.get("target_nodes"))
    kw.pop("target_nodes", None)
    if tgt is not None:
        kw["p_cont"] = fit_p_cont(tgt, seed=seed, **{k: v for k, v in _defaults(kw).items() if k != "p_cont"})
    g = public_private(seed=seed, **kw)
    g.meta["config"] = name
    return g


def _defaults(kw: dict) -> dict:
    d = dict(deal_kind=DEAL_BUCKET_PAIRS, num_buckets=3, depth=6, amin=2, amax=3, p_cont=1.0, p_chance=0.0,
             payoff_kind=PAY_UNIFORM, umax=2.0, general_sum=False, first_actor=1)
    d.update(kw)
    return d


def matrix_game(payoff: np.ndarray) -> GameDesc:
    """Zero-sum normal-form game (player-1 payoff matrix) as a one-level tree.

    Player 1 acts at the root (infoset 0); player 2 acts at one infoset (1) that holds every
    player-1 action, so player 2 does not observe it.  Node ids: 0 root, 1..m the player-2 nodes,
    then the m*n terminals.
    """
    A = np.asarray(payoff, dtype=np.float64)
    m, n = A.shape
    N = 1 + m + m * n
    parent = np.full(N, -1, np.int32)
    action = np.full(N, -1, np.int32)
    infoset = np.full(N, -1, np.int32)
    util = np.zeros((N, 2))
    infoset[0] = 0
    for i in range(m):
        parent[1 + i] = 0
        action[1 + i] = i
        infoset[1 + i] = 1
        for j in range(n):
            t = 1 + m + i * n + j
            parent[t] = 1 + i
            action[t] = j
            util[t] = (A[i, j], -A[i, j])
    return GameDesc(parent, action, infoset, np.array([1, 2], np.int8), np.array([m, n], np.int32),
                    np.zeros(0), util, dict(kind="matrix", shape=(m, n)))


def first_deals(g: GameDesc, k: int) -> GameDesc:
    """The sub-game of a ``public_private`` game holding only its first k deals.

    Nodes are emitted deal-major (root, then each deal's copy of the public tree), so the sub-game
    is the node prefix [0, 1 + k * P).  The root's chance infoset keeps k outcomes with probability
    1/k each; every other infoset keeps its id (some are left without nodes).
    """
    K, P = int(g.meta["deals"]), int(g.meta["public_nodes"])
    k = max(1, min(int(k), K))
    n = 1 + k * P
    nact = g.infoset_num_actions.copy()
    nact[0] = k
    cprob = np.concatenate([np.full(k, 1.0 / k), g.chance_prob[K:]])
    meta = dict(g.meta)
    meta.update(deals=k, sample_of=g.num_nodes)
    return GameDesc(g.parent[:n].copy(), g.action[:n].copy(), g.infoset[:n].copy(), g.infoset_player.copy(), nact,
                    cprob, g.utility[:n].copy(), meta)


def permute_nodes(g: GameDesc, seed: int) -> GameDesc:
    """Same game with node ids relabelled by a seeded permutation (tests order independence)."""
    rng = np.random.default_rng(seed)
    n = g.num_nodes
    perm = rng.permutation(n).astype(np.int64)       # new id of old node i is perm[i]
    parent = np.full(n, -1, np.int32)
    action = np.empty(n, np.int32)
    infoset = np.empty(n, np.int32)
    util = np.empty_like(g.utility)
    old_par = g.parent.astype(np.int64)
    newpar = np.where(old_par >= 0, perm[np.maximum(old_par, 0)], -1)
    parent[perm] = newpar.astype(np.int32)
    action[perm] = g.action
    infoset[perm] = g.infoset
    util[perm] = g.utility
    meta = dict(g.meta)
    meta["permutation_seed"] = seed
    meta["perm"] = perm
    return GameDesc(parent, action, infoset, g.infoset_player.copy(), g.infoset_num_actions.copy(),
                    g.chance_prob.copy(), util, meta)


def batch_subgames(count: int, seed: int = 0, min_nodes: float = 1e2, max_nodes: float = 1e5,
                   min_depth: int = 4, max_depth: int = 10) -> list:
    """Independent seeded subgames for batched solving: sizes log-uniform in [min_nodes, max_nodes],
    depth uniform over the depths in [min_depth, max_depth] whose full public tree reaches the drawn
    size (a large size rules out the shallow depths; if none reaches it, the deepest), 2..5 actions per
    public node, the 6-deal bucket game's deal and U[-2, 2] payoffs.  The size fit is the continuation
    probability's bisection (+-10%); where small trees only change size in large steps, the closest size
    on a grid of continuation probabilities that is not below min_nodes, and the size is kept within
    [min_nodes, 1.1 max_nodes]."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5B6A]))
    out = []
    kw = dict(deal_kind=DEAL_BUCKET_PAIRS, num_buckets=3, amin=2, amax=5, payoff_kind=PAY_UNIFORM, umax=2.0,
              p_chance=0.0, general_sum=False, first_actor=1)
    for i in range(count):
        target = int(round(float(np.exp(rng.uniform(np.log(min_nodes), np.log(max_nodes))))))
        sub_seed = int(rng.integers(0, 2**62))
        u = float(rng.uniform())
        # the full tree grows with the depth: the depths that reach the size are d0 .. max_depth
        full = {}
        d0 = max_depth
        for d in range(min_depth, max_depth + 1):
            full[d] = public_size(seed=sub_seed, depth=d, p_cont=1.0, **kw)
            if full[d] >= target:
                d0 = d
                break
        ok = list(range(d0, max_depth + 1))
        first = min(int(u * len(ok)), len(ok) - 1)
        depth, p = ok[first], 1.0
        for depth in ok[first:] + ok[:first][::-1]:     # the drawn depth, else the next ones that fit
            if depth not in full:
                full[depth] = public_size(seed=sub_seed, depth=depth, p_cont=1.0, **kw)
            p = _fit_subgame(target, full[depth], min_nodes, max_nodes, seed=sub_seed, depth=depth, **kw)
            if p is not None:
                break
        g = public_private(seed=sub_seed, depth=depth, p_cont=1.0 if p is None else p, **kw)
        g.meta.update(config="batch_subgame", target_nodes=target, batch_index=i, depth=depth)
        out.append(g)
    return out


def _fit_subgame(target: int, full: int, min_nodes: float, max_nodes: float, **kw):
    """Continuation probability giving about target nodes within [min_nodes, 1.1 max_nodes] (full: the
    size at p = 1), or None."""
    if full <= target * 1.1:
        return 1.0 if min_nodes <= full <= 1.1 * max_nodes else None
    try:
        return fit_p_cont(target, **kw)
    except ValueError:       # small trees change size in steps of whole subtrees: the closest allowed size
        grid = np.linspace(0.0, 1.0, 201)
        sizes = np.array([public_size(p_cont=float(q), **kw) for q in grid])
        allowed = (sizes >= min_nodes) & (sizes <= 1.1 * max_nodes)
        if not allowed.any():
            return None
        err = np.where(allowed, np.abs(np.log(sizes / target)), np.inf)
        return float(grid[int(np.argmin(err))])


def with_chance_root(games: list) -> GameDesc:
    """The games under one uniform chance root (one tree): a plain single-tree solver then runs them
    all at once, each game's regrets scaled by the root's probability (which regret matching ignores)."""
    k = len(games)
    sizes = [g.num_nodes for g in games]
    hs = [g.num_infosets for g in games]
    N = 1 + sum(sizes)
    parent = np.empty(N, np.int32)
    action = np.empty(N, np.int32)
    infoset = np.empty(N, np.int32)
    util = np.zeros((N, 2))
    parent[0], action[0], infoset[0] = -1, -1, 0
    players, nacts, probs = [np.array([0], np.int8)], [np.array([k], np.int32)], [np.full(k, 1.0 / k)]
    off, hoff = 1, 1
    for i, g in enumerate(games):
        n = g.num_nodes
        p = g.parent.astype(np.int64)
        parent[off:off + n] = np.where(p < 0, 0, p + off)
        action[off:off + n] = np.where(p < 0, i, g.action)
        infoset[off:off + n] = np.where(g.infoset < 0, -1, g.infoset + hoff)
        util[off:off + n] = g.utility
        players.append(g.infoset_player)
        nacts.append(g.infoset_num_actions)
        probs.append(g.chance_prob)
        off += n
        hoff += g.num_infosets
    return GameDesc(parent, action, infoset, np.concatenate(players).astype(np.int8),
                    np.concatenate(nacts).astype(np.int32), np.concatenate(probs), util,
                    meta=dict(config="chance_root_of_batch", games=k))
