"""TEST INFRASTRUCTURE ONLY: the plain recursive FP64 CFR oracle (``cfr_oracle.c``).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package.  The product path (``paper_2408_14778_gb300``) never does, and this package never imports
the product path.  See the header of ``cfr_oracle.c`` for what is computed and which readings of
the paper it takes.

Arrays use the caller's ids throughout: node arrays in node-id order, infoset arrays in infoset-id
order, and "Q" arrays infoset-major over *all* infosets (chance infosets included), actions in
order.  Chance slots of regret/sum arrays stay zero; chance slots of strategy arrays hold sigma_0.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

VANILLA, CFR_PLUS, LINEAR, DISCOUNTED = 0, 1, 2, 3
AVG_UNIFORM, AVG_LINEAR = 0, 1


def build(force: bool = False) -> str:
    """Compile cfr_oracle.c into liboracle.so (plain gcc -O2; no fast-math; OpenMP for the
    multi-threaded passes where the compiler has it, else those passes run on one thread)."""
    src = os.path.join(_HERE, "cfr_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-ffp-contract=off", src, "-o", tmp, "-lm"]
    try:
        subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _SO)
    return _SO


_lib_handle = None
_P = ctypes.c_void_p


def _lib():
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(_SO):
            build()
        lib = ctypes.CDLL(_SO)
        lib.orc_create.restype = _P
        lib.orc_create.argtypes = [ctypes.c_int64, _P, _P, _P, ctypes.c_int32, _P, _P, _P, _P]
        lib.orc_destroy.argtypes = [_P]
        lib.orc_num_q.restype = ctypes.c_int64
        lib.orc_num_q.argtypes = [_P]
        lib.orc_root.restype = ctypes.c_int32
        lib.orc_root.argtypes = [_P]
        lib.orc_set_record.argtypes = [_P, ctypes.c_int32]
        lib.orc_iterate.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P]
        lib.orc_iterate_mt.restype = ctypes.c_int32
        lib.orc_iterate_mt.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                       ctypes.c_int32]
        lib.orc_max_threads.restype = ctypes.c_int32
        lib.orc_max_threads.argtypes = []
        lib.orc_get_state.argtypes = [_P, _P, _P, _P, _P, _P, _P]
        lib.orc_set_state.argtypes = [_P, _P, _P, ctypes.c_int64]
        lib.orc_get_nodes.restype = ctypes.c_int32
        lib.orc_get_nodes.argtypes = [_P, _P]
        lib.orc_get_cf_reach_sum.argtypes = [_P, _P]
        lib.orc_recall_violations.restype = ctypes.c_int64
        lib.orc_recall_violations.argtypes = [_P]
        lib.orc_average_strategy.argtypes = [_P, _P]
        lib.orc_best_response.restype = ctypes.c_double
        lib.orc_best_response.argtypes = [_P, ctypes.c_int32, _P, _P]
        lib.orc_expected_value.restype = ctypes.c_double
        lib.orc_expected_value.argtypes = [_P, ctypes.c_int32, _P]
        lib.orc_exploitability.argtypes = [_P, _P, _P, _P]
        _lib_handle = lib
    return _lib_handle


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def max_threads() -> int:
    """Host threads the multi-threaded passes use by default (1 if the oracle was built without OpenMP)."""
    return int(_lib().orc_max_threads())


class Oracle:
    """Recursive FP64 CFR on one game (see module docstring for array conventions)."""

    def __init__(self, game, record: bool = False):
        self._keep = [_c(game.parent, np.int32), _c(game.action, np.int32), _c(game.infoset, np.int32),
                      _c(game.infoset_player, np.int8), _c(game.infoset_num_actions, np.int32),
                      _c(game.chance_prob, np.float64), _c(game.utility, np.float64)]
        p, a, i, pl, na, cp, u = self._keep
        self.num_nodes = int(p.shape[0])
        self.num_infosets = int(pl.shape[0])
        self._h = _lib().orc_create(self.num_nodes, p.ctypes.data, a.ctypes.data, i.ctypes.data,
                                    self.num_infosets, pl.ctypes.data, na.ctypes.data,
                                    cp.ctypes.data if cp.size else None, u.ctypes.data)
        if not self._h:
            raise ValueError("oracle: arrays do not describe a valid game tree")
        self.num_q = int(_lib().orc_num_q(self._h))
        self.player = pl
        self.num_actions = na
        self.qbase = np.concatenate([[0], np.cumsum(na, dtype=np.int64)])
        self._keep = None if not record else self._keep
        if record:
            _lib().orc_set_record(self._h, 1)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib().orc_destroy(h)
            self._h = None

    @property
    def root(self) -> int:
        return int(_lib().orc_root(self._h))

    def iterate(self, n: int = 1, variant: int = VANILLA, avg: int = AVG_UNIFORM, alternating: bool = False,
                dcfr=(1.5, 0.0, 2.0), threads: int = 1):
        """Runs n CFR iterations; returns the root payoffs (u1, u2) of the last pass.  variant: VANILLA,
        CFR_PLUS, LINEAR or DISCOUNTED (with dcfr = (alpha, beta, gamma)); avg is ignored by the last two.
        threads != 1: each pass walks the root's subtrees on that many host threads (0: all), with the
        same results bit for bit; the count used is in ``last_threads``."""
        rv = np.zeros(2)
        d = np.asarray(dcfr, dtype=np.float64)
        if threads == 1:
            _lib().orc_iterate(self._h, int(n), int(variant), int(avg), int(bool(alternating)), d.ctypes.data,
                               rv.ctypes.data)
            self.last_threads = 1
        else:
            used = _lib().orc_iterate_mt(self._h, int(n), int(variant), int(avg), int(bool(alternating)),
                                         d.ctypes.data, rv.ctypes.data, int(threads))
            if used < 0:
                raise MemoryError("oracle: no memory for the multi-threaded pass")
            self.last_threads = int(used)
        return rv

    def state(self) -> dict:
        Q, H = max(self.num_q, 1), max(self.num_infosets, 1)
        R, S, inst, sig = (np.zeros(Q) for _ in range(4))
        own = np.zeros(H)
        T = ctypes.c_int64()
        _lib().orc_get_state(self._h, R.ctypes.data, S.ctypes.data, inst.ctypes.data, sig.ctypes.data,
                             own.ctypes.data, ctypes.byref(T))
        cfs = np.zeros(H)
        _lib().orc_get_cf_reach_sum(self._h, cfs.ctypes.data)
        q, h = self.num_q, self.num_infosets
        return dict(cum_regret=R[:q], strat_sum=S[:q], inst_regret=inst[:q], sigma=sig[:q], own_reach=own[:h],
                    cf_reach_sum=cfs[:h], iteration=int(T.value))

    def set_state(self, cum_regret, strat_sum, iteration: int):
        R = _c(cum_regret, np.float64)
        S = _c(strat_sum, np.float64)
        assert R.shape == (self.num_q,) and S.shape == (self.num_q,)
        _lib().orc_set_state(self._h, R.ctypes.data, S.ctypes.data, int(iteration))

    def nodes(self) -> dict:
        """Per node of the last pass (needs record=True): node payoffs u1, u2 (Eq. 1), counterfactual
        reaches cf1, cf2 (Eq. 2) and own reaches own1, own2 (Eq. 4)."""
        out = np.zeros((self.num_nodes, 6))
        if _lib().orc_get_nodes(self._h, out.ctypes.data) != 0:
            raise RuntimeError("oracle was created without record=True")
        return dict(u1=out[:, 0], u2=out[:, 1], cf1=out[:, 2], cf2=out[:, 3], own1=out[:, 4], own2=out[:, 5])

    def recall_violations(self) -> int:
        return int(_lib().orc_recall_violations(self._h))

    def average_strategy(self) -> np.ndarray:
        out = np.zeros(max(self.num_q, 1))
        _lib().orc_average_strategy(self._h, out.ctypes.data)
        return out[: self.num_q]

    def current_strategy(self) -> np.ndarray:
        return self.state()["sigma"]

    def best_response(self, player: int, profile, with_choice: bool = False):
        prof = _c(profile, np.float64)
        choice = np.zeros(max(self.num_infosets, 1), np.int32)
        v = _lib().orc_best_response(self._h, int(player), prof.ctypes.data, choice.ctypes.data)
        return (v, choice[: self.num_infosets]) if with_choice else v

    def expected_value(self, player: int, profile) -> float:
        prof = _c(profile, np.float64)
        return float(_lib().orc_expected_value(self._h, int(player), prof.ctypes.data))

    def exploitability(self, profile=None):
        """(NashConv, exploitability) of `profile` (default: the current average strategy)."""
        prof = _c(self.average_strategy() if profile is None else profile, np.float64)
        nc, ex = ctypes.c_double(), ctypes.c_double()
        _lib().orc_exploitability(self._h, prof.ctypes.data, ctypes.byref(nc), ctypes.byref(ex))
        return float(nc.value), float(ex.value)
