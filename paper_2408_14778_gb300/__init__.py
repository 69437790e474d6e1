"""Python binding of libcfr_gb300.so (include/cfr_gb300.h): argument marshalling only.

Every step of a CFR iteration runs in the library's CUDA kernels; this module converts numpy
arrays to the C structures, passes PyTorch's current CUDA stream and (optionally) PyTorch's
caching allocator to the library, and turns status codes into exceptions.  There is no CPU
fallback: if the shared library is missing, importing the binding's entry points raises.

Functions carry the C names (``cfr_load_tree``, ``cfr_iterate``, ...).  ``Solver`` bundles them.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from ._build import LIB as _LIB_PATH
from ._build import build as _build_library

CFR_OK, CFR_ERR_INVALID, CFR_ERR_CUDA, CFR_ERR_OOM, CFR_ERR_TIMEOUT, CFR_ERR_STATE, CFR_ERR_UNSUPPORTED = range(7)
CFR_VANILLA, CFR_PLUS, CFR_LINEAR, CFR_DISCOUNTED = 0, 1, 2, 3
CFR_FP32, CFR_FP64 = 0, 1
CFR_SIMULTANEOUS, CFR_ALTERNATING = 0, 1
CFR_AVG_DEFAULT, CFR_AVG_UNIFORM, CFR_AVG_LINEAR = -1, 0, 1
CFR_PHASE_TOPDOWN, CFR_PHASE_BOTTOMUP, CFR_PHASE_FUSED, CFR_PHASE_UPDATE, CFR_PHASE_OWN = 0, 1, 2, 3, 4
CFR_PHASE_TOPDOWN_PAIR, CFR_PHASE_BOTTOMUP_PAIR = 5, 6

_STATUS_NAMES = {0: "CFR_OK", 1: "CFR_ERR_INVALID", 2: "CFR_ERR_CUDA", 3: "CFR_ERR_OOM", 4: "CFR_ERR_TIMEOUT",
                 5: "CFR_ERR_STATE", 6: "CFR_ERR_UNSUPPORTED"}


class CfrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class _GameDesc(ctypes.Structure):
    _fields_ = [
        ("num_nodes", ctypes.c_int64),
        ("parent", ctypes.c_void_p),
        ("action", ctypes.c_void_p),
        ("infoset", ctypes.c_void_p),
        ("num_infosets", ctypes.c_int32),
        ("infoset_player", ctypes.c_void_p),
        ("infoset_num_actions", ctypes.c_void_p),
        ("chance_prob", ctypes.c_void_p),
        ("num_chance_prob", ctypes.c_int64),
        ("utility", ctypes.c_void_p),
    ]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class _Config(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("update_mode", ctypes.c_int32),
        ("avg_weight", ctypes.c_int32),
        ("device", ctypes.c_int32),
        ("cuda_stream", ctypes.c_void_p),
        ("dev_alloc", _ALLOC_FN),
        ("dev_free", _FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
        ("fuse_levels", ctypes.c_int32),
        ("record_nodes", ctypes.c_int32),
        ("dcfr_alpha", ctypes.c_double),
        ("dcfr_beta", ctypes.c_double),
        ("dcfr_gamma", ctypes.c_double),
        ("head_levels", ctypes.c_int32),
        ("batch_split_nodes", ctypes.c_int64),
        ("tail_slots", ctypes.c_int32),
    ]


class _Info(ctypes.Structure):
    _fields_ = [
        ("num_nodes", ctypes.c_int64), ("num_decision", ctypes.c_int64), ("num_terminal", ctypes.c_int64),
        ("num_q", ctypes.c_int64), ("num_infosets", ctypes.c_int32), ("num_levels", ctypes.c_int32),
        ("max_depth", ctypes.c_int32), ("max_actions", ctypes.c_int32), ("single_level_infosets", ctypes.c_int32),
        ("variant", ctypes.c_int32), ("precision", ctypes.c_int32), ("update_mode", ctypes.c_int32),
        ("avg_weight", ctypes.c_int32), ("iteration", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
        ("bytes_per_iteration", ctypes.c_int64), ("kernels_per_iteration", ctypes.c_int32),
        ("kernel_launches", ctypes.c_int64), ("fused_from_depth", ctypes.c_int32), ("fused_tiles", ctypes.c_int32),
        ("head_depths", ctypes.c_int32), ("tail_kernel", ctypes.c_int32), ("pair_depth", ctypes.c_int32),
    ]


class _BatchTuning(ctypes.Structure):
    _fields_ = [("threads_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [
        ("num_games", ctypes.c_int32), ("num_nodes", ctypes.c_int64), ("num_decision", ctypes.c_int64),
        ("num_q", ctypes.c_int64), ("iteration", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
        ("threads_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("grid", ctypes.c_int32),
        ("tuned", ctypes.c_int32), ("kernel_launches", ctypes.c_int64), ("forest_games", ctypes.c_int32),
        ("forest_nodes", ctypes.c_int64), ("split_nodes", ctypes.c_int64), ("smem_bytes", ctypes.c_int64),
        ("forest_bytes_per_iteration", ctypes.c_int64), ("forest_head_depths", ctypes.c_int32),
    ]


_lib_handle = None
_P = ctypes.c_void_p


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles libcfr_gb300.so in-tree (nvcc, sm_103a)."""
    return _build_library(force=force, verbose=verbose)


def library_path() -> str:
    return _LIB_PATH


def lib():
    """The loaded shared library; raises if it has not been built."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_2408_14778_gb300.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(_LIB_PATH)
        L.cfr_config_init.argtypes = [ctypes.POINTER(_Config)]
        L.cfr_config_init.restype = None
        L.cfr_validate.argtypes = [ctypes.POINTER(_GameDesc), ctypes.c_char_p, ctypes.c_size_t]
        L.cfr_layout_digest.argtypes = [ctypes.POINTER(_GameDesc), ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_uint64)]
        L.cfr_layout_digest.restype = ctypes.c_int
        L.cfr_load_tree.argtypes = [ctypes.POINTER(_GameDesc), ctypes.POINTER(_Config), ctypes.POINTER(_P)]
        L.cfr_iterate.argtypes = [_P, ctypes.c_int32]
        L.cfr_synchronize.argtypes = [_P]
        L.cfr_average_strategy.argtypes = [_P, _P, ctypes.c_int64]
        L.cfr_current_strategy.argtypes = [_P, _P, ctypes.c_int64]
        L.cfr_exploitability.argtypes = [_P, _P, _P]
        L.cfr_get_state.argtypes = [_P, _P, _P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P]
        L.cfr_set_state.argtypes = [_P, _P, _P, ctypes.c_int64, ctypes.c_int64]
        L.cfr_get_nodes.argtypes = [_P, _P, _P, _P, ctypes.c_int64]
        L.cfr_get_info.argtypes = [_P, ctypes.POINTER(_Info)]
        L.cfr_root_value.argtypes = [_P, _P]
        L.cfr_root_value_async.argtypes = [_P, _P]
        L.cfr_phase_times.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int32, _P]
        L.cfr_phase_times.restype = ctypes.c_int
        L.cfr_exploitability_static.argtypes = [_P, _P, _P]
        L.cfr_exploitability_static.restype = ctypes.c_int
        L.cfr_last_error.argtypes = [_P]
        L.cfr_last_error.restype = ctypes.c_char_p
        L.cfr_free.argtypes = [_P]
        L.cfr_free.restype = None
        L.cfr_batch_load.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(_Config), ctypes.POINTER(_P)]
        L.cfr_batch_iterate.argtypes = [_P, ctypes.c_int32]
        L.cfr_batch_set_tuning.argtypes = [_P, ctypes.POINTER(_BatchTuning)]
        L.cfr_batch_autotune.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(_BatchTuning), _P]
        L.cfr_batch_game_times.argtypes = [_P, _P, ctypes.c_int32]
        L.cfr_batch_exploitability.argtypes = [_P, _P, ctypes.c_int32]
        L.cfr_batch_get_state.argtypes = [_P, ctypes.c_int32, _P, _P, ctypes.c_int64, _P]
        L.cfr_batch_average_strategy.argtypes = [_P, ctypes.c_int32, _P, ctypes.c_int64]
        L.cfr_batch_get_info.argtypes = [_P, ctypes.POINTER(_BatchInfo)]
        L.cfr_batch_last_error.argtypes = [_P]
        L.cfr_batch_last_error.restype = ctypes.c_char_p
        L.cfr_batch_free.argtypes = [_P]
        L.cfr_batch_free.restype = None
        L.cfr_set_range_program.argtypes = [_P, ctypes.c_int64, _P, _P, _P, _P]
        L.cfr_gather_ranges.argtypes = [_P, _P, ctypes.c_int32]
        L.cfr_set_leaves.argtypes = [_P, _P, _P, ctypes.c_int64]
        L.cfr_set_leaf_values.argtypes = [_P, _P, ctypes.c_double]
        for name in ("cfr_set_range_program", "cfr_gather_ranges", "cfr_set_leaves", "cfr_set_leaf_values"):
            getattr(L, name).restype = ctypes.c_int
        L.cfr_mlp_create.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.POINTER(_P)]
        L.cfr_mlp_num_params.argtypes = [_P]
        L.cfr_mlp_num_params.restype = ctypes.c_int64
        for name in ("cfr_mlp_set_params", "cfr_mlp_get_params", "cfr_mlp_get_grads"):
            getattr(L, name).argtypes = [_P, _P, ctypes.c_int64]
        L.cfr_mlp_forward.argtypes = [_P, _P, ctypes.c_int32, _P]
        L.cfr_mlp_backward.argtypes = [_P, _P, _P, ctypes.c_int32, _P]
        L.cfr_mlp_adam.argtypes = [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
        L.cfr_mlp_gemm_stats.argtypes = [_P, _P, _P, _P, _P]
        L.cfr_mlp_set_tensor_path.argtypes = [_P, ctypes.c_int32]
        L.cfr_mlp_synchronize.argtypes = [_P]
        L.cfr_mlp_get_intermediate.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int64]
        L.cfr_mlp_last_error.argtypes = [_P]
        L.cfr_mlp_last_error.restype = ctypes.c_char_p
        L.cfr_mlp_free.argtypes = [_P]
        L.cfr_mlp_free.restype = None
        for name in ("cfr_mlp_create", "cfr_mlp_set_params", "cfr_mlp_get_params", "cfr_mlp_get_grads",
                     "cfr_mlp_forward", "cfr_mlp_backward", "cfr_mlp_adam", "cfr_mlp_gemm_stats",
                     "cfr_mlp_set_tensor_path", "cfr_mlp_synchronize", "cfr_mlp_get_intermediate"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("cfr_batch_load", "cfr_batch_iterate", "cfr_batch_set_tuning", "cfr_batch_autotune",
                     "cfr_batch_game_times", "cfr_batch_exploitability", "cfr_batch_get_state",
                     "cfr_batch_average_strategy", "cfr_batch_get_info"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("cfr_validate", "cfr_load_tree", "cfr_iterate", "cfr_synchronize", "cfr_average_strategy",
                     "cfr_current_strategy", "cfr_exploitability", "cfr_get_state", "cfr_set_state", "cfr_get_nodes",
                     "cfr_get_info", "cfr_root_value", "cfr_root_value_async"):
            getattr(L, name).restype = ctypes.c_int
        _lib_handle = L
    return _lib_handle


def declared_functions() -> list[str]:
    """Names of the functions include/cfr_gb300.h declares (used to check the exports)."""
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "cfr_gb300.h")
    text = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(cfr_[a-z_]+)\s*\(", text)) - {"cfr_alloc_fn", "cfr_free_fn"})


def _check(st: int, solver_handle=None):
    if st != CFR_OK:
        msg = lib().cfr_last_error(solver_handle)
        raise CfrError(st, msg.decode(errors="replace") if msg else "")


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class _Desc:
    """Keeps the marshalled arrays alive for the duration of a call."""

    def __init__(self, game):
        self.arrays = [_arr(game.parent, np.int32), _arr(game.action, np.int32), _arr(game.infoset, np.int32),
                       _arr(game.infoset_player, np.int8), _arr(game.infoset_num_actions, np.int32),
                       _arr(game.chance_prob, np.float64), _arr(game.utility, np.float64)]
        p, a, i, pl, na, cp, u = self.arrays
        if u.ndim != 2 or u.shape != (p.shape[0], 2):
            raise ValueError("utility must have shape (num_nodes, 2)")
        self.c = _GameDesc(p.shape[0], p.ctypes.data, a.ctypes.data, i.ctypes.data, pl.shape[0], pl.ctypes.data,
                           na.ctypes.data, cp.ctypes.data if cp.size else None, cp.shape[0], u.ctypes.data)


def cfr_validate(game) -> tuple[int, str]:
    """(status, message) without touching the GPU."""
    d = _Desc(game)
    buf = ctypes.create_string_buffer(512)
    st = lib().cfr_validate(ctypes.byref(d.c), buf, len(buf))
    return st, buf.value.decode(errors="replace")


def cfr_layout_digest(game, builder: int, forest: bool = False) -> tuple[int, int, str]:
    """(status, hash of the host layout, message) from the one-thread (0) or multi-threaded (1) builder."""
    d = _Desc(game)
    h = ctypes.c_uint64()
    st = lib().cfr_layout_digest(ctypes.byref(d.c), int(builder), int(bool(forest)), ctypes.byref(h))
    msg = lib().cfr_last_error(None)
    return st, h.value, (msg.decode(errors="replace") if (st and msg) else "")


class _TorchAllocator:
    """Routes the library's device allocations through PyTorch's caching allocator."""

    def __init__(self, device: int, stream: int):
        import torch

        self.torch = torch
        self.device, self.stream = device, stream
        self.alloc = _ALLOC_FN(self._alloc)
        self.free = _FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
        except Exception:  # noqa: BLE001 - reported to the library as NULL (CFR_ERR_OOM)
            return None

    def _free(self, ptr, ctx):
        try:
            self.torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:  # noqa: BLE001
            pass


def cfr_load_tree(game, variant=CFR_VANILLA, precision=CFR_FP32, update_mode=CFR_SIMULTANEOUS,
                  avg_weight=CFR_AVG_DEFAULT, device=None, stream=None, allocator: str = "torch",
                  fuse_levels: int = -1, record_nodes: bool = False, dcfr=(1.5, 0.0, 2.0), head_levels: int = -1,
                  tail_slots: int = 0):
    """Loads a game and returns a Solver.  stream: None = PyTorch's current stream on the device.
    fuse_levels / record_nodes / head_levels / tail_slots: cfr_config's fields of the same names; dcfr:
    (alpha, beta, gamma) of CFR_DISCOUNTED."""
    import torch

    if not torch.cuda.is_available():
        raise CfrError(CFR_ERR_CUDA, "no CUDA device is available")
    dev = torch.cuda.current_device() if device is None else int(device)
    st_handle = torch.cuda.current_stream(dev).cuda_stream if stream is None else int(stream)
    cfg = _Config()
    lib().cfr_config_init(ctypes.byref(cfg))
    cfg.variant, cfg.precision, cfg.update_mode, cfg.avg_weight = variant, precision, update_mode, avg_weight
    cfg.device = dev
    cfg.cuda_stream = st_handle
    cfg.fuse_levels = int(fuse_levels)
    cfg.record_nodes = 1 if record_nodes else 0
    cfg.head_levels = int(head_levels)
    cfg.tail_slots = int(tail_slots)
    cfg.dcfr_alpha, cfg.dcfr_beta, cfg.dcfr_gamma = (float(x) for x in dcfr)
    alloc = None
    if allocator == "torch":
        alloc = _TorchAllocator(dev, st_handle)
        cfg.dev_alloc, cfg.dev_free = alloc.alloc, alloc.free
    elif allocator != "cuda":
        raise ValueError("allocator must be 'torch' or 'cuda'")
    d = _Desc(game)
    h = _P()
    _check(lib().cfr_load_tree(ctypes.byref(d.c), ctypes.byref(cfg), ctypes.byref(h)))
    return Solver(h, alloc)


def cfr_iterate(s: "Solver", n: int = 1):
    _check(lib().cfr_iterate(s.handle, int(n)), s.handle)


def cfr_synchronize(s: "Solver"):
    _check(lib().cfr_synchronize(s.handle), s.handle)


def cfr_average_strategy(s: "Solver") -> np.ndarray:
    out = np.empty(max(s.num_q, 1))
    _check(lib().cfr_average_strategy(s.handle, out.ctypes.data, out.shape[0]), s.handle)
    return out[: s.num_q]


def cfr_current_strategy(s: "Solver") -> np.ndarray:
    out = np.empty(max(s.num_q, 1))
    _check(lib().cfr_current_strategy(s.handle, out.ctypes.data, out.shape[0]), s.handle)
    return out[: s.num_q]


def cfr_exploitability(s: "Solver") -> tuple[float, float]:
    nc, ex = ctypes.c_double(), ctypes.c_double()
    _check(lib().cfr_exploitability(s.handle, ctypes.byref(nc), ctypes.byref(ex)), s.handle)
    return nc.value, ex.value


def cfr_exploitability_static(s: "Solver") -> tuple[float, float]:
    """cfr_exploitability with its working memory in the library's fixed per-GPU region.

    For callers that may not allocate device memory while running (fixed memory budget, real-time
    loops).  Games needing more than CFR_STATIC_SCRATCH_BYTES raise CFR_ERR_UNSUPPORTED.  The first
    call on a device performs a one-time set-up and should come before any stream capture; calls
    that overlap on the GPU share the region and race.  This wrapper allocates no device memory.
    """
    nc, ex = ctypes.c_double(), ctypes.c_double()
    _check(lib().cfr_exploitability_static(s.handle, ctypes.byref(nc), ctypes.byref(ex)), s.handle)
    return nc.value, ex.value


CFR_STATIC_SCRATCH_BYTES = 32 << 20


def cfr_get_state(s: "Solver") -> dict:
    q, h = max(s.num_q, 1), max(s.num_infosets, 1)
    R, S, inst, own = np.empty(q), np.empty(q), np.empty(q), np.empty(h)
    it = ctypes.c_int64()
    _check(lib().cfr_get_state(s.handle, R.ctypes.data, S.ctypes.data, inst.ctypes.data, q, own.ctypes.data, h,
                               ctypes.byref(it)), s.handle)
    return dict(cum_regret=R[: s.num_q], strat_sum=S[: s.num_q], inst_regret=inst[: s.num_q],
                own_reach=own[: s.num_infosets], iteration=it.value)


def cfr_set_state(s: "Solver", cum_regret, strat_sum, iteration: int):
    R, S = _arr(cum_regret, np.float64), _arr(strat_sum, np.float64)
    _check(lib().cfr_set_state(s.handle, R.ctypes.data, S.ctypes.data, R.shape[0], int(iteration)), s.handle)


def cfr_get_nodes(s: "Solver", values_only: bool = False) -> dict:
    """Per node of the last iteration: u1 (Eq. 1) and, unless values_only, the counterfactual reaches."""
    n = s.num_nodes
    u = np.empty(n)
    r1, r2 = (None, None) if values_only else (np.empty(n), np.empty(n))
    _check(lib().cfr_get_nodes(s.handle, u.ctypes.data, None if r1 is None else r1.ctypes.data,
                               None if r2 is None else r2.ctypes.data, n), s.handle)
    return dict(u1=u) if values_only else dict(u1=u, cf_reach1=r1, cf_reach2=r2)


def cfr_root_value(s: "Solver") -> float:
    """u-check(sigma^T, v_0, 1) of the last iteration (synchronises the solver's stream)."""
    v = ctypes.c_double()
    _check(lib().cfr_root_value(s.handle, ctypes.byref(v)), s.handle)
    return v.value


def cfr_root_value_async(s: "Solver", dst: int):
    """Enqueues the write of u-check(sigma^T, v_0, 1) as a float64 to dst (the address of page-locked host
    memory, e.g. a pinned torch tensor's data_ptr()) on the solver's stream; it is there once the stream
    has passed this point."""
    _check(lib().cfr_root_value_async(s.handle, ctypes.c_void_p(int(dst))), s.handle)


def cfr_phase_times(s: "Solver") -> list:
    """Runs one iteration as individually timed kernels (it counts as an iteration) and returns its
    phases in launch order, each a dict: name, kind (CFR_PHASE_*), depth, us and algorithmic bytes."""
    n = ctypes.c_int32()
    _check(lib().cfr_phase_times(s.handle, None, None, None, None, 0, ctypes.byref(n)), s.handle)
    if n.value == 0:
        return []
    us, by = np.zeros(n.value), np.zeros(n.value)
    kind, depth = np.zeros(n.value, np.int32), np.zeros(n.value, np.int32)
    _check(lib().cfr_phase_times(s.handle, us.ctypes.data, by.ctypes.data, kind.ctypes.data, depth.ctypes.data,
                                 n.value, ctypes.byref(n)), s.handle)
    names = {CFR_PHASE_TOPDOWN: "top-down depth {}", CFR_PHASE_BOTTOMUP: "bottom-up depth {}",
             CFR_PHASE_FUSED: "fused depths {}+", CFR_PHASE_UPDATE: "update", CFR_PHASE_OWN: "own reaches",
             CFR_PHASE_TOPDOWN_PAIR: "top-down depths {}-{}", CFR_PHASE_BOTTOMUP_PAIR: "bottom-up depths {}-{}"}
    return [dict(name=names[int(k)].format(int(d), int(d) + 1), kind=int(k), depth=int(d), us=float(u), bytes=float(b))
            for k, d, u, b in zip(kind, depth, us, by)]


def cfr_set_range_program(s: "Solver", seg_dst, seg_entries, entry_prod, slots):
    """Registers the range program of cfr_gather_ranges (include/cfr_gb300.h)."""
    d, e, p = _arr(seg_dst, np.int64), _arr(seg_entries, np.int64), _arr(entry_prod, np.int64)
    sl = _arr(slots, np.int32)
    _check(lib().cfr_set_range_program(s.handle, d.size, d.ctypes.data, e.ctypes.data, p.ctypes.data,
                                       sl.ctypes.data if sl.size else None), s.handle)


CFR_CURRENT_STRATEGY, CFR_AVERAGE_STRATEGY = 0, 1


def cfr_gather_ranges(s: "Solver", out, strategy: int = CFR_CURRENT_STRATEGY):
    """Writes the range program's output into out (an FP32 CUDA tensor), queued on the solver's stream,
    from the current (CFR_CURRENT_STRATEGY) or the average strategy (CFR_AVERAGE_STRATEGY)."""
    _check(lib().cfr_gather_ranges(s.handle, out.data_ptr(), int(strategy)), s.handle)


def cfr_set_leaves(s: "Solver", nodes, src_index):
    n, si = _arr(nodes, np.int32), _arr(src_index, np.int64)
    if n.size != si.size:
        raise ValueError("nodes and src_index need the same length")
    _check(lib().cfr_set_leaves(s.handle, n.ctypes.data if n.size else None, si.ctypes.data if si.size else None,
                                n.size), s.handle)


def cfr_set_leaf_values(s: "Solver", src, scale: float = 1.0):
    """Leaf utilities from src (an FP32 CUDA tensor), queued on the solver's stream."""
    _check(lib().cfr_set_leaf_values(s.handle, src.data_ptr(), float(scale)), s.handle)


def cfr_get_info(s: "Solver") -> dict:
    info = _Info()
    _check(lib().cfr_get_info(s.handle, ctypes.byref(info)), s.handle)
    return {name: getattr(info, name) for name, _ in _Info._fields_}


def cfr_free(s: "Solver"):
    s.close()


class Solver:
    """A loaded game on the GPU (owns the C handle)."""

    def __init__(self, handle, allocator=None):
        self.handle = handle
        self._allocator = allocator          # keeps the ctypes callbacks alive
        info = cfr_get_info(self)
        self.num_nodes = info["num_nodes"]
        self.num_q = info["num_q"]
        self.num_infosets = info["num_infosets"]

    def close(self):
        if self.handle:
            lib().cfr_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    iterate = cfr_iterate
    synchronize = cfr_synchronize
    average_strategy = cfr_average_strategy
    current_strategy = cfr_current_strategy
    exploitability = cfr_exploitability
    get_state = cfr_get_state
    set_state = cfr_set_state
    get_nodes = cfr_get_nodes
    root_value = cfr_root_value
    root_value_async = cfr_root_value_async
    phase_times = cfr_phase_times
    info = cfr_get_info


# ---- batched solving -------------------------------------------------------------------------------

def _check_batch(st: int, handle=None):
    if st != CFR_OK:
        msg = lib().cfr_batch_last_error(handle)
        raise CfrError(st, msg.decode(errors="replace") if msg else "")


class Batch:
    """Many independent games solved side by side on the GPU (owns the C handle)."""

    def __init__(self, handle, allocator, games):
        self.handle = handle
        self._allocator = allocator
        self.num_games = len(games)
        self.num_q = [int(np.sum(g.infoset_num_actions)) for g in games]
        self.num_nodes = [int(g.num_nodes) for g in games]

    def close(self):
        if self.handle:
            lib().cfr_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def cfr_batch_load(games, variant=CFR_PLUS, avg_weight=CFR_AVG_DEFAULT, device=None, stream=None,
                   allocator: str = "torch", dcfr=(1.5, 0.0, 2.0), split_nodes: int = 0,
                   update_mode=CFR_SIMULTANEOUS, head_levels: int = -1, fuse_levels: int = -1) -> Batch:
    """Loads a list of games for batched solving (FP32 mode).  split_nodes: cfr_config.batch_split_nodes
    (0 default, negative: every game whose image fits shared memory in the persistent kernel);
    head_levels and fuse_levels: cfr_config.head_levels and cfr_config.fuse_levels of the forest part."""
    import torch

    if not torch.cuda.is_available():
        raise CfrError(CFR_ERR_CUDA, "no CUDA device is available")
    dev = torch.cuda.current_device() if device is None else int(device)
    st_handle = torch.cuda.current_stream(dev).cuda_stream if stream is None else int(stream)
    cfg = _Config()
    lib().cfr_config_init(ctypes.byref(cfg))
    cfg.variant, cfg.precision, cfg.avg_weight = variant, CFR_FP32, avg_weight
    cfg.device, cfg.cuda_stream = dev, st_handle
    cfg.dcfr_alpha, cfg.dcfr_beta, cfg.dcfr_gamma = (float(x) for x in dcfr)
    cfg.batch_split_nodes = int(split_nodes)
    cfg.update_mode = int(update_mode)
    cfg.head_levels = int(head_levels)
    cfg.fuse_levels = int(fuse_levels)
    alloc = None
    if allocator == "torch":
        alloc = _TorchAllocator(dev, st_handle)
        cfg.dev_alloc, cfg.dev_free = alloc.alloc, alloc.free
    elif allocator != "cuda":
        raise ValueError("allocator must be 'torch' or 'cuda'")
    descs = [_Desc(g) for g in games]
    arr = (_GameDesc * len(descs))(*[d.c for d in descs])
    h = _P()
    _check_batch(lib().cfr_batch_load(arr, len(descs), ctypes.byref(cfg), ctypes.byref(h)))
    b = Batch(h, alloc, games)
    b._variant = int(variant)
    b._update_mode = int(update_mode)
    return b


def cfr_batch_iterate(b: Batch, n: int = 1):
    _check_batch(lib().cfr_batch_iterate(b.handle, int(n)), b.handle)


def cfr_batch_set_tuning(b: Batch, threads_per_block: int, blocks_per_sm: int = 0):
    t = _BatchTuning(int(threads_per_block), int(blocks_per_sm))
    _check_batch(lib().cfr_batch_set_tuning(b.handle, ctypes.byref(t)), b.handle)


_TUNE_CACHE: dict = {}


def _size_bucket(b: Batch) -> str:
    """Key of the autotuner's cache: the games' count and mean size, each rounded to a power of 2."""
    mean = float(np.mean(b.num_nodes))
    return f"games~2^{int(round(np.log2(b.num_games)))},nodes~2^{int(round(np.log2(max(mean, 1.0))))}"


def cfr_batch_autotune(b: Batch, trial_iterations: int = 3, cache_path: str | None = None) -> dict:
    """Launch shape for this batch: from the cache when one was measured for this GPU and size bucket
    (in memory, and in the JSON file cache_path when given), else measured (cfr_batch_autotune) and
    stored.  Returns {threads_per_block, blocks_per_sm, us_per_iteration (None if cached), cached}."""
    import json

    import torch

    key = (f"{torch.cuda.get_device_name()}|{_size_bucket(b)}|variant={cfr_batch_get_info(b)['variant']}"
           f"|mode={getattr(b, '_update_mode', 0)}")
    disk = {}
    if cache_path and os.path.exists(cache_path):
        try:
            disk = json.load(open(cache_path))
        except (OSError, ValueError):
            disk = {}
    hit = _TUNE_CACHE.get(key) or disk.get(key)
    if hit:
        cfr_batch_set_tuning(b, hit["threads_per_block"], hit["blocks_per_sm"])
        return dict(hit, us_per_iteration=None, cached=True, key=key)
    t = _BatchTuning()
    us = ctypes.c_double()
    _check_batch(lib().cfr_batch_autotune(b.handle, int(trial_iterations), ctypes.byref(t), ctypes.byref(us)),
                 b.handle)
    rec = {"threads_per_block": t.threads_per_block, "blocks_per_sm": t.blocks_per_sm}
    _TUNE_CACHE[key] = rec
    if cache_path:
        disk[key] = rec
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(disk, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(rec, us_per_iteration=us.value, cached=False, key=key)


def cfr_batch_game_times(b: Batch) -> np.ndarray:
    out = np.zeros(b.num_games)
    _check_batch(lib().cfr_batch_game_times(b.handle, out.ctypes.data, b.num_games), b.handle)
    return out


def cfr_batch_exploitability(b: Batch) -> np.ndarray:
    """NashConv of every game's average strategy (exploitability = NashConv / 2)."""
    out = np.zeros(b.num_games)
    _check_batch(lib().cfr_batch_exploitability(b.handle, out.ctypes.data, b.num_games), b.handle)
    return out


def cfr_batch_get_state(b: Batch, game: int) -> dict:
    q = b.num_q[game]
    R, S = np.zeros(max(q, 1)), np.zeros(max(q, 1))
    it = ctypes.c_int64()
    _check_batch(lib().cfr_batch_get_state(b.handle, int(game), R.ctypes.data, S.ctypes.data, max(q, 1),
                                           ctypes.byref(it)), b.handle)
    return dict(cum_regret=R[:q], strat_sum=S[:q], iteration=it.value)


def cfr_batch_average_strategy(b: Batch, game: int) -> np.ndarray:
    q = b.num_q[game]
    out = np.zeros(max(q, 1))
    _check_batch(lib().cfr_batch_average_strategy(b.handle, int(game), out.ctypes.data, max(q, 1)), b.handle)
    return out[:q]


def cfr_batch_get_info(b: Batch) -> dict:
    info = _BatchInfo()
    _check_batch(lib().cfr_batch_get_info(b.handle, ctypes.byref(info)), b.handle)
    d = {name: getattr(info, name) for name, _ in _BatchInfo._fields_}
    d["variant"] = getattr(b, "_variant", None)
    return d


def cfr_batch_tune(games, variant=CFR_PLUS, splits=(1, 512, 2048, -1), trial_iterations: int = 10,
                   device=None, cache_path: str | None = None, dcfr=(1.5, 0.0, 2.0),
                   update_mode=CFR_SIMULTANEOUS, fuse_candidates=(-1, 2)) -> dict:
    """The batch's size split (which games run as one forest through the per-depth kernels, which in the
    persistent kernel), the persistent launch shape and the forest part's fusion: for each candidate split
    the batch is loaded, the launch shape measured (cfr_batch_autotune), and trial_iterations timed; then
    the fastest split is timed again with each other fusion setting of fuse_candidates (cfr_config.fuse_levels
    of the forest part: -1 the last two depths and the pair above them, 2 the last two only).  The fastest is
    kept and cached per GPU and size bucket (in memory, and in the JSON file cache_path when given).  split 1
    runs every game as one forest, -1 every game whose image fits shared memory in the persistent kernel.
    Returns {split_nodes, threads_per_block, blocks_per_sm, fuse_levels, us_per_iteration (None if cached),
    cached, trials}."""
    import json

    import torch

    probe = Batch(None, None, games)
    key = f"{torch.cuda.get_device_name()}|{_size_bucket(probe)}|variant={int(variant)}|mode={int(update_mode)}|split+fuse"
    disk = {}
    if cache_path and os.path.exists(cache_path):
        try:
            disk = json.load(open(cache_path))
        except (OSError, ValueError):
            disk = {}
    hit = _TUNE_CACHE.get(key) or disk.get(key)
    if hit:
        return dict({"fuse_levels": -1}, **hit, us_per_iteration=None, cached=True, trials=None, key=key)

    def trial(split, fuse, shape=None):
        b = cfr_batch_load(games, variant=variant, device=device, dcfr=dcfr, split_nodes=split, update_mode=update_mode,
                           fuse_levels=fuse)
        if shape is None:
            t = _BatchTuning()                           # measured for this split (no cache lookup)
            _check_batch(lib().cfr_batch_autotune(b.handle, 2, ctypes.byref(t), None), b.handle)
            shape = {"threads_per_block": t.threads_per_block, "blocks_per_sm": t.blocks_per_sm}
        else:
            cfr_batch_set_tuning(b, shape["threads_per_block"], shape["blocks_per_sm"])
        cfr_batch_iterate(b, 2)                       # warm-up (graph capture)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        cfr_batch_iterate(b, trial_iterations)
        e1.record()
        torch.cuda.synchronize()
        us = 1e3 * e0.elapsed_time(e1) / trial_iterations
        b.close()
        return {"split_nodes": split, "threads_per_block": shape["threads_per_block"],
                "blocks_per_sm": shape["blocks_per_sm"], "fuse_levels": fuse, "us_per_iteration": us}

    trials = [trial(split, fuse_candidates[0]) for split in splits]
    best = min(trials, key=lambda r: r["us_per_iteration"])
    for fuse in fuse_candidates[1:]:
        trials.append(trial(best["split_nodes"], fuse, {k: best[k] for k in ("threads_per_block", "blocks_per_sm")}))
    best = min(trials, key=lambda r: r["us_per_iteration"])
    rec = {k: best[k] for k in ("split_nodes", "threads_per_block", "blocks_per_sm", "fuse_levels")}
    _TUNE_CACHE[key] = rec
    if cache_path:
        disk[key] = rec
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(disk, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(rec, us_per_iteration=best["us_per_iteration"], cached=False, trials=trials, key=key)


# ---- learned leaf values: the BF16 value network (cfr_mlp_*) ---------------------------------------------

def _check_mlp(st: int, handle=None):
    if st != CFR_OK:
        msg = lib().cfr_mlp_last_error(handle)
        raise CfrError(st, msg.decode(errors="replace") if msg else "")


class Mlp:
    """A value network on the GPU (owns the C handle).  dims: input, hidden..., output widths."""

    def __init__(self, handle, dims, device):
        self.handle = handle
        self.dims = list(dims)
        self.device = device

    @property
    def num_params(self) -> int:
        return int(lib().cfr_mlp_num_params(self.handle))

    def close(self):
        if self.handle:
            lib().cfr_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def cfr_mlp_create(dims, device=None, stream=None) -> Mlp:
    """A network of len(dims) - 1 linear layers (ReLU between them), parameters zero.  stream: None =
    PyTorch's current stream on the device."""
    import torch

    if not torch.cuda.is_available():
        raise CfrError(CFR_ERR_CUDA, "no CUDA device is available")
    dev = torch.cuda.current_device() if device is None else int(device)
    st_handle = torch.cuda.current_stream(dev).cuda_stream if stream is None else int(stream)
    d = _arr(dims, np.int32)
    h = _P()
    _check_mlp(lib().cfr_mlp_create(d.ctypes.data, len(d) - 1, dev, st_handle, ctypes.byref(h)))
    return Mlp(h, d.tolist(), dev)


def cfr_mlp_set_params(m: Mlp, params):
    p = _arr(params, np.float32)
    _check_mlp(lib().cfr_mlp_set_params(m.handle, p.ctypes.data, p.size), m.handle)


def cfr_mlp_get_params(m: Mlp) -> np.ndarray:
    out = np.zeros(m.num_params, np.float32)
    _check_mlp(lib().cfr_mlp_get_params(m.handle, out.ctypes.data, out.size), m.handle)
    return out


def cfr_mlp_get_grads(m: Mlp) -> np.ndarray:
    out = np.zeros(m.num_params, np.float32)
    _check_mlp(lib().cfr_mlp_get_grads(m.handle, out.ctypes.data, out.size), m.handle)
    return out


def _dev_f32(x, m: Mlp, width: int):
    import torch

    t = torch.as_tensor(x, dtype=torch.float32, device=f"cuda:{m.device}").contiguous()
    if t.ndim != 2 or t.shape[1] != width:
        raise ValueError(f"expected shape (batch, {width}), got {tuple(t.shape)}")
    return t


def cfr_mlp_forward(m: Mlp, x, out=None):
    """y = the network at x (batch x dims[0]); x and the result are FP32 CUDA tensors."""
    import torch

    xt = _dev_f32(x, m, m.dims[0])
    y = out if out is not None else torch.empty((xt.shape[0], m.dims[-1]), dtype=torch.float32, device=xt.device)
    _check_mlp(lib().cfr_mlp_forward(m.handle, xt.data_ptr(), xt.shape[0], y.data_ptr()), m.handle)
    return y


def cfr_mlp_backward(m: Mlp, x, target, loss=None):
    """Gradients of the mean squared error at (x, target) into the network's buffer; returns the loss
    as a one-element FP64 CUDA tensor (not synchronised)."""
    import torch

    xt, tt = _dev_f32(x, m, m.dims[0]), _dev_f32(target, m, m.dims[-1])
    if xt.shape[0] != tt.shape[0]:
        raise ValueError("x and target need the same batch")
    lt = loss if loss is not None else torch.zeros(1, dtype=torch.float64, device=xt.device)
    _check_mlp(lib().cfr_mlp_backward(m.handle, xt.data_ptr(), tt.data_ptr(), xt.shape[0], lt.data_ptr()), m.handle)
    return lt


def cfr_mlp_adam(m: Mlp, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    _check_mlp(lib().cfr_mlp_adam(m.handle, float(lr), float(beta1), float(beta2), float(eps)), m.handle)


MLP_PATH_MMA_SYNC, MLP_PATH_TCGEN05, MLP_PATH_MIXED = 0, 1, 2


def cfr_mlp_set_tensor_path(m: Mlp, path: int = MLP_PATH_MIXED):
    """0: mma.sync for every product; 1: tcgen05 for every product; 2 (default): tcgen05 with TMA operands
    for the forward and data-gradient products, mma.sync for the weight-gradient ones."""
    _check_mlp(lib().cfr_mlp_set_tensor_path(m.handle, int(path)), m.handle)


CFR_MLP_ACT, CFR_MLP_DZ, CFR_MLP_OUT = 0, 1, 2


def cfr_mlp_get_intermediate(m: Mlp, which: int, layer: int, batch: int) -> np.ndarray:
    """Test hook: one intermediate of the last forward or backward pass of ``batch`` rows, as FP32:
    CFR_MLP_ACT the input of layer ``layer`` as its product read it (BF16 values), CFR_MLP_DZ the
    gradient dL/dZ of layer ``layer`` (BF16 values, after a backward pass), CFR_MLP_OUT the output."""
    cols = {CFR_MLP_ACT: m.dims[layer] if which == CFR_MLP_ACT else 0,
            CFR_MLP_DZ: m.dims[layer + 1] if which == CFR_MLP_DZ else 0,
            CFR_MLP_OUT: m.dims[-1]}.get(which)
    if cols is None:
        raise CfrError(CFR_ERR_INVALID, f"unknown intermediate {which}")
    out = np.zeros((batch, cols), np.float32)
    _check_mlp(lib().cfr_mlp_get_intermediate(m.handle, int(which), int(layer), out.ctypes.data, out.size), m.handle)
    return out


def cfr_mlp_synchronize(m: Mlp):
    _check_mlp(lib().cfr_mlp_synchronize(m.handle), m.handle)


def cfr_mlp_gemm_stats(m: Mlp) -> dict:
    """Time (us) and FLOPs of the matrix products of the last forward and backward calls."""
    v = [ctypes.c_double() for _ in range(4)]
    _check_mlp(lib().cfr_mlp_gemm_stats(m.handle, *[ctypes.byref(x) for x in v]), m.handle)
    return dict(fwd_us=v[0].value, fwd_flops=v[1].value, bwd_us=v[2].value, bwd_flops=v[3].value)
