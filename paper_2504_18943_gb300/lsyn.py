"""Thin Python binding of the lsyn C ABI (``include/lsyn.h``).

Functions carry the C names and only marshal arguments: every step of the
enumeration runs in the CUDA library ``_lib/liblsyn.so``. There is no CPU
fallback: if the library is missing or cannot be loaded, importing this module
raises. PyTorch serves only as the device allocator and stream provider
(``torch_config``).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

LSYN_OK = 0
LSYN_NOT_FOUND = 1
LSYN_PENDING = 2
LSYN_E_INVAL = -1
LSYN_E_NOMEM = -2
LSYN_E_CUDA = -3
LSYN_E_UNSUPPORTED = -4
LSYN_E_CACHE_FULL = -5
LSYN_E_TIMEOUT = -6
LSYN_E_STATE = -7

OP_NOT, OP_AND, OP_OR, OP_X, OP_F, OP_G, OP_U = (1 << i for i in range(7))
OPS_ALL = 0x7F
OPS_PAPER = OP_NOT | OP_AND | OP_X | OP_F | OP_U

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class lsyn_problem(ctypes.Structure):
    _fields_ = [("n_props", ctypes.c_int32), ("n_pos", ctypes.c_int32), ("n_neg", ctypes.c_int32),
                ("word_bits", ctypes.c_int32), ("lengths", ctypes.POINTER(ctypes.c_int32)),
                ("atom_words", ctypes.c_void_p)]


class lsyn_config(ctypes.Structure):
    _fields_ = [("op_mask", ctypes.c_uint32), ("cache_bytes", ctypes.c_uint64), ("table_load", ctypes.c_float),
                ("full_levels", ctypes.c_int32), ("timing", ctypes.c_int32), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", ctypes.c_void_p), ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int32), ("tile_rows", ctypes.c_int32), ("defer_cap", ctypes.c_uint32),
                ("hole_cap", ctypes.c_uint32), ("time_limit_ms", ctypes.c_double)]


class lsyn_level_stats(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("solved", ctypes.c_int32), ("cache_full", ctypes.c_int32),
                ("early_exit", ctypes.c_int32), ("candidates", ctypes.c_int64), ("unique", ctypes.c_int64),
                ("total", ctypes.c_int64), ("deferred", ctypes.c_int64), ("ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double * 4), ("bytes_alg", ctypes.c_double),
                ("bytes_binary", ctypes.c_double), ("bytes_unary", ctypes.c_double), ("launches", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("kernel_ms", "reserved")}
        d["kernel_ms"] = list(self.kernel_ms)
        return d


class lsyn_result(ctypes.Structure):
    _fields_ = [("found", ctypes.c_int32), ("size", ctypes.c_int32), ("exact", ctypes.c_int32),
                ("levels_done", ctypes.c_int32), ("constructed", ctypes.c_int64), ("unique", ctypes.c_int64),
                ("ms", ctypes.c_double), ("launches", ctypes.c_int32), ("level_stats_cap", ctypes.c_int32),
                ("level_stats", ctypes.POINTER(lsyn_level_stats)), ("formula", ctypes.c_char_p),
                ("formula_cap", ctypes.c_size_t)]


class lsyn_batch_tuning(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("max_active", ctypes.c_int32),
                ("predict_pct", ctypes.c_int32), ("pool_bytes", ctypes.c_uint64),
                ("solo_candidates", ctypes.c_uint64), ("light_sms", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("rows_per_item", ctypes.c_int32), ("words_per_thread", ctypes.c_int32),
                ("table_load_pct", ctypes.c_int32)]


class lsyn_sched_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("active", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("steps", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("redos", ctypes.c_int64), ("large_levels", ctypes.c_int64), ("pool_bytes", ctypes.c_uint64),
                ("pool_in_use", ctypes.c_uint64), ("pool_peak", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class lsyn_step_trace(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("lane", ctypes.c_int32), ("active", ctypes.c_int32),
                ("solo", ctypes.c_int32), ("passes", ctypes.c_int32), ("finished", ctypes.c_int32),
                ("level", ctypes.c_int32), ("plan_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("settle_ms", ctypes.c_double), ("candidates", ctypes.c_uint64), ("pool_in_use", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class lsyn_dc_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("splits", ctypes.c_int32), ("leaves", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("parts", ctypes.c_int64), ("formula_len", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 2)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


def make_tuning(blocks_per_sm: int = 0, use_graph: int = 0, max_active: int = 0, pool_bytes: int = 0,
                predict_pct: int = 0, solo_candidates: int = 0, light_sms: int = 0, lanes: int = 0,
                rows_per_item: int = 0, words_per_thread: int = 0, table_load_pct: int = 0) -> lsyn_batch_tuning:
    t = lsyn_batch_tuning()
    t.blocks_per_sm, t.use_graph, t.max_active, t.pool_bytes = blocks_per_sm, use_graph, max_active, pool_bytes
    t.predict_pct, t.solo_candidates, t.light_sms, t.lanes = predict_pct, solo_candidates, light_sms, lanes
    t.rows_per_item, t.words_per_thread, t.table_load_pct = rows_per_item, words_per_thread, table_load_pct
    return t


class LsynError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"lsyn status {status}: {message}")
        self.status = status


def _load_library():
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"the lsyn CUDA library is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, vp, i32, i64 = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.lsyn_create.restype = i32
    lib.lsyn_create.argtypes = [P(lsyn_problem), P(lsyn_config), P(vp)]
    lib.lsyn_destroy.restype = None
    lib.lsyn_destroy.argtypes = [vp]
    lib.lsyn_last_error.restype = ctypes.c_char_p
    lib.lsyn_last_error.argtypes = [vp]
    lib.lsyn_reset.restype = i32
    lib.lsyn_reset.argtypes = [vp]
    lib.lsyn_enumerate_level.restype = i32
    lib.lsyn_enumerate_level.argtypes = [vp, i32, P(lsyn_level_stats)]
    lib.lsyn_solve.restype = i32
    lib.lsyn_solve.argtypes = [vp, i32, P(lsyn_result)]
    lib.lsyn_level_count.restype = i32
    lib.lsyn_level_count.argtypes = [vp, i32, P(i64)]
    lib.lsyn_export_level.restype = i32
    lib.lsyn_export_level.argtypes = [vp, i32, i64, i64, vp, ctypes.c_size_t]
    lib.lsyn_entry_formula.restype = i32
    lib.lsyn_entry_formula.argtypes = [vp, i32, i64, ctypes.c_char_p, ctypes.c_size_t]
    lib.lsyn_eval.restype = i32
    lib.lsyn_eval.argtypes = [P(lsyn_problem), ctypes.c_char_p, vp, P(lsyn_config)]
    lib.lsyn_eval_noalloc.restype = i32
    lib.lsyn_eval_noalloc.argtypes = [i32, i32, i32, vp, vp, ctypes.c_char_p, vp, vp]
    lib.lsyn_level_candidates.restype = i64
    lib.lsyn_level_candidates.argtypes = [P(i64), i32, ctypes.c_uint32]
    lib.lsyn_version.restype = ctypes.c_char_p
    lib.lsyn_version.argtypes = []
    lib.lsyn_batch_create.restype = i32
    lib.lsyn_batch_create.argtypes = [P(lsyn_problem), i32, P(lsyn_config), P(lsyn_batch_tuning), P(vp)]
    lib.lsyn_batch_solve.restype = i32
    lib.lsyn_batch_solve.argtypes = [vp, i32, P(lsyn_result), P(i32)]
    lib.lsyn_batch_autotune.restype = i32
    lib.lsyn_batch_autotune.argtypes = [vp, i32, P(lsyn_batch_tuning)]
    lib.lsyn_batch_problem.restype = i32
    lib.lsyn_batch_problem.argtypes = [vp, i32, P(vp)]
    lib.lsyn_batch_last_error.restype = ctypes.c_char_p
    lib.lsyn_batch_last_error.argtypes = [vp]
    lib.lsyn_batch_destroy.restype = None
    lib.lsyn_batch_destroy.argtypes = [vp]
    lib.lsyn_batch_stats.restype = i32
    lib.lsyn_batch_stats.argtypes = [vp, P(lsyn_sched_stats)]
    lib.lsyn_batch_trace.restype = i32
    lib.lsyn_batch_trace.argtypes = [vp, P(lsyn_step_trace), i32, P(i32)]
    lib.lsyn_server_trace.restype = i32
    lib.lsyn_server_trace.argtypes = [vp, P(lsyn_step_trace), i32, P(i32)]
    lib.lsyn_dc_solve.restype = i32
    lib.lsyn_dc_solve.argtypes = [P(lsyn_problem), i32, P(lsyn_config), P(lsyn_batch_tuning), P(lsyn_result),
                                  P(lsyn_dc_stats)]
    lib.lsyn_dc_last_error.restype = ctypes.c_char_p
    lib.lsyn_dc_last_error.argtypes = []
    lib.lsyn_server_create.restype = i32
    lib.lsyn_server_create.argtypes = [P(lsyn_config), P(lsyn_batch_tuning), P(vp)]
    lib.lsyn_submit.restype = i32
    lib.lsyn_submit.argtypes = [vp, P(lsyn_problem), i32, P(ctypes.c_uint64)]
    lib.lsyn_poll.restype = i32
    lib.lsyn_poll.argtypes = [vp, ctypes.c_uint64, P(lsyn_result)]
    lib.lsyn_wait.restype = i32
    lib.lsyn_wait.argtypes = [vp, ctypes.c_uint64, i32, P(lsyn_result)]
    lib.lsyn_server_stats.restype = i32
    lib.lsyn_server_stats.argtypes = [vp, P(lsyn_sched_stats)]
    lib.lsyn_server_last_error.restype = ctypes.c_char_p
    lib.lsyn_server_last_error.argtypes = [vp]
    lib.lsyn_server_destroy.restype = None
    lib.lsyn_server_destroy.argtypes = [vp]
    return lib


_lib = _load_library()


def library_path() -> str:
    return _build.LIB_PATH


def _err(ctx) -> str:
    m = _lib.lsyn_last_error(ctx)
    return m.decode() if m else ""


def _check(status: int, ctx=None, ok=(LSYN_OK,)) -> int:
    if status not in ok:
        raise LsynError(status, _err(ctx))
    return status


# ---------------------------------------------------------------------------
# Argument marshalling
# ---------------------------------------------------------------------------

class PackedProblem:
    """A problem in the ABI layout: atom words [n_props][T] (one word per trace)
    or [n_props][T][W] (W words per trace) and lengths [T].

    Holds the numpy buffers the ``lsyn_problem`` struct points to."""

    def __init__(self, n_props: int, n_pos: int, n_neg: int, word_bits: int, lengths: np.ndarray,
                 atom_words: np.ndarray):
        self.n_props, self.n_pos, self.n_neg, self.word_bits = n_props, n_pos, n_neg, word_bits
        self.lengths = np.ascontiguousarray(lengths, dtype=np.int32)
        dt = np.uint32 if word_bits == 32 else np.uint64
        self.atom_words = np.ascontiguousarray(atom_words, dtype=dt)
        self.struct = lsyn_problem(n_props, n_pos, n_neg, word_bits,
                                   self.lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   self.atom_words.ctypes.data)

    @property
    def n_traces(self) -> int:
        return self.n_pos + self.n_neg

    @property
    def planes(self) -> int:
        """Words per trace."""
        return int(self.atom_words.shape[2]) if self.atom_words.ndim == 3 else 1

    @property
    def word_dtype(self):
        return np.uint32 if self.word_bits == 32 else np.uint64

    @property
    def h2d_bytes(self) -> int:
        return int(self.lengths.nbytes + self.atom_words.nbytes)


def pack_traces(bits: np.ndarray, lengths: np.ndarray, n_pos: int, n_neg: int, word_bits: int) -> PackedProblem:
    """Pack boolean traces ``bits[i, t, p]`` into atom words: bit t of word
    (p, i) when every trace fits a word, else bit t of word (p, i, w) for
    position w * word_bits + t (W = ceil(longest / word_bits) words)."""
    bits = np.asarray(bits, dtype=bool)
    T, L, n = bits.shape
    longest = int(np.max(lengths)) if len(lengths) else 1
    planes = max(1, -(-longest // word_bits))
    if L > planes * word_bits:
        if bits[:, planes * word_bits:, :].any():
            raise ValueError("a trace has propositions past its length")
        bits = bits[:, :planes * word_bits, :]
        L = planes * word_bits
    if L < planes * word_bits:
        bits = np.concatenate([bits, np.zeros((T, planes * word_bits - L, n), dtype=bool)], axis=1)
    weights = np.left_shift(np.uint64(1), np.arange(word_bits, dtype=np.uint64))
    # [n][T][planes][word_bits] -> words
    b = bits.transpose(2, 0, 1).reshape(n, T, planes, word_bits).astype(np.uint64)
    words = (b * weights[None, None, None, :]).sum(axis=3, dtype=np.uint64)
    if planes == 1:
        words = words[:, :, 0]
    return PackedProblem(n, n_pos, n_neg, word_bits, lengths, words)


def pack_problem(problem) -> PackedProblem:
    """Pack a ``workloads.Problem``."""
    return pack_traces(problem.traces.bits, problem.traces.lengths, problem.n_pos, problem.n_neg,
                       problem.word_bits)


def make_config(op_mask: int = 0, cache_bytes: int = 0, table_load: float = 0.0, full_levels: bool = False,
                timing: bool = False, stream=None, device: int = -1, allocator=None, tile_rows: int = 0,
                defer_cap: int = 0, hole_cap: int = 0, time_limit_ms: float = 0.0) -> lsyn_config:
    cfg = lsyn_config()
    cfg.op_mask = op_mask
    cfg.cache_bytes = cache_bytes
    cfg.table_load = table_load
    cfg.full_levels = 1 if full_levels else 0
    cfg.timing = 1 if timing else 0
    cfg.stream = stream
    cfg.device = device
    cfg.tile_rows = tile_rows
    cfg.defer_cap = defer_cap
    cfg.hole_cap = hole_cap
    cfg.time_limit_ms = time_limit_ms
    if allocator is not None:
        cfg.alloc, cfg.free = allocator.alloc_fn, allocator.free_fn
    else:
        cfg.alloc = ALLOC_FN()
        cfg.free = FREE_FN()
    cfg._allocator = allocator  # keep the callbacks alive with the struct
    return cfg


class TorchAllocator:
    """Device allocation through the PyTorch caching allocator on a stream."""

    def __init__(self, device: Optional[int] = None, stream=None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream

        def _alloc(nbytes, _user):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:  # noqa: BLE001 - reported to the library as NULL
                return None

        def _free(ptr, _user):
            if ptr:
                self._torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)


def torch_config(op_mask: int = 0, cache_bytes: int = 0, full_levels: bool = False, timing: bool = False,
                 stream=None, device: Optional[int] = None, table_load: float = 0.0, **knobs) -> lsyn_config:
    """A config whose device memory comes from PyTorch and whose work goes on a
    torch stream; ``knobs`` are make_config's tile_rows, defer_cap, hole_cap
    and time_limit_ms."""
    import torch
    dev = torch.cuda.current_device() if device is None else device
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    alloc = TorchAllocator(dev, s)
    cfg = make_config(op_mask, cache_bytes, table_load, full_levels, timing, s.cuda_stream, dev, alloc, **knobs)
    cfg._torch_stream = s
    return cfg


# ---------------------------------------------------------------------------
# The C entry points, same names
# ---------------------------------------------------------------------------

def lsyn_version() -> str:
    return _lib.lsyn_version().decode()


# Configurations whose allocation callbacks a live handle (context, batch or
# server) may still call, by handle value. The library keeps the function
# pointers of a config's alloc / free callbacks and calls free when the handle
# is destroyed, so the Python callback objects must outlive that call even
# when the caller passed a temporary config.
_live_configs: dict = {}


def _hold(handle: ctypes.c_void_p, config) -> None:
    if config is not None and handle.value:
        _live_configs[handle.value] = config


def _let_go(handle) -> None:
    value = handle.value if isinstance(handle, ctypes.c_void_p) else handle
    _live_configs.pop(value, None)


def lsyn_create(problem: PackedProblem, config: Optional[lsyn_config] = None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    st = _lib.lsyn_create(ctypes.byref(problem.struct), ctypes.byref(config) if config is not None else None,
                          ctypes.byref(ctx))
    _check(st, None)
    _hold(ctx, config)
    return ctx


def lsyn_destroy(ctx) -> None:
    _lib.lsyn_destroy(ctx)
    _let_go(ctx)  # after the library's last call into the config's free callback


def lsyn_last_error(ctx=None) -> str:
    return _err(ctx)


def lsyn_reset(ctx) -> None:
    _check(_lib.lsyn_reset(ctx), ctx)


def lsyn_enumerate_level(ctx, k: int) -> lsyn_level_stats:
    st = lsyn_level_stats()
    _check(_lib.lsyn_enumerate_level(ctx, k, ctypes.byref(st)), ctx)
    return st


def lsyn_solve(ctx, max_size: int, formula_cap: int = 1 << 16):
    """Returns (status, lsyn_result, formula text or None, per-level stats of
    the levels this call built); LSYN_NOT_FOUND, LSYN_E_CACHE_FULL and LSYN_E_TIMEOUT are
    results, not exceptions."""
    buf = ctypes.create_string_buffer(formula_cap)
    levels = (lsyn_level_stats * 64)()
    res = lsyn_result()
    res.formula = ctypes.cast(buf, ctypes.c_char_p)
    res.formula_cap = formula_cap
    res.level_stats = ctypes.cast(levels, ctypes.POINTER(lsyn_level_stats))
    res.level_stats_cap = 64
    st = _check(_lib.lsyn_solve(ctx, max_size, ctypes.byref(res)), ctx,
                ok=(LSYN_OK, LSYN_NOT_FOUND, LSYN_E_CACHE_FULL, LSYN_E_TIMEOUT))
    text = buf.value.decode() if st == LSYN_OK else None
    built = [levels[i] for i in range(min(64, res.levels_done)) if levels[i].level == i + 1]
    return st, res, text, built


def lsyn_level_count(ctx, k: int) -> int:
    n = ctypes.c_int64()
    _check(_lib.lsyn_level_count(ctx, k, ctypes.byref(n)), ctx)
    return int(n.value)


def lsyn_export_level(ctx, k: int, n_traces: int, word_bits: int, first: int = 0,
                      count: Optional[int] = None, planes: int = 1) -> np.ndarray:
    """CMs of level k as an array [count, n_traces] (or [count, n_traces, planes]
    with several words per trace) of uint32/uint64 words."""
    if count is None:
        count = lsyn_level_count(ctx, k) - first
    dt = np.uint32 if word_bits == 32 else np.uint64
    out = np.empty((count, n_traces) if planes == 1 else (count, n_traces, planes), dtype=dt)
    _check(_lib.lsyn_export_level(ctx, k, first, count, out.ctypes.data if count else None, out.nbytes), ctx)
    return out


def lsyn_entry_formula(ctx, k: int, index: int, cap: int = 1 << 16) -> str:
    buf = ctypes.create_string_buffer(cap)
    _check(_lib.lsyn_entry_formula(ctx, k, index, buf, cap), ctx)
    return buf.value.decode()


def lsyn_eval(problem: PackedProblem, formula: str, config: Optional[lsyn_config] = None) -> np.ndarray:
    """The formula's CM: [n_traces] words, or [n_traces, planes] with several words per trace."""
    shape = problem.n_traces if problem.planes == 1 else (problem.n_traces, problem.planes)
    out = np.zeros(shape, dtype=problem.word_dtype)
    st = _lib.lsyn_eval(ctypes.byref(problem.struct), formula.encode(), out.ctypes.data,
                        ctypes.byref(config) if config is not None else None)
    _check(st, None)
    return out


def lsyn_eval_noalloc(n_props: int, n_traces: int, word_bits: int, atom_words_dev: int, lengths_dev: int,
                      formula: str, dst_dev: int, stream: int = 0) -> None:
    """Evaluate a formula on traces already on the device, into a device buffer,
    without allocating device memory (pointers are device addresses as ints).
    Only enqueues work on ``stream``."""
    st = _lib.lsyn_eval_noalloc(n_props, n_traces, word_bits, atom_words_dev, lengths_dev, formula.encode(),
                                dst_dev, stream or None)
    _check(st, None)


def lsyn_level_candidates(level_sizes: Sequence[int], k: int, op_mask: int = OPS_ALL) -> int:
    arr = (ctypes.c_int64 * max(1, len(level_sizes)))(*level_sizes)
    return int(_lib.lsyn_level_candidates(arr, k, op_mask))


# ---------------------------------------------------------------------------
# Conveniences
# ---------------------------------------------------------------------------

def labeller(formula: str, traces, n_props: int) -> np.ndarray:
    """Workload labeller on the GPU: True where trace, 0 |= formula (lsyn_eval)."""
    p = pack_traces(traces.bits, traces.lengths, len(traces.lengths), 0, 64)
    cm = lsyn_eval(p, formula).reshape(p.n_traces, -1)
    return (cm[:, 0] & np.uint64(1)).astype(bool)  # position 0: bit 0 of a trace's first word


def cm_strings(words: np.ndarray, lengths: Sequence[int]) -> str:
    """One CM row as '0'/'1' characteristic sequences joined by ',' (position 0 first)."""
    parts = []
    for w, L in zip(words, lengths):
        w = int(w)
        parts.append("".join("1" if (w >> t) & 1 else "0" for t in range(int(L))))
    return ",".join(parts)


class Synthesizer:
    """Owns one lsyn context: ``with Synthesizer(problem, cfg) as s: s.solve(12)``."""

    def __init__(self, problem: PackedProblem, config: Optional[lsyn_config] = None):
        self.problem = problem
        self.config = config
        self.ctx = lsyn_create(problem, config)

    def close(self):
        if self.ctx:
            lsyn_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def level(self, k: int) -> lsyn_level_stats:
        return lsyn_enumerate_level(self.ctx, k)

    def solve(self, max_size: int):
        return lsyn_solve(self.ctx, max_size)

    def reset(self):
        lsyn_reset(self.ctx)

    def count(self, k: int) -> int:
        return lsyn_level_count(self.ctx, k)

    def export(self, k: int, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        return lsyn_export_level(self.ctx, k, self.problem.n_traces, self.problem.word_bits, first, count,
                                 self.problem.planes)

    def formula(self, k: int, index: int) -> str:
        return lsyn_entry_formula(self.ctx, k, index)


# ---------------------------------------------------------------------------
# Batched solving
# ---------------------------------------------------------------------------

def _batch_err(b) -> str:
    m = _lib.lsyn_batch_last_error(b)
    return m.decode() if m else ""


def lsyn_batch_create(problems: Sequence[PackedProblem], config: Optional[lsyn_config] = None,
                      tuning: Optional[lsyn_batch_tuning] = None) -> ctypes.c_void_p:
    arr = (lsyn_problem * len(problems))(*[p.struct for p in problems])
    b = ctypes.c_void_p()
    st = _lib.lsyn_batch_create(arr, len(problems), ctypes.byref(config) if config is not None else None,
                                ctypes.byref(tuning) if tuning is not None else None, ctypes.byref(b))
    if st != LSYN_OK:
        raise LsynError(st, _batch_err(None))
    _hold(b, config)
    return b


def lsyn_batch_solve(batch, n: int, max_size: int, formula_cap: int = 4096):
    """Returns (statuses, results, formulas) for the n problems of the batch."""
    results = (lsyn_result * n)()
    bufs = [ctypes.create_string_buffer(formula_cap) for _ in range(n)]
    for r, buf in zip(results, bufs):
        r.formula = ctypes.cast(buf, ctypes.c_char_p)
        r.formula_cap = formula_cap
    statuses = (ctypes.c_int32 * n)()
    st = _lib.lsyn_batch_solve(batch, max_size, results, statuses)
    if st != LSYN_OK:
        raise LsynError(st, _batch_err(batch))
    formulas = [bufs[i].value.decode() if statuses[i] == LSYN_OK else None for i in range(n)]
    return list(statuses), list(results), formulas


def lsyn_batch_autotune(batch, max_size: int) -> lsyn_batch_tuning:
    t = lsyn_batch_tuning()
    st = _lib.lsyn_batch_autotune(batch, max_size, ctypes.byref(t))
    if st != LSYN_OK:
        raise LsynError(st, _batch_err(batch))
    return t


def lsyn_batch_problem(batch, i: int) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(_lib.lsyn_batch_problem(batch, i, ctypes.byref(ctx)), None)
    return ctx


def lsyn_batch_destroy(batch) -> None:
    _lib.lsyn_batch_destroy(batch)
    _let_go(batch)


def _trace(fn, handle, cap: int = 4096) -> list:
    buf = (lsyn_step_trace * cap)()
    n = ctypes.c_int32()
    _check(fn(handle, buf, cap, ctypes.byref(n)), None)
    return [buf[i].as_dict() for i in range(n.value)]


def lsyn_batch_trace(batch) -> list:
    return _trace(_lib.lsyn_batch_trace, batch)


def lsyn_server_trace(server) -> list:
    return _trace(_lib.lsyn_server_trace, server)


def lsyn_batch_stats(batch) -> dict:
    st = lsyn_sched_stats()
    _check(_lib.lsyn_batch_stats(batch, ctypes.byref(st)), None)
    return st.as_dict()


class Batch:
    """Owns a batch: ``with Batch(problems, cfg) as b: statuses, results, formulas = b.solve(13)``."""

    def __init__(self, problems: Sequence[PackedProblem], config: Optional[lsyn_config] = None,
                 tuning: Optional[lsyn_batch_tuning] = None):
        self.problems = list(problems)
        self.config = config
        self.handle = lsyn_batch_create(self.problems, config, tuning)

    def close(self):
        if self.handle:
            lsyn_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def solve(self, max_size: int):
        return lsyn_batch_solve(self.handle, len(self.problems), max_size)

    def autotune(self, max_size: int) -> lsyn_batch_tuning:
        return lsyn_batch_autotune(self.handle, max_size)

    def count(self, i: int, k: int) -> int:
        return lsyn_level_count(lsyn_batch_problem(self.handle, i), k)

    def export(self, i: int, k: int) -> np.ndarray:
        p = self.problems[i]
        return lsyn_export_level(lsyn_batch_problem(self.handle, i), k, p.n_traces, p.word_bits, planes=p.planes)

    def stats(self) -> dict:
        return lsyn_batch_stats(self.handle)

    def trace(self) -> list:
        return lsyn_batch_trace(self.handle)


# ---------------------------------------------------------------------------
# Divide-and-conquer
# ---------------------------------------------------------------------------

def lsyn_dc_solve(problem: PackedProblem, max_size: int, config: Optional[lsyn_config] = None,
                  tuning: Optional[lsyn_batch_tuning] = None, formula_cap: int = 1 << 20):
    """(status, result, formula, stats): status LSYN_OK or LSYN_NOT_FOUND; the
    formula separates the specification (minimal when result.exact)."""
    r = lsyn_result()
    buf = ctypes.create_string_buffer(formula_cap)
    r.formula = ctypes.cast(buf, ctypes.c_char_p)
    r.formula_cap = formula_cap
    stats = lsyn_dc_stats()
    st = _lib.lsyn_dc_solve(ctypes.byref(problem.struct), max_size, ctypes.byref(config) if config is not None else None,
                            ctypes.byref(tuning) if tuning is not None else None, ctypes.byref(r), ctypes.byref(stats))
    if st not in (LSYN_OK, LSYN_NOT_FOUND):
        raise LsynError(st, (_lib.lsyn_dc_last_error() or b"").decode())
    return st, r, (buf.value.decode() if st == LSYN_OK else None), stats.as_dict()


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------

def _server_err(sv) -> str:
    m = _lib.lsyn_server_last_error(sv)
    return m.decode() if m else ""


def lsyn_server_create(config: Optional[lsyn_config] = None,
                       tuning: Optional[lsyn_batch_tuning] = None) -> ctypes.c_void_p:
    sv = ctypes.c_void_p()
    st = _lib.lsyn_server_create(ctypes.byref(config) if config is not None else None,
                                 ctypes.byref(tuning) if tuning is not None else None, ctypes.byref(sv))
    if st != LSYN_OK:
        raise LsynError(st, _server_err(None))
    _hold(sv, config)
    return sv


def lsyn_submit(server, problem: PackedProblem, max_size: int) -> int:
    t = ctypes.c_uint64()
    st = _lib.lsyn_submit(server, ctypes.byref(problem.struct), max_size, ctypes.byref(t))
    if st != LSYN_OK:
        raise LsynError(st, _server_err(server))
    return t.value


def _answer(fn, server, ticket, *args, formula_cap: int = 4096):
    r = lsyn_result()
    buf = ctypes.create_string_buffer(formula_cap)
    r.formula = ctypes.cast(buf, ctypes.c_char_p)
    r.formula_cap = formula_cap
    st = fn(server, ticket, *args, ctypes.byref(r))
    if st == LSYN_E_INVAL:
        raise LsynError(st, _server_err(server))
    return st, r, (buf.value.decode() if st == LSYN_OK else None)


def lsyn_poll(server, ticket: int):
    """(status, result, formula); status LSYN_PENDING while the problem runs."""
    return _answer(_lib.lsyn_poll, server, ticket)


def lsyn_wait(server, ticket: int, timeout_ms: int = -1):
    """(status, result, formula); LSYN_E_TIMEOUT if still pending after timeout_ms."""
    return _answer(_lib.lsyn_wait, server, ticket, timeout_ms)


def lsyn_server_stats(server) -> dict:
    st = lsyn_sched_stats()
    _check(_lib.lsyn_server_stats(server, ctypes.byref(st)), None)
    return st.as_dict()


def lsyn_server_destroy(server) -> None:
    _lib.lsyn_server_destroy(server)
    _let_go(server)


class Server:
    """Owns a server: ``with Server(cfg) as s: t = s.submit(p, 13); st, res, f = s.wait(t)``."""

    def __init__(self, config: Optional[lsyn_config] = None, tuning: Optional[lsyn_batch_tuning] = None):
        self.config = config
        self.handle = lsyn_server_create(config, tuning)
        self._keep = {}  # problems stay alive until answered (the library copies them anyway)

    def close(self):
        if self.handle:
            lsyn_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def submit(self, problem: PackedProblem, max_size: int) -> int:
        return lsyn_submit(self.handle, problem, max_size)

    def poll(self, ticket: int):
        return lsyn_poll(self.handle, ticket)

    def wait(self, ticket: int, timeout_ms: int = -1):
        return lsyn_wait(self.handle, ticket, timeout_ms)

    def stats(self) -> dict:
        return lsyn_server_stats(self.handle)

    def trace(self) -> list:
        return lsyn_server_trace(self.handle)
