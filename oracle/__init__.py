"""Python access to the plain CPU oracle (``oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The product path (the CUDA
library and its binding) never imports this package.

The oracle evaluates formulae by the LTLf definition on '0'/'1' strings and
deduplicates with an ordered set of characteristic matrices; see the header of
``oracle.cpp`` for the passages of the paper each part follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Operator mask bits (shared interface): 0 not, 1 and, 2 or, 3 X, 4 F, 5 G, 6 U.
OP_NOT, OP_AND, OP_OR, OP_X, OP_F, OP_G, OP_U = (1 << i for i in range(7))
ALL_OPS = 0x7F
PAPER_OPS = OP_NOT | OP_AND | OP_X | OP_F | OP_U  # the grammar printed in the paper


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (g++, no GPU code)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load_library(path: str):
    """Load an oracle library from ``path`` (the default build, or a test variant)."""
    lib = ctypes.CDLL(path)
    _configure(lib)
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
        return _lib


def _configure(lib) -> None:
    vp, cp, i32, i64, sz = ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    ip = ctypes.POINTER(ctypes.c_int32)
    lib.oracle_spec_new.restype = vp
    lib.oracle_spec_new.argtypes = [i32, i32, i32, ip, ip, i32]
    lib.oracle_spec_free.argtypes = [vp]
    for name in ("oracle_eval", "oracle_eval_seq"):
        getattr(lib, name).restype = i32
        getattr(lib, name).argtypes = [vp, cp, ctypes.c_char_p, sz]
    lib.oracle_separates.restype = i32
    lib.oracle_separates.argtypes = [vp, cp]
    for name in ("oracle_enumerate", "oracle_bruteforce"):
        getattr(lib, name).restype = vp
        getattr(lib, name).argtypes = [vp, i32, ctypes.c_uint]
    lib.oracle_enumerate_threads.restype = vp
    lib.oracle_enumerate_threads.argtypes = [vp, i32, ctypes.c_uint, i32]
    lib.oracle_run_free.argtypes = [vp]
    lib.oracle_run_levels.restype = i32
    lib.oracle_run_levels.argtypes = [vp]
    lib.oracle_level_size.restype = i64
    lib.oracle_level_size.argtypes = [vp, i32]
    lib.oracle_level_candidates.restype = i64
    lib.oracle_level_candidates.argtypes = [vp, i32]
    for name in ("oracle_level_cm", "oracle_level_formula"):
        getattr(lib, name).restype = i32
        getattr(lib, name).argtypes = [vp, i32, i64, ctypes.c_char_p, sz]
    lib.oracle_level_cm_rows.restype = i64
    lib.oracle_level_cm_rows.argtypes = [vp, i32, i64, i64, ctypes.c_char_p, sz]
    lib.oracle_solve.restype = i32
    lib.oracle_solve.argtypes = [vp, i32, ctypes.c_uint, ctypes.c_char_p, sz, ctypes.POINTER(i64)]


class Spec:
    """A specification (P, N) held by the oracle; positives first."""

    def __init__(self, n_props: int, lengths, masks, n_pos: int, lib=None):
        lib = lib if lib is not None else _load()
        lengths = np.ascontiguousarray(lengths, dtype=np.int32)
        masks = np.ascontiguousarray(masks, dtype=np.int32)
        if masks.ndim != 2 or masks.shape[0] != lengths.shape[0]:
            raise ValueError("masks must be [n_traces, stride]")
        self.n_traces = int(lengths.shape[0])
        self.lengths = lengths
        self.n_pos = n_pos
        stride = max(1, masks.shape[1])
        if masks.shape[1] == 0:
            masks = np.zeros((self.n_traces, 1), dtype=np.int32)
        self._h = lib.oracle_spec_new(n_props, self.n_traces, n_pos,
                                      lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      masks.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), stride)
        if not self._h:
            raise ValueError("invalid specification")
        self._lib = lib

    @classmethod
    def from_problem(cls, problem, lib=None) -> "Spec":
        return cls(problem.n_props, problem.traces.lengths, problem.position_masks(), problem.n_pos, lib)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_spec_free(h)
            self._h = None

    def _cm_buf(self) -> ctypes.Array:
        return ctypes.create_string_buffer(int(self.lengths.sum()) + self.n_traces + 16)

    def eval(self, formula: str) -> str:
        """Characteristic matrix by the recursive satisfaction definition."""
        buf = self._cm_buf()
        r = self._lib.oracle_eval(self._h, formula.encode(), buf, len(buf))
        if r < 0:
            raise ValueError(f"bad formula {formula!r}")
        return buf.value.decode()

    def eval_seq(self, formula: str) -> str:
        """Characteristic matrix by the characteristic-sequence operators."""
        buf = self._cm_buf()
        r = self._lib.oracle_eval_seq(self._h, formula.encode(), buf, len(buf))
        if r < 0:
            raise ValueError(f"bad formula {formula!r}")
        return buf.value.decode()

    def separates(self, formula: str) -> bool:
        r = self._lib.oracle_separates(self._h, formula.encode())
        if r < 0:
            raise ValueError(f"bad formula {formula!r}")
        return bool(r)

    def enumerate(self, max_level: int, op_mask: int = ALL_OPS) -> "Run":
        return Run(self, self._lib.oracle_enumerate(self._h, max_level, op_mask))

    def enumerate_threads(self, max_level: int, threads: int, op_mask: int = ALL_OPS) -> "Run":
        """The levels of ``enumerate``, each level's candidates shared out among
        ``threads`` host threads (same sets; entry order may differ)."""
        return Run(self, self._lib.oracle_enumerate_threads(self._h, max_level, op_mask, threads))

    def bruteforce(self, max_size: int, op_mask: int = ALL_OPS) -> "Run":
        return Run(self, self._lib.oracle_bruteforce(self._h, max_size, op_mask))

    def solve(self, max_size: int, op_mask: int = ALL_OPS) -> Tuple[int, Optional[str], int]:
        """(size, formula, constructed): size 0 and formula None if nothing up to max_size."""
        buf = ctypes.create_string_buffer(1 << 16)
        c = ctypes.c_int64(0)
        r = self._lib.oracle_solve(self._h, max_size, op_mask, buf, len(buf), ctypes.byref(c))
        if r < 0:
            raise RuntimeError("formula buffer too small")
        return r, (buf.value.decode() if r > 0 else None), int(c.value)


class Run:
    """Levels of one enumeration (or brute force) held by the oracle."""

    def __init__(self, spec: Spec, h):
        self.spec = spec
        self._h = h
        self._lib = spec._lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_run_free(h)
            self._h = None

    @property
    def n_levels(self) -> int:
        return self._lib.oracle_run_levels(self._h)

    def size(self, k: int) -> int:
        return int(self._lib.oracle_level_size(self._h, k))

    def candidates(self, k: int) -> int:
        return int(self._lib.oracle_level_candidates(self._h, k))

    def cms(self, k: int) -> List[str]:
        buf = self.spec._cm_buf()
        out = []
        for i in range(self.size(k)):
            if self._lib.oracle_level_cm(self._h, k, i, buf, len(buf)) < 0:
                raise RuntimeError("cm export failed")
            out.append(buf.value.decode())
        return out

    def cm_rows(self, k: int, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        """Characteristic matrices of entries [first, first + count) of level k
        as a uint8 array [count, stride]: each row is one matrix's '0'/'1'
        text (traces joined by ','), padded with zero bytes."""
        n = self.size(k) - first if count is None else count
        stride = int(self.spec.lengths.sum()) + self.spec.n_traces
        buf = ctypes.create_string_buffer(max(1, n * stride))
        if self._lib.oracle_level_cm_rows(self._h, k, first, n, buf, stride) != n:
            raise RuntimeError("cm export failed")
        return np.frombuffer(buf, dtype=np.uint8, count=n * stride).reshape(n, stride)

    def formulas(self, k: int) -> List[str]:
        buf = ctypes.create_string_buffer(1 << 16)
        out = []
        for i in range(self.size(k)):
            if self._lib.oracle_level_formula(self._h, k, i, buf, len(buf)) < 0:
                raise RuntimeError("formula export failed")
            out.append(buf.value.decode())
        return out


def labeller(formula: str, traces, n_props: int) -> np.ndarray:
    """Label traces by a formula (True where trace, 0 |= formula) for the workload generator."""
    bits = np.asarray(traces.bits, dtype=np.int64)
    masks = (bits << np.arange(n_props, dtype=np.int64)[None, None, :]).sum(axis=2)
    s = Spec(n_props, traces.lengths, masks.astype(np.int32), len(traces.lengths))
    cm = s.eval_seq(formula)  # bottom-up, O(length^2) per node; pinned equal to the recursive definition
    return np.array([seq[:1] == "1" for seq in cm.split(",")], dtype=bool)


def dc_solve(problem, max_size: int, op_mask: int = ALL_OPS):
    """Divide-and-conquer (paragraph "Divide-and-conquer" of section "Parallel
    enumeration of LTLf formulae on GPUs"), on the oracle's exact solver.

    A specification (P, N) that has a separating formula of size <= max_size is
    answered by it (``Spec.solve``). Otherwise it is split into (P_i, N_j),
    i, j = 1, 2, with P the disjoint union of P_1 and P_2 and N of N_1 and N_2,
    the phi_ij are synthesised recursively from the (P_i, N_j), and the answer
    is (phi_11 and phi_12) or (phi_21 and phi_22). Readings where the paragraph
    is silent: P_1 is the first ceil(|P| / 2) positives in input order and P_2
    the rest (N likewise); a part with one positive trace splits N only
    (phi_1 and phi_2), one with one negative trace splits P only
    (phi_1 or phi_2); a part of one positive and one negative trace without an
    answer has none.

    Returns (size, formula, stats): size 0 and formula None when some part has
    no answer; stats counts splits, leaves and the deepest part.
    """
    lengths = np.asarray(problem.traces.lengths, dtype=np.int32)
    masks = problem.position_masks()
    n_props = problem.n_props
    stats = {"splits": 0, "leaves": 0, "depth": 0}

    def halves(v):
        h = (len(v) + 1) // 2
        return v[:h], v[h:]

    def solve(pos, neg, depth):
        stats["depth"] = max(stats["depth"], depth)
        idx = pos + neg
        spec = Spec(n_props, lengths[idx], masks[idx], len(pos))
        size, formula, _ = spec.solve(max_size, op_mask)
        if size > 0:
            stats["leaves"] += 1
            return size, formula
        if len(pos) >= 2 and len(neg) >= 2:
            (p1, p2), (n1, n2) = halves(pos), halves(neg)
            parts = [solve(p1, n1, depth + 1), solve(p1, n2, depth + 1),
                     solve(p2, n1, depth + 1), solve(p2, n2, depth + 1)]
            if any(x is None for x in parts):
                return None
            stats["splits"] += 1
            (s11, f11), (s12, f12), (s21, f21), (s22, f22) = parts
            return 3 + s11 + s12 + s21 + s22, f"(| (& {f11} {f12}) (& {f21} {f22}))"
        if len(pos) >= 2:
            p1, p2 = halves(pos)
            parts = [solve(p1, neg, depth + 1), solve(p2, neg, depth + 1)]
            if any(x is None for x in parts):
                return None
            stats["splits"] += 1
            return 1 + parts[0][0] + parts[1][0], f"(| {parts[0][1]} {parts[1][1]})"
        if len(neg) >= 2:
            n1, n2 = halves(neg)
            parts = [solve(pos, n1, depth + 1), solve(pos, n2, depth + 1)]
            if any(x is None for x in parts):
                return None
            stats["splits"] += 1
            return 1 + parts[0][0] + parts[1][0], f"(& {parts[0][1]} {parts[1][1]})"
        return None

    T = len(lengths)
    got = solve(list(range(problem.n_pos)), list(range(problem.n_pos, T)), 0)
    if got is None:
        return 0, None, stats
    return got[0], got[1], stats
