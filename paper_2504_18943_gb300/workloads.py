"""Seeded synthetic workloads for LTLf synthesis from examples.

This module draws random numbers and random syntax trees. It holds none of the
method's arithmetic: it never evaluates a formula. Labelling a trace (does the
hidden formula hold at position 0?) is delegated to a caller-supplied
``labeller`` callable, so the same recipe serves the CUDA library (which labels
with its own evaluator) and the CPU oracle used by the tests.

Random numbers come from SplitMix64 used as a counter-based generator: output
``i`` of stream ``s`` is ``mix64(s + (i + 1) * 0x9E3779B97F4A7C15)`` with the
SplitMix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014). Every stream is keyed by (seed, purpose, indices),
so a trace or formula never depends on how many were drawn before it.

Workload recipes follow the problem statement of the paper's section
"Synthesising linear temporal logic formulae from examples": a specification
(P, N) is a pair of finite sets of finite traces over the powerset of the
propositions, positives first in a fixed order.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

# Operator spelling of the prefix formula text shared by every component:
# atoms p0..p{n-1}; unary "(! f)", "(X f)", "(F f)", "(G f)"; binary
# "(& f g)", "(| f g)", "(U f g)".
UNARY_OPS = ("!", "X", "F", "G")
BINARY_OPS = ("&", "|", "U")


def mix64(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, *path: int) -> int:
    """Derive an independent stream key from a seed and a path of integers."""
    k = mix64(seed ^ 0x5EED5EED5EED5EED)
    for p in path:
        k = mix64(k ^ mix64((p + 0x1234567) & MASK64))
    return k


class Stream:
    """Counter-based SplitMix64 stream."""

    def __init__(self, key: int):
        self.key = key & MASK64
        self.ctr = 0

    def u64(self) -> int:
        self.ctr += 1
        return mix64(self.key + self.ctr * GOLDEN)

    def block(self, n: int) -> np.ndarray:
        """n outputs as a uint64 array (advances the counter by n)."""
        idx = np.arange(self.ctr + 1, self.ctr + 1 + n, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            x = np.uint64(self.key) + idx * np.uint64(GOLDEN)
        return _mix64_np(x)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (multiply-high mapping)."""
        span = hi - lo + 1
        return lo + ((self.u64() * span) >> 64)

    def uniform(self) -> float:
        return (self.u64() >> 11) * (1.0 / (1 << 53))

    def randint_block(self, n: int, lo: int, hi: int) -> np.ndarray:
        span = hi - lo + 1
        x = self.block(n)
        # (x * span) >> 64 without 128-bit numpy: split x into 32-bit halves.
        hi32 = (x >> np.uint64(32)).astype(np.float64)
        lo32 = (x & np.uint64(0xFFFFFFFF)).astype(np.float64)
        v = np.floor((hi32 * span + np.floor(lo32 * span / 4294967296.0)) / 4294967296.0)
        return (lo + v).astype(np.int64)

    def uniform_block(self, n: int) -> np.ndarray:
        return (self.block(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


# ----------------------------------------------------------------------------
# Random formulas (syntax only)
# ----------------------------------------------------------------------------

def random_formula(st: Stream, size: int, n_props: int) -> str:
    """A random formula with exactly ``size`` syntax-tree nodes, as prefix text.

    Recipe: size 1 is an atom drawn uniformly; size 2 is a unary operator over
    an atom; larger sizes are unary (probability 4/7, child size - 1) or a
    binary operator drawn uniformly from {&, |, U} whose left child size is
    uniform in [1, size - 2].
    """
    if size < 1:
        raise ValueError("size must be >= 1")
    if size == 1:
        return f"p{st.randint(0, n_props - 1)}"
    if size == 2 or st.randint(0, 6) < 4:
        op = UNARY_OPS[st.randint(0, 3)]
        return f"({op} {random_formula(st, size - 1, n_props)})"
    op = BINARY_OPS[st.randint(0, 2)]
    left = st.randint(1, size - 2)
    a = random_formula(st, left, n_props)
    b = random_formula(st, size - 1 - left, n_props)
    return f"({op} {a} {b})"


def formula_size(text: str) -> int:
    """Number of syntax-tree nodes of a prefix formula (counts atoms and operators)."""
    toks = text.replace("(", " ( ").replace(")", " ) ").split()
    return sum(1 for t in toks if t not in ("(", ")"))


# ----------------------------------------------------------------------------
# Traces and problems
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class TraceBatch:
    """Traces as booleans: ``bits[i, t, p]`` says proposition p holds at position t of trace i."""

    bits: np.ndarray      # bool [n, max_len, n_props]
    lengths: np.ndarray   # int32 [n]

    def __len__(self) -> int:
        return int(self.lengths.shape[0])

    def take(self, idx: Sequence[int]) -> "TraceBatch":
        idx = np.asarray(idx, dtype=np.int64)
        return TraceBatch(self.bits[idx], self.lengths[idx])


Labeller = Callable[[str, TraceBatch, int], np.ndarray]
"""labeller(formula_text, traces, n_props) -> bool array, True where trace, 0 |= formula."""


@dataclasses.dataclass
class Problem:
    """A specification (P, N): positives first, then negatives, in a fixed order."""

    name: str
    n_props: int
    traces: TraceBatch
    n_pos: int
    n_neg: int
    word_bits: int
    hidden: Optional[str] = None
    seed: Optional[int] = None

    @property
    def n_traces(self) -> int:
        return self.n_pos + self.n_neg

    @property
    def max_len(self) -> int:
        return int(self.traces.lengths.max()) if len(self.traces) else 0

    def position_masks(self) -> np.ndarray:
        """int32 [T, max_len]: bit p of entry (i, t) is set iff p holds at position t of trace i."""
        T, L, n = self.traces.bits.shape
        w = (np.int64(1) << np.arange(n, dtype=np.int64))
        m = (self.traces.bits.astype(np.int64) * w[None, None, :]).sum(axis=2)
        return m.astype(np.int32)


def draw_traces(st: Stream, count: int, n_props: int, len_lo: int, len_hi: int,
                probs: np.ndarray) -> TraceBatch:
    lengths = st.randint_block(count, len_lo, len_hi).astype(np.int32)
    u = st.uniform_block(count * len_hi * n_props).reshape(count, len_hi, n_props)
    bits = u < probs[None, None, :]
    pos = np.arange(len_hi)[None, :, None]
    bits &= pos < lengths[:, None, None]
    return TraceBatch(bits, lengths)


def labelled_problem(name: str, seed: int, n_props: int, n_pos: int, n_neg: int,
                     len_lo: int, len_hi: int, hidden_size: int, word_bits: int,
                     labeller: Labeller, prob_lo: float = 0.5, prob_hi: float = 0.5,
                     block: int = 1024, max_attempts: int = 64) -> Problem:
    """Traces labelled by a seeded hidden formula of size ``hidden_size``.

    Candidate traces are drawn in a fixed order; each goes to P if the hidden
    formula holds at position 0, else to N, until both classes are full. If the
    classes cannot be filled within ``10**4 + 40 * (n_pos + n_neg)`` draws the
    formula is redrawn. Per-proposition probabilities are uniform in
    [prob_lo, prob_hi] (a constant when the two are equal).
    """
    if len_hi > 16 * word_bits:
        raise ValueError("traces longer than 16 words")
    cap = 10 ** 4 + 40 * (n_pos + n_neg)
    for attempt in range(max_attempts):
        fst = Stream(stream_key(seed, 1, attempt))
        hidden = random_formula(fst, hidden_size, n_props)
        pst = Stream(stream_key(seed, 2, attempt))
        if prob_lo == prob_hi:
            probs = np.full(n_props, prob_lo)
        else:
            probs = prob_lo + (prob_hi - prob_lo) * pst.uniform_block(n_props)
        pos_idx: List[int] = []
        neg_idx: List[int] = []
        batches: List[TraceBatch] = []
        drawn = 0
        while drawn < cap and (len(pos_idx) < n_pos or len(neg_idx) < n_neg):
            nb = min(block, cap - drawn)
            tst = Stream(stream_key(seed, 3, attempt, drawn))
            tb = draw_traces(tst, nb, n_props, len_lo, len_hi, probs)
            lab = np.asarray(labeller(hidden, tb, n_props), dtype=bool)
            if lab.shape != (nb,):
                raise ValueError("labeller returned a wrong shape")
            for i in range(nb):
                if lab[i] and len(pos_idx) < n_pos:
                    pos_idx.append(drawn + i)
                elif not lab[i] and len(neg_idx) < n_neg:
                    neg_idx.append(drawn + i)
            batches.append(tb)
            drawn += nb
        if len(pos_idx) == n_pos and len(neg_idx) == n_neg:
            allbits = np.concatenate([b.bits for b in batches])
            alllen = np.concatenate([b.lengths for b in batches])
            sel = pos_idx + neg_idx
            traces = TraceBatch(allbits[sel], alllen[sel])
            return Problem(name, n_props, traces, n_pos, n_neg, word_bits, hidden, seed)
    raise RuntimeError(f"could not fill both classes for seed {seed}")


# ----------------------------------------------------------------------------
# The workloads
# ----------------------------------------------------------------------------

def tiny_problem(seed: int, labeller: Labeller) -> Problem:
    """2 propositions; 4 + 4 traces, lengths uniform in [3, 8], Bernoulli(0.5);
    hidden formula of size 5; one uint32 word per trace."""
    return labelled_problem("tiny", seed, 2, 4, 4, 3, 8, 5, 32, labeller)


def mid_problem(seed: int, labeller: Labeller) -> Problem:
    """5 propositions; 64 + 64 traces, lengths uniform in [8, 32], Bernoulli(0.5);
    hidden formula of size 11; 128 uint32 words (512 B) per characteristic matrix."""
    return labelled_problem("mid", seed, 5, 64, 64, 8, 32, 11, 32, labeller)


def large_problem(seed: int, labeller: Labeller) -> Problem:
    """10 propositions; 1024 + 1024 traces, lengths uniform in [16, 64],
    per-proposition probability uniform in [0.2, 0.8]; hidden size 15; uint64 words."""
    return labelled_problem("large", seed, 10, 1024, 1024, 16, 64, 15, 64, labeller,
                            prob_lo=0.2, prob_hi=0.8)


def batched_problem(seed: int, index: int, labeller: Labeller) -> Problem:
    """One problem of the batched distribution: propositions uniform in [2, 8],
    trace count uniform in [8, 512] split evenly, lengths uniform in [8, 64]
    (uint64 words), hidden size uniform in [5, 13]."""
    st = Stream(stream_key(seed, 7, index))
    n = st.randint(2, 8)
    half = st.randint(4, 256)
    hs = st.randint(5, 13)
    sub = stream_key(seed, 8, index) & 0x7FFFFFFFFFFFFFFF
    p = labelled_problem("batched", sub, n, half, half, 8, 64, hs, 64, labeller)
    return p


def poisson_arrivals(seed: int, rate: float, duration: float) -> np.ndarray:
    """Arrival times (seconds) of an open-loop Poisson process."""
    st = Stream(stream_key(seed, 9, int(rate * 1000)))
    out = []
    t = 0.0
    while True:
        u = st.uniform()
        t += -math.log(1.0 - u) / rate
        if t >= duration:
            break
        out.append(t)
    return np.asarray(out)


def problem_from_strings(name: str, pos: Sequence[Sequence[str]], neg: Sequence[Sequence[str]],
                         props: str, word_bits: int = 32) -> Problem:
    """Build a problem from traces written as lists of letter sets, e.g.
    ``[["a", "b"], [], ["a"]]`` is the trace <ab, {}, a>; ``props`` gives the
    proposition order (``"ab"`` makes a = p0, b = p1)."""
    traces = list(pos) + list(neg)
    n = len(props)
    L = max(len(t) for t in traces)
    bits = np.zeros((len(traces), L, n), dtype=bool)
    lengths = np.zeros(len(traces), dtype=np.int32)
    for i, tr in enumerate(traces):
        lengths[i] = len(tr)
        for t, letters in enumerate(tr):
            for ch in letters:
                bits[i, t, props.index(ch)] = True
    return Problem(name, n, TraceBatch(bits, lengths), len(pos), len(neg), word_bits)
