"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare its levels with the CPU oracle's, element by element."""
from __future__ import annotations

import numpy as np

import oracle


def lib():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA GPU")
    from paper_2504_18943_gb300 import build
    build.build()
    from paper_2504_18943_gb300 import lsyn
    return lsyn


def oracle_rows(cms, word_bits: int, n_traces: int, planes: int = 1) -> np.ndarray:
    """Oracle CM strings ('0'/'1', position 0 first, traces joined by ',') as
    words: [rows, traces], or [rows, traces, planes] with word w of a trace
    holding positions w * word_bits + t in bit t."""
    dt = np.uint32 if word_bits == 32 else np.uint64
    mask = (1 << word_bits) - 1
    out = np.zeros((len(cms), n_traces, planes), dtype=dt)
    for r, cm in enumerate(cms):
        seqs = cm.split(",")
        assert len(seqs) == n_traces
        for i, s in enumerate(seqs):
            v = int(s[::-1], 2) if s else 0
            for w in range(planes):
                out[r, i, w] = (v >> (w * word_bits)) & mask
    return out[:, :, 0] if planes == 1 else out


def oracle_level_words(run, k: int, lengths, word_bits: int, planes: int = 1, chunk: int = 1 << 15) -> np.ndarray:
    """Level k of an oracle run as words, like oracle_rows, for large levels:
    the oracle's '0'/'1' rows are exported in bulk and packed with numpy."""
    lengths = np.asarray(lengths, dtype=np.int64)
    T = len(lengths)
    width = planes * word_bits
    stride = int(lengths.sum()) + T
    off = np.concatenate([[0], np.cumsum(lengths + 1)[:-1]])  # where trace i's sequence starts
    t = np.arange(width)
    idx = np.where(t[None, :] < lengths[:, None], off[:, None] + t[None, :], stride)  # past the end: a '0'
    dt = np.dtype("<u4") if word_bits == 32 else np.dtype("<u8")
    n = run.size(k)
    out = np.empty((n, T, planes), dtype=dt)
    for first in range(0, n, chunk):
        c = min(chunk, n - first)
        text = run.cm_rows(k, first, c)
        text = np.concatenate([text, np.full((c, 1), ord("0"), dtype=np.uint8)], axis=1)
        bits = text[:, idx] == ord("1")                            # [c, T, width], position t at index t
        out[first:first + c] = np.packbits(bits, axis=2, bitorder="little").view(dt)
    out = out.astype(np.uint32 if word_bits == 32 else np.uint64, copy=False)
    return out[:, :, 0] if planes == 1 else out


def sorted_rows(rows: np.ndarray) -> np.ndarray:
    """Rows as one opaque byte string each, sorted: equal multisets of rows give
    equal arrays, and a duplicate row shows up as two equal neighbours."""
    a = np.ascontiguousarray(rows.reshape(rows.shape[0], -1))
    return np.sort(a.view(np.dtype((np.void, a.shape[1] * a.itemsize))).ravel())


def has_duplicates(srt: np.ndarray) -> bool:
    return bool(srt.shape[0] > 1 and np.any(srt[1:] == srt[:-1]))


def planes_of(problem) -> int:
    """Words per trace of a workloads.Problem."""
    return max(1, -(-int(np.max(problem.traces.lengths)) // problem.word_bits))


def canon(rows: np.ndarray) -> np.ndarray:
    if rows.shape[0] == 0:
        return rows
    return np.unique(rows, axis=0)


def assert_levels_match(L, problem, depth, op_mask=0x7F, cache_bytes=256 << 20, config=None, spec=None):
    """GPU levels 1..depth (built completely) equal the oracle's, as sets of CMs,
    with no duplicate inside a level or across levels."""
    spec = spec or oracle.Spec.from_problem(problem)
    run = spec.enumerate(depth, op_mask)
    packed = L.pack_problem(problem)
    cfg = config or L.make_config(op_mask=op_mask, full_levels=True, cache_bytes=cache_bytes)
    seen = []
    with L.Synthesizer(packed, cfg) as s:
        for k in range(1, depth + 1):
            st = s.level(k)
            assert not st.cache_full, f"cache full at level {k}"
            rows = s.export(k)
            assert rows.shape[0] == run.size(k), (k, rows.shape[0], run.size(k))
            got = canon(rows)
            assert got.shape[0] == rows.shape[0], f"duplicate CMs inside level {k}"
            want = canon(oracle_rows(run.cms(k), problem.word_bits, problem.n_traces, planes_of(problem)))
            assert np.array_equal(got, want), f"level {k} differs from the oracle"
            seen.append(rows)
        allrows = np.concatenate(seen) if seen else np.zeros((0, problem.n_traces))
        assert canon(allrows).shape[0] == allrows.shape[0], "a CM appears in two levels"
        # every entry's reconstructed formula re-evaluates (by the oracle) to its CM
        for k in range(1, depth + 1):
            n = s.count(k)
            for idx in sorted(set([0, n // 2, n - 1])) if n else []:
                f = s.formula(k, idx)
                cm = oracle_rows([spec.eval(f)], problem.word_bits, problem.n_traces, planes_of(problem))[0]
                assert np.array_equal(cm, s.export(k, idx, 1)[0]), (k, idx, f)
                from paper_2504_18943_gb300.workloads import formula_size
                assert formula_size(f) == k, (k, f)
    return run
