"""Traces longer than a word (several words per trace) through the C ABI
against the oracle (needs a GPU): formula evaluation, every level as a set of
CMs, minimal solution sizes, and batches."""
import numpy as np
import pytest

import oracle
from paper_2504_18943_gb300 import workloads as W
from tests.gpu_util import assert_levels_match, canon, lib, oracle_rows, planes_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


def _long(seed, n_props, n_pos, n_neg, lo, hi, hidden, word_bits):
    return W.labelled_problem("long", seed, n_props, n_pos, n_neg, lo, hi, hidden, word_bits, oracle.labeller)


@pytest.mark.parametrize("word_bits,lo,hi", [(64, 60, 200), (32, 20, 150), (32, 1, 40)])
def test_eval_long_traces(L, word_bits, lo, hi):
    p = _long(3, 3, 24, 24, lo, hi, 5, word_bits)
    packed = L.pack_problem(p)
    spec = oracle.Spec.from_problem(p)
    planes = planes_of(p)
    assert packed.planes == planes
    st = W.Stream(W.stream_key(11, word_bits, hi))
    for i in range(80):
        f = W.random_formula(st, 1 + i % 9, p.n_props)
        got = L.lsyn_eval(packed, f).reshape(p.n_traces, -1)
        want = oracle_rows([spec.eval(f)], word_bits, p.n_traces, planes)[0].reshape(p.n_traces, -1)
        assert np.array_equal(got, want), f


@pytest.mark.parametrize("word_bits,lo,hi,depth", [(64, 40, 140, 6), (32, 30, 150, 5), (64, 70, 128, 6)])
def test_levels_long_traces(L, word_bits, lo, hi, depth):
    p = _long(5, 2, 4, 4, lo, hi, 5, word_bits)
    assert planes_of(p) > 1
    assert_levels_match(L, p, depth)


def test_levels_long_traces_many(L):
    """128 traces of 60..130 positions in 32-bit words: five words per trace,
    five 512-byte planes per CM."""
    p = _long(2, 4, 64, 64, 60, 130, 7, 32)
    assert planes_of(p) == 5
    assert_levels_match(L, p, 5, cache_bytes=1 << 30)


@pytest.mark.parametrize("seed", range(6))
def test_solve_long_traces(L, seed):
    p = _long(seed, 3, 8, 8, 50, 120, 6, 64)
    spec = oracle.Spec.from_problem(p)
    size, _, _ = spec.solve(7)
    with L.Synthesizer(L.pack_problem(p), L.make_config(cache_bytes=256 << 20)) as s:
        st, res, f, _ = s.solve(7)
    if size == 0:
        assert st == L.LSYN_NOT_FOUND
    else:
        assert st == L.LSYN_OK and res.size == size and spec.separates(f) and W.formula_size(f) == size


def test_batch_long_traces_equals_plain(L):
    probs = [_long(s, 3, 16, 16, 30 + 10 * s, 90 + 20 * s, 6, 64) for s in range(5)]
    probs += [W.batched_problem(1000, i, oracle.labeller) for i in range(3)]
    packed = [L.pack_problem(p) for p in probs]
    cfg = L.make_config(cache_bytes=512 << 20, full_levels=True)
    with L.Batch(packed, cfg) as b:
        statuses, results, formulas = b.solve(6)
        for i, q in enumerate(packed):
            with L.Synthesizer(q, cfg) as s:
                st, res, f, _ = s.solve(6)
                assert statuses[i] == st
                done = res.levels_done if st != L.LSYN_OK else res.levels_done - 1
                for k in range(1, done + 1):
                    assert np.array_equal(canon(b.export(i, k)), canon(s.export(k))), (i, k)
            if st == L.LSYN_OK:
                assert oracle.Spec.from_problem(probs[i]).separates(formulas[i])
