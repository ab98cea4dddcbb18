"""Divide-and-conquer (lsyn_dc_solve) through the C ABI against the oracle's
recursion (needs a GPU).

With the same split rule and the same size bound, the parts answered
directly have unique minimal sizes, so the recombined size is fixed: the GPU
must return the oracle's status and size, and a formula of that size that the
oracle confirms separates the specification."""
import pytest

import oracle
from paper_2504_18943_gb300 import workloads as W
from tests.gpu_util import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("bound", [3, 4])
def test_dc_matches_oracle(L, seed, bound):
    p = W.tiny_problem(seed, oracle.labeller)
    spec = oracle.Spec.from_problem(p)
    osize, of, ost = oracle.dc_solve(p, bound)
    st, res, f, stats = L.lsyn_dc_solve(L.pack_problem(p), bound, L.make_config(cache_bytes=64 << 20))
    if of is None:
        assert st == L.LSYN_NOT_FOUND and not res.found
        return
    assert st == L.LSYN_OK and res.size == osize, (seed, bound, res.size, osize)
    assert spec.separates(f) and W.formula_size(f) == res.size
    assert res.exact == (1 if ost["splits"] == 0 else 0)
    assert stats["formula_len"] == len(f)


def test_dc_direct_answer_is_minimal(L):
    p = W.mid_problem(0, oracle.labeller)
    packed = L.pack_problem(p)
    cfg = L.make_config(cache_bytes=1 << 30)
    st, res, f, stats = L.lsyn_dc_solve(packed, 9, cfg)
    with L.Synthesizer(packed, cfg) as s:
        st2, res2, f2, _ = s.solve(9)
    assert st == st2 == L.LSYN_OK and res.exact == 1 and res.size == res2.size and stats["splits"] == 0


def test_dc_mid_split_matches_oracle(L):
    p = W.mid_problem(2, oracle.labeller)  # minimal size 11; a bound of 6 forces splits
    spec = oracle.Spec.from_problem(p)
    osize, of, _ = oracle.dc_solve(p, 6)
    st, res, f, stats = L.lsyn_dc_solve(L.pack_problem(p), 6, L.make_config(cache_bytes=1 << 30))
    assert st == L.LSYN_OK and res.size == osize and spec.separates(f) and stats["splits"] >= 1


def test_dc_equal_traces_not_found(L):
    p = W.problem_from_strings("same", [["a"], ["b", "a"]], [["b"], ["b", "a"]], "ab")
    st, res, f, _ = L.lsyn_dc_solve(L.pack_problem(p), 6, L.make_config(cache_bytes=64 << 20))
    assert st == L.LSYN_NOT_FOUND and f is None


def test_dc_splits_parts_whose_cache_fills(L):
    """A small cache makes the whole specification fill its cache; the parts
    (fewer traces, fewer distinct CMs) fit, and the recombined formula
    separates."""
    p = W.batched_problem(1000, 2, oracle.labeller)  # minimal size 9, ~6 M CMs of 3 KB
    spec = oracle.Spec.from_problem(p)
    st, res, f, stats = L.lsyn_dc_solve(L.pack_problem(p), 10, L.make_config(cache_bytes=256 << 20))
    assert st == L.LSYN_OK and stats["splits"] >= 1 and res.exact == 0
    assert spec.separates(f) and W.formula_size(f) == res.size
