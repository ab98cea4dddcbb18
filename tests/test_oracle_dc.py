"""The oracle's divide-and-conquer (paragraph "Divide-and-conquer") against
what the paragraph fixes: the recombined formula separates (P, N); it is the
direct answer when one exists within the size bound; it is never smaller than
the minimal formula; a part of one positive and one negative trace with no
answer leaves the whole specification without one; and the recombination
(phi_11 and phi_12) or (phi_21 and phi_22) is the one that works (its mirror
image does not)."""
import numpy as np
import pytest

import oracle
from paper_2504_18943_gb300 import workloads as W


def _sub(problem, pos, neg):
    lengths = np.asarray(problem.traces.lengths, dtype=np.int32)
    masks = problem.position_masks()
    idx = list(pos) + list(neg)
    return oracle.Spec(problem.n_props, lengths[idx], masks[idx], len(pos))


@pytest.mark.parametrize("seed", range(8))
def test_dc_is_the_direct_answer_when_one_exists(seed):
    p = W.tiny_problem(seed, oracle.labeller)
    spec = oracle.Spec.from_problem(p)
    size, f, _ = spec.solve(7)
    assert size > 0
    dsize, df, st = oracle.dc_solve(p, 7)
    assert dsize == size and st["splits"] == 0 and spec.separates(df)


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("bound", [3, 4])
def test_dc_split_answers_separate(seed, bound):
    p = W.tiny_problem(seed, oracle.labeller)
    spec = oracle.Spec.from_problem(p)
    minimal, _, _ = spec.solve(8)
    size, f, st = oracle.dc_solve(p, bound)
    if f is None:
        return  # some 1 x 1 part has no formula within the bound
    assert spec.separates(f)
    assert W.formula_size(f) == size
    assert size >= minimal
    if minimal > bound:
        assert st["splits"] >= 1 and st["depth"] >= 1


def test_dc_mid_problem_separates():
    p = W.mid_problem(2, oracle.labeller)  # minimal size 11: a bound of 6 forces splits
    spec = oracle.Spec.from_problem(p)
    size, f, st = oracle.dc_solve(p, 6)
    assert f is not None and spec.separates(f) and W.formula_size(f) == size and st["splits"] >= 1


def test_dc_equal_traces_have_no_answer():
    p = W.problem_from_strings("same", [["a"], ["b", "a"]], [["b"], ["b", "a"]], "ab")
    size, f, _ = oracle.dc_solve(p, 6)
    assert size == 0 and f is None


def test_recombination_rule_has_teeth():
    """Solve the four parts directly and recombine them both ways: the paper's
    form separates every specification; the mirrored form
    (phi_11 or phi_12) and (phi_21 or phi_22) fails on some."""
    mirrored_fails = 0
    for seed in range(12):
        p = W.tiny_problem(seed, oracle.labeller)
        pos = list(range(p.n_pos))
        neg = list(range(p.n_pos, p.n_pos + p.n_neg))
        h = lambda v: (v[:(len(v) + 1) // 2], v[(len(v) + 1) // 2:])
        (p1, p2), (n1, n2) = h(pos), h(neg)
        f = {}
        for name, (a, b) in {"11": (p1, n1), "12": (p1, n2), "21": (p2, n1), "22": (p2, n2)}.items():
            size, formula, _ = _sub(p, a, b).solve(8)
            assert size > 0
            f[name] = formula
        spec = oracle.Spec.from_problem(p)
        assert spec.separates(f"(| (& {f['11']} {f['12']}) (& {f['21']} {f['22']}))")
        if not spec.separates(f"(& (| {f['11']} {f['12']}) (| {f['21']} {f['22']}))"):
            mirrored_fails += 1
    assert mirrored_fails > 0
