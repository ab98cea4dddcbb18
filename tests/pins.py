"""Pins for the CPU oracle: facts fixed by the paper and by mathematics.

Each ``pin_*`` function takes an oracle library handle (the default build or a
deliberately broken variant) and raises AssertionError when the oracle
disagrees with what the paper prints, with a closed form, with an LTLf
identity, or with brute force over all syntax trees. ``tests/test_oracle.py``
runs them against the real oracle; ``tests/test_oracle_mutants.py`` plants
plausible mistakes in a copy of the oracle source and checks that each one
fails at least one pin.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2504_18943_gb300 import workloads as W  # noqa: E402

GOLDEN = json.load(open(os.path.join(HERE, "golden", "paper_examples.json")))


def spec_from_letters(pos, neg, props, lib):
    p = W.problem_from_strings("golden", pos, neg, props)
    return oracle.Spec.from_problem(p, lib)


def random_spec(seed, n_props, n_traces, len_lo, len_hi, lib):
    st = W.Stream(W.stream_key(seed, 101))
    tb = W.draw_traces(st, n_traces, n_props, len_lo, len_hi, np.full(n_props, 0.5))
    p = W.Problem("random", n_props, tb, n_traces // 2, n_traces - n_traces // 2, 64)
    return oracle.Spec.from_problem(p, lib)


def random_formulas(seed, count, n_props, max_size):
    st = W.Stream(W.stream_key(seed, 102))
    return [W.random_formula(st, st.randint(1, max_size), n_props) for _ in range(count)]


# --- values printed in the paper -------------------------------------------

def pin_squeegee(lib):
    g = GOLDEN["squeegee"]
    s = spec_from_letters([g["trace"]], [], g["props"], lib)
    for f in g["facts"]:
        cs = s.eval(f["formula"])
        assert len(cs) == len(g["trace"])
        assert (cs[f["position"]] == "1") == f["holds"], f


def pin_abcaa(lib):
    g = GOLDEN["abcaa"]
    s = spec_from_letters([g["trace"]], [], g["props"], lib)
    for f, cs in g["cs"].items():
        assert s.eval(f) == cs, (f, s.eval(f), cs)
        assert s.eval_seq(f) == cs, (f, s.eval_seq(f), cs)


def pin_suffix_closure(lib):
    g = GOLDEN["suffix_closure"]
    s = spec_from_letters([g["trace"]], [], g["props"], lib)
    for f, cs in g["cs"].items():
        assert s.eval(f) == cs and s.eval_seq(f) == cs, f


def pin_not_b_until_a(lib):
    g = GOLDEN["not_b_until_a"]
    s = spec_from_letters(g["positive"], g["negative"], g["props"], lib)
    assert s.separates(g["formula"])
    assert W.formula_size(g["formula"]) == g["size"]
    size, f, _ = s.solve(6, oracle.PAPER_OPS)
    assert size == g["min_size_paper_grammar"], (size, f)
    assert s.separates(f) and W.formula_size(f) == size
    # no syntax tree of a smaller size separates
    bf = s.bruteforce(size, oracle.PAPER_OPS)
    for k in range(1, size):
        assert not any(s.separates(t) for t in bf.formulas(k)), k


def pin_size16(lib):
    g = GOLDEN["size16"]
    s = spec_from_letters(g["positive"], g["negative"], g["props"], lib)
    assert W.formula_size(g["formula"]) == g["size"]
    assert s.separates(g["formula"])
    # dropping the outer negation (or the innermost one) breaks separation
    assert not s.separates("(U (& p1 (X p1)) (U p0 (! (X (U (X (! (X p1))) p0)))))")
    assert not s.separates("(U (! (& p1 (X p1))) (U p0 (! (X (U (X (X p1)) p0)))))")


# --- closed forms ------------------------------------------------------------

def pin_tree_counts(lib):
    g = GOLDEN["tree_counts"]
    s = random_spec(5, g["n_props"], 3, 1, 3, lib)
    bf = s.bruteforce(len(g["counts"]) - 1, oracle.ALL_OPS)
    for k, c in enumerate(g["counts"][:-1], start=1):
        assert bf.candidates(k) == c, (k, bf.candidates(k), c)


def pin_listing_counts(lib):
    # The generic listing builds, per level k, one candidate per unary
    # operator and program of size k-1, and one per binary operator and
    # ordered pair of programs whose sizes sum to k-1.
    s = random_spec(6, 2, 6, 2, 6, lib)
    for mask, nu, nb in ((oracle.ALL_OPS, 4, 3), (oracle.PAPER_OPS, 3, 2)):
        run = s.enumerate(6, mask)
        L = [0] + [run.size(k) for k in range(1, 7)]
        assert run.candidates(1) == 2
        for k in range(2, 7):
            expect = nu * L[k - 1] + nb * sum(L[i] * L[k - 1 - i] for i in range(1, k - 1))
            assert run.candidates(k) == expect, (k, run.candidates(k), expect)


def pin_length_one(lib):
    # On traces of length 1: X f is false, F f = G f = f, f U g = g.
    s = random_spec(7, 3, 10, 1, 1, lib)
    for f in random_formulas(8, 40, 3, 5):
        v = s.eval(f)
        assert s.eval(f"(X {f})").replace("1", "0") == s.eval(f"(X {f})")
        assert s.eval(f"(F {f})") == v and s.eval(f"(G {f})") == v
        assert s.eval(f"(U p2 {f})") == v


# --- LTLf identities on random formulas and traces ------------------------

def pin_identities(lib):
    for seed in range(3):
        s = random_spec(10 + seed, 3, 12, 1, 9, lib)
        fs = random_formulas(20 + seed, 60, 3, 6)
        for a, b in zip(fs, fs[1:] + fs[:1]):
            ev = s.eval
            va, vb = ev(a), ev(b)
            assert s.eval_seq(a) == va
            assert ev(f"(! (! {a}))") == va
            assert ev(f"(G {a})") == ev(f"(! (F (! {a})))")
            assert ev(f"(F {a})") == ev(f"(U (| p0 (! p0)) {a})")
            assert ev(f"(F {a})") == ev(f"(| {a} (X (F {a})))")
            assert ev(f"(G {a})") == ev(f"(& {a} (! (X (! (G {a})))))")
            assert ev(f"(U {a} {b})") == ev(f"(| {b} (& {a} (X (U {a} {b}))))")
            assert ev(f"(! (& {a} {b}))") == ev(f"(| (! {a}) (! {b}))")
            assert ev(f"(X (& {a} {b}))") == ev(f"(& (X {a}) (X {b}))")
            assert ev(f"(F (| {a} {b}))") == ev(f"(| (F {a}) (F {b}))")
            # U is not symmetric: on some pair the operand order matters
        assert any(s.eval(f"(U {a} {b})") != s.eval(f"(U {b} {a})") for a, b in zip(fs, fs[1:]))


# --- brute force over syntax trees --------------------------------------------

def pin_levels_vs_bruteforce(lib):
    cases = [(30, 2, 6, 1, 5, 6, oracle.ALL_OPS), (31, 2, 8, 3, 8, 6, oracle.ALL_OPS),
             (32, 3, 5, 1, 4, 5, oracle.ALL_OPS), (33, 2, 6, 2, 6, 7, oracle.PAPER_OPS)]
    for seed, n, T, lo, hi, depth, mask in cases:
        s = random_spec(seed, n, T, lo, hi, lib)
        dp = s.enumerate(depth, mask)
        bf = s.bruteforce(depth, mask)
        for k in range(1, depth + 1):
            a, b = sorted(dp.cms(k)), bf.cms(k)
            assert a == b, (seed, k, len(a), len(b))
            # each exported formula re-evaluates to its characteristic matrix
            for f, cm in zip(dp.formulas(k)[:50], dp.cms(k)[:50]):
                assert s.eval(f) == cm and W.formula_size(f) == k


def pin_solve_vs_bruteforce(lib):
    for seed in range(6):
        p = W.tiny_problem(seed, lambda f, tb, n: oracle.labeller(f, tb, n))
        s = oracle.Spec.from_problem(p, lib)
        size, f, _ = s.solve(7)
        assert size >= 1 and s.separates(f) and W.formula_size(f) == size
        assert size <= W.formula_size(p.hidden)
        assert s.separates(p.hidden)
        bf = s.bruteforce(size, oracle.ALL_OPS)
        first = next(k for k in range(1, size + 1) if any(s.separates(t) for t in bf.formulas(k)))
        assert first == size, (seed, first, size)


ALL_PINS = [pin_squeegee, pin_abcaa, pin_suffix_closure, pin_not_b_until_a, pin_size16,
            pin_tree_counts, pin_listing_counts, pin_length_one, pin_identities,
            pin_levels_vs_bruteforce, pin_solve_vs_bruteforce]


def run_all(lib_path):
    """Run every pin against the library at ``lib_path``; exit status 1 if any fails."""
    lib = oracle.load_library(lib_path)
    failed = []
    for pin in ALL_PINS:
        try:
            pin(lib)
        except Exception as e:  # noqa: BLE001 - any failure counts
            failed.append(f"{pin.__name__}: {type(e).__name__}")
    print(json.dumps({"failed": failed}))
    return 1 if failed else 0


if __name__ == "__main__":
    sys.exit(run_all(sys.argv[1]))
