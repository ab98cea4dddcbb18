"""The seeded workload generator: determinism, shapes and the labelling recipe."""
import numpy as np

import oracle
from paper_2504_18943_gb300 import workloads as W


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator.
    st = W.Stream(0)
    assert [st.u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    blk = W.Stream(0).block(3)
    assert [int(x) for x in blk] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_randint_block_matches_scalar():
    a = W.Stream(123).randint_block(1000, 3, 8)
    st = W.Stream(123)
    b = [st.randint(3, 8) for _ in range(1000)]
    assert list(a) == b and a.min() == 3 and a.max() == 8


def test_random_formula_has_requested_size():
    st = W.Stream(9)
    for s in range(1, 16):
        for _ in range(20):
            assert W.formula_size(W.random_formula(st, s, 4)) == s


def test_tiny_problem_deterministic_and_labelled():
    p1 = W.tiny_problem(3, oracle.labeller)
    p2 = W.tiny_problem(3, oracle.labeller)
    assert p1.hidden == p2.hidden
    assert np.array_equal(p1.traces.bits, p2.traces.bits)
    assert p1.n_pos == 4 and p1.n_neg == 4 and p1.traces.lengths.min() >= 3 and p1.traces.lengths.max() <= 8
    s = oracle.Spec.from_problem(p1)
    assert s.separates(p1.hidden)


def test_mid_problem_shape():
    p = W.mid_problem(0, oracle.labeller)
    assert p.n_traces == 128 and p.n_props == 5
    assert 8 <= p.traces.lengths.min() and p.traces.lengths.max() <= 32
    assert W.formula_size(p.hidden) == 11
    assert oracle.Spec.from_problem(p).separates(p.hidden)


def test_poisson_arrivals_rate():
    t = W.poisson_arrivals(0, 200.0, 60.0)
    assert abs(len(t) / 60.0 - 200.0) < 15 and np.all(np.diff(t) > 0)
