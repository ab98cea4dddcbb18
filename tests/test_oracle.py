"""The CPU oracle against the paper's printed values, closed forms, LTLf
identities and brute force over all syntax trees (see ``tests/pins.py``)."""
import pytest

import oracle
from tests import pins


@pytest.fixture(scope="module")
def lib():
    return oracle.load_library(oracle.build())


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin, lib):
    pin(lib)


def test_bulk_level_export_matches_per_entry_export():
    """The bulk row export that the large parity tests use gives the same
    words as converting each exported matrix string on its own."""
    import numpy as np
    from paper_2504_18943_gb300 import workloads as W
    from tests.gpu_util import oracle_level_words, oracle_rows, planes_of
    cases = [W.tiny_problem(3, oracle.labeller), W.mid_problem(2, oracle.labeller),
             W.labelled_problem("mw", 5, 2, 6, 6, 20, 150, 4, 32, oracle.labeller)]
    for p in cases:
        run = oracle.Spec.from_problem(p).enumerate(4)
        planes = planes_of(p)
        for k in range(1, 5):
            got = oracle_level_words(run, k, p.traces.lengths, p.word_bits, planes, chunk=7)
            want = oracle_rows(run.cms(k), p.word_bits, p.n_traces, planes)
            assert got.dtype == want.dtype and np.array_equal(got, want), (p.name, k)


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_enumeration_equals_sequential(threads):
    """The all-cores baseline's enumeration builds the same candidates and the
    same level sets as the sequential listing (which brute force pins)."""
    from paper_2504_18943_gb300 import workloads as W
    for p, depth, mask in [(W.tiny_problem(11, oracle.labeller), 7, oracle.ALL_OPS),
                           (W.tiny_problem(12, oracle.labeller), 7, oracle.PAPER_OPS),
                           (W.mid_problem(2, oracle.labeller), 5, oracle.ALL_OPS)]:
        spec = oracle.Spec.from_problem(p)
        seq = spec.enumerate(depth, mask)
        par = spec.enumerate_threads(depth, threads, mask)
        for k in range(1, depth + 1):
            assert par.candidates(k) == seq.candidates(k), (p.name, k)
            assert sorted(par.cms(k)) == sorted(seq.cms(k)), (p.name, k)
        bf = spec.bruteforce(5, mask) if p.n_traces <= 8 else None
        if bf is not None:
            for k in range(1, 6):
                assert sorted(par.cms(k)) == sorted(bf.cms(k)), (p.name, k)
