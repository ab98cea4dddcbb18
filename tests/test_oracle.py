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
