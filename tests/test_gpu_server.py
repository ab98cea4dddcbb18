"""Serving (lsyn_server_*, lsyn_submit, lsyn_poll, lsyn_wait) through the C ABI
(needs a GPU).

A problem's answer must not depend on what else the server is running: the
same status, the same minimal size with a separating formula of that size,
and, when no formula exists up to max_size, the same number of distinct CMs,
whether it runs alone, among others admitted while it runs, or through the
one-problem path."""
import time

import pytest

import oracle
from paper_2504_18943_gb300 import workloads as W
from tests.gpu_util import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def problems():
    return [W.batched_problem(1000, i, oracle.labeller) for i in range(24)]


def _same(L, p, a, b):
    assert a[0] == b[0]
    if a[0] == L.LSYN_OK:
        assert a[1].size == b[1].size
        spec = oracle.Spec.from_problem(p)
        for f in (a[2], b[2]):
            assert spec.separates(f) and W.formula_size(f) == a[1].size
    elif a[0] == L.LSYN_NOT_FOUND:
        assert a[1].unique == b[1].unique


def test_server_answers_equal_alone_and_in_the_mix(L, problems):
    packed = [L.pack_problem(p) for p in problems]
    cfg = L.make_config(cache_bytes=512 << 20)
    alone = []
    with L.Server(cfg) as s:
        for q in packed:
            alone.append(s.wait(s.submit(q, 9)))
    # Arrivals while others run, at most 8 admitted at once, a pool that
    # cannot hold every cache at its cap.
    with L.Server(cfg, L.make_tuning(max_active=8, pool_bytes=3 << 30)) as s:
        tickets = []
        for q in packed:
            tickets.append(s.submit(q, 9))
            time.sleep(0.0005)
        mixed = [s.wait(t) for t in tickets]
        stats = s.stats()
    assert stats["completed"] == len(packed) and stats["submitted"] == len(packed)
    assert stats["active"] == 0 and stats["queued"] == 0
    for i, p in enumerate(problems):
        _same(L, p, alone[i], mixed[i])
        with L.Synthesizer(packed[i], cfg) as syn:
            st, res, f, _ = syn.solve(9)
        _same(L, p, alone[i], (st, res, f))
        assert mixed[i][1].ms > 0


def test_server_tickets(L, problems):
    q = L.pack_problem(problems[3])
    with L.Server(L.make_config(cache_bytes=256 << 20)) as s:
        t = s.submit(q, 9)
        st, _, _ = s.poll(t)
        assert st in (L.LSYN_PENDING, L.LSYN_OK)
        st, res, f = s.wait(t, 60_000)
        assert st == L.LSYN_OK and res.found and f
        with pytest.raises(L.LsynError):  # retired
            s.poll(t)
        with pytest.raises(L.LsynError):  # never issued
            s.poll(t + 1000)
        with pytest.raises(L.LsynError) as ei:
            s.submit(q, 0)
        assert ei.value.status == L.LSYN_E_INVAL
        bad = L.pack_problem(problems[4])
        bad.struct.word_bits = 16
        with pytest.raises(L.LsynError):
            s.submit(bad, 5)
        t2 = s.submit(q, 2)  # too small a bound: answered NOT_FOUND
        st, res, f = s.wait(t2)
        assert st == L.LSYN_NOT_FOUND and res.levels_done == 2 and f is None
