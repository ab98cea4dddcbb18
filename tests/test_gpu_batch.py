"""Batched solving (lsyn_batch_*) against the plain one-problem path and the
CPU oracle, through the C ABI (needs a GPU).

Each problem of a batch must give what it gives alone: the same status, the
same minimal size, a separating formula of that size, and, level by level, the
same set of characteristic matrices for every level built completely."""
import numpy as np
import pytest

import oracle
from paper_2504_18943_gb300 import workloads as W
from tests.gpu_util import canon, lib, oracle_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def problems():
    return [W.batched_problem(1000, i, oracle.labeller) for i in range(24)]


def _complete_levels(status, res):
    # the answering level may stop early (solution) or be partial (cache full)
    return range(1, res.levels_done) if status in (0, -5) else range(1, res.levels_done + 1)


def test_batch_equals_plain_path(L, problems):
    packed = [L.pack_problem(p) for p in problems]
    cfg = L.make_config(cache_bytes=1 << 30)
    with L.Batch(packed, cfg) as b:
        statuses, results, formulas = b.solve(9)
        for i, p in enumerate(problems):
            spec = oracle.Spec.from_problem(p)
            with L.Synthesizer(packed[i], L.make_config(cache_bytes=1 << 30)) as s:
                st, res, f, _ = s.solve(9)
                assert statuses[i] == st, (i, statuses[i], st)
                if st == L.LSYN_OK:
                    assert results[i].size == res.size, (i, results[i].size, res.size)
                    assert spec.separates(formulas[i]) and W.formula_size(formulas[i]) == res.size
                for k in _complete_levels(st, res):
                    assert np.array_equal(canon(b.export(i, k)), canon(s.export(k))), (i, k)
    assert any(s == L.LSYN_OK for s in statuses)


def test_full_batch_answers_equal_plain_path(L):
    """The 256-problem batch at its benchmark settings (8 GiB cap per problem,
    sizes up to 13; a few problems fill their cap, several need gigabytes):
    every problem's status and size equal the one-problem path's. Ids that
    warps reserve and leave unused count against a cache until its level
    closes, so the scheduler's path-D unary launches and deferred passes
    reserve exactly each batch's ids, as the one-problem path does; with
    per-warp chunks, three of these problems filled their cap one level before
    the answer the one-problem path finds."""
    import torch
    packed = [L.pack_problem(W.batched_problem(1000, i, L.labeller)) for i in range(256)]
    # the scheduler's pool takes most of the free device memory, as in the
    # benchmark: nothing cached by earlier tests may shrink it
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    with L.Batch(packed, L.make_config(cache_bytes=8 << 30)) as b:
        statuses, results, formulas = b.solve(13)
    assert statuses.count(L.LSYN_OK) > 200
    torch.cuda.empty_cache()
    cfg = L.torch_config(cache_bytes=8 << 30)
    for i, q in enumerate(packed):
        with L.Synthesizer(q, cfg) as s:
            st, res, f, _ = s.solve(13)
        assert statuses[i] == st, (i, statuses[i], st)
        if st == L.LSYN_OK:
            assert results[i].size == res.size, (i, results[i].size, res.size)


def test_batch_levels_equal_oracle(L, problems):
    small = [p for p in problems if p.n_traces <= 120][:4]
    packed = [L.pack_problem(p) for p in small]
    with L.Batch(packed, L.make_config(cache_bytes=256 << 20, full_levels=True)) as b:
        statuses, results, _ = b.solve(4)
        for i, p in enumerate(small):
            run = oracle.Spec.from_problem(p).enumerate(results[i].levels_done)
            for k in range(1, results[i].levels_done + 1):
                want = canon(oracle_rows(run.cms(k), 64, p.n_traces))
                assert np.array_equal(canon(b.export(i, k)), want), (i, k)


def test_batch_graph_and_autotune(L, problems):
    packed = [L.pack_problem(p) for p in problems[:12]]
    cfg = L.make_config(cache_bytes=512 << 20)
    with L.Batch(packed, cfg) as b:
        ref = b.solve(8)
    tuning = L.lsyn_batch_tuning()
    tuning.blocks_per_sm = 2
    tuning.use_graph = 1
    with L.Batch(packed, cfg, tuning) as b:
        got = b.solve(8)
        got2 = b.solve(8)  # the captured graph is replayed
        t = b.autotune(8)
        got3 = b.solve(8)
    for g in (got, got2, got3):
        assert g[0] == ref[0]
        assert [r.size for r in g[1]] == [r.size for r in ref[1]]
    assert t.blocks_per_sm in (2, 4, 6, 8) and t.use_graph in (0, 1)
    assert t.rows_per_item in (2, 4, 8) and t.words_per_thread in (1, 2) and t.table_load_pct in (25, 50, 75)


@pytest.mark.parametrize("rows", [2, 4, 8])
@pytest.mark.parametrize("wpt", [1, 2])
@pytest.mark.parametrize("load", [25, 75])
def test_every_tuning_point_gives_the_plain_answers(L, problems, rows, wpt, load):
    """Each point of the autotuner's kernel axes (formulas per warp, words
    per thread, table sizing) gives every problem the plain path's status,
    minimal size and complete levels; small caches make some problems fill
    theirs, so the entry limit must not move with the table's load."""
    packed = [L.pack_problem(p) for p in problems[:16]]
    cfg = L.make_config(cache_bytes=64 << 20)
    tun = L.make_tuning(rows_per_item=rows, words_per_thread=wpt, table_load_pct=load, use_graph=1)
    plain = test_every_tuning_point_gives_the_plain_answers.plain
    if not plain:
        for q in packed:
            with L.Synthesizer(q, cfg) as s:
                st, res, f, _ = s.solve(9)
                plain.append((st, res.size, res.levels_done,
                              [canon(s.export(k)) for k in _complete_levels(st, res)]))
    with L.Batch(packed, cfg, tun) as b:
        statuses, results, formulas = b.solve(9)
        for i, (st, size, done, levels) in enumerate(plain):
            assert statuses[i] == st, (i, statuses[i], st)
            if st == L.LSYN_OK:
                assert results[i].size == size
            for k, want in zip(_complete_levels(st, results[i]), levels):
                assert np.array_equal(canon(b.export(i, k)), want), (i, k)


test_every_tuning_point_gives_the_plain_answers.plain = []


def test_tuning_out_of_range_rejected(L, problems):
    packed = [L.pack_problem(problems[0])]
    for bad in (dict(rows_per_item=3), dict(words_per_thread=4), dict(table_load_pct=95)):
        with pytest.raises(L.LsynError) as ei:
            L.Batch(packed, L.make_config(cache_bytes=64 << 20), L.make_tuning(**bad))
        assert ei.value.status == L.LSYN_E_INVAL


def _plain(L, packed, cfg, max_size):
    with L.Synthesizer(packed, cfg) as s:
        st, res, f, _ = s.solve(max_size)
        return st, res.size, res.unique


def _assert_matches_plain(L, problems, packed, got, cfg_plain, max_size):
    statuses, results, formulas = got
    for i, p in enumerate(problems):
        st, size, unique = _plain(L, packed[i], cfg_plain, max_size)
        assert statuses[i] == st, (i, statuses[i], st)
        if st == L.LSYN_OK:
            assert results[i].size == size, (i, results[i].size, size)
            spec = oracle.Spec.from_problem(p)
            assert spec.separates(formulas[i]) and W.formula_size(formulas[i]) == size
        elif st == L.LSYN_NOT_FOUND:
            assert results[i].unique == unique, (i, results[i].unique, unique)


def test_batch_mixed_word_sizes(L):
    """32- and 64-bit problems in one batch (one launch per word size a step)."""
    small = [W.mid_problem(s, oracle.labeller) for s in range(4)]
    packed = [L.pack_traces(p.traces.bits, p.traces.lengths, p.n_pos, p.n_neg, 32 if n % 2 else 64)
              for n, p in enumerate(small)]
    cfg = L.make_config(cache_bytes=1 << 30)
    with L.Batch(packed, cfg) as b:
        got = b.solve(6)
    _assert_matches_plain(L, small, packed, got, cfg, 6)


def test_small_pool_evicts_and_caps_like_the_plain_path(L, problems):
    """A pool of 1 GiB shared by 24 problems capped at 256 MiB each: problems
    wait, are evicted and restarted, yet each answers as it does alone with a
    256 MiB cache (cache-full ones included)."""
    packed = [L.pack_problem(p) for p in problems]
    cfg = L.make_config(cache_bytes=256 << 20)
    with L.Batch(packed, cfg, L.make_tuning(pool_bytes=1 << 30)) as b:
        got = b.solve(10)
        stats = b.stats()
    assert stats["pool_peak"] <= 1 << 30
    _assert_matches_plain(L, problems, packed, got, cfg, 10)
    assert any(s == L.LSYN_E_CACHE_FULL for s in got[0])


def test_underpredicted_levels_are_redone(L, problems):
    """With a 5% prediction margin most growing levels overflow their first
    allocation; undone and re-run, they give the plain path's levels."""
    packed = [L.pack_problem(p) for p in problems[:12]]
    cfg = L.make_config(cache_bytes=1 << 30, full_levels=True)
    with L.Batch(packed, cfg, L.make_tuning(predict_pct=5)) as b:
        statuses, results, _ = b.solve(7)
        stats = b.stats()
        assert stats["redos"] > 0
        for i in range(len(packed)):
            with L.Synthesizer(packed[i], cfg) as s:
                st, res, f, _ = s.solve(7)
                assert statuses[i] == st
                for k in _complete_levels(st, res):
                    assert np.array_equal(canon(b.export(i, k)), canon(s.export(k))), (i, k)


def test_large_level_lane_matches_plain(L, problems):
    """With a low threshold most levels run in the large-level lane (one-problem
    kernels on their own stream, beside the batch steps on a few SMs); answers
    and complete levels stay those of the plain path."""
    packed = [L.pack_problem(p) for p in problems]
    cfg = L.make_config(cache_bytes=1 << 30)
    with L.Batch(packed, cfg, L.make_tuning(solo_candidates=2000, light_sms=8)) as b:
        got = b.solve(9)
        assert b.stats()["large_levels"] > 0
        _assert_matches_plain(L, problems, packed, got, cfg, 9)
        statuses, results, _ = got
        for i in range(len(packed)):
            if statuses[i] not in (L.LSYN_OK, L.LSYN_NOT_FOUND):
                continue
            with L.Synthesizer(packed[i], cfg) as s:
                st, res, f, _ = s.solve(9)
                for k in _complete_levels(st, res):
                    assert np.array_equal(canon(b.export(i, k)), canon(s.export(k))), (i, k)
