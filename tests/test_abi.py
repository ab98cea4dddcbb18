"""The C-ABI library without a GPU: it builds for sm_103a, loads, exports every
symbol include/lsyn.h declares, and its host-only logic and argument checks
behave (no compute call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2504_18943_gb300 import build
    build.build()
    from paper_2504_18943_gb300 import lsyn
    return lsyn


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lsyn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsyn_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lsyn_create", "lsyn_enumerate_level", "lsyn_solve", "lsyn_destroy", "lsyn_export_level",
                     "lsyn_eval", "lsyn_submit", "lsyn_poll", "lsyn_batch_create", "lsyn_batch_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    lib = ctypes.CDLL(L.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version(L):
    assert "sm_103a" in L.lsyn_version()


def _py_candidates(sizes, k, mask):
    nu = sum(bool(mask & b) for b in (1, 8, 16, 32))
    nb = bool(mask & 2) + bool(mask & 4) + 2 * bool(mask & 64)
    c = nu * sizes[k - 2]
    for i in range(1, k):
        j = k - 1 - i
        if i > j or j < 1:
            continue
        c += nb * (sizes[i - 1] * (sizes[i - 1] - 1) // 2 if i == j else sizes[i - 1] * sizes[j - 1])
    return c


@pytest.mark.parametrize("mask", [0x7F, 0x5B, 0x02, 0x40, 0x01])
def test_level_candidate_schedule(L, mask):
    rng = np.random.default_rng(mask)
    sizes = [int(x) for x in rng.integers(0, 5000, size=12)]
    for k in range(2, 13):
        assert L.lsyn_level_candidates(sizes, k, mask) == _py_candidates(sizes, k, mask)


def test_schedule_counts_match_listing_on_oracle_levels(L):
    """The schedule builds and/or once per unordered pair of distinct entries,
    U once per ordered pair of distinct entries, unary once per entry: the
    listing's count minus the pairs it builds twice or on equal operands."""
    import oracle
    from paper_2504_18943_gb300 import workloads as W
    p = W.tiny_problem(4, oracle.labeller)
    run = oracle.Spec.from_problem(p).enumerate(6)
    sizes = [run.size(k) for k in range(1, 7)]
    for k in range(2, 7):
        ordered = sum(sizes[i - 1] * sizes[k - 2 - i] for i in range(1, k - 1))
        diag = sizes[(k - 1) // 2 - 1] if (k - 1) % 2 == 0 else 0
        listing = run.candidates(k)
        assert listing == 4 * sizes[k - 2] + 3 * ordered
        ours = 4 * sizes[k - 2] + 2 * ((ordered - diag) // 2) + (ordered - diag)
        assert L.lsyn_level_candidates(sizes, k, 0x7F) == ours


@pytest.mark.parametrize("bad", ["n_props", "word_bits", "length", "empty"])
def test_create_rejects_bad_problems_before_touching_a_gpu(L, bad):
    lengths = np.array([3, 4], dtype=np.int32)
    words = np.zeros((2, 2), dtype=np.uint32)
    n_props, wb, n_pos, n_neg = 2, 32, 1, 1
    if bad == "n_props":
        n_props = 0
    elif bad == "word_bits":
        wb = 16
    elif bad == "length":
        lengths[1] = 16 * 32 + 1  # more than 16 words
    elif bad == "empty":
        n_pos = n_neg = 0
    p = L.PackedProblem(n_props, n_pos, n_neg, 32, lengths, words)
    p.struct.word_bits = wb
    with pytest.raises(L.LsynError) as ei:
        L.lsyn_create(p)
    assert ei.value.status == L.LSYN_E_INVAL
    assert L.lsyn_last_error(None)


def test_eval_rejects_bad_formulas(L):
    p = L.PackedProblem(2, 1, 0, 32, np.array([3], dtype=np.int32), np.zeros((2, 1), dtype=np.uint32))
    for f in ["", "(& p0)", "(Q p0)", "p2", "(! p0", "p0 p1", "(U p0 p1 p0)"]:
        with pytest.raises(L.LsynError) as ei:
            L.lsyn_eval(p, f)
        assert ei.value.status == L.LSYN_E_INVAL, f


def test_pack_traces_layout(L):
    bits = np.zeros((2, 5, 3), dtype=bool)
    bits[0, 0, 1] = bits[0, 4, 1] = True   # p1 at positions 0 and 4 of trace 0
    bits[1, 2, 2] = True                    # p2 at position 2 of trace 1
    p = L.pack_traces(bits, np.array([5, 3], dtype=np.int32), 1, 1, 32)
    assert p.atom_words.shape == (3, 2)
    assert p.atom_words[1, 0] == 0b10001 and p.atom_words[2, 1] == 0b100 and p.atom_words[0].sum() == 0


def test_scheduler_entry_points_check_arguments_without_a_gpu(L):
    lib = L._lib
    r = L.lsyn_result()
    assert lib.lsyn_poll(None, 1, ctypes.byref(r)) == L.LSYN_E_INVAL
    assert lib.lsyn_wait(None, 1, 0, ctypes.byref(r)) == L.LSYN_E_INVAL
    t = ctypes.c_uint64()
    assert lib.lsyn_submit(None, None, 5, ctypes.byref(t)) == L.LSYN_E_INVAL
    assert lib.lsyn_batch_solve(None, 5, None, None) == L.LSYN_E_INVAL
    assert lib.lsyn_batch_stats(None, None) == L.LSYN_E_INVAL
    assert lib.lsyn_server_stats(None, None) == L.LSYN_E_INVAL
    out = ctypes.c_void_p()
    assert lib.lsyn_batch_create(None, 0, None, None, ctypes.byref(out)) == L.LSYN_E_INVAL
    assert L._batch_err(None)
    lib.lsyn_batch_destroy(None)
    lib.lsyn_server_destroy(None)


def test_server_create_fails_cleanly_without_a_gpu(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.LsynError) as ei:
        L.lsyn_server_create(L.make_config(cache_bytes=1 << 26))
    assert ei.value.status < 0


def test_binding_structs_match_the_header_layout(L, tmp_path):
    """Every ctypes struct of the binding has the size and field offsets the C
    compiler gives the header's struct (compiled with gcc, no GPU)."""
    structs = {"lsyn_problem": L.lsyn_problem, "lsyn_config": L.lsyn_config,
               "lsyn_level_stats": L.lsyn_level_stats, "lsyn_result": L.lsyn_result,
               "lsyn_batch_tuning": L.lsyn_batch_tuning, "lsyn_sched_stats": L.lsyn_sched_stats,
               "lsyn_step_trace": L.lsyn_step_trace, "lsyn_dc_stats": L.lsyn_dc_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lsyn.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} :sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for name, cls in structs.items():
        assert got[(name, ":sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


@pytest.mark.parametrize("knobs", [{"tile_rows": 12}, {"tile_rows": 64}, {"time_limit_ms": -1.0}])
def test_config_knobs_out_of_range_rejected_before_any_device_call(L, knobs):
    import oracle
    from paper_2504_18943_gb300 import workloads as W
    p = L.pack_problem(W.tiny_problem(0, oracle.labeller))
    with pytest.raises(L.LsynError) as ei:
        L.lsyn_create(p, L.make_config(**knobs))
    assert ei.value.status == L.LSYN_E_INVAL
    assert "tile_rows" in L.lsyn_last_error() or "time_limit" in L.lsyn_last_error()
