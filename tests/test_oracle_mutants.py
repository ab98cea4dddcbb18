"""Plant plausible mistakes in copies of the oracle source and check that each
one fails at least one pin of ``tests/pins.py``.

A pin suite that passes on a broken oracle proves nothing, so every mistake
below (a wrong index, a strict/non-strict bound, transposed operands, a
dropped term, a skipped cache level) must be caught. Each mutant is compiled
with g++ into a temporary directory and run in a child process, so a crash
also counts as caught. Nothing here touches a GPU.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in oracle.cpp, replacement, which occurrence)
MUTANTS = [
    ("next_wrong_index", "case NEXT: return i + 1 < len && sat(t, x.a, tr, i + 1);",
     "case NEXT: return i + 1 < len && sat(t, x.a, tr, i);", 0),
    ("until_non_strict", "for (int k = i; k < j; ++k)\n          if (!sat(t, x.a, tr, k))",
     "for (int k = i; k <= j; ++k)\n          if (!sat(t, x.a, tr, k))", 0),
    ("until_swapped_witness", "if (!sat(t, x.b, tr, j)) continue;", "if (!sat(t, x.a, tr, j)) continue;", 0),
    ("future_strict", "for (int j = i; j < len; ++j)\n        if (sat(t, x.a, tr, j)) return true;",
     "for (int j = i + 1; j < len; ++j)\n        if (sat(t, x.a, tr, j)) return true;", 0),
    ("globally_strict", "for (int j = i; j < len; ++j)\n        if (!sat(t, x.a, tr, j)) return false;",
     "for (int j = i + 1; j < len; ++j)\n        if (!sat(t, x.a, tr, j)) return false;", 0),
    ("not_dropped", "case NOT: return !sat(t, x.a, tr, i);", "case NOT: return sat(t, x.a, tr, i);", 0),
    ("or_as_and", "case OR: return sat(t, x.a, tr, i) || sat(t, x.b, tr, i);",
     "case OR: return sat(t, x.a, tr, i) && sat(t, x.b, tr, i);", 0),
    ("seq_next_wrong_index", "if (op == NEXT) v = i + 1 < n && a[i + 1] == '1';",
     "if (op == NEXT) v = i + 1 < n && a[i] == '1';", 0),
    ("seq_until_non_strict", "for (int k = i; k < j; ++k) if (a[k] != '1') left_all = false;",
     "for (int k = i; k <= j; ++k) if (a[k] != '1') left_all = false;", 0),
    ("seq_until_transposed", "if (b[j] != '1') continue;", "if (a[j] != '1') continue;", 0),
    ("seq_future_strict", "for (int j = i; j < n; ++j) if (a[j] == '1') v = true;",
     "for (int j = i + 1; j < n; ++j) if (a[j] == '1') v = true;", 0),
    ("seq_globally_strict", "for (int j = i; j < n; ++j) if (a[j] != '1') v = false;",
     "for (int j = i + 1; j < n; ++j) if (a[j] != '1') v = false;", 0),
    ("seq_not_dropped", "if (op == NOT) v = a[i] != '1';", "if (op == NOT) v = a[i] == '1';", 0),
    ("seq_or_as_and", "if (op == OR) v = a[i] == '1' || b[i] == '1';",
     "if (op == OR) v = a[i] == '1' && b[i] == '1';", 0),
    ("atom_negated", "r[i] = tr.holds[i][p] ? '1' : '0';", "r[i] = tr.holds[i][p] ? '0' : '1';", 0),
    ("split_off_by_one", "const int j = size - 1 - i;\n        for (int x = 0;",
     "const int j = size - i;\n        for (int x = 0;", 0),
    ("cache_per_level_only", "const bool is_new = cache.insert(key).second;",
     "const bool is_new = cache.insert(key + \"#\" + std::to_string(level)).second;", 0),
    ("separation_ignores_negatives", "if (at0 != positive) return false;",
     "if (positive && !at0) return false;", 0),
    ("separation_last_position", "const bool at0 = !cm[k].empty() && cm[k][0] == '1';",
     "const bool at0 = !cm[k].empty() && cm[k].back() == '1';", 0),
    ("solve_size_off_by_one", "r->solved_size = level;", "r->solved_size = level + 1;", 0),
    ("parser_transposes_operands", "return add({op, 0, a, b});",
     "return add({op, 0, is_binary(op) ? b : a, is_binary(op) ? a : b});", 0),
    ("unary_reads_wrong_level", "const int i = size - 1;\n        for (int x = 0;",
     "const int i = size > 2 ? size - 2 : 1;\n        for (int x = 0;", 0),
]


def _mutate(src, old, new, occ):
    pos = -1
    for _ in range(occ + 1):
        pos = src.index(old, pos + 1)
    return src[:pos] + new + src[pos + len(old):]


def _build(tmpdir, name, old, new, occ):
    src = open(os.path.join(ROOT, "oracle", "oracle.cpp")).read()
    assert old in src, f"mutation anchor for {name} not found"
    mut = _mutate(src, old, new, occ)
    assert mut != src
    cpp = os.path.join(tmpdir, f"{name}.cpp")
    so = os.path.join(tmpdir, f"{name}.so")
    with open(cpp, "w") as f:
        f.write(mut)
    subprocess.run(["g++", "-O1", "-std=c++17", "-pthread", "-shared", "-fPIC", "-o", so, cpp], check=True)
    return so


def test_real_oracle_passes_all_pins():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "pins.py"), oracle.build()],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout + r.stderr


def test_every_mutant_fails_a_pin(tmp_path):
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        libs = dict(zip([m[0] for m in MUTANTS],
                        ex.map(lambda m: _build(str(tmp_path), *m), MUTANTS)))

        def run(name):
            r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "pins.py"), libs[name]],
                               capture_output=True, text=True, timeout=600, cwd=ROOT)
            return name, r.returncode, r.stdout[-400:]

        results = list(ex.map(run, libs))
    survivors = [(n, out) for n, rc, out in results if rc == 0]
    assert not survivors, f"mutants not caught by any pin: {survivors}"
