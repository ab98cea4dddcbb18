"""lsyn_eval_noalloc against the CPU oracle, through the C ABI (needs a GPU).

lsyn_eval_noalloc serves callers that cannot allocate device memory (their
process's memory manager owns every allocation, or an allocation that may
synchronise the device is not acceptable on their path): it reads traces the
caller holds on the device, writes into the caller's device buffer, and keeps
its scratch in a fixed array inside the library. Its output must equal the
oracle's evaluation by the LTLf definition bit for bit, and lsyn_eval's, on
consecutive calls that reuse that array.

The file name makes pytest collect it last, so a run that stops at the first
failure has run every other test before this one.
"""
import numpy as np
import pytest

import oracle
from paper_2504_18943_gb300 import workloads as W
from tests.gpu_util import lib, oracle_rows

pytestmark = pytest.mark.gpu


def _device_inputs(packed, lengths=None):
    import torch
    words = packed.atom_words
    view = np.int32 if packed.word_bits == 32 else np.int64
    atoms = torch.from_numpy(np.ascontiguousarray(words).view(view)).cuda()
    lens = torch.from_numpy(np.ascontiguousarray(packed.lengths if lengths is None else lengths,
                                                 dtype=np.int32)).cuda()
    out = torch.zeros(packed.n_traces, dtype=torch.int32 if packed.word_bits == 32 else torch.int64, device="cuda")
    return atoms, lens, out


def _noalloc(L, packed, atoms, lengths, out, f):
    import torch
    out.fill_(-1)
    L.lsyn_eval_noalloc(packed.n_props, packed.n_traces, packed.word_bits, atoms.data_ptr(), lengths.data_ptr(), f,
                        out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(packed.word_dtype)


@pytest.mark.parametrize("word_bits", [32, 64])
def test_noalloc_eval_equals_oracle_on_consecutive_calls(word_bits):
    L = lib()
    st = W.Stream(4242 + word_bits)
    tb = W.draw_traces(st, 777, 4, 1, word_bits, np.full(4, 0.45))
    problem = W.Problem("noalloc", 4, tb, 400, 377, word_bits)
    spec = oracle.Spec.from_problem(problem)
    packed = L.pack_problem(problem)
    atoms, lengths, out = _device_inputs(packed)
    formulas = ["(U (! p1) (& p0 (X p3)))", "(G (| p2 (F (& p0 (X (X p1))))))"]
    formulas += [W.random_formula(st, st.randint(1, 14), 4) for _ in range(6)]
    for f in formulas:  # consecutive calls share the scratch array
        got = _noalloc(L, packed, atoms, lengths, out, f)
        want = oracle_rows([spec.eval(f)], word_bits, problem.n_traces)[0]
        assert np.array_equal(got, want), f
        assert np.array_equal(got, L.lsyn_eval(packed, f)), f


@pytest.mark.parametrize("word_bits", [32, 64])
def test_noalloc_eval_clamps_lengths_to_one_word(word_bits):
    """Lengths above the word are clamped to it: the result is the oracle's on
    the traces cut to their first word_bits positions."""
    L = lib()
    st = W.Stream(99 + word_bits)
    tb = W.draw_traces(st, 300, 3, word_bits // 2, 2 * word_bits, np.full(3, 0.5))
    cut_len = np.minimum(tb.lengths, word_bits).astype(np.int32)
    cut = W.TraceBatch(tb.bits[:, :word_bits, :], cut_len)
    problem = W.Problem("clamp", 3, cut, 150, 150, word_bits)
    spec = oracle.Spec.from_problem(problem)
    packed = L.pack_problem(problem)
    assert (tb.lengths > word_bits).any()
    atoms, lengths, out = _device_inputs(packed, tb.lengths)  # the uncut lengths
    for f in ["(F p0)", "(G p1)", "(U p0 (X p2))", "(X p1)", "(! (F (& p0 p1)))"]:
        got = _noalloc(L, packed, atoms, lengths, out, f)
        want = oracle_rows([spec.eval(f)], word_bits, problem.n_traces)[0]
        assert np.array_equal(got, want), f


def test_noalloc_eval_rejects_requests_above_its_scratch():
    import torch
    L = lib()
    n = 40000  # 40 nodes x 40000 traces x 8 bytes > 8 MiB
    atoms = torch.zeros((2, n), dtype=torch.int64, device="cuda")
    lengths = torch.full((n,), 5, dtype=torch.int32, device="cuda")
    out = torch.zeros(n, dtype=torch.int64, device="cuda")
    f = "p0"
    for _ in range(13):
        f = f"(& {f} (X p1))"
    with pytest.raises(L.LsynError) as ei:
        L.lsyn_eval_noalloc(2, n, 64, atoms.data_ptr(), lengths.data_ptr(), f, out.data_ptr(), 0)
    assert ei.value.status == L.LSYN_E_INVAL and "scratch" in L.lsyn_last_error(None)
