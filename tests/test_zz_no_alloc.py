"""lsyn_eval_noalloc against lsyn_eval, through the C ABI (needs a GPU).

lsyn_eval_noalloc serves callers that cannot allocate device memory (their
process's memory manager owns every allocation, or an allocation that may
synchronise the device is not acceptable on their path): it reads traces the
caller holds on the device, writes into the caller's device buffer, and keeps
its scratch in a fixed array inside the library. Its output must equal
lsyn_eval's bit for bit, on consecutive calls that reuse that array.

The file name makes pytest collect it last, so a run that stops at the first
failure has run every other test before this one.
"""
import numpy as np
import pytest

from paper_2504_18943_gb300 import workloads as W
from tests.gpu_util import lib

pytestmark = pytest.mark.gpu


def _device_inputs(packed):
    import torch
    words = packed.atom_words
    view = np.int32 if packed.word_bits == 32 else np.int64
    atoms = torch.from_numpy(np.ascontiguousarray(words).view(view)).cuda()
    lengths = torch.from_numpy(packed.lengths).cuda()
    out = torch.zeros(packed.n_traces, dtype=torch.int32 if packed.word_bits == 32 else torch.int64, device="cuda")
    return atoms, lengths, out


@pytest.mark.parametrize("word_bits", [32, 64])
def test_noalloc_eval_equals_eval_on_consecutive_calls(word_bits):
    import torch
    L = lib()
    st = W.Stream(4242 + word_bits)
    tb = W.draw_traces(st, 777, 4, 1, word_bits, np.full(4, 0.45))
    problem = W.Problem("noalloc", 4, tb, 400, 377, word_bits)
    packed = L.pack_problem(problem)
    atoms, lengths, out = _device_inputs(packed)
    stream = torch.cuda.current_stream()
    formulas = ["(U (! p1) (& p0 (X p3)))", "(G (| p2 (F (& p0 (X (X p1))))))"]
    formulas += [W.random_formula(st, st.randint(1, 14), 4) for _ in range(6)]
    for f in formulas:  # consecutive calls share the scratch array
        out.fill_(-1)
        L.lsyn_eval_noalloc(4, packed.n_traces, word_bits, atoms.data_ptr(), lengths.data_ptr(), f,
                            out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(packed.word_dtype)
        want = L.lsyn_eval(packed, f)
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
