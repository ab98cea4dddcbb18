"""The binding keeps a context's configuration (and with it the Python
allocation callbacks whose function pointers the library holds) alive until
the context is destroyed, even when the caller passed a temporary config:
the library calls the free callback from lsyn_destroy. No GPU: the C entry
points are replaced by stubs that record what they are given."""
import ctypes
import gc
import weakref

import oracle
from paper_2504_18943_gb300 import lsyn as L
from paper_2504_18943_gb300 import workloads as W


class _Alloc:
    def __init__(self):
        self.alloc_fn = L.ALLOC_FN(lambda n, u: None)
        self.free_fn = L.FREE_FN(lambda p, u: None)


class _StubLib:
    def __init__(self):
        self.destroyed = []

    def lsyn_create(self, problem, config, out):
        ctypes.cast(out, ctypes.POINTER(ctypes.c_void_p))[0] = 0x1234
        return L.LSYN_OK

    def lsyn_destroy(self, ctx):
        self.destroyed.append(ctx.value)


def test_temporary_config_lives_until_destroy(monkeypatch):
    stub = _StubLib()
    monkeypatch.setattr(L, "_lib", stub)
    packed = L.pack_problem(W.tiny_problem(0, oracle.labeller))
    alloc = _Alloc()
    probe = weakref.ref(alloc)

    def temporary_config():
        return L.make_config(cache_bytes=1 << 20, allocator=alloc)

    ctx = L.lsyn_create(packed, temporary_config())
    del alloc
    gc.collect()
    assert probe() is not None, "the allocator callbacks were freed while the context lives"
    L.lsyn_destroy(ctx)
    gc.collect()
    assert stub.destroyed == [0x1234]
    assert probe() is None, "the context's config was not released after destroy"
