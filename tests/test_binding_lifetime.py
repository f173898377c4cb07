"""Host-side rules of the Python binding, on CPU with a stand-in for
the library: a context must outlive every batch that holds it (the C ABI's
contract), so closing it while a batch is live raises, and each handle is
destroyed exactly once, the batch before its contexts; without the built
library every call raises (no CPU fallback)."""
import ctypes as C

import pytest

from paper_2109_07527_gb300 import crmc


class _FakeLib:
    def __init__(self):
        self.calls = []

    def cr_batch_create(self, out, arr, n):
        out._obj.value = 0xB0
        self.calls.append(("batch_create", [arr[i] for i in range(n)]))
        return 0

    def cr_batch_destroy(self, h):
        self.calls.append(("batch_destroy", h.value))

    def cr_destroy(self, h):
        self.calls.append(("destroy", h.value))

    def cr_strerror(self, code):
        return b"stand-in error"


@pytest.fixture
def fake(monkeypatch):
    lib = _FakeLib()
    monkeypatch.setattr(crmc, "_L", lib)
    return lib


def _context(lib, addr):
    c = crmc.Context.__new__(crmc.Context)
    c._h, c._lib, c._nbatch = C.c_void_p(addr), lib, 0
    return c


def test_context_cannot_close_under_a_live_batch(fake):
    a, b = _context(fake, 0x10), _context(fake, 0x20)
    bt = crmc.Batch([a, b])
    assert fake.calls == [("batch_create", [0x10, 0x20])]
    with pytest.raises(RuntimeError, match="live Batch"):
        a.close()
    assert a._h is not None
    bt.close()
    a.close()
    b.close()
    bt.close()  # idempotent
    a.close()
    assert fake.calls[1:] == [("batch_destroy", 0xB0), ("destroy", 0x10), ("destroy", 0x20)]


def test_context_in_two_batches(fake):
    a = _context(fake, 0x10)
    b1, b2 = crmc.Batch([a]), crmc.Batch([a])
    b1.close()
    with pytest.raises(RuntimeError):
        a.close()
    b2.close()
    a.close()
    assert [c[0] for c in fake.calls] == ["batch_create", "batch_create", "batch_destroy", "batch_destroy",
                                          "destroy"]


def test_garbage_collection_order(fake):
    a = _context(fake, 0x30)
    bt = crmc.Batch([a])
    del a  # the batch still holds the context
    assert ("destroy", 0x30) not in fake.calls
    del bt  # the batch goes first, then its context
    assert [c[0] for c in fake.calls] == ["batch_create", "batch_destroy", "destroy"]


def test_failed_batch_creation_leaves_contexts_free(fake):
    a = _context(fake, 0x40)
    fake.cr_batch_create = lambda out, arr, n: -1
    with pytest.raises(crmc.CrError):
        crmc.Batch([a])
    a.close()
    assert fake.calls == [("destroy", 0x40)]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every call raises; nothing falls back to a
    CPU path."""
    monkeypatch.setattr(crmc, "_L", None)
    monkeypatch.setattr(crmc, "LIB_PATH", str(tmp_path / "libcrmc.so"))
    with pytest.raises(ImportError, match="not built"):
        crmc._lib()
    with pytest.raises(ImportError):
        crmc.philox(0, 0, 0, 0, 0, 0, 1)
