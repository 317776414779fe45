"""Helpers for the GPU parity tests (comparison rules, library setup)."""
import numpy as np
import pytest


def same_f32(a, b):
    """Bit equality of float32 arrays, except that any NaN equals any NaN
    (NaN payloads differ between the GPU and the host C library)."""
    a = np.asarray(a, dtype=np.float32)
    b = np.asarray(b, dtype=np.float32)
    if a.shape != b.shape:
        return False
    nan = np.isnan(a) & np.isnan(b)
    return bool(np.all(nan | (a.view(np.uint32) == b.view(np.uint32))))


def first_mismatch(a, b):
    a = np.asarray(a, dtype=np.float32).ravel()
    b = np.asarray(b, dtype=np.float32).ravel()
    nan = np.isnan(a) & np.isnan(b)
    bad = np.nonzero(~(nan | (a.view(np.uint32) == b.view(np.uint32))))[0]
    if bad.size == 0:
        return None
    i = int(bad[0])
    return i, float(a[i]), float(b[i]), int(bad.size)


@pytest.fixture(scope="session")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1902_09215_gb300 import gp
    gp.lib()
    torch.cuda.set_device(0)
    return gp
