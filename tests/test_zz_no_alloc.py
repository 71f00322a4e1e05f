"""The allocation-free dense QR entry point (hodlr_dense_qr_noalloc) against hodlr_dense_qr.

Some callers may not allocate device memory after start-up (cudaMalloc/cudaFree synchronize
the device; some services reserve all memory up front).  hodlr_dense_qr_noalloc serves them
from a fixed static device scratch array.  This file is collected last on purpose: if it
fails, a run that stops at the first failure has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from tests import gpu_util as U  # noqa: E402


def _run(fn, A, w):
    from paper_1809_10585_gb300 import binding as B
    h = A.shape[0]
    ta, pa, lda = U.dev(A)
    tt, pt, ldt = U.empty(w, w)
    rc = getattr(B.lib(), fn)(U.ctx().h, h, w, B._VP(pa), lda, B._VP(pt), ldt)
    assert rc == 0, (fn, rc)
    return U.host(ta, h, w), U.host(tt, w, w)


def test_noalloc_dense_qr_matches_allocating_entry_point_twice():
    rng = np.random.default_rng(11)
    # two calls in a row with different shapes: the shared scratch keeps the first call's data
    for (h, w) in ((300, 256), (129, 64)):
        A = rng.standard_normal((h, w))
        A[:, 1] *= 1e-9
        Ar, Tr = _run("hodlr_dense_qr", A, w)
        An, Tn = _run("hodlr_dense_qr_noalloc", A, w)
        sc = max(1.0, np.abs(A).max())
        np.testing.assert_allclose(np.triu(An[:w]), np.triu(Ar[:w]), atol=1e-13 * sc * np.sqrt(h))
        np.testing.assert_allclose(np.tril(An, -1), np.tril(Ar, -1), atol=1e-11)
        np.testing.assert_allclose(np.triu(Tn), np.triu(Tr), atol=1e-12)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1809_10585_gb300 import binding as B
    A = np.zeros((400, 300))
    ta, pa, lda = U.dev(A)
    tt, pt, ldt = U.empty(300, 300)
    rc = B.lib().hodlr_dense_qr_noalloc(U.ctx().h, 400, 300, B._VP(pa), lda, B._VP(pt), ldt)
    assert rc == B.HODLR_EINVAL
