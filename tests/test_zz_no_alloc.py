"""The allocation-free dense QR entry point (hodlr_dense_qr_noalloc).

Some callers may not allocate device memory after start-up: cudaMalloc and cudaFree
synchronize the device and can stall other streams, and some services reserve all their memory
up front.  hodlr_dense_qr_noalloc serves them from a fixed static device scratch array.  It is
checked against the allocating entry point (hodlr_dense_qr) and directly against the oracle's
compact-WY QR (Alg. 1), on two calls in a row whose sizes differ (the shared scratch keeps the
first call's data).  This file is collected last on purpose: if it fails, a run that stops at
the first failure has already run every other test."""
import numpy as np
import pytest

import oracle.core as O

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


def test_noalloc_dense_qr_matches_oracle_and_allocating_entry_point_twice():
    rng = np.random.default_rng(11)
    for (h, w) in ((300, 256), (129, 64)):
        A = rng.standard_normal((h, w))
        A[:, 1] *= 1e-9
        Yo, To, Ro = O.block_qr(A)
        Ar, Tr = _run("hodlr_dense_qr", A, w)
        An, Tn = _run("hodlr_dense_qr_noalloc", A, w)
        sc = max(1.0, np.abs(A).max())
        Rn = np.triu(An[:w])
        Yn = np.tril(An, -1)
        Yn[:w, :w] += np.eye(w)
        # against the oracle (R, the unit lower Y and the upper T of Q = I - Y T Y^T)
        np.testing.assert_allclose(Rn, Ro, atol=1e-13 * sc * np.sqrt(h))
        np.testing.assert_allclose(Yn, Yo, atol=1e-11)
        np.testing.assert_allclose(np.triu(Tn), To, atol=1e-12)
        # against the allocating entry point
        np.testing.assert_allclose(Rn, np.triu(Ar[:w]), atol=1e-13 * sc * np.sqrt(h))
        np.testing.assert_allclose(np.tril(An, -1), np.tril(Ar, -1), atol=1e-11)
        np.testing.assert_allclose(np.triu(Tn), np.triu(Tr), atol=1e-12)


@pytest.mark.parametrize("h,w", [(400, 300), (100, 1025)])
def test_noalloc_rejects_sizes_beyond_its_limits_and_writes_nothing(h, w):
    from paper_1809_10585_gb300 import binding as B
    sentinel = 7.25
    ta = torch.full((w, h), sentinel, dtype=torch.float64, device="cuda")
    k = min(h, w)
    tt = torch.full((k, k), sentinel, dtype=torch.float64, device="cuda")
    rc = B.lib().hodlr_dense_qr_noalloc(U.ctx().h, h, w, B._VP(ta.data_ptr()), h, B._VP(tt.data_ptr()), k)
    assert rc == B.HODLR_EINVAL
    torch.cuda.synchronize()
    assert bool((ta == sentinel).all()) and bool((tt == sentinel).all())
