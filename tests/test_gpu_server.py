"""Continuously batched service: requests of mixed size arriving while others run give the
same results as when each is served alone, and repeat right-hand sides reuse resident factors."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from tests import gpu_util as U  # noqa: E402


def _requests():
    from paper_1809_10585_gb300 import server as S
    specs = [(1024, 128, 5, 0.0), (2048, 256, 10, 10.0), (777, 64, 6, 0.0), (4096, 256, 12, 14.0),
             (1500, 128, 8, 6.0), (512, 64, 4, 0.0)]
    reqs = []
    for i, (n, nmin, k, dec) in enumerate(specs):
        inp = W.random_hodlr(n, nmin, k, seed=100 + i, col_scale_decades=dec)
        reqs.append(S.FactorSolve(inp, W.rhs(n, 1 + i % 3, seed=i), tol=1e-12, keep=(i % 2 == 0),
                                  key=f"m{i}", arrival=0.002 * i))
    for i in (0, 2, 4):
        reqs.append(S.Solve(f"m{i}", W.rhs(specs[i][0], 2, seed=50 + i), arrival=0.02 + 0.001 * i))
    return reqs


def test_results_alone_equal_results_in_the_mix():
    from paper_1809_10585_gb300 import server as S
    U.ctx()
    mix = S.Server(0, slots=6, hbm_budget=60e9)
    got = mix.run(_requests())
    lat = mix.latencies()
    mix.close()
    assert lat["count"] == len(got) and lat["p99_s"] >= lat["p50_s"] > 0
    alone = S.Server(0, slots=6, hbm_budget=60e9)     # same slots, one request at a time
    ref = []
    for r in _requests():
        r.arrival = 0.0
        ref.extend(alone.run([r]))
    alone.close()
    for a, b in zip(got, ref):
        assert a.kind == b.kind and np.array_equal(a.x, b.x)
    # the solutions solve the systems
    reqs = _requests()
    dense = {}
    for r in reqs:
        if isinstance(r, S.FactorSolve):
            dense[r.key] = W.to_dense(r.inp)
    for r, res in zip(reqs, got):
        A = dense[r.key] if isinstance(r, S.Solve) else dense[r.key]
        b = r.rhs
        resid = np.linalg.norm(A @ res.x - b) / (np.linalg.norm(A, 1) * np.linalg.norm(res.x) + np.linalg.norm(b))
        assert resid <= 1e-9


def test_admission_respects_the_memory_budget():
    from paper_1809_10585_gb300 import server as S
    U.ctx()
    reqs = [S.FactorSolve(W.random_hodlr(2048, 256, 8, seed=s), W.rhs(2048, 2, seed=s), 1e-12) for s in range(4)]
    need = S.footprint_bytes(reqs[0].inp, 256, 2)
    srv = S.Server(0, slots=4, hbm_budget=need * 1.5)      # room for one request at a time
    out = srv.run([S.FactorSolve(r.inp, r.rhs, r.tol, False, None, 0.0) for r in reqs])
    st = srv.stats()
    srv.close()
    assert len(out) == 4 and srv.max_running == 1
    assert st["bytes"] == 0 and st["running"] == 0


def test_server_c_abi_errors_and_eviction():
    """Through the C ABI: a solve under a key nobody factors is refused, a request that can
    never fit the budget fails with HODLR_ENOMEM, and resident factors are evicted (least
    recently used first) when a new factorization needs their memory; a solve whose factors
    were evicted fails with HODLR_ESTATE."""
    import ctypes as C
    from paper_1809_10585_gb300 import binding as B
    from paper_1809_10585_gb300 import server as S
    U.ctx()
    inp = W.random_hodlr(1024, 128, 5, seed=1)
    need = S.footprint_bytes(inp, 64, 1)
    h = B._VP()
    B.check(B.lib().hodlr_server_create(0, 2, C.c_size_t(int(need * 1.6)), 64, C.byref(h)))
    try:
        rid = C.c_longlong()
        b = np.ones((1024, 1), order="F")
        assert B.lib().hodlr_server_submit_solve(h, 99, 1, B._VP(b.ctypes.data), 1024, C.byref(rid)) == B.HODLR_ESTATE

        def submit(x, key):
            sizes, leaves, U12, V12, r12, U21, V21, r21, keep = B._marshal(x)
            B.check(B.lib().hodlr_server_submit(h, x.n, len(x.leaf_sizes), sizes, leaves, U12, V12, r12, U21, V21,
                                                r21, 1e-12, 1, B._VP(b.ctypes.data), x.n, key, C.byref(rid)))
            return rid.value

        def wait(r, n):
            st, lat = C.c_int(), C.c_double()
            x = np.zeros((n, 1), order="F")
            for _ in range(200000):
                B.check(B.lib().hodlr_server_poll(h, r, C.byref(st), B._VP(x.ctypes.data), n, C.byref(lat)))
                if st.value == 2 or st.value < 0:
                    return st.value, x
            raise AssertionError("request did not finish")
        big = W.random_hodlr(8192, 256, 10, seed=2)
        st, _ = wait(submit(big, -1), 8192)                 # far beyond the budget
        assert st == -B.HODLR_ENOMEM
        st, x0 = wait(submit(inp, 7), 1024)                  # kept under key 7
        assert st == 2
        inp2 = W.random_hodlr(1024, 128, 5, seed=3)
        st, _ = wait(submit(inp2, 8), 1024)                  # needs key 7's memory: evicts it
        assert st == 2
        r = C.c_int()
        B.check(B.lib().hodlr_server_stats(h, None, None, C.byref(r), None))
        assert r.value == 1
        B.check(B.lib().hodlr_server_submit_solve(h, 7, 1, B._VP(b.ctypes.data), 1024, C.byref(rid)))
        st, _ = wait(rid.value, 1024)
        assert st == -B.HODLR_ESTATE
        # the solve on the surviving factors equals the library's solve of the same matrix
        B.check(B.lib().hodlr_server_submit_solve(h, 8, 1, B._VP(b.ctypes.data), 1024, C.byref(rid)))
        st, x2 = wait(rid.value, 1024)
        assert st == 2
        M = U.gpu_qr(inp2, 1e-12, anorm=0.0, rank_cap=64)
        tb = torch.ones(1, 1024, dtype=torch.float64, device="cuda")
        assert M.solve(1, tb.data_ptr(), 1024) == 0
        np.testing.assert_allclose(x2[:, 0], tb.cpu().numpy()[0], rtol=1e-10, atol=1e-12)
    finally:
        B.lib().hodlr_server_destroy(h)
