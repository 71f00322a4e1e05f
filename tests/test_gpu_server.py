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
    need = S.footprint_bytes(2048, 8, 256, 256, 2)
    srv = S.Server(0, slots=4, hbm_budget=need * 1.5)      # room for one request at a time
    peak = []
    orig = srv._admit

    def admit():
        orig()
        peak.append(len(srv.active))
    srv._admit = admit
    out = srv.run([S.FactorSolve(r.inp, r.rhs, r.tol, False, None, 0.0) for r in reqs])
    srv.close()
    assert len(out) == 4 and max(peak) == 1
