"""Host-side scheduling of the continuously batched service, on the CPU: the library binding is
replaced by a fake whose work completes after a fixed number of polls, so admission order,
deferral of solves whose factors are not ready, slot reuse and the memory budget can be checked
without a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_10585_gb300 import server as S  # noqa: E402


class _Ctx:
    def __init__(self, device=0):
        self.left = 0

    def ready(self):
        self.left = max(0, self.left - 1)
        return self.left == 0

    def close(self):
        pass


class _Matrix:
    log = []

    def __init__(self, ctx, inp, rank_cap=256):
        self.ctx, self.n, self.nleaf, self.key = ctx, inp["n"], 4, inp["key"]

    def qr(self, tol, anorm):
        self.ctx.left += 3
        _Matrix.log.append(("qr", self.key))

    def solve_async(self, nrhs, ptr, ld, ctx=None):
        (ctx or self.ctx).left += 2
        _Matrix.log.append(("solve", self.key))

    def status(self):
        return 0, 1.0

    def free(self):
        pass


class _Fake:
    Context = _Ctx
    Matrix = _Matrix
    HodlrError = RuntimeError


@pytest.fixture
def server(monkeypatch):
    monkeypatch.setattr(S, "B", _Fake)
    monkeypatch.setattr(S, "footprint_bytes", lambda n, nleaf, leaf, cap, nrhs: 1000)
    _Matrix.log = []
    srv = S.Server(0, slots=3, hbm_budget=10_000)
    srv.dev = "cpu"
    srv._bytes_of = lambda req: 1000
    yield srv


def _fs(key, keep=True):
    inp = {"n": 8, "key": key}
    return S.FactorSolve(inp, np.ones((8, 1)), keep=keep, key=key)


def _drain(srv, limit=200):
    for _ in range(limit):
        srv.step()
        if not srv.waiting and not srv.active:
            return
    raise AssertionError("service did not drain")


def test_solve_waits_for_its_factorization(server):
    a = server.submit(_fs("m0"))
    b = server.submit(S.Solve("m0", np.ones((8, 2))))
    c = server.submit(_fs("m1", keep=False))
    server.step()
    # the solve on m0 cannot start yet; the later factorization passes it
    assert ("qr", "m1") in _Matrix.log and ("solve", "m0") in _Matrix.log
    assert sum(1 for x in _Matrix.log if x == ("solve", "m0")) == 1
    _drain(server)
    assert set(server.results) == {a, b, c}
    assert server.results[b].kind == "solve" and server.results[b].x.shape == (8, 2)
    assert "m0" in server.resident and "m1" not in server.resident


def test_solve_without_a_producer_is_an_error(server):
    server.submit(S.Solve("nope", np.ones((8, 1))))
    with pytest.raises(KeyError):
        server.step()


def test_one_solve_per_resident_matrix_at_a_time(server):
    server.submit(_fs("m0"))
    _drain(server)
    s1 = server.submit(S.Solve("m0", np.ones((8, 1))))
    s2 = server.submit(S.Solve("m0", np.ones((8, 1))))
    server.step()
    assert len(server.active) == 1 and len(server.waiting) == 1
    _drain(server)
    assert {s1, s2} <= set(server.results)


def test_budget_limits_concurrency(server):
    server.budget = 2500             # two requests of 1000 bytes fit, the third waits
    ids = [server.submit(_fs(f"m{i}", keep=False)) for i in range(3)]
    server.step()
    assert len(server.active) == 2 and len(server.waiting) == 1
    assert server.used <= server.budget
    _drain(server)
    assert set(ids) <= set(server.results) and server.used == 0
