"""Continuously batched factorize/solve service on one GPU, over the C ABI.

Requests
  * FactorSolve(inp, rhs, tol, keep): build the HODLR matrix on the device, hQR, solve with the
    right-hand sides, return x; keep=True keeps the factors resident under `key` for later
    Solve requests (repeat right-hand sides hit resident factors).
  * Solve(key, rhs): solve with resident factors.

Continuous batching: every admitted request gets a slot — a library context with its own
streams — so work of requests that arrive while others are on the GPU overlaps on the device.
Requests are admitted as soon as a slot is free and their estimated HBM footprint fits the
budget (least recently used resident factors are evicted to make room).  Completion is
polled without blocking (hodlr_ready).  Latency is measured from arrival to completion.

Every numeric step runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import itertools
import time
from collections import OrderedDict, deque

import numpy as np

from . import binding as B


@dataclasses.dataclass
class FactorSolve:
    inp: object
    rhs: np.ndarray
    tol: float = 1e-12
    keep: bool = False
    key: str | None = None
    arrival: float = 0.0


@dataclasses.dataclass
class Solve:
    key: str
    rhs: np.ndarray
    arrival: float = 0.0


@dataclasses.dataclass
class Result:
    rid: int
    x: np.ndarray
    latency_s: float
    kind: str
    n: int


def footprint_bytes(n: int, nleaf: int, leaf: int, rank_cap: int, nrhs: int) -> int:
    """HBM estimate of one factorization: storage of A/Y/R and T (leaves and rank_cap
    factors on every level), planner scratch (about four times the factor storage at these
    shapes) and the right-hand sides."""
    levels = max(0, nleaf.bit_length() - 1)
    leaves = 2 * nleaf * leaf * leaf * 8
    factors = 3 * n * levels * rank_cap * 8
    scratch = 4 * factors + 16 * n * rank_cap * 8
    return int(leaves + factors + scratch + 3 * n * max(nrhs, 1) * 8)


class Server:
    def __init__(self, device: int = 0, slots: int = 8, hbm_budget: float = 120e9, rank_cap: int = 256):
        import torch
        self.torch = torch
        self.device = device
        self.dev = f"cuda:{device}"      # where right-hand sides are staged
        self.slots = [B.Context(device) for _ in range(slots)]
        for c in self.slots:             # several factorizations share the SMs
            c.concurrency = slots
        self.free = deque(range(slots))
        self.budget = float(hbm_budget)
        self.used = 0.0
        self.rank_cap = rank_cap
        self.waiting: deque = deque()
        self.active = {}                 # slot -> (rid, req, matrix, rhs tensor, t_arrival, bytes, kind)
        self.resident: OrderedDict = OrderedDict()   # key -> (matrix, bytes)
        self.results: dict[int, Result] = {}
        self.ids = itertools.count()
        self.t0 = time.perf_counter()

    # ------------------------------------------------------------------------------ API
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req) -> int:
        rid = next(self.ids)
        self.waiting.append((rid, req, self.now() if req.arrival <= 0 else req.arrival))
        return rid

    def run(self, requests, poll_sleep=2e-4):
        """Replay requests with their arrival times (seconds from now) and serve them all."""
        pending = sorted(((r.arrival, i, r) for i, r in enumerate(requests)), key=lambda t: (t[0], t[1]))
        self.t0 = time.perf_counter()
        order = []
        k = 0
        while k < len(pending) or self.waiting or self.active:
            now = self.now()
            while k < len(pending) and pending[k][0] <= now:
                order.append(self.submit(pending[k][2]))
                k += 1
            self.step()
            if not self.active and not self.waiting and k < len(pending):
                time.sleep(max(0.0, min(pending[k][0] - self.now(), 0.01)))
            else:
                time.sleep(poll_sleep)
        return [self.results[r] for r in order]

    def step(self):
        self._poll()
        self._admit()

    def latencies(self):
        lat = np.array([r.latency_s for r in self.results.values()])
        if lat.size == 0:
            return {"p50_s": None, "p99_s": None, "count": 0}
        return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "count": int(lat.size)}

    def close(self):
        for _, (M, _) in list(self.resident.items()):
            M.free()
        self.resident.clear()
        for c in self.slots:
            c.close()

    # ------------------------------------------------------------------------- internals
    def _bytes_of(self, req):
        if isinstance(req, Solve):
            return 3 * req.rhs.shape[0] * max(1, req.rhs.shape[1]) * 8
        inp = req.inp
        return footprint_bytes(inp.n, len(inp.leaf_sizes), max(inp.leaf_sizes), self.rank_cap,
                               req.rhs.shape[1] if req.rhs.ndim > 1 else 1)

    def _evict_for(self, need):
        while self.used + need > self.budget and self.resident:
            key, (M, b) = self.resident.popitem(last=False)
            if any(a[2] is M for a in self.active.values()):
                self.resident[key] = (M, b)     # in use: keep, stop evicting
                self.resident.move_to_end(key, last=False)
                break
            M.free()
            self.used -= b

    def _producer_pending(self, key):
        """A FactorSolve that will keep factors under `key` is waiting or running."""
        if any(isinstance(r, FactorSolve) and r.keep and r.key == key for _, r, _ in self.waiting):
            return True
        return any(a[6] == "factor_solve" and a[1].keep and a[1].key == key for a in self.active.values())

    def _admit(self):
        torch = self.torch
        # first come, first served, except that a solve whose factors are not ready yet (still
        # being factored, or busy with another solve) lets later requests pass
        for item in list(self.waiting):
            if not self.free:
                return
            rid, req, t_arr = item
            if isinstance(req, Solve):
                if req.key not in self.resident:
                    if self._producer_pending(req.key):
                        continue
                    raise KeyError(f"no resident factors under {req.key!r}")
                if any(a[2] is self.resident[req.key][0] for a in self.active.values()):
                    continue                     # one solve per resident matrix at a time
            need = self._bytes_of(req)
            self._evict_for(need)
            if self.used + need > self.budget and self.active:
                return                           # wait for memory to free up
            self.waiting = deque(x for x in self.waiting if x[0] != rid)
            slot = self.free.popleft()
            ctx = self.slots[slot]
            rhs = np.asarray(req.rhs, dtype=np.float64)
            if rhs.ndim == 1:
                rhs = rhs[:, None]
            nrhs = rhs.shape[1]
            bt = torch.from_numpy(np.ascontiguousarray(rhs.T)).to(self.dev)
            if isinstance(req, Solve):
                M, _ = self.resident[req.key]
                self.resident.move_to_end(req.key)
                M.solve_async(nrhs, bt.data_ptr(), rhs.shape[0], ctx=ctx)
                kind = "solve"
            else:
                M = B.Matrix(ctx, req.inp, rank_cap=self.rank_cap)
                M.qr(req.tol, 0.0)
                M.solve_async(nrhs, bt.data_ptr(), rhs.shape[0])
                kind = "factor_solve"
            self.used += need
            self.active[slot] = (rid, req, M, bt, t_arr, need, kind)

    def _poll(self):
        for slot in list(self.active):
            ctx = self.slots[slot]
            if not ctx.ready():
                continue
            rid, req, M, bt, t_arr, need, kind = self.active.pop(slot)
            st, _ = (0, 0.0) if kind == "solve" else M.status()
            if st not in (0,):
                raise B.HodlrError(st, "factorization")
            x = bt.cpu().numpy().T.copy()
            self.results[rid] = Result(rid, x, self.now() - t_arr, kind, M.n)
            self.used -= need
            if kind == "factor_solve":
                if req.keep and req.key:
                    old = self.resident.pop(req.key, None)
                    if old is not None and old[0] is not M:
                        old[0].free()
                        self.used -= old[1]
                    fb = footprint_bytes(M.n, M.nleaf, 0, self.rank_cap, 0)
                    self.resident[req.key] = (M, fb)
                    self.used += fb
                else:
                    M.free()
            self.free.append(slot)
