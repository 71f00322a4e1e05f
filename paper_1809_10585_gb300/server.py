"""Continuously batched factorize/solve service on one GPU: a thin Python client of the C ABI
server (hodlr_server_* in include/hodlr_qr.h; scheduling policy in csrc/serve_sched.h).

Requests
  * FactorSolve(inp, rhs, tol, keep, key): build the HODLR matrix on the device, hQR, solve with
    the right-hand sides, return x; keep=True keeps the factors resident under `key` for later
    Solve requests (repeat right-hand sides hit resident factors).
  * Solve(key, rhs): solve with resident factors.

The server admits a request as soon as a slot is free and its exact device footprint
(hodlr_footprint plus its right-hand sides) fits the HBM budget, evicting least recently used
resident factors to make room; requests admitted while others run overlap on the device.
Latency runs from submission to completion.  This module only marshals arguments and replays
arrival times: scheduling and every numeric step run in the library.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import time

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


def footprint_bytes(inp, rank_cap: int, nrhs: int) -> int:
    """Device bytes the server charges a FactorSolve request: the exact footprint of build +
    factorization + solve (hodlr_footprint) plus its right-hand sides."""
    return B.footprint(inp.n, inp.leaf_sizes, rank_cap, estimate_norm=True, nrhs=nrhs) + 8 * inp.n * nrhs


def _rhs(a):
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    return np.asfortranarray(a)


class Server:
    def __init__(self, device: int = 0, slots: int = 8, hbm_budget: float = 120e9, rank_cap: int = 256):
        self.rank_cap = rank_cap
        self.h = B._VP()
        B.check(B.lib().hodlr_server_create(device, slots, C.c_size_t(int(hbm_budget)), rank_cap, C.byref(self.h)),
                "hodlr_server_create")
        self.keys: dict[str, int] = {}
        self.results: dict[int, Result] = {}
        self.pending: dict[int, tuple] = {}       # id -> (kind, n, nrhs)
        self.max_running = 0

    # ------------------------------------------------------------------------------ API
    def _key(self, name):
        if name not in self.keys:
            self.keys[name] = len(self.keys)
        return self.keys[name]

    def submit(self, req) -> int:
        rid = C.c_longlong()
        rhs = _rhs(req.rhs)
        nrhs = rhs.shape[1]
        if isinstance(req, Solve):
            if req.key not in self.keys:
                raise KeyError(f"no factorization was submitted under {req.key!r}")
            B.check(B.lib().hodlr_server_submit_solve(self.h, self.keys[req.key], nrhs, B._VP(rhs.ctypes.data),
                                                      rhs.shape[0], C.byref(rid)), "hodlr_server_submit_solve")
            self.pending[rid.value] = ("solve", rhs.shape[0], nrhs)
        else:
            sizes, leaves, U12, V12, r12, U21, V21, r21, keep = B._marshal(req.inp)
            key = self._key(req.key) if (req.keep and req.key is not None) else -1
            B.check(B.lib().hodlr_server_submit(self.h, req.inp.n, len(req.inp.leaf_sizes), sizes, leaves, U12, V12,
                                                r12, U21, V21, r21, req.tol, nrhs, B._VP(rhs.ctypes.data),
                                                rhs.shape[0], key, C.byref(rid)), "hodlr_server_submit")
            self.pending[rid.value] = ("factor_solve", req.inp.n, nrhs)
        return rid.value

    def poll(self):
        """Progress the server; collect finished requests into self.results."""
        running = C.c_int()
        B.check(B.lib().hodlr_server_stats(self.h, None, C.byref(running), None, None), "hodlr_server_stats")
        self.max_running = max(self.max_running, running.value)
        for rid in list(self.pending):
            kind, n, nrhs = self.pending[rid]
            st, lat = C.c_int(), C.c_double()
            B.check(B.lib().hodlr_server_poll(self.h, rid, C.byref(st), None, n, C.byref(lat)), "hodlr_server_poll")
            if st.value < 0:
                del self.pending[rid]
                raise B.HodlrError(-st.value, f"request {rid}")
            if st.value == 2:
                x = np.zeros((n, nrhs), order="F")
                B.check(B.lib().hodlr_server_poll(self.h, rid, C.byref(st), B._VP(x.ctypes.data), n, C.byref(lat)),
                        "hodlr_server_poll")
                self.results[rid] = Result(rid, x, lat.value, kind, n)
                del self.pending[rid]

    def run(self, requests, poll_sleep=2e-4):
        """Replay requests with their arrival times (seconds from now) and serve them all."""
        order_in = sorted(range(len(requests)), key=lambda i: (requests[i].arrival, i))
        t0 = time.perf_counter()
        ids = {}
        k = 0
        while k < len(order_in) or self.pending:
            now = time.perf_counter() - t0
            while k < len(order_in) and requests[order_in[k]].arrival <= now:
                i = order_in[k]
                ids[i] = self.submit(requests[i])
                k += 1
            self.poll()
            if not self.pending and k < len(order_in):
                time.sleep(max(0.0, min(requests[order_in[k]].arrival - (time.perf_counter() - t0), 0.01)))
            else:
                time.sleep(poll_sleep)
        return [self.results[ids[i]] for i in range(len(requests))]

    def latencies(self):
        lat = np.array([r.latency_s for r in self.results.values()])
        if lat.size == 0:
            return {"p50_s": None, "p99_s": None, "count": 0}
        return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "count": int(lat.size)}

    def stats(self):
        w, r, res = C.c_int(), C.c_int(), C.c_int()
        b = C.c_size_t()
        B.check(B.lib().hodlr_server_stats(self.h, C.byref(w), C.byref(r), C.byref(res), C.byref(b)),
                "hodlr_server_stats")
        return {"waiting": w.value, "running": r.value, "resident": res.value, "bytes": int(b.value)}

    def close(self):
        if self.h:
            B.lib().hodlr_server_destroy(self.h)
            self.h = B._VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
