"""Parity at the benchmark's full size and launch configuration: the n = 8192, nmin = 256,
rank-10, column-scaled (condition ~1e14) workload at tol = 1e-12, factored by the CUDA-graph
path that bench.py times, with ||A||_2 estimated on the device.  Compared with the CPU oracle
on the same seeded input and with a dense FP64 QR of the assembled matrix."""
import numpy as np
import pytest

import oracle.core as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from tests import gpu_util as U  # noqa: E402


def test_fullsize_workload_matches_oracle():
    tol = 1e-12
    inp = W.config1()
    n = inp.n
    res = O.hqr(O.from_input(inp), tol)
    M = U.gpu_qr(inp, tol, anorm=0.0, rank_cap=128, graph=True)
    st, anorm = M.status()
    assert st == 0
    assert abs(anorm - res.anorm) <= 1e-10 * res.anorm     # same power iteration on both sides
    A = torch.from_numpy(W.to_dense(inp)).cuda()
    an = U.norm2(A)
    Y, T, R = U.factors_dense(M)
    eo, ea = U.errors_torch(Y, T, R, A)
    eoF, eaF = U.errors_torch(Y, T, R, A, upper=True)
    del Y, T
    Yo, To, Ro = (torch.from_numpy(x).cuda() for x in (res.Y_dense(), res.T_dense(), res.R_dense()))
    eoo, eao = U.errors_torch(Yo, To, Ro, A)
    del Yo, To
    floor = 1e-14 * np.sqrt(n)
    assert eoF <= 100 * tol and eaF / an <= 100 * tol, (eoF, eaF / an)
    assert eo <= 10 * eoo + floor and ea <= 10 * eao + floor * an, (eo, eoo, ea, eao)
    dg = torch.diagonal(R).abs()
    assert (dg - torch.diagonal(Ro).abs()).abs().max().item() <= 1e3 * tol * an
    # dense Householder QR of the assembled matrix (sign-normalised diagonal)
    Rd = torch.linalg.qr(A, mode="r")[1]
    assert (dg - torch.diagonal(Rd).abs()).abs().max().item() <= 1e3 * tol * an
    big = torch.diagonal(Rd).abs() >= 1e-6 * an
    rel = ((dg - torch.diagonal(Rd).abs()).abs() / torch.diagonal(Rd).abs())[big].max().item()
    assert rel <= 1e3 * tol * 1e6
    # ranks stay within capacity and the flop count matches the oracle's
    O.reset_counters()
    O.hqr(O.from_input(inp), tol)
    f = M.flops()
    assert abs(f["total"] - sum(O.FLOPS.values())) <= 0.2 * sum(O.FLOPS.values())
