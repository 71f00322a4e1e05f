"""Helpers for the GPU tests: run the CUDA path through the C ABI and bring results back as
numpy/torch arrays.  Test infrastructure only."""
import numpy as np
import torch

from paper_1809_10585_gb300 import binding as B
from paper_1809_10585_gb300 import build as BUILD

_CTX = None


def ctx():
    global _CTX
    if _CTX is None:
        BUILD.build()
        _CTX = B.Context(0)
    return _CTX


def dev(a):
    """float64 column-major device copy of a numpy array, returned as (tensor, ptr, ld)."""
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    t = torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda")   # rows of t = columns of a
    return t, t.data_ptr(), a.shape[0]


def host(t, rows, cols):
    """numpy (rows x cols) from a column-major device tensor made by dev()/empty()."""
    torch.cuda.synchronize()
    return t.cpu().numpy().T[:rows, :cols].copy()


def empty(rows, cols):
    t = torch.zeros((cols, rows), dtype=torch.float64, device="cuda")
    return t, t.data_ptr(), rows


def gpu_qr(inp, tol, anorm=0.0, rank_cap=128, graph=False):
    c = ctx()
    M = B.Matrix(c, inp, rank_cap=rank_cap)
    if graph:
        M.snapshot()
        M.qr_graph(tol, anorm)
    else:
        M.qr(tol, anorm)
    c.sync()
    return M


def dense_of(M, which):
    n = M.n
    t, p, ld = empty(n, n)
    M.to_dense(which, p, ld)
    return t


def factors_dense(M):
    """(Y, T, R) dense as torch float64 cuda tensors in the natural (row, col) orientation."""
    Y = dense_of(M, 1).T
    R = dense_of(M, 2).T
    T = dense_of(M, 3).T
    return Y, T, R


def errors_torch(Y, T, R, A):
    """e_orth = ||Q^T Q - I||_2, e_acc = ||Q R - A||_2 (Sec. 5), dense on the GPU."""
    n = Y.shape[0]
    I = torch.eye(n, dtype=torch.float64, device=Y.device)
    Q = I - Y @ T @ Y.T
    e_orth = torch.linalg.matrix_norm(Q.T @ Q - I, ord=2).item()
    e_acc = torch.linalg.matrix_norm(Q @ R - A, ord=2).item()
    return e_orth, e_acc
