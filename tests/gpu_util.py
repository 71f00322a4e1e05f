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


def norm2(E, iters=60):
    """||E||_2 by power iteration on E^T E from a fixed start (dense, on E's device).  A lower
    bound that converges to ||E||_2; the Frobenius norm gives the upper bound when needed."""
    x = torch.ones(E.shape[1], 1, dtype=E.dtype, device=E.device)
    x /= torch.linalg.vector_norm(x)
    s = 0.0
    for _ in range(iters):
        z = E.T @ (E @ x)
        nz = torch.linalg.vector_norm(z).item()
        if nz == 0.0:
            return 0.0
        x = z / nz
        s = nz
    return float(np.sqrt(s))


def errors_torch(Y, T, R, A, upper=False):
    """e_orth = ||Q^T Q - I||_2, e_acc = ||Q R - A||_2 (Sec. 5), dense on the GPU; with
    upper=True the Frobenius norms (upper bounds of the 2-norms) are returned."""
    n = Y.shape[0]
    I = torch.eye(n, dtype=torch.float64, device=Y.device)
    Q = I - Y @ (T @ Y.T)
    E1 = Q.T @ Q - I
    E2 = Q @ R - A
    if upper:
        return torch.linalg.matrix_norm(E1).item(), torch.linalg.matrix_norm(E2).item()
    return norm2(E1), norm2(E2)


def errors_both(Y, T, R, A):
    """((e_orth, e_acc) in the 2-norm, (e_orth, e_acc) in the Frobenius norm) with each error
    matrix formed once (dense, on the GPU)."""
    n = Y.shape[0]
    I = torch.eye(n, dtype=torch.float64, device=Y.device)
    Q = I - Y @ (T @ Y.T)
    E1 = Q.T @ Q - I
    E2 = Q @ R - A
    del Q
    two = (norm2(E1), norm2(E2))
    fro = (torch.linalg.matrix_norm(E1).item(), torch.linalg.matrix_norm(E2).item())
    return two, fro
