"""ctypes binding of the hQR C ABI (include/hodlr_qr.h).

Argument marshalling only: every step of the factorization, apply and solve runs in the CUDA
library.  Device buffers are passed as raw pointers (e.g. ``torch.Tensor.data_ptr()``), host
buffers as numpy arrays.  Loading fails loudly when the library has not been built — there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

HODLR_OK, HODLR_EINVAL, HODLR_ENOMEM, HODLR_ERANK, HODLR_ESINGULAR, HODLR_ETIMEOUT, HODLR_ECUDA, HODLR_ESTATE = range(8)

_lib = None


class HodlrError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {lib().hodlr_strerror(code).decode()} ({code})")


_PD = C.POINTER(C.c_double)
_PPD = C.POINTER(_PD)
_PI = C.POINTER(C.c_int)
_VP = C.c_void_p

_SIGS = {
    "hodlr_strerror": (C.c_char_p, [C.c_int]),
    "hodlr_ctx_create": (C.c_int, [C.c_int, C.POINTER(_VP)]),
    "hodlr_ctx_destroy": (None, [_VP]),
    "hodlr_ctx_set_stream": (C.c_int, [_VP, _VP]),
    "hodlr_ctx_set_cluster": (C.c_int, [_VP, C.c_int]),
    "hodlr_ctx_get_cluster": (C.c_int, [_VP, _PI]),
    "hodlr_ctx_set_cluster_large": (C.c_int, [_VP, C.c_int]),
    "hodlr_ctx_set_concurrency": (C.c_int, [_VP, C.c_int]),
    "hodlr_ctx_get_concurrency": (C.c_int, [_VP, _PI]),
    "hodlr_ctx_set_batch_group": (C.c_int, [_VP, C.c_int]),
    "hodlr_sync": (C.c_int, [_VP]),
    "hodlr_build": (C.c_int, [_VP, C.c_int, C.c_int, _PI, _PPD, _PPD, _PPD, _PI, _PPD, _PPD, _PI, C.c_int, C.POINTER(_VP)]),
    "hodlr_build_dense": (C.c_int, [_VP, C.c_int, C.c_int, _PI, _VP, C.c_int, C.c_double, C.c_int, C.c_ulonglong,
                                    C.POINTER(_VP)]),
    "hodlr_stats": (C.c_int, [_VP, _VP, _PI, _PI, _PI, C.POINTER(C.c_size_t)]),
    "hodlr_free": (None, [_VP]),
    "hodlr_upload": (C.c_int, [_VP, _VP, _PPD, _PPD, _PPD, _PI, _PPD, _PPD, _PI]),
    "hodlr_snapshot": (C.c_int, [_VP, _VP]),
    "hodlr_restore": (C.c_int, [_VP, _VP]),
    "hodlr_qr": (C.c_int, [_VP, _VP, C.c_double, C.c_double]),
    "hodlr_qr_graph": (C.c_int, [_VP, _VP, C.c_double, C.c_double]),
    "hodlr_qr_batched": (C.c_int, [_VP, C.c_int, C.POINTER(_VP), C.c_double, C.c_double]),
    "hodlr_qr_batched_graph": (C.c_int, [_VP, C.c_int, C.POINTER(_VP), C.c_double, C.c_double]),
    "hodlr_qr_profile": (C.c_int, [_VP, _VP, C.c_double, C.c_double, _PD, _PI, _PD]),
    "hodlr_autotune_batched": (C.c_int, [_VP, C.c_int, C.POINTER(_VP), C.c_double, C.c_double, C.c_int, _PI, _PI, _PD]),
    "hodlr_status": (C.c_int, [_VP, _VP, _PI, _PD]),
    "hodlr_ranks": (C.c_int, [_VP, _VP, _PI, _PI, _PI]),
    "hodlr_flops": (C.c_int, [_VP, _VP, _PD]),
    "hodlr_to_dense": (C.c_int, [_VP, _VP, C.c_int, _VP, C.c_int]),
    "hodlr_matvec": (C.c_int, [_VP, _VP, C.c_int, C.c_int, C.c_int, _VP, C.c_int, _VP, C.c_int]),
    "hodlr_apply_q": (C.c_int, [_VP, _VP, C.c_int, _VP, C.c_int]),
    "hodlr_apply_qt": (C.c_int, [_VP, _VP, C.c_int, _VP, C.c_int]),
    "hodlr_solve": (C.c_int, [_VP, _VP, C.c_int, _VP, C.c_int]),
    "hodlr_solve_async": (C.c_int, [_VP, _VP, C.c_int, _VP, C.c_int]),
    "hodlr_ready": (C.c_int, [_VP, _PI]),
    "hodlr_norm2_estimate": (C.c_int, [_VP, _VP, C.c_int, _PD]),
    "hodlr_storage_bytes": (C.c_size_t, [_VP]),
    "hodlr_download": (C.c_int, [_VP, _VP, _VP, C.c_size_t]),
    "hodlr_compact_bytes": (C.c_int, [_VP, _VP, C.POINTER(C.c_size_t)]),
    "hodlr_download_compact": (C.c_int, [_VP, _VP, _VP, C.c_size_t]),
    "hodlr_dense_qr": (C.c_int, [_VP, C.c_int, C.c_int, _VP, C.c_int, _VP, C.c_int]),
    "hodlr_truncate": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int, _VP, _VP, C.c_double, C.c_int, _VP, _VP, _PI]),
    "hodlr_dense_qr_noalloc": (C.c_int, [_VP, C.c_int, C.c_int, _VP, C.c_int, _VP, C.c_int]),
    "hodlr_fp64_peak": (C.c_int, [C.c_int, C.c_int, C.c_int, _PD, _PD]),
    "hodlr_server_create": (C.c_int, [C.c_int, C.c_int, C.c_size_t, C.c_int, C.POINTER(_VP)]),
    "hodlr_server_destroy": (None, [_VP]),
    "hodlr_server_submit": (C.c_int, [_VP, C.c_int, C.c_int, _PI, _PPD, _PPD, _PPD, _PI, _PPD, _PPD, _PI,
                                      C.c_double, C.c_int, _VP, C.c_int, C.c_longlong, C.POINTER(C.c_longlong)]),
    "hodlr_server_submit_solve": (C.c_int, [_VP, C.c_longlong, C.c_int, _VP, C.c_int, C.POINTER(C.c_longlong)]),
    "hodlr_server_poll": (C.c_int, [_VP, C.c_longlong, _PI, _VP, C.c_int, _PD]),
    "hodlr_server_stats": (C.c_int, [_VP, _PI, _PI, _PI, C.POINTER(C.c_size_t)]),
    "hodlr_ctx_set_memory_limit": (C.c_int, [_VP, C.c_size_t]),
    "hodlr_ctx_memory_used": (C.c_int, [_VP, C.POINTER(C.c_size_t)]),
    "hodlr_ctx_set_memory_pool": (C.c_int, [_VP, C.c_size_t]),
    "hodlr_ctx_share_memory": (C.c_int, [_VP, _VP]),
    "hodlr_device_bytes": (C.c_int, [_VP, C.POINTER(C.c_size_t)]),
    "hodlr_footprint": (C.c_int, [C.c_int, C.c_int, _PI, C.c_int, C.c_int, C.c_int, C.c_int,
                                  C.POINTER(C.c_size_t)]),
    "hodlr_permuted_qr": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int, _PI, _PI, _VP, C.c_int, _VP, C.c_int]),
    "hodlr_rect_compress": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int, _PI, _PI, _VP, C.c_int, C.c_double, C.c_int,
                                      C.c_ulonglong, C.POINTER(_VP)]),
    "hodlr_rect_qr": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int, _PI, _PI, _VP, C.c_int, C.c_double, C.c_double,
                                C.c_int, C.c_ulonglong, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP), _PD]),
    "hodlr_rect_permutation": (C.c_int, [C.c_int, _PI, _PI, _PI]),
    "hodlr_rect_to_dense": (C.c_int, [_VP, _VP, _VP, C.c_int]),
    "hodlr_rect_ranks": (C.c_int, [_VP, _VP, _PI, _PI]),
    "hodlr_rect_free": (None, [_VP]),
}

SYMBOLS = tuple(_SIGS)


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libhodlrqr.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run paper_1809_10585_gb300.build.build()")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc, what=""):
    if rc != HODLR_OK:
        raise HodlrError(rc, what)
    return rc


def _ptr_array(arrs):
    """Array of double* for a list of C-contiguous-in-Fortran-order numpy arrays (None -> NULL)."""
    out = (_PD * len(arrs))()
    keep = []
    for i, a in enumerate(arrs):
        if a is None or a.size == 0:
            out[i] = _PD()
            continue
        a = np.asfortranarray(a, dtype=np.float64)
        keep.append(a)
        out[i] = a.ctypes.data_as(_PD)
    return out, keep


class Context:
    def __init__(self, device: int = 0):
        self.h = _VP()
        check(lib().hodlr_ctx_create(device, C.byref(self.h)), "hodlr_ctx_create")

    def set_stream(self, stream_handle: int | None):
        check(lib().hodlr_ctx_set_stream(self.h, _VP(stream_handle or 0)), "hodlr_ctx_set_stream")

    @property
    def cluster(self) -> int:
        v = C.c_int()
        check(lib().hodlr_ctx_get_cluster(self.h, C.byref(v)), "hodlr_ctx_get_cluster")
        return v.value

    @cluster.setter
    def cluster(self, size: int):
        check(lib().hodlr_ctx_set_cluster(self.h, int(size)), "hodlr_ctx_set_cluster")

    def set_cluster_large(self, size: int):
        check(lib().hodlr_ctx_set_cluster_large(self.h, int(size)), "hodlr_ctx_set_cluster_large")

    @property
    def concurrency(self) -> int:
        v = C.c_int()
        check(lib().hodlr_ctx_get_concurrency(self.h, C.byref(v)), "hodlr_ctx_get_concurrency")
        return v.value

    @concurrency.setter
    def concurrency(self, factorizations: int):
        check(lib().hodlr_ctx_set_concurrency(self.h, int(factorizations)), "hodlr_ctx_set_concurrency")

    def set_batch_group(self, max_matrices: int):
        check(lib().hodlr_ctx_set_batch_group(self.h, int(max_matrices)), "hodlr_ctx_set_batch_group")

    def sync(self):
        check(lib().hodlr_sync(self.h), "hodlr_sync")

    def set_memory_limit(self, nbytes: int):
        check(lib().hodlr_ctx_set_memory_limit(self.h, int(nbytes)), "hodlr_ctx_set_memory_limit")

    def set_memory_pool(self, nbytes: int):
        check(lib().hodlr_ctx_set_memory_pool(self.h, int(nbytes)), "hodlr_ctx_set_memory_pool")

    def share_memory(self, other: "Context"):
        check(lib().hodlr_ctx_share_memory(self.h, other.h), "hodlr_ctx_share_memory")

    def memory_used(self) -> int:
        v = C.c_size_t()
        check(lib().hodlr_ctx_memory_used(self.h, C.byref(v)), "hodlr_ctx_memory_used")
        return int(v.value)

    def ready(self) -> bool:
        r = C.c_int()
        check(lib().hodlr_ready(self.h, C.byref(r)), "hodlr_ready")
        return bool(r.value)

    def close(self):
        if self.h:
            lib().hodlr_ctx_destroy(self.h)
            self.h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _marshal(inp):
    nleaf = len(inp.leaf_sizes)
    nn = nleaf - 1
    sizes = (C.c_int * nleaf)(*inp.leaf_sizes)
    leaves, k1 = _ptr_array(list(inp.leaves))
    U12, k2 = _ptr_array(list(inp.U12) if nn else [None])
    V12, k3 = _ptr_array(list(inp.V12) if nn else [None])
    U21, k4 = _ptr_array(list(inp.U21) if nn else [None])
    V21, k5 = _ptr_array(list(inp.V21) if nn else [None])
    r12 = (C.c_int * max(1, nn))(*[int(np.shape(u)[1]) for u in inp.U12] if nn else [0])
    r21 = (C.c_int * max(1, nn))(*[int(np.shape(u)[1]) for u in inp.U21] if nn else [0])
    return sizes, leaves, U12, V12, r12, U21, V21, r21, (k1, k2, k3, k4, k5)


class Matrix:
    """A device-resident HODLR matrix built from a host description with the fields
    n, leaf_sizes, leaves, U12, V12, U21, V21 (see workloads.HodlrInput)."""

    def __init__(self, ctx: Context, inp, rank_cap: int = 128):
        self.ctx = ctx
        self.n = int(inp.n)
        self.nleaf = len(inp.leaf_sizes)
        self.h = _VP()
        sizes, leaves, U12, V12, r12, U21, V21, r21, keep = _marshal(inp)
        check(lib().hodlr_build(ctx.h, self.n, self.nleaf, sizes, leaves, U12, V12, r12, U21, V21, r21,
                                rank_cap, C.byref(self.h)), "hodlr_build")
        self.rank_cap = rank_cap

    @classmethod
    def from_dense(cls, ctx: Context, n: int, leaf_sizes, A_ptr: int, lda: int, tol: float, rank_cap: int = 128,
                   seed: int = 0):
        """HODLR approximation of a dense column-major device matrix (hodlr_build_dense)."""
        self = cls.__new__(cls)
        self.ctx = ctx
        self.n = int(n)
        self.nleaf = len(leaf_sizes)
        self.h = _VP()
        sizes = (C.c_int * self.nleaf)(*[int(x) for x in leaf_sizes])
        check(lib().hodlr_build_dense(ctx.h, self.n, self.nleaf, sizes, _VP(A_ptr), lda, tol, rank_cap, seed,
                                      C.byref(self.h)), "hodlr_build_dense")
        self.rank_cap = rank_cap
        return self

    def stats(self):
        y, t, r = C.c_int(), C.c_int(), C.c_int()
        b = C.c_size_t()
        check(lib().hodlr_stats(self.ctx.h, self.h, C.byref(y), C.byref(t), C.byref(r), C.byref(b)), "hodlr_stats")
        return {"max_rank_Y": y.value, "max_rank_T": t.value, "max_rank_R": r.value, "bytes": b.value}

    def upload(self, inp):
        sizes, leaves, U12, V12, r12, U21, V21, r21, keep = _marshal(inp)
        check(lib().hodlr_upload(self.ctx.h, self.h, leaves, U12, V12, r12, U21, V21, r21), "hodlr_upload")

    def snapshot(self):
        check(lib().hodlr_snapshot(self.ctx.h, self.h), "hodlr_snapshot")

    def restore(self):
        check(lib().hodlr_restore(self.ctx.h, self.h), "hodlr_restore")

    def qr(self, tol: float, anorm: float = 0.0):
        check(lib().hodlr_qr(self.ctx.h, self.h, tol, anorm), "hodlr_qr")

    def qr_graph(self, tol: float, anorm: float = 0.0):
        check(lib().hodlr_qr_graph(self.ctx.h, self.h, tol, anorm), "hodlr_qr_graph")

    KINDS = ("gemm", "gemm_reduce", "cluster_qr", "cluster_jacobi", "select", "data_movement", "norm", "other")

    def qr_profile(self, tol: float, anorm: float = 0.0):
        ms, ln, fl = (C.c_double * 8)(), (C.c_int * 8)(), (C.c_double * 8)()
        check(lib().hodlr_qr_profile(self.ctx.h, self.h, tol, anorm, ms, ln, fl), "hodlr_qr_profile")
        return {k: {"ms": ms[i], "launches": ln[i], "flops": fl[i]} for i, k in enumerate(self.KINDS)}

    def status(self):
        st = C.c_int()
        an = C.c_double()
        check(lib().hodlr_status(self.ctx.h, self.h, C.byref(st), C.byref(an)), "hodlr_status")
        return st.value, an.value

    def ranks(self):
        nn = max(1, self.nleaf - 1)
        a, b, c = (C.c_int * nn)(), (C.c_int * nn)(), (C.c_int * nn)()
        check(lib().hodlr_ranks(self.ctx.h, self.h, a, b, c), "hodlr_ranks")
        k = self.nleaf - 1
        return np.array(a[:k]), np.array(b[:k]), np.array(c[:k])

    def flops(self):
        out = (C.c_double * 8)()
        check(lib().hodlr_flops(self.ctx.h, self.h, out), "hodlr_flops")
        keys = ["a2_norm", "a3_left_orth", "a4_leaf_qr", "a5_S", "a6_TS", "a7_update", "a8_T12", "total"]
        return dict(zip(keys, list(out)))

    def to_dense(self, which: int, out_ptr: int, ld: int):
        check(lib().hodlr_to_dense(self.ctx.h, self.h, which, _VP(out_ptr), ld), "hodlr_to_dense")

    def matvec(self, which, trans, nrhs, X_ptr, ldx, Y_ptr, ldy):
        check(lib().hodlr_matvec(self.ctx.h, self.h, which, int(trans), nrhs, _VP(X_ptr), ldx, _VP(Y_ptr), ldy),
              "hodlr_matvec")

    def apply_q(self, nrhs, B_ptr, ldb):
        check(lib().hodlr_apply_q(self.ctx.h, self.h, nrhs, _VP(B_ptr), ldb), "hodlr_apply_q")

    def apply_qt(self, nrhs, B_ptr, ldb):
        check(lib().hodlr_apply_qt(self.ctx.h, self.h, nrhs, _VP(B_ptr), ldb), "hodlr_apply_qt")

    def solve(self, nrhs, B_ptr, ldb):
        return lib().hodlr_solve(self.ctx.h, self.h, nrhs, _VP(B_ptr), ldb)

    def solve_async(self, nrhs, B_ptr, ldb, ctx=None):
        c = ctx or self.ctx
        check(lib().hodlr_solve_async(c.h, self.h, nrhs, _VP(B_ptr), ldb), "hodlr_solve_async")

    def norm2_estimate(self, iters=30):
        out = C.c_double()
        check(lib().hodlr_norm2_estimate(self.ctx.h, self.h, iters, C.byref(out)), "hodlr_norm2_estimate")
        return out.value

    def device_bytes(self) -> int:
        v = C.c_size_t()
        check(lib().hodlr_device_bytes(self.h, C.byref(v)), "hodlr_device_bytes")
        return int(v.value)

    def storage_bytes(self):
        return int(lib().hodlr_storage_bytes(self.h))

    def download(self, host: np.ndarray):
        check(lib().hodlr_download(self.ctx.h, self.h, _VP(host.ctypes.data), host.nbytes), "hodlr_download")

    def compact_bytes(self) -> int:
        v = C.c_size_t()
        check(lib().hodlr_compact_bytes(self.ctx.h, self.h, C.byref(v)), "hodlr_compact_bytes")
        return int(v.value)

    def download_compact(self, host: np.ndarray):
        check(lib().hodlr_download_compact(self.ctx.h, self.h, _VP(host.ctypes.data), host.nbytes),
              "hodlr_download_compact")

    def free(self):
        if self.h:
            lib().hodlr_free(self.h)
            self.h = _VP()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def qr_batched(ctx: Context, mats, tol: float, anorm: float = 0.0, graph: bool = False):
    arr = (_VP * len(mats))(*[m.h for m in mats])
    fn = lib().hodlr_qr_batched_graph if graph else lib().hodlr_qr_batched
    check(fn(ctx.h, len(mats), arr, tol, anorm), "hodlr_qr_batched")


def autotune_batched(ctx: Context, mats, tol: float, anorm: float = 0.0, reps: int = 2):
    """Pick the cluster size and batch group of the context by timing the batched graph."""
    arr = (_VP * len(mats))(*[m.h for m in mats])
    c, g, ms = C.c_int(), C.c_int(), C.c_double()
    check(lib().hodlr_autotune_batched(ctx.h, len(mats), arr, tol, anorm, reps, C.byref(c), C.byref(g), C.byref(ms)),
          "hodlr_autotune_batched")
    return {"cluster": c.value, "group": g.value, "ms": ms.value}


def dense_qr(ctx: Context, h, w, A_ptr, lda, T_ptr, ldt):
    check(lib().hodlr_dense_qr(ctx.h, h, w, _VP(A_ptr), lda, _VP(T_ptr), ldt), "hodlr_dense_qr")


def fp64_peak(device=0, iters=2000, reps=5):
    """Measured FP64 TFLOP/s of the device: {"dfma": .., "dmma": ..}."""
    a, b = C.c_double(), C.c_double()
    check(lib().hodlr_fp64_peak(device, iters, reps, C.byref(a), C.byref(b)), "hodlr_fp64_peak")
    return {"dfma": a.value, "dmma": b.value}


def unpack_compact(buf):
    """Parse a hodlr_download_compact buffer into (leaf_sizes, ranks (r12, r21, rT), leaves A,
    leaves T, per-node dict of factor arrays).  Marshalling only: no arithmetic."""
    ints = np.frombuffer(buf, dtype=np.int32)
    n, nleaf, nn = int(ints[0]), int(ints[1]), int(ints[2])
    ls = [int(x) for x in ints[4:4 + nleaf]]
    rk = ints[4 + nleaf:4 + nleaf + 3 * nn].reshape(3, nn) if nn else np.zeros((3, 0), dtype=np.int32)
    off = ((4 + nleaf + 3 * nn) * 4 + 7) // 8 * 8
    dbl = np.frombuffer(buf, dtype=np.float64, offset=off)
    pos = 0

    def take(rows, cols):
        nonlocal pos
        a = dbl[pos:pos + rows * cols].reshape(cols, rows).T
        pos += rows * cols
        return a
    leavesA = [take(w, w) for w in ls]
    leavesT = [take(w, w) for w in ls]
    lo = np.concatenate([[0], np.cumsum(ls)])
    rng = [None] * (2 * nleaf - 1)
    for j in range(nleaf):
        rng[nleaf - 1 + j] = (lo[j], lo[j + 1])
    for v in range(nleaf - 2, -1, -1):
        rng[v] = (rng[2 * v + 1][0], rng[2 * v + 2][1])
    nodes = []
    for v in range(nn):
        a = rng[2 * v + 1][1] - rng[2 * v + 1][0]
        b = rng[2 * v + 2][1] - rng[2 * v + 2][0]
        r12, r21, rT = int(rk[0, v]), int(rk[1, v]), int(rk[2, v])
        nodes.append({"U12": take(a, r12), "V12": take(b, r12), "U21": take(b, r21), "V21": take(a, r21),
                      "TU": take(a, rT), "TV": take(b, rT)})
    return ls, rk, leavesA, leavesT, nodes


def footprint(n, leaf_sizes, rank_cap, estimate_norm=True, with_snapshot=False, nrhs=0):
    """Device bytes of hodlr_build (+ snapshot) + hodlr_qr (+ hodlr_solve_async), from the host."""
    sizes = (C.c_int * len(leaf_sizes))(*[int(x) for x in leaf_sizes])
    out = C.c_size_t()
    check(lib().hodlr_footprint(int(n), len(leaf_sizes), sizes, int(rank_cap), int(bool(estimate_norm)),
                                int(bool(with_snapshot)), int(nrhs), C.byref(out)), "hodlr_footprint")
    return int(out.value)


def truncate(ctx: Context, nL, nR, K, L_ptr, Rt_ptr, thr, kmax, Lout_ptr, Rout_ptr):
    k = C.c_int()
    rc = lib().hodlr_truncate(ctx.h, nL, nR, K, _VP(L_ptr), _VP(Rt_ptr), thr, kmax, _VP(Lout_ptr),
                              _VP(Rout_ptr), C.byref(k))
    return rc, k.value


# ------------------------------------------------------------ rectangular HODLR (Sec. 6)
def _ints(xs):
    return (C.c_int * len(xs))(*[int(x) for x in xs])


def rect_permutation(m_sizes, n_sizes):
    """Row permutation of the permuted QR (hodlr_rect_permutation, host only): p[i] is the row
    of A that is row i of P A."""
    m = int(sum(m_sizes))
    p = (C.c_int * max(m, 1))()
    check(lib().hodlr_rect_permutation(len(m_sizes), _ints(m_sizes), _ints(n_sizes), p), "hodlr_rect_permutation")
    return np.array(p[:m])


def permuted_qr(ctx: Context, m_sizes, n_sizes, A_ptr, lda, T_ptr, ldt):
    """Dense permuted QR of Sec. 6 in place on the device (hodlr_permuted_qr)."""
    m, n = int(sum(m_sizes)), int(sum(n_sizes))
    check(lib().hodlr_permuted_qr(ctx.h, m, n, len(m_sizes), _ints(m_sizes), _ints(n_sizes), _VP(A_ptr), lda,
                                  _VP(T_ptr), ldt), "hodlr_permuted_qr")


class RectMatrix:
    """A device-resident rectangular HODLR matrix (hodlr_rect)."""

    def __init__(self, ctx: Context, h, m_sizes, n_sizes):
        self.ctx, self.h = ctx, h
        self.m_sizes, self.n_sizes = list(m_sizes), list(n_sizes)
        self.m, self.n = int(sum(m_sizes)), int(sum(n_sizes))

    @classmethod
    def compress(cls, ctx: Context, m_sizes, n_sizes, A_ptr, lda, thr, rank_cap=128, seed=0):
        h = _VP()
        rc = lib().hodlr_rect_compress(ctx.h, int(sum(m_sizes)), int(sum(n_sizes)), len(m_sizes), _ints(m_sizes),
                                       _ints(n_sizes), _VP(A_ptr), lda, thr, rank_cap, seed, C.byref(h))
        if rc not in (0, HODLR_ERANK):
            raise HodlrError(rc, "hodlr_rect_compress")
        return cls(ctx, h, m_sizes, n_sizes), rc

    def to_dense(self, out_ptr, ld):
        check(lib().hodlr_rect_to_dense(self.ctx.h, self.h, _VP(out_ptr), ld), "hodlr_rect_to_dense")

    def ranks(self):
        nn = max(1, len(self.m_sizes) - 1)
        a, b = (C.c_int * nn)(), (C.c_int * nn)()
        check(lib().hodlr_rect_ranks(self.ctx.h, self.h, a, b), "hodlr_rect_ranks")
        k = len(self.m_sizes) - 1
        return np.array(a[:k]), np.array(b[:k])

    def storage(self):
        """Doubles stored at the actual ranks: dense leaves plus the low-rank factors."""
        import math
        L = len(self.m_sizes)
        s = sum(a * b for a, b in zip(self.m_sizes, self.n_sizes))
        r12, r21 = self.ranks()
        ro = np.concatenate([[0], np.cumsum(self.m_sizes)])
        co = np.concatenate([[0], np.cumsum(self.n_sizes)])

        def span(off, v):                       # extent of heap node v in a partition
            d = int(math.floor(math.log2(v + 1)))
            width = L >> d
            first = (v - ((1 << d) - 1)) * width
            return int(off[first + width] - off[first])
        for v in range(L - 1):
            a, b = 2 * v + 1, 2 * v + 2
            s += r12[v] * (span(ro, a) + span(co, b)) + r21[v] * (span(ro, b) + span(co, a))
        return int(s)

    def free(self):
        if self.h:
            lib().hodlr_rect_free(self.h)
            self.h = _VP()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rect_qr(ctx: Context, m_sizes, n_sizes, A_ptr, lda, tol, anorm=0.0, rank_cap=128, seed=0):
    """Sec. 6 factorization (hodlr_rect_qr): returns (Y, T, R, anorm_used, rc) with rc 0 or
    HODLR_ERANK."""
    y, t, r = _VP(), _VP(), _VP()
    an = C.c_double()
    rc = lib().hodlr_rect_qr(ctx.h, int(sum(m_sizes)), int(sum(n_sizes)), len(m_sizes), _ints(m_sizes),
                             _ints(n_sizes), _VP(A_ptr), lda, tol, anorm, rank_cap, seed, C.byref(y), C.byref(t),
                             C.byref(r), C.byref(an))
    if rc not in (0, HODLR_ERANK):
        raise HodlrError(rc, "hodlr_rect_qr")
    return (RectMatrix(ctx, y, m_sizes, n_sizes), RectMatrix(ctx, t, n_sizes, n_sizes),
            RectMatrix(ctx, r, m_sizes, n_sizes), an.value, rc)
