"""CPU checks of the CUDA library: it builds for sm_103a, loads, and exports every entry point
that include/hodlr_qr.h declares; the binding covers them; the product package never reaches
the oracle.  No GPU calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hodlr_qr.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hodlr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1809_10585_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hodlr_build", "hodlr_qr", "hodlr_apply_q", "hodlr_apply_qt", "hodlr_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1809_10585_gb300 import binding
    assert set(declared_functions()) == set(binding.SYMBOLS)


def test_strerror_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.hodlr_strerror.restype = ctypes.c_char_p
    assert lib.hodlr_strerror(0) == b"ok"
    assert b"rank" in lib.hodlr_strerror(3)


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1809_10585_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, re.M), f


# --------------------------------------------------------------- memory footprint (host only)
def _children(leaf_sizes):
    """(range of child 1, range of child 2) of every internal node of the cluster tree."""
    import workloads as W
    rng = W.node_ranges(leaf_sizes)
    return [(rng[2 * v + 1], rng[2 * v + 2]) for v in range(len(leaf_sizes) - 1)]


def _storage_doubles(n, leaf_sizes, kc):
    """Storage of the flattened HODLR container (Sec. 2.1, O(k n log n)): dense leaves of A and
    T padded to the largest leaf, plus four factor blocks of A and two of T per internal node at
    rank capacity kc."""
    import workloads as W
    nleaf = len(leaf_sizes)
    maxw = max(leaf_sizes)
    leafd = nleaf * maxw * maxw
    fac = 0
    for (lo1, hi1), (lo2, hi2) in _children(leaf_sizes):
        fac += 3 * ((hi1 - lo1) + (hi2 - lo2)) * kc
    return 2 * leafd + fac


@pytest.mark.parametrize("n,nmin,kc", [(1024, 128, 64), (8192, 256, 128), (1000, 100, 32), (96, 128, 16)])
def test_footprint_counts_storage_and_grows_with_rank_capacity(libpath, n, nmin, kc):
    import workloads as W
    from paper_1809_10585_gb300 import binding as B
    ls = W.balanced_leaf_sizes(n, nmin)
    base = B.footprint(n, ls, kc, estimate_norm=True)
    store = 8 * _storage_doubles(n, ls, kc)
    assert base > store                               # storage plus tables, plans and scratch
    # a snapshot adds exactly the A part of the storage and the rank table
    snap = B.footprint(n, ls, kc, estimate_norm=True, with_snapshot=True) - base
    leafd = len(ls) * max(ls) ** 2
    afac = sum(2 * ((h1 - l1) + (h2 - l2)) * kc for (l1, h1), (l2, h2) in _children(ls))
    assert snap == 8 * (leafd + afac) + 4 * max(1, 3 * (len(ls) - 1))
    # more rank capacity, more bytes; a solve plan adds at least its staging buffer
    if len(ls) > 1:
        assert B.footprint(n, ls, 2 * kc) > base
    else:                                             # one dense leaf: no factors, no ranks
        assert B.footprint(n, ls, 2 * kc) == base
    assert B.footprint(n, ls, kc, nrhs=8) - base >= 8 * n * 8
    # the norm estimate's plan is extra work, never less memory
    assert B.footprint(n, ls, kc, estimate_norm=False) <= base


def test_footprint_rejects_bad_partitions(libpath):
    import ctypes as C
    from paper_1809_10585_gb300 import binding as B
    out = C.c_size_t()
    sizes = (C.c_int * 3)(100, 100, 100)                       # not a power of two of leaves
    assert B.lib().hodlr_footprint(300, 3, sizes, 32, 1, 0, 0, C.byref(out)) == B.HODLR_EINVAL
    sizes = (C.c_int * 2)(100, 100)
    assert B.lib().hodlr_footprint(201, 2, sizes, 32, 1, 0, 0, C.byref(out)) == B.HODLR_EINVAL   # sum != n
    assert B.lib().hodlr_footprint(200, 2, sizes, 0, 1, 0, 0, C.byref(out)) == B.HODLR_EINVAL    # rank_cap
    assert B.lib().hodlr_footprint(200, 2, sizes, 32, 1, 0, 2000, C.byref(out)) == B.HODLR_EINVAL


@pytest.mark.parametrize("m_sizes,n_sizes", [([5, 4, 6, 3], [2, 4, 1, 3]), ([500] * 16, [250] * 16),
                                             ([7], [7]), ([9, 12], [9, 3]), ([31, 40, 22, 50], [30, 1, 22, 17])])
def test_rect_permutation_matches_oracle(libpath, m_sizes, n_sizes):
    """The host-side row permutation of the permuted QR (Sec. 6) equals the oracle's."""
    import oracle.rect as OR
    from paper_1809_10585_gb300 import binding as B
    assert B.rect_permutation(m_sizes, n_sizes).tolist() == OR.row_permutation(m_sizes, n_sizes).tolist()


def test_rect_permutation_rejects_bad_partitions(libpath):
    import ctypes as C
    from paper_1809_10585_gb300 import binding as B
    p = (C.c_int * 64)()
    bad = [([4, 6], [5, 5]),            # m_1 < n_1
           ([4, 4, 4], [2, 2, 2]),      # not a power of two of leaves
           ([4, 4], [0, 2])]            # empty column block
    for ms, ns in bad:
        rc = B.lib().hodlr_rect_permutation(len(ms), (C.c_int * len(ms))(*ms), (C.c_int * len(ns))(*ns), p)
        assert rc == B.HODLR_EINVAL
