"""CPU checks of the index arithmetic and warp-exchange patterns of the CUDA kernels.

Each check restates, in plain Python over a 32-lane warp, one mapping the kernels rely on and
verifies its invariant on every size the kernels meet: that each output, operand element,
column pair or partial sum is produced exactly once and lands where the kernel reads it.  These
are the properties that make the kernels' accesses stay in bounds; the parity tests then check
the numbers on the GPU."""
import bisect
import itertools

import numpy as np

GT, BM, BN, BK, MR, NR = 256, 64, 32, 16, 4, 2   # gemm_kernel: threads, tile, k chunk, micro-tile
LDA_S, LDB_S = BM + 2, BN + 2                      # shared-memory row strides of the operand tiles


def shfl_xor(vals, o):
    return [vals[l ^ o] for l in range(32)]


def test_gemm_micro_tiles_cover_outputs_once():
    """gemm_kernel: the ma x na outputs of a tile are covered by MR x NR micro-tiles dealt to
    threads in column-major order; every existing output is stored by exactly one thread, every
    micro-tile lies inside the BM x BN tile (shared reads stay in bounds), only warps holding a
    micro-tile issue FMAs, and the FMAs spent beyond ma x na are those of the edge micro-tiles."""
    for ma in range(1, BM + 1):
        for na in range(1, BN + 1):
            mrow, mcol = -(-ma // MR), -(-na // NR)
            nmic = mrow * mcol
            assert nmic <= GT
            stored = []
            computing_warps = set()
            for t in range(GT):
                active = t < nmic
                if (t & ~31) < nmic:
                    computing_warps.add(t // 32)
                if not active:
                    continue
                mi, nj = t % mrow, t // mrow
                r0, c0 = mi * MR, nj * NR
                assert r0 + MR <= BM and c0 + NR <= BN
                assert (r0 * 8) % 16 == 0 and (c0 * 8) % 16 == 0          # double2 reads aligned
                for v in range(NR):
                    for u in range(MR):
                        if r0 + u < ma and c0 + v < na:
                            stored.append((r0 + u, c0 + v))
            assert sorted(stored) == [(i, j) for i in range(ma) for j in range(na)]
            assert computing_warps == set(range(-(-nmic // 32)))
            waste = nmic * MR * NR - ma * na
            assert waste <= (MR - 1) * mcol * NR + (NR - 1) * mrow * MR


def test_gemm_dense_form_deals_outputs_once():
    """gemm_kernel dense form (ma x na <= 4 GT): output o = t + GT u goes to thread t in pass u,
    column-major; the packed (row << 8 | column) code round-trips; every output is stored once;
    only warps holding an output issue FMAs, and only the last warp of a pass has idle lanes."""
    for ma in range(1, BM + 1):
        for na in range(1, BN + 1):
            nout = ma * na
            if nout > 4 * GT:
                continue
            stored = []
            for u in range(4):
                busy = 0
                for t in range(GT):
                    o = min(t + GT * u, nout - 1)
                    oj = o // ma
                    code = ((o - oj * ma) << 8) | oj
                    i, j = code >> 8, code & 255
                    assert 0 <= i < ma and 0 <= j < na and (i, j) == (o % ma, o // ma)
                    computes = (t & ~31) + GT * u < nout
                    busy += computes
                    if t + GT * u < nout:
                        assert computes
                        stored.append((i, j))
                assert busy - max(0, min(GT, nout - GT * u)) < 32
            assert sorted(stored) == [(i, j) for i in range(ma) for j in range(na)]


def test_gemm_form_choice_covers_every_tile():
    """A tile takes the dense form up to 4 GT outputs and the micro-tile form beyond; the micro
    form then keeps every thread of at least 4 warps busy (all four sub-partitions)."""
    for ma in range(1, BM + 1):
        for na in range(1, BN + 1):
            if ma * na > 4 * GT:
                nmic = -(-ma // MR) * -(-na // NR)
                assert nmic >= 4 * 32


def test_gemm_persistent_loop_visits_every_item_once():
    """gemm_kernel: CTA b takes items b, b + grid, ...; every item is taken exactly once."""
    for total in (1, 7, 911, 5000):
        for grid in (min(total, 6 * 152), 1, 3):
            seen = [i for b in range(grid) for i in range(b, total, grid)]
            assert sorted(seen) == list(range(total))


def test_gemm_shared_strides_keep_vector_reads_aligned():
    """Rows of As / Bs start on 16-byte boundaries, so the double2 reads of a micro-tile's rows
    and columns are aligned for every k in the chunk."""
    for l in range(BK):
        assert (l * LDA_S * 8) % 16 == 0 and (l * LDB_S * 8) % 16 == 0


def test_gemm_operand_tiles_covered_once_and_coalesced():
    """gemm_kernel prefetch: element e = t + 256 p of the 64 x 16 A tile (p < 4) and of the
    16 x 32 B tile (p < 2); consecutive threads read consecutive addresses of the stored operand."""
    PA, PB = BM * BK // GT, BN * BK // GT
    for ta in (0, 1):
        cells = []
        for e in range(PA * GT):
            i, l = (e // BK, e % BK) if ta else (e % BM, e // BM)
            cells.append((i, l))
        assert sorted(cells) == [(i, l) for i in range(BM) for l in range(BK)]
        lda = 1000
        for w in range(0, PA * GT, 32):          # a warp's 32 consecutive elements
            addr = [(l + i * lda) if ta else (i + l * lda) for i, l in cells[w:w + 32]]
            runs = sum(1 for a, b in zip(addr, addr[1:]) if b != a + 1)
            assert runs <= 1                     # at most two contiguous runs per warp
    for tb in (0, 1):
        cells = []
        for e in range(PB * GT):
            j, lb = (e % BN, e // BN) if tb else (e // BK, e % BK)
            cells.append((j, lb))
        assert sorted(cells) == [(j, l) for j in range(BN) for l in range(BK)]
        ldb = 1000
        for w in range(0, PB * GT, 32):
            addr = [(j + lb * ldb) if tb else (lb + j * ldb) for j, lb in cells[w:w + 32]]
            runs = sum(1 for a, b in zip(addr, addr[1:]) if b != a + 1)
            assert runs <= 1


def _vote_search(work0, item):
    """gemm_kernel descriptor lookup: a 32-lane vote at stride s, then a scan of s entries."""
    nd = len(work0)
    stride = (nd + 31) >> 5
    m = 0
    for lane in range(32):
        idx = lane * stride
        if idx < nd and work0[idx] <= item:
            m |= 1 << lane
    lo = (m.bit_length() - 1) * stride            # lane 0 always votes yes
    if stride > 1:
        end = min(lo + stride, nd)
        b = lo
        while b < end:
            m = 0
            for lane in range(32):
                idx = b + lane
                if idx < end and work0[idx] <= item:
                    m |= 1 << lane
            lo = b + m.bit_length() - 1           # m == 0 gives b - 1: the previous chunk's last
            if m != 0xFFFFFFFF:
                break
            b += 32
    return lo


def test_gemm_descriptor_vote_equals_bisection():
    rng = np.random.default_rng(3)
    for nd in list(range(1, 70)) + [1023, 1024, 1025, 2000]:
        work = rng.integers(1, 9, size=nd)
        work0 = [0] + list(np.cumsum(work)[:-1])
        total = int(np.sum(work))
        items = range(total) if total < 600 else rng.integers(0, total, size=600)
        for item in items:
            assert _vote_search(work0, int(item)) == bisect.bisect_right(work0, int(item)) - 1


def test_qr_two_column_reduction():
    """qr_dsmem_kernel pair update: one exchange at offset 16 moves column A's partial sums to
    lanes 0-15 and column B's to lanes 16-31, then four levels finish both sums at once."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        tA, tB = rng.standard_normal(32), rng.standard_normal(32)
        lo = [l < 16 for l in range(32)]
        send = [tB[l] if lo[l] else tA[l] for l in range(32)]
        recv = shfl_xor(send, 16)
        tm = [(tA[l] if lo[l] else tB[l]) + recv[l] for l in range(32)]
        for o in (8, 4, 2, 1):
            other = shfl_xor(tm, o)
            tm = [tm[l] + other[l] for l in range(32)]
        assert np.allclose(tm[:16], tA.sum(), rtol=1e-13) and np.allclose(tm[16:], tB.sum(), rtol=1e-13)


def test_T_build_halving_exchange():
    """qr_build_T: each lane holds 16 partial sums of a 4 x 4 block of G; after halving
    exchanges at offsets 16, 8, 4, 2 and a final add at offset 1, lane l holds entry q(l)
    summed over all lanes, q(l) = 8 b4 + 4 b3 + 2 b2 + b1 of l's bits."""
    rng = np.random.default_rng(7)
    acc = [list(rng.standard_normal(16)) for _ in range(32)]
    total = np.sum(np.array(acc), axis=0)
    for o, half in ((16, 8), (8, 4), (4, 2), (2, 1)):
        new = []
        for l in range(32):
            hi = bool(l & o)
            row = acc[l][:]
            partner = acc[l ^ o]
            for q in range(half):
                send_p = partner[q] if (l ^ o) & o else partner[q + half]   # what the partner sends
                keep = row[q + half] if hi else row[q]
                row[q] = keep + send_p
            new.append(row)
        acc = new
    final = [acc[l][0] + acc[l ^ 1][0] for l in range(32)]
    for l in range(32):
        q = ((l >> 4) & 1) * 8 + ((l >> 3) & 1) * 4 + ((l >> 2) & 1) * 2 + ((l >> 1) & 1)
        assert np.isclose(final[l], total[q], rtol=1e-12)


def _rr_pair(r, i, P):
    if i == 0:
        return P - 1, r
    m = P - 1
    a = r + i
    a -= m if a >= m else 0
    b = r - i
    b += m if b < 0 else 0
    return a, b


def test_jacobi_round_robin_schedules():
    """rr_pair (remote-store and global forms) and the owner form's partner y = 2r - x mod m:
    every round pairs all P players, and the P - 1 rounds meet every pair exactly once."""
    for P in range(2, 42, 2):
        m = P - 1
        seen = set()
        for r in range(P - 1):
            players = []
            for i in range(P // 2):
                a, b = _rr_pair(r, i, P)
                assert 0 <= a < P and 0 <= b < P and a != b
                players += [a, b]
                seen.add((min(a, b), max(a, b)))
            assert sorted(players) == list(range(P))
            # owner form: each player finds its partner alone, consistently with rr_pair
            partner = {}
            for x in range(P):
                y = 2 * r - x
                y += m if y < 0 else 0
                y -= m if y >= m else 0
                y = r if x == m else (m if x == r else y)
                partner[x] = y
            for x in range(P):
                assert partner[partner[x]] == x and partner[x] != x
            pairs_owner = {(min(x, y), max(x, y)) for x, y in partner.items()}
            pairs_rr = {(min(*_rr_pair(r, i, P)), max(*_rr_pair(r, i, P))) for i in range(P // 2)}
            assert pairs_owner == pairs_rr
        assert seen == set(itertools.combinations(range(P), 2))


def test_jacobi_packed_active_columns():
    """jacobi owner form: act[x] = (slot << 5) | owner CTA, with owner = j % C < 32."""
    for C in (1, 2, 4, 8, 16):
        for j in range(4096):
            p = ((j // C) << 5) | (j % C)
            assert (p & 31) == j % C and (p >> 5) == j // C and (p >> 5) * C + (p & 31) == j
