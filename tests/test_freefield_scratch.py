"""The free-field pair-sum scratch is large enough for every slot the kernels touch.

vpm_freefield_scratch_bytes(n) sizes the scratch by a closed formula. This test walks the
indices the one-evaluation-per-pair kernels write and read, following their loops (rows of
1024 particles, 512-source tiles, off-diagonal segments of 32 tiles, the combine's reads), for
many field sizes, and checks that each lies inside the scratch and that no two writers share a
slot. It runs on the host only (the size query needs no device)."""
import ctypes as C

import pytest

ROW, TILE, SEG = 1024, 512, 32


def _slots_used(n):
    """Every float2 slot index written (with its writer) and read, following the kernels."""
    rows = -(-n // ROW)
    ntiles = -(-n // TILE)
    max_seg = max(0, -(-(ntiles - ROW // TILE) // SEG))
    f_seg = 2 * n
    r_slot = f_seg + rows * max_seg * ROW
    span = ntiles * TILE

    def rev_base(I):
        return r_slot + I * span - ROW * I * (I + 1) // 2 - ROW * (I + 1)

    writes, reads = {}, set()
    for I in range(rows):
        tr0 = I * (ROW // TILE)
        units = [(0, tr0, min(tr0 + ROW // TILE, ntiles))]
        for u in range(1, 1 + max_seg):
            t0 = tr0 + ROW // TILE + (u - 1) * SEG
            t1 = min(t0 + SEG, ntiles)
            if t0 < t1:
                units.append((u, t0, t1))
        for unit, t0, t1 in units:
            for t in range(t0, t1):
                for q in range(TILE):
                    j = t * TILE + q
                    if j >= n:
                        continue
                    idx = n + j if unit == 0 else rev_base(I) + j
                    assert idx not in writes, (n, I, unit, j)
                    writes[idx] = (I, unit, j)
            for li in range(ROW):
                i = I * ROW + li
                if i >= n:
                    continue
                idx = i if unit == 0 else f_seg + (I * max_seg + unit - 1) * ROW + li
                assert idx not in writes, (n, I, unit, i)
                writes[idx] = (I, unit, i)
    for j in range(n):                                       # the combine kernel's reads
        T, li = j // ROW, j % ROW
        reads.add(j)
        reads.add(n + j)
        t_after = ntiles - (T + 1) * (ROW // TILE)
        segs = max(0, -(-t_after // SEG))
        for s in range(segs):
            reads.add(f_seg + (T * max_seg + s) * ROW + li)
        for I in range(T):
            reads.add(rev_base(I) + j)
    return writes, reads


@pytest.mark.parametrize("n", [1, 2, 31, 511, 512, 513, 1023, 1024, 1025, 1536, 2047, 2048, 2049,
                               3000, 17 * 1024 + 5, 34 * 512 + 100])
def test_scratch_covers_every_slot(n):
    import paper_2509_16079_b300 as V
    b = C.c_size_t()
    V.check(V.lib().vpm_freefield_scratch_bytes(n, C.byref(b)))
    total = b.value // 8                                     # float2 slots
    writes, reads = _slots_used(n)
    assert max(writes) < total and max(reads) < total
    assert reads <= set(writes)                              # nothing is read that no one wrote
