"""The binary32 rollout kernel's pair-sum scratch is large enough for every slot it touches.

rollout blocks size their scratch by a closed formula (vpm_rollout_scratch_bytes_cap). This test
walks the float2 slot indices the pair phase writes and the finalize phase reads, following the
kernel's loops (rows of 128 particles with the compensated forward sums of their targets as
float4 = two slots each, reverse sums per row and later source, the per-particle combination),
for field sizes up to the capacity, and checks that each lies inside the scratch, that no two
writers share a slot and that nothing is read that was not written. Host only."""
import ctypes as C

import pytest

ROW = 128


def _walk(n, cap):
    cap32 = (cap + 31) & ~31
    rows = -(-n // ROW)
    rows_off = max(0, rows - 1)

    def row_base(a):
        return cap32 * (a + 2) - (ROW // 2) * a * (a + 1)

    writes, reads = {}, set()
    for a in range(rows_off):                                # off-diagonal row units
        for t in range(ROW):                                 # the targets' float4 sums
            i = ROW * a + t
            assert i < n
            for q in (2 * i, 2 * i + 1):
                assert q not in writes, (n, cap, a, i)
                writes[q] = ("fwd", a, i)
        for j in range(ROW * (a + 1), n):                    # reverse sums of later sources
            q = row_base(a) - ROW * (a + 1) + j
            assert q not in writes, (n, cap, a, j)
            writes[q] = ("rev", a, j)
    for i in range(n):                                       # finalize: old_sum
        row = i // ROW
        if row < rows_off:
            reads.update((2 * i, 2 * i + 1))
        for a in range(row):
            reads.add(row_base(a) - ROW * (a + 1) + i)
    return writes, reads


@pytest.mark.parametrize("cap", [129, 160, 255, 256, 257, 1040, 1200, 2100, 3000, 5400])
def test_rollout_scratch_covers_every_slot(cap):
    import paper_2509_16079_b300 as V
    b = C.c_size_t()
    V.check(V.lib().vpm_rollout_scratch_bytes_cap(V.FP32, cap, 1, C.byref(b)))
    slots = b.value // 8
    assert slots % 2 == 0                                    # 16-byte aligned blocks
    for n in sorted({1, 128, 129, cap // 2, cap - 33, cap - 1, cap} - {0}):
        if n < 1 or n > cap:
            continue
        writes, reads = _walk(n, cap)
        if writes:
            assert max(writes) < slots, (cap, n)
        assert reads <= set(writes), (cap, n)


def test_small_fields_and_binary64_need_no_scratch():
    import paper_2509_16079_b300 as V
    b = C.c_size_t()
    V.check(V.lib().vpm_rollout_scratch_bytes_cap(V.FP32, 128, 4, C.byref(b)))
    assert b.value == 0
    V.check(V.lib().vpm_rollout_scratch_bytes_cap(V.FP64, 5000, 4, C.byref(b)))
    assert b.value == 0
