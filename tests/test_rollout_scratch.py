"""The binary32 rollout kernel's pair-sum scratch is large enough for every slot it touches.

rollout blocks size their scratch by a closed formula (vpm_rollout_scratch_bytes_cap). This test
walks the slots the pair phase writes and the finalize phase reads, following the kernel's loops
(rows of 128 particles with the compensated forward sums of their targets as float4 = two float2
slots each, reverse sums per row and later source, the per-particle combination). The slot of
each (row, particle) comes from the kernel's own index functions through
vpm_rollout_scratch_slot, so a change of the kernel's layout is walked as it is. For field sizes
up to the capacity it checks that each slot lies inside the scratch, that no two writers share a
slot and that nothing is read that was not written. Host only."""
import ctypes as C

import pytest

ROW = 128


def _slot(V, cap, kind, row, particle):
    s = C.c_longlong()
    V.check(V.lib().vpm_rollout_scratch_slot(cap, kind, row, particle, C.byref(s)))
    return s.value


def _walk(V, n, cap):
    rows = -(-n // ROW)
    rows_off = max(0, rows - 1)
    fwd = lambda i: _slot(V, cap, 0, 0, i)
    rev = lambda a, j: _slot(V, cap, 1, a, j)
    writes, reads = {}, set()
    for a in range(rows_off):                                # off-diagonal row units
        for t in range(ROW):                                 # the targets' float4 sums
            i = ROW * a + t
            assert i < n
            q0 = fwd(i)
            assert q0 % 2 == 0                               # float4-aligned
            for q in (q0, q0 + 1):
                assert q not in writes, (n, cap, a, i)
                writes[q] = ("fwd", a, i)
        for j in range(ROW * (a + 1), n):                    # reverse sums of later sources
            q = rev(a, j)
            assert q not in writes, (n, cap, a, j)
            writes[q] = ("rev", a, j)
    for i in range(n):                                       # finalize: old_sum
        row = i // ROW
        if row < rows_off:
            q0 = fwd(i)
            reads.update((q0, q0 + 1))
        for a in range(row):
            reads.add(rev(a, i))
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
        writes, reads = _walk(V, n, cap)
        if writes:
            assert min(writes) >= 0 and max(writes) < slots, (cap, n)
        assert reads <= set(writes), (cap, n)


def test_scratch_slot_rejects_slots_that_do_not_exist():
    import paper_2509_16079_b300 as V
    s = C.c_longlong()
    L = V.lib()
    assert L.vpm_rollout_scratch_slot(1200, 1, 0, 100, C.byref(s)) == V.VPM_ERR_INVALID  # inside row 0
    assert L.vpm_rollout_scratch_slot(1200, 0, 0, 1199, C.byref(s)) == V.VPM_ERR_INVALID  # last row
    assert L.vpm_rollout_scratch_slot(1200, 1, 9, 1199, C.byref(s)) == V.VPM_ERR_INVALID  # no row 9
    assert L.vpm_rollout_scratch_slot(1200, 2, 0, 500, C.byref(s)) == V.VPM_ERR_INVALID
    assert L.vpm_rollout_scratch_slot(1200, 1, 0, 500, None) == V.VPM_ERR_INVALID


def test_small_fields_and_binary64_need_no_scratch():
    import paper_2509_16079_b300 as V
    b = C.c_size_t()
    V.check(V.lib().vpm_rollout_scratch_bytes_cap(V.FP32, 128, 4, C.byref(b)))
    assert b.value == 0
    V.check(V.lib().vpm_rollout_scratch_bytes_cap(V.FP64, 5000, 4, C.byref(b)))
    assert b.value == 0
