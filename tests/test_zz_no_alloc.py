"""The allocation-free Heun entry point gives the same fields as the ordinary one and as the
FP64 oracle's Heun steps.

vpm_freefield_heun_noalloc exists for callers that cannot let the library allocate device
memory while they run (a control loop with memory fixed in advance, or a host whose device
memory belongs to another owner). It keeps its scratch in a fixed array inside the library.
This file is collected last so that a run stopping at its first failure has already run
every other test; it also passes on its own in a fresh process.

Tolerance: both entry points store positions in binary32 after each of the two Heun stages, so
they agree with each other and with the binary64 oracle to a few units in the last place of the
largest coordinate per step: tol = 4 x steps x ulp(max |x|). The test checks that the gap
between the oracle's Heun and forward-Euler results on the same input exceeds 2 tol, so an
entry point that skipped or miswired the second stage (an error of about that gap) would fail.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import cuda

pytestmark = pytest.mark.gpu

MAX_N = 262144
R_CORE, DT = 0.05, 0.01


def _field(torch, seed, n):
    a = np.zeros((n, 4), np.float32)
    a[:, :3] = W.background_field(seed, n)
    return a, torch.tensor(a, device="cuda")


def test_noalloc_matches_allocating_heun_and_oracle():
    import oracle
    oracle.build()
    torch, V = cuda()
    L = V.lib()
    sh = V.stream_handle()
    # three calls in a row with different sizes and data (a smaller field after a larger one):
    # no call may see an earlier call's leftovers in the shared scratch array
    for seed, n, steps in ((11, 1500, 5), (12, 4097, 3), (13, 700, 4)):
        host, ref = _field(torch, seed, n)
        got = ref.clone()
        V.check(L.vpm_freefield_heun(V.ptr(ref), n, V.KERNEL_VATISTAS, R_CORE, DT, steps, sh))
        V.check(L.vpm_freefield_heun_noalloc(V.ptr(got), n, V.KERNEL_VATISTAS, R_CORE, DT, steps, sh))
        torch.cuda.synchronize()
        start = host[:, :3].astype(np.float64)
        heun = oracle.free_heun(start, oracle.VATISTAS, R_CORE, DT, steps)
        euler = oracle.free_euler(start, oracle.VATISTAS, R_CORE, DT, steps)
        tol = 4 * steps * float(np.spacing(np.float32(np.abs(heun[:, :2]).max())))
        gap = np.abs(heun[:, :2] - euler[:, :2]).max()
        assert gap > 2 * tol, (n, gap, tol)
        g = got.cpu().numpy().astype(np.float64)
        r = ref.cpu().numpy().astype(np.float64)
        assert np.abs(g[:, :2] - r[:, :2]).max() <= tol, (n, "noalloc vs allocating")
        assert np.abs(g[:, :2] - heun[:, :2]).max() <= tol, (n, "noalloc vs oracle")
        assert np.abs(r[:, :2] - heun[:, :2]).max() <= tol, (n, "allocating vs oracle")
        assert np.array_equal(g[:, 2], r[:, 2])


def test_noalloc_rejects_fields_beyond_its_scratch():
    torch, V = cuda()
    L = V.lib()
    _, small = _field(torch, 1, 8)
    st = L.vpm_freefield_heun_noalloc(V.ptr(small), MAX_N + 1, V.KERNEL_VATISTAS, R_CORE, DT, 1,
                                      V.stream_handle())
    assert st == V.VPM_ERR_CAPACITY
    assert b"262144" in L.vpm_last_error()
