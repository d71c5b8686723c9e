"""The allocation-free Heun entry point gives the same fields as the ordinary one.

vpm_freefield_heun_noalloc exists for callers that cannot let the library allocate device
memory while they run (a control loop with memory fixed in advance, or a host whose device
memory belongs to another owner). It keeps its scratch in a fixed array inside the library.
This file is collected last so that a run stopping at its first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from tests.gpu_common import POS_TOL, cuda

pytestmark = pytest.mark.gpu

MAX_N = 262144


def _field(torch, seed, n):
    a = np.zeros((n, 4), np.float32)
    a[:, :3] = W.background_field(seed, n)
    return torch.tensor(a, device="cuda")


def test_noalloc_matches_allocating_heun_twice():
    torch, V = cuda()
    L = V.lib()
    sh = V.stream_handle()
    # two calls in a row with different sizes and data: the second must not see the first's
    # leftovers in the shared scratch array
    for seed, n, steps in ((11, 1500, 5), (12, 4097, 3)):
        ref = _field(torch, seed, n)
        got = ref.clone()
        V.check(L.vpm_freefield_heun(V.ptr(ref), n, V.KERNEL_VATISTAS, 0.05, 0.01, steps, sh))
        V.check(L.vpm_freefield_heun_noalloc(V.ptr(got), n, V.KERNEL_VATISTAS, 0.05, 0.01, steps, sh))
        torch.cuda.synchronize()
        diff = (got[:, :2] - ref[:, :2]).abs().max().item()
        assert diff <= POS_TOL, (n, diff)
        assert torch.equal(got[:, 2], ref[:, 2])


def test_noalloc_rejects_fields_beyond_its_scratch():
    torch, V = cuda()
    L = V.lib()
    small = _field(torch, 1, 8)
    st = L.vpm_freefield_heun_noalloc(V.ptr(small), MAX_N + 1, V.KERNEL_VATISTAS, 0.05, 0.01, 1,
                                      V.stream_handle())
    assert st == V.VPM_ERR_CAPACITY
    assert b"262144" in L.vpm_last_error()
