"""The C-ABI library builds, loads without a GPU and exports every function include/vpm.h
declares; host-side argument checks run before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def vlib():
    from paper_2509_16079_b300 import build
    build.build()
    import paper_2509_16079_b300 as V
    return V.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("vpm_state_create", "vpm_step", "vpm_rollout_batch", "mppi_weights",
                 "mppi_update", "vpm_freefield_velocity", "vpm_state_save", "vpm_state_load"):
        assert must in names


def test_every_declared_symbol_is_exported(vlib):
    missing = [n for n in sorted(_declared()) if not hasattr(vlib, n)]
    assert not missing, missing


def test_version(vlib):
    assert b"sm_103a" in vlib.vpm_version()


def test_host_side_rejections(vlib):
    import paper_2509_16079_b300 as V
    import workloads as W
    h = C.c_void_p()
    xg = np.zeros(7)
    xp = xg.ctypes.data_as(C.c_void_p)
    assert vlib.vpm_state_create(None, None, 0, 4, xp, C.byref(h), None) == V.VPM_ERR_INVALID
    bad = V.make_params(dict(W.glider_params(), n_b=1))
    assert vlib.vpm_state_create(C.byref(bad), None, 0, 4, xp, C.byref(h), None) == V.VPM_ERR_INVALID
    bad = V.make_params(dict(W.glider_params(), dt=float("nan")))
    assert vlib.vpm_state_create(C.byref(bad), None, 0, 4, xp, C.byref(h), None) == V.VPM_ERR_INVALID
    ok = V.make_params(W.glider_params())
    assert vlib.vpm_state_create(C.byref(ok), None, 5, 4, xp, C.byref(h), None) == V.VPM_ERR_INVALID
    assert vlib.mppi_weights(None, 4, 1.0, None, None) == V.VPM_ERR_INVALID
    assert vlib.vpm_rollout_batch(None, 1, 1, None, None, None, None, None, None, None) == V.VPM_ERR_INVALID
    assert b"null" in vlib.vpm_last_error()
    assert vlib.vpm_batch_set_ctas(None, 0, 0, 2) == V.VPM_ERR_INVALID
    assert vlib.vpm_batch_set_schedule(None, 0, 0, 128, 2) == V.VPM_ERR_INVALID
    r = C.c_double(0.0)
    assert vlib.vpm_probe_rate(99, 1, C.byref(r)) == V.VPM_ERR_INVALID
    assert vlib.vpm_probe_rate(V.PROBE_PAIRS_SYM + 1, 1, C.byref(r)) == V.VPM_ERR_INVALID
    assert vlib.vpm_probe_rate(V.PROBE_FFMA, 0, C.byref(r)) == V.VPM_ERR_INVALID
    assert vlib.vpm_probe_rate(V.PROBE_FFMA, 8, C.byref(r)) == V.VPM_ERR_INVALID
    # NMPC: a latency longer than the replanning period would replace plans before they act
    N, K = 20, 8
    noise = W.nmpc_noise(1, 2, 1, K, N)
    for latency, want in ((6, V.VPM_ERR_INVALID), (-1, V.VPM_ERR_INVALID)):
        with pytest.raises(V.VpmError) as e:
            V.NMPC(W.glider_params(), np.zeros((0, 3)), 40, W.GLIDER_X0, np.zeros(N, np.float32),
                   noise, horizon=N, replan_every=5, latency=latency, rollouts=K, iterations=1,
                   lam=10.0, qc=W.TVLQR_QC, qf=W.TVLQR_QF, rc=W.TVLQR_RC)
        assert e.value.status == want and "configuration" in str(e.value)


def test_no_silent_cpu_fallback(vlib):
    """Without a usable CUDA device a well-formed call reports VPM_ERR_CUDA."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import paper_2509_16079_b300 as V
    import workloads as W
    h = C.c_void_p()
    ok = V.make_params(W.glider_params())
    xg = np.zeros(7)
    st = vlib.vpm_state_create(C.byref(ok), None, 0, 4, xg.ctypes.data_as(C.c_void_p), C.byref(h), None)
    assert st == V.VPM_ERR_CUDA
