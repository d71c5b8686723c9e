"""Replanning server: results alone and in a mix, the plain per-request form, supersession of
queued requests, admission by the memory budget and by the device memory free at admission,
resident fields advanced between replans."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import cuda

pytestmark = pytest.mark.gpu

SIZES = [300, 500, 800, 400, 1000, 600]


def _server(V, max_inflight, budget=0, H=20, max_rollouts_inflight=0, **admission):
    srv = V.Server(max_inflight=max_inflight, max_rollouts=2048, max_horizon=100, hbm_budget=budget,
                   max_inflight_rollouts=max_rollouts_inflight, **admission)
    p = W.glider_params()
    fields = [W.background_field(50 + i, n) for i, n in enumerate(SIZES)]
    for f in fields:
        srv.add_scenario(p, f, W.GLIDER_X0, len(f) + 2 * 100 + 10)
    return srv, p, fields


def _direct_mu(V, torch, p, field, eps, lam):
    st = V.State(p, field, W.GLIDER_X0, len(field) + 2 * eps.shape[1])
    c = V.mppi_perturb(torch.zeros(eps.shape[1], device="cuda"), torch.tensor(eps, device="cuda"))
    out = st.rollout_batch(c, want_final=False)
    mu = V.mppi_update(V.mppi_weights(out["costs"], lam), c)
    return mu.cpu().numpy(), out["costs"].min().item()


@pytest.mark.parametrize("admission", ["arrival", "least_work", "least_work_lane"])
def test_same_result_alone_in_mix_and_per_request(admission):
    """Under every admission policy (least work first with the small-request lane runs the
    128-rollout request on its own high-priority stream) the result does not depend on what
    else is on the device."""
    torch, V = cuda()
    eps_x = W.mppi_noise(1, 128, 20, W.MPPI_SIGMA_U)
    kw = {"arrival": {}, "least_work": dict(policy=V.ADMIT_LEAST_WORK),
          "least_work_lane": dict(policy=V.ADMIT_LEAST_WORK, small_rollouts=256)}[admission]
    srv, p, fields = _server(V, 8, max_rollouts_inflight=100000, **kw)
    res_a, mu_a = srv.poll(srv.submit(0, eps_x))
    assert res_a["status"] == V.VPM_OK
    # the same request among others on the device
    tickets = [srv.submit(0, eps_x)]
    for s in range(1, len(SIZES)):
        tickets.append(srv.submit(s, W.mppi_noise(10 + s, 256 * (1 + s % 3), 20, W.MPPI_SIGMA_U)))
    results = [srv.poll(t) for t in tickets]
    assert all(r[0]["status"] == V.VPM_OK for r in results)
    assert np.array_equal(results[0][1], mu_a) and results[0][0]["j_min"] == res_a["j_min"]
    # requests overlapped on the device
    spans = sorted((r[0]["t_start_ms"], r[0]["t_done_ms"]) for r in results)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    srv.close()
    # the plain per-request form and the direct library calls give the same numbers
    srv1, _, _ = _server(V, 1)
    res_1, mu_1 = srv1.poll(srv1.submit(0, eps_x))
    srv1.close()
    assert np.array_equal(mu_1, mu_a)
    mu_d, jmin_d = _direct_mu(V, torch, p, fields[0], eps_x, 10.0)
    assert np.array_equal(mu_d, mu_a) and jmin_d == res_a["j_min"]


def test_newer_request_supersedes_queued_one():
    torch, V = cuda()
    srv, p, fields = _server(V, 1)
    long_t = srv.submit(4, W.mppi_noise(2, 2048, 100, W.MPPI_SIGMA_U))
    a = srv.submit(1, W.mppi_noise(3, 64, 20, W.MPPI_SIGMA_U))
    b = srv.submit(1, W.mppi_noise(4, 64, 20, W.MPPI_SIGMA_U))
    ra, rb, rl = srv.poll(a), srv.poll(b), srv.poll(long_t)
    assert ra[0]["status"] == V.VPM_ERR_BUSY
    assert rb[0]["status"] == V.VPM_OK and rl[0]["status"] == V.VPM_OK
    srv.close()


def test_admission_by_rollouts_in_flight():
    torch, V = cuda()
    srv, p, fields = _server(V, 8, max_rollouts_inflight=600)
    ks = [512, 512, 64, 64]
    tickets = [srv.submit(s, W.mppi_noise(60 + s, k, 20, W.MPPI_SIGMA_U)) for s, k in enumerate(ks)]
    res = [srv.poll(t)[0] for t in tickets]
    assert all(r["status"] == V.VPM_OK for r in res)
    # the two 512-rollout requests never share the device; the 64-rollout ones may join
    assert res[1]["t_start_ms"] >= res[0]["t_done_ms"]
    srv.close()


def test_admission_by_memory_budget():
    torch, V = cuda()
    K, H = 512, 20
    scen = [0, 3, 1]                                   # fields of 300, 400 and 500 particles
    probe, _, _ = _server(V, 1)
    need = [probe.request_bytes(s, K, H) for s in scen]
    probe.close()
    buffers = 4 * (2 * K * H + 2 * K + H)            # noise, controls, costs, weights, controls out
    assert all(b > buffers for b in need)              # plus the rollouts' pair-sum scratch
    two = sum(sorted(need)[:2])                        # the smallest pair of requests together
    assert max(need) < two
    srv, p, fields = _server(V, 4, budget=(max(need) + two) // 2)   # any one fits, no two do
    tickets = [srv.submit(s, W.mppi_noise(20 + s, K, H, W.MPPI_SIGMA_U)) for s in scen]
    res = [srv.poll(t)[0] for t in tickets]
    assert all(r["status"] == V.VPM_OK for r in res)
    spans = sorted((r["t_start_ms"], r["t_done_ms"]) for r in res)
    assert all(spans[i + 1][0] >= spans[i][1] for i in range(len(spans) - 1))   # one at a time
    with pytest.raises(V.VpmError) as e:
        srv.submit(1, W.mppi_noise(30, 2048, H, W.MPPI_SIGMA_U))
    assert e.value.status == V.VPM_ERR_CAPACITY
    srv.close()


def test_resident_field_advances_like_vpm_step():
    torch, V = cuda()
    srv, p, fields = _server(V, 2)
    t = srv.submit(2, W.mppi_noise(40, 32, 10, W.MPPI_SIGMA_U), advance_steps=3, advance_u=0.75)
    assert srv.poll(t)[0]["status"] == V.VPM_OK
    parts, xg = srv.read_scenario(2, SIZES[2] + 210)
    st = V.State(p, fields[2], W.GLIDER_X0, SIZES[2] + 210)
    for _ in range(3):
        st.step(0.75)
    ref_parts, ref_xg, _ = st.read()
    assert np.array_equal(parts, ref_parts) and np.array_equal(xg, ref_xg)
    srv.close()


def test_admission_waits_for_memory_taken_after_creation():
    """Device memory that other code takes after the server was made holds a request in the queue
    (no out-of-memory failure) until it is freed; then the request runs. The library's scratch
    comes from its own pool, so the device's default pool (torch's allocations here) is untouched."""
    torch, V = cuda()
    srv, p, fields = _server(V, 2)
    K, H = 512, 20
    need = srv.request_bytes(4, K, H)
    V.pool_trim()
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info()
    reserve = max(1 << 30, total // 50)                # the server keeps this much free
    hog_bytes = free - reserve - need // 2               # leaves half the request's bytes
    assert hog_bytes > 0
    hog = torch.empty(hog_bytes, dtype=torch.uint8, device="cuda")
    t = srv.submit(4, W.mppi_noise(70, K, H, W.MPPI_SIGMA_U))
    assert srv.poll(t, timeout_ms=1500) is None          # waiting, not failed
    st = srv.stats()
    assert st["queued"] == 1 and st["in_flight"] == 0
    del hog
    torch.cuda.empty_cache()
    res = srv.poll(t, timeout_ms=60000)
    assert res is not None and res[0]["status"] == V.VPM_OK
    srv.close()


@pytest.mark.parametrize("policy,max_wait_ms,small_first", [(0, 0.0, False), (1, 0.0, True), (1, 1.0, False)])
def test_admission_order_by_policy(policy, max_wait_ms, small_first):
    """One slot: while a long request runs, a large request B and then a small one C queue up.
    In arrival order B starts first; least work first starts C first (it needs about 1/30 of B's
    pair interactions); with a 1 ms bound on waiting, both have waited longer when the slot frees,
    so arrival order holds again. C's result is the same bits under every policy."""
    torch, V = cuda()
    srv = V.Server(max_inflight=1, max_rollouts=2048, max_horizon=100, policy=policy, max_wait_ms=max_wait_ms)
    p = W.glider_params()
    fields = [W.background_field(80, 1000), W.background_field(81, 1000), W.background_field(82, 300)]
    for f in fields:
        srv.add_scenario(p, f, W.GLIDER_X0, len(f) + 2 * 100 + 10)
    ta = srv.submit(0, W.mppi_noise(90, 2048, 100, W.MPPI_SIGMA_U))
    tb = srv.submit(1, W.mppi_noise(91, 2048, 100, W.MPPI_SIGMA_U))
    eps_c = W.mppi_noise(92, 256, 100, W.MPPI_SIGMA_U)
    tc = srv.submit(2, eps_c)
    (ra, _), (rb, _), (rc, mu_c) = srv.poll(ta), srv.poll(tb), srv.poll(tc)
    srv.close()
    assert ra["status"] == rb["status"] == rc["status"] == V.VPM_OK
    assert (rc["t_start_ms"] < rb["t_start_ms"]) == small_first, (policy, rb, rc)
    mu_d, jmin_d = _direct_mu(V, torch, p, fields[2], eps_c, 10.0)
    assert np.array_equal(mu_c, mu_d) and rc["j_min"] == jmin_d


def test_unknown_admission_policy_is_rejected():
    torch, V = cuda()
    with pytest.raises(V.VpmError):
        V.Server(max_inflight=1, policy=7)


@pytest.mark.parametrize("lane", [False, True])
def test_small_request_lane_overtakes_a_large_launch(lane):
    """Least work first with and without the small requests' lane. A request of 4096 rollouts
    (four waves of blocks) runs; a request of 256 rollouts arrives just after. Without the lane it
    waits until the large one is done (the device's rollout budget is full); with the lane it is
    admitted at once on a high-priority stream, its blocks start as the first wave's blocks
    finish, and it completes before the large request. Its result is the same bits either way."""
    torch, V = cuda()
    srv = V.Server(max_inflight=4, max_rollouts=4096, max_horizon=100, policy=V.ADMIT_LEAST_WORK,
                   small_rollouts=256 if lane else 0)
    p = W.glider_params()
    fields = [W.background_field(85, 1000), W.background_field(86, 300)]
    for f in fields:
        srv.add_scenario(p, f, W.GLIDER_X0, len(f) + 2 * 100 + 10)
    ta = srv.submit(0, W.mppi_noise(95, 4096, 100, W.MPPI_SIGMA_U))
    eps_c = W.mppi_noise(96, 256, 20, W.MPPI_SIGMA_U)
    tc = srv.submit(1, eps_c)
    (ra, _), (rc, mu_c) = srv.poll(ta), srv.poll(tc)
    srv.close()
    assert ra["status"] == rc["status"] == V.VPM_OK
    if lane:
        assert rc["t_done_ms"] < ra["t_done_ms"], (ra, rc)
    else:
        assert rc["t_start_ms"] >= ra["t_done_ms"], (ra, rc)
    mu_d, jmin_d = _direct_mu(V, torch, p, fields[1], eps_c, 10.0)
    assert np.array_equal(mu_c, mu_d) and rc["j_min"] == jmin_d


def test_small_lane_needs_least_work_policy():
    torch, V = cuda()
    with pytest.raises(V.VpmError):
        V.Server(max_inflight=2, small_rollouts=256)
