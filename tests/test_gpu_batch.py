"""Uneven batches (many roots with different particle counts in persistent class launches)
against single-root rollouts and the FP64 oracle."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import cuda

pytestmark = pytest.mark.gpu


def _roots(counts, seed=0):
    fields = [W.background_field(seed * 1000 + i, int(n)) for i, n in enumerate(counts)]
    rng = np.random.default_rng(seed)
    gliders = np.tile(np.array(W.GLIDER_X0), (len(counts), 1))
    gliders[:, 4] += rng.uniform(-0.5, 0.5, len(counts))
    return fields, gliders


def _singles(V, torch, p, fields, gliders, controls, precision):
    H = controls.shape[1]
    res = []
    for i, f in enumerate(fields):
        st = V.State(p, f, gliders[i], len(f) + 2 * H, precision)
        out = st.rollout_batch(controls[i:i + 1].contiguous(), want_field=True)
        res.append((out["costs"][0].item(), int(out["count"][0]), out["final_glider"][0].cpu().numpy()))
        st.close()
    return res


@pytest.mark.parametrize("counts", [
    list(W.uneven_counts(3, 24, 64, 1500)),
    [60, 900, 1500, 2200, 2600, 4000, 7000, 0, 130, 3100],
])
def test_batch_matches_single_rollouts(counts):
    torch, V = cuda()
    p = W.glider_params()
    H = 6
    fields, gliders = _roots(counts)
    controls = torch.tensor(W.mppi_noise(5, len(counts), H, W.MPPI_SIGMA_U), device="cuda")
    b = V.Batch(p, fields, gliders, H)
    out = b.rollout(controls)
    torch.cuda.synchronize()
    b.status()
    ref = _singles(V, torch, p, fields, gliders, controls, V.FP32)
    for i, (c, n, xg) in enumerate(ref):
        assert out["costs"][i].item() == c, i
        assert int(out["count"][i]) == n == counts[i] + 2 * H
        assert np.array_equal(out["final_glider"][i].cpu().numpy(), xg), i
    if max(counts) > 2300:
        assert len(b.schedule()) >= 3


def test_graph_replay_and_tuning_do_not_change_results():
    torch, V = cuda()
    p = W.glider_params()
    H = 5
    counts = list(W.uneven_counts(4, 40, 64, 3000))
    fields, gliders = _roots(counts, 1)
    controls = torch.tensor(W.mppi_noise(6, len(counts), H, W.MPPI_SIGMA_U), device="cuda")
    b = V.Batch(p, fields, gliders, H)
    base = {k: v.clone() for k, v in b.rollout(controls).items()}
    outs = [dict(costs=torch.empty_like(base["costs"]), count=torch.empty_like(base["count"]),
                 final_glider=torch.empty_like(base["final_glider"]))]
    for _ in range(2):                  # capture, then replay into the same buffers
        b.rollout(controls, use_graph=True, out=outs[0])
        torch.cuda.synchronize()
        for k in base:
            assert torch.equal(outs[0][k], base[k])
    b.tune(controls)
    sched = b.schedule()
    assert all(s["threads"] in (128, 256, 512) and s["tuned_ms"] > 0 and s["diag_t"] in (1, 2, 4)
               and s["ctas"] in (1, 2, 4) for s in sched)
    assert all(s["ctas"] == 1 for s in sched if s["cap"] <= 2300)
    tuned = b.rollout(controls)
    torch.cuda.synchronize()
    for k in base:
        assert torch.equal(tuned[k], base[k])


def test_every_schedule_gives_the_same_bits():
    """Each class launch at every block size and diagonal-unit size, and all rollouts in one merged
    launch at every size, give the bits of the default schedule."""
    torch, V = cuda()
    p = W.glider_params()
    H = 4
    counts = list(W.uneven_counts(8, 30, 64, 3000)) + [2500, 1400, 90]
    fields, gliders = _roots(counts, 3)
    controls = torch.tensor(W.mppi_noise(9, len(counts), H, W.MPPI_SIGMA_U), device="cuda")
    b = V.Batch(p, fields, gliders, H)
    base = {k: v.clone() for k, v in b.rollout(controls).items()}
    checked = 0
    for merged in (False, True):
        nl = 1 if merged else len(b.schedule())
        assert nl >= (1 if merged else 3)
        for cls in range(nl):
            for threads in (128, 256, 512):
                for diag_t in (1, 2, 4):
                    try:
                        b.set_schedule(merged, cls, threads, diag_t)
                    except V.VpmError:
                        continue                        # the size does not fit this class
                    out = b.rollout(controls)
                    torch.cuda.synchronize()
                    assert b.schedule()[0]["merged"] == merged
                    for k in base:
                        assert torch.equal(out[k], base[k]), (merged, cls, threads, diag_t, k)
                    checked += 1
    assert checked >= 20
    b.status()


def test_cluster_schedules_give_the_same_bits():
    """Each launch of both schedules with every rollout spread over a cluster of 2 and of 4 CTAs,
    at every block and diagonal-unit size that fits, gives the bits of one CTA per rollout. The
    fields cover a single row (up to 128 particles), ragged last rows, the once-per-target and
    once-per-pair diagonal units (below and from 1300 particles) and the 512-thread classes."""
    torch, V = cuda()
    p = W.glider_params()
    H = 4
    counts = [90, 127, 600, 1299, 1400, 2500, 2999, 4100, 6000, 8100, 0, 33]
    fields, gliders = _roots(counts, 5)
    controls = torch.tensor(W.mppi_noise(13, len(counts), H, W.MPPI_SIGMA_U), device="cuda")
    b = V.Batch(p, fields, gliders, H)
    base = {k: v.clone() for k, v in b.rollout(controls).items()}
    checked = set()
    for merged in (False, True):
        nl = 1 if merged else len(b.schedule())
        assert nl >= (1 if merged else 5)
        for cls in range(nl):
            for threads in (128, 256, 512):
                for diag_t in (1, 2, 4):
                    for ctas in (2, 4):
                        try:
                            b.set_ctas(merged, cls, 1)
                            b.set_schedule(merged, cls, threads, diag_t)
                            b.set_ctas(merged, cls, ctas)
                        except V.VpmError:
                            continue                # does not fit this class
                        out = b.rollout(controls)
                        torch.cuda.synchronize()
                        s = b.schedule()[cls]
                        assert (s["ctas"], s["threads"], s["diag_t"], s["merged"]) == \
                            (ctas, threads, diag_t, merged)
                        for k in base:
                            assert torch.equal(out[k], base[k]), (merged, cls, threads, diag_t, ctas, k)
                        checked.add((merged, cls, ctas))
            b.set_ctas(merged, cls, 1)
    # every class launch (5) and the merged launch ran on clusters of both sizes
    assert len(checked) == 2 * 6, sorted(checked)
    b.status()


def test_tuner_spreads_few_large_rollouts_over_clusters():
    """16 rollouts of 7000 particles use 16 of the SMs with one CTA each; the autotuner moves them
    to clusters (2.5x faster measured at this shape) and the results keep their bits."""
    torch, V = cuda()
    p = W.glider_params()
    H = 4
    counts = [7000] * 16
    fields, gliders = _roots(counts, 9)
    controls = torch.tensor(W.mppi_noise(17, len(counts), H, W.MPPI_SIGMA_U), device="cuda")
    b = V.Batch(p, fields, gliders, H)
    base = {k: v.clone() for k, v in b.rollout(controls).items()}
    b.tune(controls)
    sched = b.schedule()
    assert len(sched) == 1 and sched[0]["ctas"] in (2, 4), sched
    out = b.rollout(controls, use_graph=True)
    torch.cuda.synchronize()
    for k in base:
        assert torch.equal(out[k], base[k]), k
    b.status()


def test_clusters_at_the_largest_field_one_cta_holds():
    """Fields that fill a CTA's shared memory (9200 + 2H particles: about 224 of 227 KB) on clusters of 2
    and 4 CTAs give the bits of one CTA per rollout."""
    torch, V = cuda()
    p = W.glider_params()
    H = 3
    counts = [9200, 9290 - 2 * H]
    fields, gliders = _roots(counts, 4)
    controls = torch.tensor(W.mppi_noise(19, len(counts), H, W.MPPI_SIGMA_U), device="cuda")
    b = V.Batch(p, fields, gliders, H)
    base = {k: v.clone() for k, v in b.rollout(controls).items()}
    assert len(b.schedule()) == 1 and b.schedule()[0]["cap"] == 9290
    for ctas in (2, 4):
        b.set_ctas(False, 0, ctas)
        out = b.rollout(controls)
        torch.cuda.synchronize()
        assert b.schedule()[0]["ctas"] == ctas
        for k in base:
            assert torch.equal(out[k], base[k]), (ctas, k)
    b.status()


def test_cluster_ctas_rejected_where_they_cannot_run():
    torch, V = cuda()
    p = W.glider_params()
    fields, gliders = _roots([300, 2600], 1)
    b = V.Batch(p, fields, gliders, 2)
    for bad in (0, 3, 8):
        with pytest.raises(V.VpmError):
            b.set_ctas(False, 0, bad)
    with pytest.raises(V.VpmError):
        b.set_ctas(False, 5, 2)                     # no such launch
    b64 = V.Batch(p, fields, gliders, 2, precision=V.FP64)
    with pytest.raises(V.VpmError):
        b64.set_ctas(False, 0, 2)                   # clusters are a binary32 schedule
    b.set_ctas(False, 1, 2)
    assert b.schedule()[1]["ctas"] == 2


@pytest.mark.parametrize("K,n", [(1, 7000), (16, 3000), (40, 5000)])
def test_rollout_batch_on_clusters_gives_the_bits_of_one_block(K, n, monkeypatch):
    """vpm_rollout_batch spreads a few rollouts of large fields over clusters of CTAs (the largest
    C in {4, 2} with K C <= SMs); costs, final and per-step glider states, final fields and counts
    are the same bits as with one block per rollout (VPM_ROLLOUT_CLUSTERS=0), also with per-rollout
    initial states; the profiler shows the cluster kernel ran."""
    from torch.profiler import ProfilerActivity, profile
    torch, V = cuda()
    p = W.glider_params()
    H = 5
    st = V.State(p, W.background_field(77 + K, n), W.GLIDER_X0, n + 2 * H, V.FP32)
    controls = torch.tensor(W.mppi_noise(8, K, H, W.MPPI_SIGMA_U), device="cuda")
    x0 = torch.tensor(np.tile(np.array(W.GLIDER_X0), (K, 1)) +
                      np.random.default_rng(K).uniform(-0.1, 0.1, (K, 7)), device="cuda")
    for kw in ({}, {"x0": x0}):
        monkeypatch.setenv("VPM_ROLLOUT_CLUSTERS", "0")
        one = st.rollout_batch(controls, want_traj=True, want_field=True, **kw)
        torch.cuda.synchronize()
        monkeypatch.delenv("VPM_ROLLOUT_CLUSTERS")
        with profile(activities=[ProfilerActivity.CUDA], acc_events=True) as prof:
            cl = st.rollout_batch(controls, want_traj=True, want_field=True, **kw)
            torch.cuda.synchronize()
        names = [e.name for e in prof.events()]
        assert any("uneven_cluster_kernel" in nm for nm in names), names[:20]
        for k in one:
            assert torch.equal(cl[k], one[k]), (K, n, k, bool(kw))
    st.status()
    st.close()


def test_rollout_batch_on_clusters_under_graph_capture():
    """A few rollouts of a large field captured into a CUDA graph (torch.cuda.graph, global capture
    mode) and replayed give the bits of the eager launch. A launch shape that ran eagerly before
    the capture replays on clusters; a shape first seen during capture keeps one block per rollout
    (the library makes no occupancy query while a capture is open)."""
    from torch.profiler import ProfilerActivity, profile
    torch, V = cuda()
    p = W.glider_params()
    H = 4
    for n, K, eager_first in ((3000, 4, True), (5200, 2, False)):
        st = V.State(p, W.background_field(300 + n, n), W.GLIDER_X0, n + 2 * H, V.FP32)
        controls = torch.tensor(W.mppi_noise(21, K, H, W.MPPI_SIGMA_U), device="cuda")
        if eager_first:
            eager = st.rollout_batch(controls, want_traj=True)
            torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cap = st.rollout_batch(controls, want_traj=True)
        with profile(activities=[ProfilerActivity.CUDA], acc_events=True) as prof:
            g.replay()
            torch.cuda.synchronize()
        names = [e.name for e in prof.events()]
        on_clusters = any("uneven_cluster_kernel" in nm for nm in names)
        assert on_clusters == eager_first, names[:20]
        if not eager_first:
            eager = st.rollout_batch(controls, want_traj=True)
            torch.cuda.synchronize()
        for k in eager:
            assert torch.equal(cap[k], eager[k]), (n, k)
        g.replay()
        torch.cuda.synchronize()
        for k in eager:
            assert torch.equal(cap[k], eager[k]), (n, k)
        del g
        st.status()
        st.close()


def test_batch_fp64_against_oracle(ora):
    torch, V = cuda()
    p = W.glider_params()
    H = 20
    counts = [0, 50, 300, 700, 64]
    fields, gliders = _roots(counts, 2)
    eps = W.mppi_noise(7, len(counts), H, W.MPPI_SIGMA_U)
    b = V.Batch(p, fields, gliders, H, precision=V.FP64)
    out = b.rollout(torch.tensor(eps, device="cuda"))
    torch.cuda.synchronize()
    for i in range(len(counts)):
        ref = ora.rollout(p, fields[i], gliders[i], eps[i].astype(np.float64))
        assert np.abs(out["final_glider"][i].cpu().numpy() - ref["xg"]).max() <= 1e-6
        assert abs(out["costs"][i].item() - ref["cost"]) <= 1e-6 * abs(ref["cost"]) + 1e-5


def test_batch_rejects_fields_beyond_shared_memory():
    torch, V = cuda()
    fields, gliders = _roots([100, 9400])
    with pytest.raises(V.VpmError) as e:
        V.Batch(W.glider_params(), fields, gliders, 10)
    assert e.value.status == V.VPM_ERR_CAPACITY
