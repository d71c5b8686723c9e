"""Benchmark of the batched VPM-MPPI hot path on B300.

Workload (the MPPI batch): K = 1024 rollouts x H = 100 steps of dt = 0.01 from a shared
1000-particle root field (uniform in a 6c x 3c box, Gamma ~ N(0, 0.01^2), Vatistas core
0.05 c); every step sheds an LEV and a TEV, so each field grows to 1200 particles. One
benchmark step is one MPPI iteration: perturb the nominal controls with stored noise, run the
K rollouts (binary32 pair sums, binary64 plate solve and glider), reduce costs to weights,
and form the reweighted control sequence. A replan is three iterations.

Metric: Biot-Savart pair interactions per second (every evaluated target-source pair of
Eqs. 12 and 16 counted once), plus replan p50/p99 latency in ms.

The default line also carries, as entries of their own: the replan latency on ~2000-particle
fields next to the one-rollout-per-launch form, the serving loop at two arrival rates, the
uneven batch (4096 rollouts of 64-8192 particles, autotuned persistent launches), the 2^20
free field (two Heun steps, error on 4096 sampled targets) and the FP64 oracle on the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--replans R] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import math
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

K_ROLL, H, N0 = 1024, 100, 1000
LAMBDA = 10.0
FLOPS_PER_PAIR = 12        # 2 FADD, 2 FMUL, 4 FFMA per pair (FMA = 2 flops), plus one MUFU.RSQ
PEAK_SM_MHZ = 2032.0
N_SM = 148


def pairs_per_rollout(n0: int, H: int, n_b: int = 8, shed: int = 2) -> int:
    """Target-source pairs of one rollout: per step N(n_c + n_b) plate pairs from the
    N pre-shed wake particles, then N'(N' + n_b) convection pairs with N' = N + shed."""
    total, n = 0, n0
    for _ in range(H):
        total += n * (2 * n_b + 1)
        n2 = n + shed
        total += n2 * (n2 + n_b)
        n = n2
    return total


def fp32_peak_tflops() -> float:
    return N_SM * 128 * 2 * PEAK_SM_MHZ * 1e6 / 1e12


def profiled_traffic(summary: str, source: str):
    """DRAM bytes per full-size launch recorded in profiles/<summary> by an ncu capture, or None
    when the kernel source has changed since (the summary records the source's hash)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", summary)
    src = os.path.join(ROOT, "paper_2509_16079_b300", "csrc", source)
    if not (os.path.exists(path) and os.path.exists(src)):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*(\d+)\s+source\s+([0-9a-f]{16})", text)
    if not m:
        return None
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return int(m.group(1)) if digest == m.group(2) else None


def profiled_pipes(summary: str, source: str):
    """Pipe utilisation (% of peak) of the kernel's ncu full-set capture recorded in
    profiles/<summary>, or None when the kernel source has changed since."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", summary)
    src = os.path.join(ROOT, "paper_2509_16079_b300", "csrc", source)
    if not (os.path.exists(path) and os.path.exists(src)):
        return None
    m = re.search(r"pipes_pct:\s*fma ([0-9.]+) xu ([0-9.]+) fp64 ([0-9.]+) issue ([0-9.]+) source ([0-9a-f]{16})",
                  open(path).read())
    if not m:
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != m.group(5):
        return None
    return {"fma_pipe_pct": float(m.group(1)), "mufu_pipe_pct": float(m.group(2)),
            "fp64_pipe_pct": float(m.group(3)), "issue_active_pct": float(m.group(4)),
            "capture": "ncu --set full on the small case of profiles/%s" % summary}


def graph_replans(V, L, stream, flush, replans, body, state):
    """Replan latency of the graph-captured form: body(stream_handle) enqueues one replan; it is
    captured once into a CUDA graph and replayed `replans` times (L2 flushed in between, outside
    the events). The replayed replan must give the same bits as the eager one from the same
    state. Returns p50/p99 ms, or the reason capture failed."""
    import torch
    try:
        cs = torch.cuda.Stream()
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            body(V.stream_handle(cs))                       # warm-up on the capture stream
        stream.wait_stream(cs)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cs, capture_error_mode="thread_local"):
            body(V.stream_handle(cs))
        torch.cuda.synchronize()
        s0 = state.clone()
        body(V.stream_handle(stream))                       # eager replan from s0
        torch.cuda.synchronize()
        eager = state.clone()
        state.copy_(s0)
        g.replay()
        torch.cuda.synchronize()
        same = bool(torch.equal(state, eager))
        lat = []
        for r in range(replans):
            flush.fill_(float(r))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b.record(stream)
            b.synchronize()
            lat.append(a.elapsed_time(b))
        return {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                "replans": len(lat), "same_bits_as_eager": same}
    except Exception as e:                                   # report, keep the eager numbers
        torch.cuda.synchronize()
        return {"unavailable": str(e)[:200]}


# ------------------------------------------------------------------ clocks during the run
class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU baseline (oracle)
ERR_ROLLOUTS = (0, 5, 10, 15)          # sampled rollouts whose per-result errors are reported
ERR_STEPS = (0, 33, 66, 99)            # steps compared from identical states
VEL_TOL, POS_TOL = 1e-5, 1e-4


def _oracle_rollout_stepped(oracle, p, field, xg0, u, cap, snap_steps):
    """One oracle rollout advanced step by step (the same C arithmetic as oracle.rollout), keeping
    the full state before each step in snap_steps and that step's velocities."""
    st = oracle.State(p, field, xg0, cap)
    snaps = {}
    for k in range(len(u)):
        if k in snap_steps:
            snaps[k] = dict(parts=st.particles.copy(), xg=st.xg.copy(), gb=st.gb_prev.copy(),
                            glev=st.glev_prev, hp=st.has_prev)
        out = st.step(float(u[k]))
        if k in snap_steps:
            snaps[k]["vel"] = out["vel"].copy()
    return st.particles.copy(), snaps


def _oracle_binary32_spread(oracle, p, field, xg0, u, cap):
    """Distance after len(u) steps between the oracle and the same oracle whose state is rounded
    to binary32 after every step: the deviation that binary32 storage alone picks up from the
    model's own sensitivity."""
    a = oracle.State(p, field, xg0, cap)
    b = oracle.State(p, field, xg0, cap)
    for k in range(len(u)):
        a.step(float(u[k]))
        b.step(float(u[k]))
        for arr in (b.x, b.z, b.g):
            arr[:b.n] = arr[:b.n].astype(np.float32).astype(np.float64)
    if a.n != b.n:
        return float("nan")
    return float(np.abs(a.particles[:, :2] - b.particles[:, :2]).max())


def cpu_baseline(rollouts: int = 16, threads: int | None = None, V=None):
    """FP64 oracle rollouts of the same workload on the host cores (one rollout per thread at a
    time; the C oracle releases the GIL), timed. With the library V given, the same oracle
    results also give the per-result errors of the binary32 GPU path on this sample: each step
    of ERR_STEPS of the rollouts ERR_ROLLOUTS run on the GPU from the oracle's own state (normwise
    velocity error), and every sampled rollout's 100-step positions from a GPU launch of the same
    16 controls (a rollout's bits do not depend on the batch it runs in) beside the spread of the
    binary32-rounded oracle."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    oracle.build()
    p, field, xg0, eps = W.mppi_batch_inputs(0, K=rollouts, H=H, n=N0)
    cap = N0 + 2 * H
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        runs = list(ex.map(lambda i: _oracle_rollout_stepped(
            oracle, p, field, xg0, eps[i].astype(np.float64), cap,
            ERR_STEPS if (V is not None and i in ERR_ROLLOUTS) else ()), range(rollouts)))
    dt = time.perf_counter() - t0
    pairs = pairs_per_rollout(N0, H) * rollouts
    cores = min(threads, rollouts)
    out = {"value": pairs / dt, "unit": "pair-interactions/s", "cores": cores,
           "kind": "oracle",
           "sample": "%d of the %d rollouts (1000 particles, 100 steps, FP64 C oracle stepped from Python), "
                     "%.1f s wall" % (rollouts, K_ROLL, dt),
           "per_core": pairs / dt / cores, "cpu_model": cpu_model(),
           "hardware_threads": os.cpu_count(),
           "iteration_s_extrapolated": dt * K_ROLL / rollouts}
    if V is None:
        return out, None
    import torch
    sel = [i for i in ERR_ROLLOUTS if i < rollouts]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        spreads = list(ex.map(lambda i: _oracle_binary32_spread(
            oracle, p, field, xg0, eps[i].astype(np.float64), cap), sel))
    root = V.State(p, field, xg0, cap, V.FP32)
    res = root.rollout_batch(torch.tensor(eps, device="cuda"), want_final=False, want_field=True)
    torch.cuda.synchronize()
    root.status()
    fields = res["field"].cpu().numpy()
    counts = res["count"].cpu().numpy()
    root.close()
    vel_err, pos = [], []
    for r, i in enumerate(sel):
        final, snaps = runs[i]
        n = int(counts[i])
        perr = float(np.abs(fields[i, :n, :2] - final[:, :2]).max()) if n == len(final) else float("nan")
        pos.append({"rollout": i, "max_position_error": perr, "binary32_envelope": spreads[r]})
        for k in ERR_STEPS:
            sn = snaps[k]
            st = V.State(p, sn["parts"], sn["xg"], cap, V.FP32)
            st.set_history(sn["gb"], sn["glev"], bool(sn["hp"]))
            pr = st.step(float(eps[i, k]), probe=True)
            m = len(sn["vel"])
            v = pr["vel"].cpu().numpy()[:2 * m].reshape(-1, 2)
            st.close()
            den = np.linalg.norm(sn["vel"], axis=1).max()
            vel_err.append(float(np.linalg.norm(v - sn["vel"], axis=1).max() / den))
    errors = {
        "per_step_velocity_normwise": {"max": max(vel_err), "tolerance": VEL_TOL,
                                       "cases": len(vel_err), "rollouts": sel, "steps": list(ERR_STEPS),
                                       "form": "one binary32 GPU step from the oracle's own state"},
        "positions_after_100_steps": {"per_rollout": pos, "tolerance": POS_TOL,
                                      "note": "the ungated workload is chaotic; binary32_envelope is the "
                                              "distance between the oracle and the oracle rounded to binary32 "
                                              "after every step (the model's own sensitivity to binary32 state)"},
    }
    return out, errors


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ------------------------------------------------------------------ distributed helpers
def dist_setup(n_gpus: int, backend: str = None):
    """Rank, world size and local rank from the launcher's environment; for N > 1 a process
    group over NCCL (one GPU per rank), or gloo where no GPU is present."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = backend or ("nccl" if torch.cuda.is_available() else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job rate of independent replicas: every rank processes the same units, the job
    ends with the slowest rank."""
    return units_per_rank * world / max_seconds


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    rank, world, local = dist_setup(args.gpus)
    if rank == 0:
        build.build()
    barrier(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    V.lib()

    p, field, xg0, eps_np = W.mppi_batch_inputs(rank, K=K_ROLL, H=H, n=N0)
    n_iter_noise = 4
    eps_all = [torch.tensor(W.mppi_noise(1000 + 7 * j + rank, K_ROLL, H, W.MPPI_SIGMA_U), device=dev)
               for j in range(n_iter_noise)]
    root = V.State(p, field, xg0, N0 + 2 * H, V.FP32)
    mu = torch.zeros(H, dtype=torch.float32, device=dev)
    controls = torch.empty((K_ROLL, H), dtype=torch.float32, device=dev)
    costs = torch.empty(K_ROLL, dtype=torch.float32, device=dev)
    weights = torch.empty(K_ROLL, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    sh = V.stream_handle(stream)
    L = V.lib()

    def iteration_on(j, hs):
        V.check(L.mppi_perturb(V.ptr(mu), V.ptr(eps_all[j % n_iter_noise]), K_ROLL, H, V.ptr(controls), hs))
        V.check(L.vpm_rollout_batch(root.handle, K_ROLL, H, V.ptr(controls), V.ptr(costs), None, None,
                                    None, None, hs))
        V.check(L.mppi_weights(V.ptr(costs), K_ROLL, LAMBDA, V.ptr(weights), hs))
        V.check(L.mppi_update(V.ptr(weights), V.ptr(controls), K_ROLL, H, V.ptr(mu), hs))

    def iteration(j):
        iteration_on(j, sh)

    for j in range(args.warmup):
        iteration(j)
    torch.cuda.synchronize()
    root.status()

    # timed iterations: events around each iteration (and around the rollout kernel alone),
    # L2 flushed between iterations outside the events
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for j in range(args.steps):
            flush.fill_(float(j))
            a, b, c = ev[j]
            a.record(stream)
            V.check(L.mppi_perturb(V.ptr(mu), V.ptr(eps_all[j % n_iter_noise]), K_ROLL, H, V.ptr(controls), sh))
            V.check(L.vpm_rollout_batch(root.handle, K_ROLL, H, V.ptr(controls), V.ptr(costs), None,
                                        None, None, None, sh))
            b.record(stream)
            V.check(L.mppi_weights(V.ptr(costs), K_ROLL, LAMBDA, V.ptr(weights), sh))
            V.check(L.mppi_update(V.ptr(weights), V.ptr(controls), K_ROLL, H, V.ptr(mu), sh))
            c.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    roll_ms = [a.elapsed_time(b) for a, b, c in ev]
    total_ms = max_over_ranks(sum(step_ms), world)
    root.status()

    pairs_iter = pairs_per_rollout(N0, H) * K_ROLL
    value = job_throughput(pairs_iter * args.steps, world, total_ms / 1e3)

    # replan latency: 3 iterations per replan, events per replan
    rep = []
    for r in range(args.replans):
        flush.fill_(float(r))
        a, _, c = ev[r % len(ev)]
        a.record(stream)
        for j in range(3):
            iteration(j)
        c.record(stream)
        c.synchronize()
        rep.append(a.elapsed_time(c))
    rep.sort()
    p50 = float(np.percentile(rep, 50)) if rep else None
    p99 = float(np.percentile(rep, 99)) if rep else None
    replan_graph = graph_replans(V, L, stream, flush, args.replans,
                                 lambda hs: [iteration_on(j, hs) for j in range(3)], mu)

    # end-to-end: host noise -> device each iteration, nominal controls back to the host
    eps_host = [torch.tensor(W.mppi_noise(2000 + j, K_ROLL, H, W.MPPI_SIGMA_U)).pin_memory()
                for j in range(2)]
    mu_host = torch.empty(H, dtype=torch.float32).pin_memory()
    eps_dev = torch.empty((K_ROLL, H), dtype=torch.float32, device=dev)
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(e2e_steps):
        eps_dev.copy_(eps_host[j % 2], non_blocking=True)
        V.check(L.mppi_perturb(V.ptr(mu), V.ptr(eps_dev), K_ROLL, H, V.ptr(controls), sh))
        V.check(L.vpm_rollout_batch(root.handle, K_ROLL, H, V.ptr(controls), V.ptr(costs), None, None,
                                    None, None, sh))
        V.check(L.mppi_weights(V.ptr(costs), K_ROLL, LAMBDA, V.ptr(weights), sh))
        V.check(L.mppi_update(V.ptr(weights), V.ptr(controls), K_ROLL, H, V.ptr(mu), sh))
        mu_host.copy_(mu, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = job_throughput(pairs_iter * e2e_steps, world, e2e_s)

    replan2000 = None
    if args.replan2000_replans > 0:
        with ClockSampler(local) as clk_ns:
            replan2000 = replans_2000_particles(V, torch, args.n0, args.replan2000_replans, args.per_launch_subset)
        replan2000["clocks"] = clk_ns.summary()

    serving = None
    if args.serve_line_seconds > 0 and world == 1:
        with ClockSampler(local) as clk_sv:
            serving = serving_at_rates(V, args.serve_line_rates, args.serve_line_seconds)
        serving = {"workload": "16 scenarios of 500-5000 resident particles, K in {256, 1024, 4096}, "
                               "H=100, Poisson arrivals; continuous batching (16 in flight; arrival "
                               "order, and least estimated work first with a 4 s bound on waiting and a "
                               "high-priority lane for K <= 256) "
                               "against the plain per-request form (1 in flight) on the same trace",
                   "seconds_of_arrivals": args.serve_line_seconds, "runs": serving,
                   "clocks": clk_sv.summary()}

    # the uneven batch and the large free field, each measured as its own workload would be
    uneven = freefield = None
    if world == 1 and args.uneven_line_steps > 0:
        uneven = uneven_result(V, torch, args.rollouts_uneven, args.uneven_line_steps, args.sample)
    if world == 1 and args.ff_line_steps > 0:
        freefield = freefield_result(V, torch, args.n, args.ff_line_steps)

    if rank != 0:
        return
    clocks = clk.summary()
    roll_avg_s = statistics.mean(roll_ms) / 1e3
    achieved = pairs_iter * FLOPS_PER_PAIR / roll_avg_s / 1e12
    peak = fp32_peak_tflops()
    traffic = profiled_traffic("rollout_kernel_mppi_batch.md", "vpm_rollout.cu")
    pipes = profiled_pipes("rollout_kernel_mppi_batch.md", "vpm_rollout.cu")
    line = {
        "metric": "Biot-Savart pair-interactions/s",
        "value": value,
        "unit": "pair-interactions/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 pair sums (f64 plate solve, Kelvin sum, loads, glider)",
        "data": "synthetic",
        "config": {
            "workload": "MPPI batch: K=1024 rollouts x H=100 steps, dt=0.01, root field 1000 "
                        "particles growing to 1200, Vatistas core 0.05c, one MPPI iteration per step",
            "K": K_ROLL, "H": H, "n0": N0, "lambda": LAMBDA,
            "pairs_per_step": pairs_iter,
            "l2": "flushed between timed iterations (256 MB write outside the events)",
            "parallelism": "replicas" if world > 1 else "single GPU",
        },
        "replan_ms": {"p50": p50, "p99": p99, "replans": len(rep), "iterations_per_replan": 3,
                      "form": "eager launches", "graph": replan_graph},
        "e2e": {"value": e2e_value, "unit": "pair-interactions/s",
                "h2d_bytes_per_step": K_ROLL * H * 4, "d2h_bytes_per_step": H * 4,
                "steps": e2e_steps},
        "gpu_launches": 4 * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "rollout_kernel<float, Vatistas>", "pipes": pipes,
                     "peak_basis": "148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz (FMA = 2 flops)",
                     "rollout_ms": statistics.mean(roll_ms)},
        "clocks": clocks,
    }
    if replan2000 is not None:
        line["replan2000_ms"] = replan2000
    if serving is not None:
        line["serving"] = serving
    if uneven is not None:
        line["uneven_batch"] = uneven
    if freefield is not None:
        line["free_field"] = freefield
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"], line["error_vs_fp64_oracle"] = cpu_baseline(V=V)
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """A few launches of the MPPI iteration at a reduced size, for ncu captures."""
    import torch
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    build.build()
    K, Hh, n0 = args.rollouts, args.horizon, args.profile_n0
    p, field, xg0, _ = W.mppi_batch_inputs(0, K=1, H=1, n=n0)
    eps = torch.tensor(W.mppi_noise(1000, K, Hh, W.MPPI_SIGMA_U), device="cuda")
    root = V.State(p, field, xg0, n0 + 2 * Hh, V.FP32)
    mu = torch.zeros(Hh, dtype=torch.float32, device="cuda")
    for j in range(args.warmup + args.steps):
        c = V.mppi_perturb(mu, eps)
        out = root.rollout_batch(c, want_final=False)
        w = V.mppi_weights(out["costs"], LAMBDA)
        mu = V.mppi_update(w, c)
    torch.cuda.synchronize()
    root.status()
    print(json.dumps({"profile_case": True, "K": K, "H": Hh, "n0": n0, "launches": 4 * (args.warmup + args.steps)}))



# ------------------------------------------------------------------ extra workloads
def freefield_result(V, torch, n: int, steps: int, targets: int = 4096) -> dict:
    """Large free field: n regularised vortices (64 Gaussian blobs, core 1e-3), `steps` Heun
    steps in binary32 with one evaluation per particle pair; error of the final velocities
    against the FP64 oracle on `targets` sampled targets, which also times the oracle."""
    rc, dt = 1e-3, 1e-3
    P = W.blob_field(0, n)
    a = np.zeros((n, 4), np.float32)
    a[:, :3] = P
    d = torch.tensor(a, device="cuda")
    V.freefield_heun(d.clone(), V.KERNEL_VATISTAS, rc, dt, 1)   # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record()
        V.freefield_heun(d, V.KERNEL_VATISTAS, rc, dt, steps)
        e1.record()
        e1.synchronize()
    ms = e0.elapsed_time(e1)
    pairs = 2.0 * steps * n * n
    # one velocity evaluation for the error check and the per-launch timing of the kernel alone
    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    v0.record()
    vel = V.freefield_velocity(d, V.KERNEL_VATISTAS, rc)
    v1.record()
    v1.synchronize()
    kern_ms = v0.elapsed_time(v1)
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    oracle.build()
    Pf = d[:, :3].double().cpu().numpy()
    idx = W.sample_indices(1, n, targets)
    chunks = np.array_split(idx, os.cpu_count() or 1)
    t_ora = time.perf_counter()
    with ThreadPoolExecutor(max_workers=len(chunks)) as ex:
        parts = list(ex.map(lambda c: oracle.velocity_at(Pf, Pf[c, :2], 1, rc, skip=c), chunks))
    t_ora = time.perf_counter() - t_ora
    ref = np.concatenate(parts)
    ora_pairs = float(len(idx)) * n
    got = vel.cpu().numpy()[idx].astype(np.float64)
    err = np.linalg.norm(got - ref, axis=1).max() / np.linalg.norm(ref, axis=1).max()
    achieved = n * float(n) * FLOPS_PER_PAIR / (kern_ms / 1e3) / 1e12
    peak = fp32_peak_tflops()
    return {
        "metric": "Biot-Savart pair-interactions/s", "value": pairs / (ms / 1e3),
        "unit": "pair-interactions/s", "n_gpus": 1, "steps": steps, "ms_per_step": ms / steps,
        "higher_is_better": True, "dtype": "f32 (Kahan-compensated tile sums)", "data": "synthetic",
        "config": {"workload": "free field N=%d, 64 Gaussian blobs sigma 0.1 in a 10x10 box, "
                               "Vatistas core 1e-3, Heun dt=1e-3" % n, "pairs_per_step": 2 * n * n,
                   "l2": "not flushed: the %d MB field stays L2-resident across the Heun steps of "
                         "one call; each evaluation is ALU-bound (%d x %d pairs)" % (16 * n >> 20, n, n)},
        "error_vs_fp64_oracle": {"normwise_velocity": err, "targets": int(len(idx)),
                                 "tolerance": 1e-5},
        "cpu_baseline": {"value": ora_pairs / t_ora, "unit": "pair-interactions/s",
                         "cores": len(chunks), "kind": "oracle",
                         "per_core": ora_pairs / t_ora / len(chunks), "cpu_model": cpu_model(),
                         "sample": "%d sampled targets against all %d sources (FP64 C oracle), %.1f s wall"
                                   % (len(idx), n, t_ora)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "kernel": "freefield_sym_kernel<Vatistas> + freefield_combine_kernel (one velocity "
                               "evaluation; one evaluation per particle pair)",
                     "traffic": profiled_traffic("freefield_kernel_2pow20.md", "vpm_freefield.cu"),
                     "pipes": profiled_pipes("freefield_kernel_2pow20.md", "vpm_freefield.cu"),
                     "launch_ms": kern_ms},
        "clocks": clk.summary()}


def run_freefield(args):
    """The large free field alone: N = 2^20 by default, 10 Heun steps."""
    import torch
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    build.build()
    print(json.dumps(freefield_result(V, torch, args.n, args.ff_steps)), flush=True)


def run_alu(args):
    """Measured ceilings of the binary32 pair kernels: FP32 FMA, MUFU rsqrt and ex2 rates, the
    pair loop that evaluates every pair once per target (1, 2, 4 targets per lane) and the
    rollout kernel's pair phase (one evaluation per pair across rows) alone, 1 and 7 blocks per SM."""
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    build.build()
    V.probe_rate(V.PROBE_FFMA, 7)          # first-launch warm-up
    with ClockSampler(0) as clk:
        rates = {
            "ffma_per_s": V.probe_rate(V.PROBE_FFMA, 7),
            "mufu_rsqrt_per_s": V.probe_rate(V.PROBE_RSQRT, 7),
            "mufu_ex2_per_s": V.probe_rate(V.PROBE_EX2, 7),
        }
        loop = {}
        for name, pr in (("t1", V.PROBE_PAIRS_T1), ("t2", V.PROBE_PAIRS_T2), ("t4", V.PROBE_PAIRS_T4),
                         ("sym", V.PROBE_PAIRS_SYM)):
            for bps in (1, 7):
                loop["%s_%dblk" % (name, bps)] = V.probe_rate(pr, bps)
    clocks = clk.summary()
    mhz = clocks.get("sm_mhz") or PEAK_SM_MHZ
    per_clk = lambda r: r / (N_SM * mhz * 1e6)
    fp32_ops_per_pair = 8          # 2 FADD, 2 FMUL, 4 FFMA
    ceiling = min(rates["ffma_per_s"] / fp32_ops_per_pair, rates["mufu_rsqrt_per_s"])
    # one evaluation for two pairs: 2 FADD, 3 FMUL, 6 FFMA and one MUFU (rows only; the
    # diagonal blocks are evaluated once per target)
    ceiling_sym = min(rates["ffma_per_s"] / 5.5, 2.0 * rates["mufu_rsqrt_per_s"])
    directed = {k: v for k, v in loop.items() if not k.startswith("sym")}
    best = max(loop.values())
    print(json.dumps({
        "metric": "pair-loop ceiling (pair-interactions/s)", "value": best, "unit": "pair-interactions/s",
        "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "throughput probes: 8 independent chains per thread, 128-thread blocks; "
                               "pair loop over a 1024-particle field in shared memory"},
        "unit_rates": rates,
        "unit_rates_per_sm_per_clock": {k: per_clk(v) for k, v in rates.items()},
        "pair_loop_rates": loop,
        "issue_free_ceiling_pairs_per_s": ceiling,
        "loop_fraction_of_issue_free_ceiling": max(directed.values()) / ceiling,
        "issue_free_ceiling_one_evaluation_per_pair": ceiling_sym,
        "pair_phase_fraction_of_its_ceiling": max(loop["sym_1blk"], loop["sym_7blk"]) / ceiling_sym,
        "fp32_peak_tflops": fp32_peak_tflops(),
        "clocks": clocks}), flush=True)


def run_table1(args):
    """The perch benchmark's shape (Table I): clean wake, merging above N_max = 60 particles, 80
    steps at dt = 0.01, batch sizes 1 ... 1024; wall time of one batched rollout launch."""
    import torch
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    build.build()
    p = dict(W.glider_params(), n_wake_max=60)
    Hh = 80
    root = V.State(p, np.zeros((0, 3)), W.GLIDER_X0, 62, V.FP32)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    rows = {}
    with ClockSampler(0) as clk:
        for K in (1, 128, 256, 512, 1024):
            eps = torch.tensor(W.mppi_noise(40 + K, K, Hh, W.MPPI_SIGMA_U), device="cuda")
            for _ in range(3):
                root.rollout_batch(eps, want_final=False)
            ts = []
            for _ in range(20):
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                out = root.rollout_batch(eps, want_final=False)
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            assert bool(torch.isfinite(out["costs"]).all())
            pairs = K * sum(min(2 * k, 60) * 17 + (min(2 * k, 60) + 2) * (min(2 * k, 60) + 2 + 8)
                            for k in range(Hh))
            rows[str(K)] = {"ms_p50": statistics.median(ts), "ms_min": min(ts),
                            "pairs_per_s": pairs / (statistics.median(ts) / 1e3)}
    paper = {"1": 8.0, "128": 10.3, "256": 12.2, "512": 16.3, "1024": 27.2}
    print(json.dumps({
        "metric": "batched rollout wall time (ms)", "value": rows["1024"]["ms_p50"], "unit": "ms",
        "n_gpus": 1, "steps": 20, "higher_is_better": False, "dtype": "f32 pair sums (f64 plate work)",
        "data": "synthetic",
        "config": {"workload": "perch benchmark shape: clean wake, merging above 60 particles, 80 steps, "
                               "dt 0.01, batch 1..1024", "l2": "flushed between timed launches (256 MB)"},
        "by_batch": rows,
        "paper_rtx5080_ms_context_only": paper,
        "clocks": clk.summary()}), flush=True)


def run_policy(args):
    """Policy construction of §IV-B at the NMPC settings of §V-A (batch 256, 77-step nominal
    trajectory, perch wake with merging above 60 particles): perturbed rollouts with their
    trajectories, least-squares Jacobians and TVLQR gains, each timed with CUDA events."""
    import torch
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    build.build()
    p = dict(W.glider_params(), n_wake_max=60)
    K, Hh = 256, 77
    root = V.State(p, np.zeros((0, 3)), W.GLIDER_X0, 62, V.FP32)
    ubar = W.mppi_noise(51, 1, Hh, 2.0)[0]
    x0, u = W.policy_samples(52, K, W.GLIDER_X0, ubar)
    d_x0, d_u, d_ub = (torch.tensor(a, device="cuda") for a in (x0, u, ubar))
    nom = root.rollout_batch(d_ub[None, :], want_traj=True)
    xbar = torch.cat([torch.tensor([W.GLIDER_X0], dtype=torch.float64, device="cuda"), nom["traj"][0]])
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    times = {"rollouts": [], "least_squares": [], "tvlqr": [], "total": []}
    with ClockSampler(0) as clk:
        for it in range(args.warmup + args.steps):
            ev[0].record()
            out = root.rollout_batch(d_u, want_final=False, want_traj=True, x0=d_x0)
            ev[1].record()
            A, B, info = V.ls_jacobians(d_x0, out["traj"], d_u, xbar, d_ub, p["dt"])
            ev[2].record()
            g, s0 = V.tvlqr(A, B, p["dt"], W.TVLQR_QC, W.TVLQR_QF, W.TVLQR_RC)
            ev[3].record()
            ev[3].synchronize()
            if it >= args.warmup:
                times["rollouts"].append(ev[0].elapsed_time(ev[1]))
                times["least_squares"].append(ev[1].elapsed_time(ev[2]))
                times["tvlqr"].append(ev[2].elapsed_time(ev[3]))
                times["total"].append(ev[0].elapsed_time(ev[3]))
    assert not bool(info.any()) and bool(torch.isfinite(g).all())
    med = {k: statistics.median(v) for k, v in times.items()}
    print(json.dumps({
        "metric": "policy construction time (ms)", "value": med["total"], "unit": "ms", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
        "dtype": "f32 pair sums (f64 plate work, least squares and Riccati in f64)", "data": "synthetic",
        "config": {"workload": "policy synthesis: K=256 perturbed rollouts x 77 steps (perch wake, merging "
                               "above 60 particles), least squares per step, TVLQR with the weights of §V-A"},
        "median_ms": med, "paper_ms_context_only": 9.0, "clocks": clk.summary()}), flush=True)


def run_nmpc(args):
    """Timing of the NMPC of §IV-C at the settings of §V-A: a 77-step manoeuvre, replanning every
    10 steps (10 Hz at dt = 0.01) with a 10-step projection, 256 rollouts x 3 MPPI iterations and
    the least-squares / TVLQR synthesis per plan, planning on its own thread while the control
    loop runs paced at 100 Hz against a plant model. Reports the longest plan (each replan must
    finish within the 100 ms between replans; the first plan, made at the first control call,
    is timed by that call too) and the control call's time. The library is warmed up first."""
    import torch  # noqa: F401
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    build.build()
    p = dict(W.glider_params(), n_wake_max=60)
    N, P_, L, K, IT = 77, 10, 10, 256, 3
    cap = 64
    x0 = np.array(W.GLIDER_X0)
    mu0 = np.zeros(N, np.float32)
    noise = W.nmpc_noise(61, 8, IT, K, N)
    cfg = dict(horizon=N, replan_every=P_, latency=L, rollouts=K, iterations=IT, lam=LAMBDA,
               qc=W.TVLQR_QC, qf=W.TVLQR_QF, rc=W.TVLQR_RC)
    # a throwaway controller's first plan loads every kernel the plans launch, so the timed
    # controller's plans carry no first-launch cost
    warm = V.NMPC(p, np.zeros((0, 3)), cap, x0, mu0, noise, threaded=False, **cfg)
    warm.control(0, x0)
    warm.close()
    with ClockSampler(0) as clk:
        nm = V.NMPC(p, np.zeros((0, 3)), cap, x0, mu0, noise, threaded=True, **cfg)
        plant = V.State(p, np.zeros((0, 3)), x0, cap)
        ctl_ms = []
        t_start = time.perf_counter()
        for t in range(N):
            wait = t_start + t * p["dt"] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            x = plant.glider()
            c0 = time.perf_counter()
            u = nm.control(t, x)
            ctl_ms.append((time.perf_counter() - c0) * 1e3)
            plant.step(u)
        st = nm.stats()
        nm.close()
        plant.close()
    print(json.dumps({
        "metric": "NMPC replan time", "value": st["max_plan_ms"], "unit": "ms", "n_gpus": 1,
        "higher_is_better": False, "dtype": "f32 pair sums (f64 plate work, policy in f64)",
        "data": "synthetic",
        "config": {"workload": "perch manoeuvre in simulation: 77 steps at dt 0.01, replan every 10 steps with a "
                               "10-step projection, 256 rollouts x 3 MPPI iterations, planner thread, control "
                               "paced at 100 Hz"},
        "plans": st, "first_plan_ms": ctl_ms[0],
        "control_call_ms": {"p50": statistics.median(ctl_ms[1:]), "max": max(ctl_ms[1:])},
        "clocks": clk.summary()}), flush=True)


def run_plate(args):
    """The fixed flat plate at 45 degrees in a unit stream with the disturbance pair
    (Gaussian core 0.05 c, no decay, shedding every step), 200 steps in binary64 on the GPU, one
    block; the FP64 oracle runs the same input on the host for the error and the CPU time."""
    import torch
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    import oracle
    build.build()
    oracle.build()
    p = W.fixed_plate_params()
    steps = 200
    parts, xg, cap = W.fixed_plate_initial(0, steps)
    st = V.State(p, parts, xg, cap, V.FP64)
    zero = torch.zeros((1, steps), dtype=torch.float32, device="cuda")
    st.rollout_batch(zero, want_final=False)                      # warm-up
    torch.cuda.synchronize()
    ts = []
    with ClockSampler(0) as clk:
        for _ in range(max(3, args.steps // 4)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = st.rollout_batch(zero, want_final=False, want_field=True)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    n = int(out["count"][0])
    field = out["field"][0, :n].cpu().numpy()
    t0 = time.perf_counter()
    ref = oracle.rollout(p, parts, xg, np.zeros(steps), capacity=cap, want_field=True)
    cpu_s = time.perf_counter() - t0
    err = float(np.abs(field[:, :2] - ref["field"][:, :2]).max())
    pairs = 0
    m = len(parts)
    for _ in range(steps):
        pairs += m * (2 * int(p["n_b"]) + 1)
        m += 2
        pairs += m * (m + int(p["n_b"]))
    ms = statistics.median(ts)
    print(json.dumps({
        "metric": "Biot-Savart pair-interactions/s", "value": pairs / (ms / 1e3),
        "unit": "pair-interactions/s", "n_gpus": 1, "steps": len(ts), "ms_per_step": ms,
        "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fixed plate at 45 deg, unit stream, disturbance pair 2c upstream, Gaussian core "
                               "0.05c, 200 steps (2 -> 402 particles), binary64, one rollout (one cluster of SMs)",
                   "pairs_per_run": pairs},
        "error_vs_fp64_oracle": {"max_position_difference": err, "particles": n},
        "cpu_baseline": {"value": pairs / cpu_s, "unit": "pair-interactions/s", "cores": 1, "kind": "oracle",
                         "sample": "the same 200-step run, FP64 C oracle, one thread, %.2f s" % cpu_s},
        "clocks": clk.summary()}), flush=True)


def replans_2000_particles(V, torch, n0: int, replans: int, per_launch_subset: int):
    """Replan latency at K = 1024 rollouts x H = 100 steps with ~2000-particle fields (n0 -> n0 +
    200), three MPPI iterations per replan: eager launches and one CUDA graph replayed, against the
    one-rollout-per-launch form. The latter issues K x H single-block launches per iteration on
    one stream, so its time is linear in K: it is timed on per_launch_subset rollouts and scaled."""
    K, Hh = 1024, 100
    p, field, xg0, _ = W.mppi_batch_inputs(0, K=1, H=1, n=n0)
    root = V.State(p, field, xg0, n0 + 2 * Hh, V.FP32)
    eps = [torch.tensor(W.mppi_noise(3000 + j, K, Hh, W.MPPI_SIGMA_U), device="cuda") for j in range(3)]
    mu = torch.zeros(Hh, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def replan(mu):
        for j in range(3):
            c = V.mppi_perturb(mu, eps[j])
            out = root.rollout_batch(c, want_final=False)
            mu = V.mppi_update(V.mppi_weights(out["costs"], LAMBDA), c)
        return mu

    for _ in range(2):
        replan(mu)
    torch.cuda.synchronize()
    lat = []
    for r in range(replans):
        flush.fill_(float(r))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        replan(mu)
        b.record()
        b.synchronize()
        lat.append(a.elapsed_time(b))
    mu_s = mu.clone()

    def body(hs):
        m = mu_s
        for j in range(3):
            c = V.mppi_perturb(m, eps[j])
            out = root.rollout_batch(c, want_final=False)
            m = V.mppi_update(V.mppi_weights(out["costs"], LAMBDA), c)
        mu_s.copy_(m)

    graph = graph_replans(V, V.lib(), torch.cuda.current_stream(), flush, replans, body, mu_s)
    del flush
    ks = per_launch_subset
    c = V.mppi_perturb(mu, eps[0])[:ks].contiguous()
    root.rollout_batch_per_launch(c[:2].contiguous())
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    pl = root.rollout_batch_per_launch(c)
    b.record()
    b.synchronize()
    per_launch_iter_ms = a.elapsed_time(b) * K / ks
    ref = root.rollout_batch(c, want_final=False)
    same = bool(torch.equal(ref["costs"], pl["costs"]))
    root.close()
    pairs_iter = pairs_per_rollout(n0, Hh) * K
    p50 = float(np.percentile(lat, 50))
    return {
        "workload": "K=1024 x H=100, fields %d -> %d particles, 3 MPPI iterations per replan" % (n0, n0 + 2 * Hh),
        "persistent": {"p50": p50, "p99": float(np.percentile(lat, 99)), "replans": len(lat),
                       "pairs_per_s": 3 * pairs_iter / (p50 / 1e3), "form": "eager launches",
                       "l2": "flushed between replans",
                       # 12 flops per pair interaction over the whole replan (the MPPI kernels
                       # between the rollout launches included), against the derived FP32 peak
                       "fp32_frac_of_replan": 3 * pairs_iter * FLOPS_PER_PAIR / (p50 / 1e3) / 1e12
                       / fp32_peak_tflops()},
        "persistent_graph": graph,
        "one_rollout_per_launch": {"replan_ms_scaled": 3 * per_launch_iter_ms,
                                   "timed_rollouts": ks, "scaled_to": K,
                                   "launches_per_iteration": K * Hh,
                                   "bitwise_equal_costs": same},
        "speedup_p50": 3 * per_launch_iter_ms / p50}


def run_replan2000(args):
    """The replan latency on ~2000-particle fields alone (see replans_2000_particles)."""
    import torch
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    build.build()
    with ClockSampler(0) as clk:
        r = replans_2000_particles(V, torch, args.n0, args.replans, args.per_launch_subset)
    print(json.dumps({"metric": "MPPI replan latency (3 iterations)", "unit": "ms",
                      "higher_is_better": False, **r, "clocks": clk.summary()}), flush=True)


def uneven_result(V, torch, R: int, steps: int, sample: int) -> dict:
    """Uneven batching: R rollouts with particle counts log-uniform in [64, 8192], H = 50,
    binary32, persistent launches (class launches side by side or one merged launch) with
    autotuned block and diagonal-unit sizes, the horizon replayed from a CUDA graph, L2 flushed
    between timed horizons; against one launch per rollout (timed on a systematic sample of the
    rollouts sorted by size and scaled to all of them: the launches are serial on one stream)."""
    Hh = 50
    counts = W.uneven_counts(0, R, 64, 8192)
    fields = [W.background_field(10_000 + i, int(n)) for i, n in enumerate(counts)]
    gliders = np.tile(np.array(W.GLIDER_X0), (R, 1))
    p = W.glider_params()
    controls = torch.tensor(W.mppi_noise(11, R, Hh, W.MPPI_SIGMA_U), device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    b = V.Batch(p, fields, gliders, Hh)
    b.tune(controls)
    out = b.rollout(controls, use_graph=True)
    torch.cuda.synchronize()
    b.status()
    times = []
    with ClockSampler(0) as clk:
        for j in range(steps):
            flush.fill_(float(j))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.rollout(controls, use_graph=True, out=out)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    b.status()
    schedule, modes = b.schedule(), b.tuned_modes()
    b.close()
    del flush
    pairs = sum(pairs_per_rollout(int(n), Hh) for n in counts)
    ms = float(np.median(times))
    # one launch per rollout, systematic sample
    order = np.argsort(counts)
    picked = order[len(order) // (2 * sample) :: max(1, len(order) // sample)][: sample]
    single_ms = []
    for i in picked:
        st = V.State(p, fields[i], gliders[i], int(counts[i]) + 2 * Hh, V.FP32)
        c = controls[i:i + 1].contiguous()
        st.rollout_batch(c, want_final=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st.rollout_batch(c, want_final=False)
        e1.record()
        e1.synchronize()
        single_ms.append(e0.elapsed_time(e1))
        st.close()
    per_launch_ms = float(np.sum(single_ms)) * R / len(picked)
    return {
        "metric": "Biot-Savart pair-interactions/s", "value": pairs / (ms / 1e3),
        "unit": "pair-interactions/s", "n_gpus": 1, "steps": steps, "ms_per_step": ms,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "uneven batch: %d rollouts, counts log-uniform in [64, 8192], H=50" % R,
                   "pairs_per_step": pairs, "max_count": int(counts.max()),
                   "schedule": schedule, "tuner_whole_batch_ms": modes, "graph": True,
                   "l2": "flushed between timed horizons (256 MB write outside the events)"},
        "one_launch_per_rollout": {"ms_scaled": per_launch_ms, "sampled_rollouts": int(len(picked)),
                                   "pairs_per_s": pairs / (per_launch_ms / 1e3)},
        "speedup": per_launch_ms / ms, "clocks": clk.summary()}


def run_uneven(args):
    """The uneven batch alone: 4096 rollouts by default."""
    import torch
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    build.build()
    print(json.dumps(uneven_result(V, torch, args.rollouts_uneven, args.steps, args.sample)), flush=True)


def run_clusters(args):
    """A few rollouts of large fields through vpm_rollout_batch, one block per rollout
    (VPM_ROLLOUT_CLUSTERS=0) against the automatic choice of a 2- or 4-CTA cluster per rollout;
    the same bits either way (checked here on the costs and final glider states)."""
    import torch
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    build.build()
    p = W.glider_params()
    Hh = args.cluster_horizon
    rows = []
    with ClockSampler(0) as clk:
        for case in args.cluster_cases:
            K, n = (int(x) for x in case.split("x"))
            st = V.State(p, W.background_field(5 + K, n), W.GLIDER_X0, n + 2 * Hh, V.FP32)
            c = torch.tensor(W.mppi_noise(2, K, Hh, W.MPPI_SIGMA_U), device="cuda")
            row, outs = {"K": K, "n": n}, {}
            for mode in ("0", "1"):
                os.environ["VPM_ROLLOUT_CLUSTERS"] = mode
                outs[mode] = st.rollout_batch(c)
                torch.cuda.synchronize()
                ts = []
                for _ in range(max(1, args.steps)):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    st.rollout_batch(c)
                    e1.record()
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                row["one_block_ms" if mode == "0" else "auto_ms"] = float(np.median(ts))
            os.environ.pop("VPM_ROLLOUT_CLUSTERS", None)
            row["same_bits"] = all(torch.equal(outs["0"][k], outs["1"][k]) for k in outs["0"])
            rows.append(row)
            st.close()
    print(json.dumps({"workload": "vpm_rollout_batch, few rollouts of large fields, H=%d, binary32, "
                                  "Vatistas core 0.05c" % Hh, "cases": rows, "clocks": clk.summary()}),
          flush=True)


SERVE_H = 100
SERVE_MAX_WAIT_MS = 4000.0   # least-work-first admission: a request queued this long goes first
SERVE_SMALL_ROLLOUTS = 256   # and requests of up to this many rollouts take the high-priority lane


def serving_setup(V):
    """The serving workload's 16 scenarios (500-5000 particles, merging caps growth at n + 300)
    and its noise per request size K in {256, 1024, 4096}."""
    fields = W.serving_scenarios(0)
    noise = {k: [W.mppi_noise(100 + 7 * j + k, k, SERVE_H, W.MPPI_SIGMA_U) for j in range(3)]
             for k in (256, 1024, 4096)}
    return fields, noise


def serve_trace(V, fields, noise, arrivals, streams, sizes, slots, policy=0, max_wait_ms=0.0,
                small_rollouts=0):
    """Replays an arrival trace in real time against a server with `slots` requests in flight
    (16: continuous batching; 1: the plain per-request form) and the given admission policy.
    Each request first advances its scenario by 2 steps, then replans with K = sizes[j] rollouts
    over SERVE_H steps."""
    srv = V.Server(max_inflight=slots, max_rollouts=4096, max_horizon=SERVE_H, policy=policy,
                   max_wait_ms=max_wait_ms, small_rollouts=small_rollouts)
    for f in fields:
        p = W.glider_params(n_wake_max=len(f) + 300)
        srv.add_scenario(p, f, W.GLIDER_X0, len(f) + 300 + 2 * SERVE_H + 8)
    tickets, t0 = [], time.perf_counter()
    for j, (ta, sc) in enumerate(zip(arrivals, streams)):
        dt = ta - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        k = int(sizes[j])
        tickets.append(srv.submit(int(sc), noise[k][j % 3], advance_steps=2, advance_u=0.0))
    lat, done_k, superseded = [], 0, 0
    for tk in tickets:
        r = srv.poll(tk)
        if r[0]["status"] == V.VPM_OK:
            lat.append(r[0]["t_done_ms"] - r[0]["t_submit_ms"])
            done_k += r[0]["K"]
        else:
            superseded += 1
    wall = time.perf_counter() - t0
    srv.close()
    return {"offered": int(len(arrivals)), "completed": len(lat), "superseded": superseded,
            "p50_ms": float(np.percentile(lat, 50)) if lat else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat else None,
            "rollouts_per_s": done_k / wall, "wall_s": wall}


def serving_at_rates(V, rates, seconds):
    """Continuous batching (arrival order, and least estimated work first with a 4 s bound on
    waiting and a high-priority lane for requests of up to 256 rollouts) against the per-request form at total request rates around one GPU's capacity (same
    scenarios, request mix and arrival seeds as the sweep of --workload serving)."""
    fields, noise = serving_setup(V)
    out = []
    for rate in rates:
        arr, strm = W.poisson_arrivals(11, rate / len(fields), seconds, len(fields))
        ks = W.request_sizes(12, len(arr))
        out.append({"offered_hz": rate,
                    "continuous": serve_trace(V, fields, noise, arr, strm, ks, 16),
                    "continuous_least_work": serve_trace(V, fields, noise, arr, strm, ks, 16,
                                                         V.ADMIT_LEAST_WORK, SERVE_MAX_WAIT_MS,
                                                         SERVE_SMALL_ROLLOUTS),
                    "per_request": serve_trace(V, fields, noise, arr, strm, ks, 1)})
    return out


def run_serving(args):
    """Serving: 16 scenarios with resident fields of 500-5000 particles (merging caps growth
    at n + 300), replanning requests arriving as Poisson streams at 50 Hz each, K drawn from
    {256, 1024, 4096}, H = 100, each request first advancing its scenario by 2 steps. The
    arrival trace is replayed in real time against the continuous-batching server (16 slots)
    and then against the plain per-request form (1 slot). The offered load is far above one
    GPU's capacity, so a newer request for a scenario supersedes its queued one."""
    import torch
    import paper_2509_16079_b300 as V
    from paper_2509_16079_b300 import build
    build.build()
    T = args.serve_seconds
    fields, noise = serving_setup(V)
    arrivals, streams = W.poisson_arrivals(1, 50.0, T, len(fields))
    sizes = W.request_sizes(2, len(arrivals))
    out = {"metric": "MPPI replan latency under load", "unit": "ms", "higher_is_better": False,
           "config": {"workload": "serving: 16 scenarios, 500-5000 particles, Poisson 50 Hz each, "
                                  "K in {256, 1024, 4096}, H=100", "seconds": T,
                      "offered_requests": int(len(arrivals))}}
    pol = (V.ADMIT_LEAST_WORK, SERVE_MAX_WAIT_MS, SERVE_SMALL_ROLLOUTS) if args.serve_policy == "least_work" \
        else (V.ADMIT_ARRIVAL, 0.0, 0)
    out["config"]["policy"] = args.serve_policy
    out["continuous"] = serve_trace(V, fields, noise, arrivals, streams, sizes, 16, *pol)
    out["per_request"] = serve_trace(V, fields, noise, arrivals, streams, sizes, 1)
    # sustainable-rate sweep: the same scenarios and request mix at total rates around one GPU's
    # capacity (a request averages ~1.7e12 pair interactions, ~0.5 s of the device); a rate is
    # sustained when no request is superseded and the p99 latency stays within twice the p99
    # at the lowest rate
    sweep, base_p99, sustained = [], None, None
    for rate in args.serve_rates:
        arr, strm = W.poisson_arrivals(11, rate / len(fields), args.serve_sweep_seconds, len(fields))
        ks = W.request_sizes(12, len(arr))
        r = serve_trace(V, fields, noise, arr, strm, ks, 16, *pol)
        p99 = r["p99_ms"]
        if base_p99 is None:
            base_p99 = p99
        ok = r["superseded"] == 0 and p99 is not None and base_p99 is not None and p99 <= 2.0 * base_p99
        if ok:
            sustained = rate
        sweep.append({"offered_hz": rate, "offered": r["offered"], "completed": r["completed"],
                      "superseded": r["superseded"], "p50_ms": r["p50_ms"], "p99_ms": p99,
                      "rollouts_per_s": r["rollouts_per_s"], "sustained": ok})
    out["rate_sweep"] = sweep
    out["sustainable_rate_hz"] = sustained
    print(json.dumps(out), flush=True)

# ------------------------------------------------------------------ reference arm (oracle)
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(8, os.cpu_count() or 1)      # one rollout per host core
    vals = []
    t_all = 0.0
    for j in range(args.warmup + args.steps):
        cb, _ = cpu_baseline(rollouts=per_step)
        if j >= args.warmup:
            vals.append(cb["value"])
            t_all += pairs_per_rollout(N0, H) * per_step / cb["value"]
    value = pairs_per_rollout(N0, H) * per_step * args.steps / t_all
    line = {
        "impl": "reference",
        "metric": "Biot-Savart pair-interactions/s",
        "value": value,
        "unit": "pair-interactions/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_all / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "MPPI batch: K=1024 rollouts x H=100 steps, dt=0.01, root field 1000 "
                               "particles growing to 1200, Vatistas core 0.05c, one MPPI iteration per step",
                   "sample_per_step": "%d rollouts of the 1024" % per_step},
        "cpu_baseline": {"value": value, "unit": "pair-interactions/s",
                         "cores": min(os.cpu_count() or 1, per_step), "kind": "oracle",
                         "sample": "%d rollouts per step (FP64 C oracle on host threads)" % per_step},
        "e2e": {"value": value, "unit": "pair-interactions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--replans", type=int, default=200)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", action="store_true",
                    help="small case for profilers: K rollouts x --horizon steps, one timed iteration")
    ap.add_argument("--horizon", type=int, default=H)
    ap.add_argument("--workload", default="mppi", choices=["mppi", "freefield", "replan2000", "uneven", "serving", "alu", "table1", "policy", "nmpc", "plate", "clusters"])
    ap.add_argument("--cluster-cases", nargs="*", default=["1x8000", "8x6000", "32x8000", "64x6000", "74x4000", "128x4000"],
                    help="K x field-size cases of the clusters workload")
    ap.add_argument("--cluster-horizon", type=int, default=50)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[0.5, 1.0, 1.5, 2.0, 3.0],
                    help="total request rates (Hz) of the serving workload's sustainable-rate sweep")
    ap.add_argument("--serve-sweep-seconds", type=float, default=12.0)
    ap.add_argument("--serve-policy", default="arrival", choices=["arrival", "least_work"],
                    help="admission of the continuous-batching server in --workload serving")
    ap.add_argument("--rollouts-uneven", type=int, default=4096)
    ap.add_argument("--sample", type=int, default=64, help="rollouts timed one launch each (uneven)")
    ap.add_argument("--n", type=int, default=1 << 20, help="free-field particle count")
    ap.add_argument("--ff-steps", type=int, default=10)
    ap.add_argument("--ff-line-steps", type=int, default=2,
                    help="Heun steps of the free-field entry in the default line (0: leave it out)")
    ap.add_argument("--uneven-line-steps", type=int, default=5,
                    help="timed horizons of the uneven-batch entry in the default line (0: leave it out)")
    ap.add_argument("--n0", type=int, default=1900, help="root field size of the ~2000-particle replans")
    ap.add_argument("--per-launch-subset", type=int, default=16)
    ap.add_argument("--replan2000-replans", type=int, default=200,
                    help="replans of ~2000-particle fields timed in the main line (0: skip)")
    ap.add_argument("--rollouts", type=int, default=K_ROLL)
    ap.add_argument("--profile-n0", type=int, default=N0, help="root field size of --profile-case")
    ap.add_argument("--serve-line-seconds", type=float, default=8.0,
                    help="seconds of arrivals per serving run in the main line (0: skip)")
    ap.add_argument("--serve-line-rates", type=float, nargs="*", default=[1.5, 4.0],
                    help="total request rates (Hz) of the main line's serving runs")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_case:
        run_profile_case(args)
    elif args.workload == "freefield":
        run_freefield(args)
    elif args.workload == "replan2000":
        run_replan2000(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "alu":
        run_alu(args)
    elif args.workload == "table1":
        run_table1(args)
    elif args.workload == "policy":
        run_policy(args)
    elif args.workload == "nmpc":
        run_nmpc(args)
    elif args.workload == "clusters":
        run_clusters(args)
    elif args.workload == "plate":
        run_plate(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
