"""Helpers shared by the GPU parity tests (comparison metrics and state transfer).

Tolerances (binary32 path), fixed by the workload definition:
  per-step velocities      normwise relative error <= 1e-5
                           (max_i |v_gpu - v_ref| / max_i |v_ref|)
  100-step positions       max_i |r_gpu - r_ref| <= 1e-4 chord
  MPPI weights             max_i |w_gpu - w_ref| <= 1e-5 (weights sum to 1)
"""
import numpy as np
import pytest

VEL_TOL = 1e-5
POS_TOL = 1e-4
W_TOL = 1e-5


def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2509_16079_b300 import build
    build.build()
    import paper_2509_16079_b300 as V
    V.lib()
    return torch, V


def normwise(a, ref):
    a = np.asarray(a, dtype=np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    if len(ref) == 0:
        return 0.0
    den = np.linalg.norm(ref, axis=1).max()
    num = np.linalg.norm(a - ref, axis=1).max()
    return num / den if den > 0 else num


def snapshot(s):
    """Copy of an oracle State's full content."""
    return dict(parts=s.particles.copy(), xg=s.xg.copy(), gb=s.gb_prev.copy(),
                glev=s.glev_prev, hp=s.has_prev)


def gpu_state(V, params, snap, capacity, precision):
    st = V.State(params, snap["parts"], snap["xg"], capacity, precision)
    st.set_history(snap["gb"], snap["glev"], bool(snap["hp"]))
    return st


def oracle_state(ora, params, snap, capacity):
    return ora.State(params, snap["parts"], snap["xg"], capacity, snap["gb"], snap["glev"],
                     snap["hp"])
