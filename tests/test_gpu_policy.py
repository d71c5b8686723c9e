"""Tracking policy of §IV-B on the GPU (least-squares Jacobians, TVLQR) against the FP64
oracle: on shared unstructured inputs, and end to end from rollouts of perturbed initial
states and controls (binary64 rollouts on both sides)."""
import numpy as np
import pytest

import workloads as W
from oracle import policy as OP
from tests.gpu_common import cuda

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_ls_matches_oracle_on_shared_inputs():
    torch, V = cuda()
    x0, traj, u, xbar, ubar = W.policy_random_data(3, 300, 24)
    A, B, info = V.ls_jacobians(*(torch.tensor(a, device="cuda") for a in (x0, traj, u, xbar, ubar)), 0.01)
    Ar, Br = OP.ls_jacobians(x0, traj, u.astype(np.float64), xbar, ubar.astype(np.float64), 0.01)
    assert not info.any()
    assert _rel(A.cpu().numpy(), Ar) <= 1e-10 and _rel(B.cpu().numpy(), Br) <= 1e-10


def test_ls_flags_singular_steps():
    torch, V = cuda()
    x0, traj, u, xbar, ubar = W.policy_random_data(4, 8, 3)
    u[:, 1] = ubar[1]                        # no control variation at step 1
    A, B, info = V.ls_jacobians(*(torch.tensor(a, device="cuda") for a in (x0, traj, u, xbar, ubar)), 0.01)
    assert info.tolist() == [0, 1, 0]
    assert torch.isnan(A[1]).all() and torch.isfinite(A[0]).all() and torch.isfinite(A[2]).all()
    with pytest.raises(V.VpmError):
        V.ls_jacobians(*(torch.tensor(a[:5], device="cuda") for a in (x0, traj, u)),
                       torch.tensor(xbar, device="cuda"), torch.tensor(ubar, device="cuda"), 0.01)


def test_tvlqr_matches_oracle():
    torch, V = cuda()
    rng = np.random.default_rng(9)
    H = 80
    Ah = rng.normal(0.0, 2.0, (H, 3, 5))
    Bh = rng.normal(0.0, 2.0, (H, 3))
    g, s0 = V.tvlqr(torch.tensor(Ah, device="cuda"), torch.tensor(Bh, device="cuda"), 0.01,
                    W.TVLQR_QC, W.TVLQR_QF, W.TVLQR_RC)
    gr, Sr = OP.tvlqr(Ah, Bh, 0.01, W.TVLQR_QC, W.TVLQR_QF, W.TVLQR_RC)
    assert _rel(g.cpu().numpy(), gr) <= 1e-11
    assert _rel(s0.cpu().numpy(), Sr[0]) <= 1e-11
    with pytest.raises(V.VpmError):
        V.tvlqr(torch.tensor(Ah, device="cuda"), torch.tensor(Bh, device="cuda"), 0.01,
                W.TVLQR_QC, W.TVLQR_QF, 0.0)


def test_policy_from_rollouts_end_to_end(ora):
    """Nominal rollout, K perturbed rollouts (initial state and controls), least squares and
    TVLQR: GPU (binary64 rollouts) against the oracle run on its own rollouts."""
    torch, V = cuda()
    p = W.glider_params()
    field = W.background_field(21, 120)
    K, H = 48, 30
    ubar = W.mppi_noise(22, 1, H, 2.0)[0]
    x0, u = W.policy_samples(23, K, W.GLIDER_X0, ubar)
    cap = len(field) + 2 * H
    # oracle
    nom = ora.rollout(p, field, np.array(W.GLIDER_X0), ubar.astype(np.float64), want_traj=True)
    xbar_r = np.vstack([W.GLIDER_X0, nom["traj"]])
    traj_r = np.stack([ora.rollout(p, field, x0[i], u[i].astype(np.float64), want_traj=True)["traj"]
                       for i in range(K)])
    Ar, Br = OP.ls_jacobians(x0, traj_r, u.astype(np.float64), xbar_r, ubar.astype(np.float64), p["dt"])
    gr, Sr = OP.tvlqr(Ar, Br, p["dt"], W.TVLQR_QC, W.TVLQR_QF, W.TVLQR_RC)
    # GPU
    st = V.State(p, field, W.GLIDER_X0, cap, V.FP64)
    nom_g = st.rollout_batch(torch.tensor(ubar[None, :], device="cuda"), want_traj=True)
    xbar = torch.cat([torch.tensor([W.GLIDER_X0], dtype=torch.float64, device="cuda"), nom_g["traj"][0]])
    out = st.rollout_batch(torch.tensor(u, device="cuda"), want_traj=True,
                           x0=torch.tensor(x0, device="cuda"))
    A, B, info = V.ls_jacobians(torch.tensor(x0, device="cuda"), out["traj"], torch.tensor(u, device="cuda"),
                                xbar, torch.tensor(ubar, device="cuda"), p["dt"])
    g, s0 = V.tvlqr(A, B, p["dt"], W.TVLQR_QC, W.TVLQR_QF, W.TVLQR_RC)
    torch.cuda.synchronize()
    st.close()
    assert not info.any()
    assert np.abs(out["traj"].cpu().numpy() - traj_r).max() <= 1e-9
    assert _rel(A.cpu().numpy(), Ar) <= 1e-6 and _rel(B.cpu().numpy(), Br) <= 1e-6
    assert _rel(g.cpu().numpy(), gr) <= 1e-6
