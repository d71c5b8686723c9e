"""Parity of the free-field velocity and Heun kernels and of the MPPI kernels against the FP64
oracle."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import POS_TOL, VEL_TOL, W_TOL, cuda, normwise

pytestmark = pytest.mark.gpu


def _dev_particles(torch, P):
    a = np.zeros((len(P), 4), np.float32)
    a[:, :3] = P
    return torch.tensor(a, device="cuda")


@pytest.mark.parametrize("kernel", [0, 1, 2])
@pytest.mark.parametrize("n", [0, 1, 2, 511, 512, 513, 1023, 1024, 1025, 1500, 2049, 4097])
def test_freefield_velocity(ora, kernel, n):
    torch, V = cuda()
    P = W.background_field(n, n)
    if kernel == 0:
        P[:, 2] *= 1e-2  # keep the singular kernel's close pairs moderate
    d = _dev_particles(torch, P)
    v = V.freefield_velocity(d, kernel, 0.05).cpu().numpy()
    # the oracle sees the binary32 positions the kernel sees
    Pf = d[:, :3].double().cpu().numpy()
    ref = ora.free_velocity(Pf, kernel, 0.05)
    if n:
        assert normwise(v, ref) <= VEL_TOL


@pytest.mark.parametrize("n", [1 << 20, 1 << 22])
def test_freefield_large_sampled(ora, n):
    """2^20 and 2^22 blob-field particles (core 1e-3): 256 sampled targets against all sources.
    The scratch is 32 bytes per particle (134 MB at 2^22)."""
    torch, V = cuda()
    P = W.blob_field(0, n, gamma_std=1e-3)
    d = _dev_particles(torch, P)
    v = V.freefield_velocity(d, 1, 1e-3).cpu().numpy()
    Pf = d[:, :3].double().cpu().numpy()
    idx = W.sample_indices(1, n, 256)
    ref = ora.velocity_at(Pf, Pf[idx, :2], 1, 1e-3, skip=idx)
    assert normwise(v[idx], ref) <= VEL_TOL


def test_freefield_velocity_is_deterministic():
    """The CTAs add their partial sums into the exact accumulators in whatever order they run;
    integer addition makes the result the same bits every time."""
    torch, V = cuda()
    d = _dev_particles(torch, W.blob_field(2, 300000, gamma_std=1e-3))
    a = V.freefield_velocity(d, 1, 1e-3)
    for _ in range(3):
        assert torch.equal(V.freefield_velocity(d, 1, 1e-3), a)


def test_freefield_heun(ora):
    torch, V = cuda()
    P = W.background_field(3, 1500)
    d = _dev_particles(torch, P)
    Pf = d[:, :3].double().cpu().numpy()
    V.freefield_heun(d, 1, 0.05, 0.01, 20)
    ref = ora.free_heun(Pf, 1, 0.05, 0.01, 20)
    got = d[:, :2].double().cpu().numpy()
    assert np.abs(got - ref[:, :2]).max() <= POS_TOL


@pytest.mark.parametrize("K", [1, 2, 37, 1024, 4096, 5000])
def test_mppi_weights(ora, K):
    torch, V = cuda()
    J = W.costs_synthetic(K, K)
    Jd = torch.tensor(J, device="cuda")
    for lam in (1.0, 10.0, float(np.median(np.abs(J - J.min()))) or 1.0):
        w = V.mppi_weights(Jd, lam).cpu().numpy()
        ref = ora.mppi_weights(J.astype(np.float64), float(np.float32(lam)))
        assert np.abs(w - ref).max() <= W_TOL
        assert abs(w.astype(np.float64).sum() - 1.0) <= 1e-5


@pytest.mark.parametrize("K", [5, 1024, 5000])
def test_mppi_weights_with_diverged_rollouts(ora, K):
    """Costs that are NaN (a diverged rollout) or infinite get weight 0 on both sides; the
    others match the oracle; with no finite cost every weight is NaN."""
    torch, V = cuda()
    J = W.costs_synthetic(K + 7, K)
    rng = np.random.default_rng(K)
    bad = rng.choice(K, size=max(2, K // 50), replace=False)
    J[bad[0::3]] = np.nan
    J[bad[1::3]] = np.inf
    J[bad[2::3]] = -np.inf
    w = V.mppi_weights(torch.tensor(J, device="cuda"), 10.0).cpu().numpy()
    ref = ora.mppi_weights(J.astype(np.float64), 10.0)
    assert np.all(w[bad] == 0.0) and np.all(ref[bad] == 0.0)
    assert np.abs(w - ref).max() <= W_TOL
    assert abs(w.astype(np.float64).sum() - 1.0) <= 1e-5
    none = np.full(K, np.nan, np.float32)
    none[: K // 2] = np.inf
    assert np.isnan(V.mppi_weights(torch.tensor(none, device="cuda"), 10.0).cpu().numpy()).all()


@pytest.mark.parametrize("K,H", [(1, 1), (16, 100), (1024, 100), (4096, 37)])
def test_mppi_update_and_perturb(ora, K, H):
    torch, V = cuda()
    rng = np.random.default_rng(K + H)
    w = rng.random(K).astype(np.float32)
    w /= w.sum()
    mu = rng.normal(size=H).astype(np.float32)
    eps = W.mppi_noise(K, K, H, 10.0)
    c = V.mppi_perturb(torch.tensor(mu, device="cuda"), torch.tensor(eps, device="cuda"))
    assert np.array_equal(c.cpu().numpy(), mu[None, :] + eps)
    m = V.mppi_update(torch.tensor(w, device="cuda"), c).cpu().numpy()
    ref = ora.mppi_update(w.astype(np.float64), (mu[None, :] + eps).astype(np.float64))
    assert np.abs(m - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())
