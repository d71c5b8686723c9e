"""Python binding of the B300 VPM rollout library (libvpm.so, C ABI in include/vpm.h).

The binding only marshals arguments: every step of the model runs in the library's CUDA
kernels. PyTorch provides device memory (tensors) and streams (the current stream of the
current device). If libvpm.so is missing, the first call raises; there is no CPU fallback.

Build the library with `python -m paper_2509_16079_b300.build`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# VPM_DEBUG_BOUNDS=1 selects the build with device-side bounds checks (build.py --debug-bounds)
LIB_PATH = os.path.join(_HERE, "libvpm_debug.so" if os.environ.get("VPM_DEBUG_BOUNDS") == "1"
                        else "libvpm.so")

VPM_OK, VPM_ERR_INVALID, VPM_ERR_OOM, VPM_ERR_CAPACITY, VPM_ERR_NONFINITE, VPM_ERR_TIMEOUT, \
    VPM_ERR_CUDA, VPM_ERR_BUSY, VPM_ERR_SINGULAR = range(9)
KERNEL_SINGULAR, KERNEL_VATISTAS, KERNEL_GAUSSIAN = 0, 1, 2
FP32, FP64 = 0, 1
GATE_OFF, GATE_BOTH, GATE_LEV = 0, 1, 2
N_B_MAX = 32

_STATUS_NAMES = {0: "VPM_OK", 1: "VPM_ERR_INVALID", 2: "VPM_ERR_OOM", 3: "VPM_ERR_CAPACITY",
                 4: "VPM_ERR_NONFINITE", 5: "VPM_ERR_TIMEOUT", 6: "VPM_ERR_CUDA",
                 7: "VPM_ERR_BUSY", 8: "VPM_ERR_SINGULAR"}


class VpmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class Params(C.Structure):
    """Mirror of vpm_params."""
    _fields_ = [
        ("n_b", C.c_int), ("chord", C.c_double), ("span", C.c_double), ("rho", C.c_double),
        ("wake_kernel", C.c_int), ("r_core", C.c_double), ("shed_offset", C.c_double),
        ("gamma_decay", C.c_double), ("shed_gate", C.c_int), ("alpha_crit", C.c_double),
        ("n_wake_max", C.c_int), ("u_inf", C.c_double * 2), ("dt", C.c_double),
        ("fixed_plate", C.c_int), ("mass", C.c_double), ("inertia", C.c_double),
        ("g", C.c_double), ("l", C.c_double), ("l_w", C.c_double), ("l_e", C.c_double),
        ("s_e", C.c_double), ("q", C.c_double * 7), ("x_d", C.c_double * 7),
        ("precision", C.c_int),
    ]


def make_params(d: dict, precision: int = FP32) -> Params:
    p = Params()
    for k in ("n_b", "wake_kernel", "shed_gate", "n_wake_max", "fixed_plate"):
        setattr(p, k, int(d[k]))
    for k in ("chord", "span", "rho", "r_core", "shed_offset", "gamma_decay", "alpha_crit",
              "dt", "mass", "inertia", "g", "l", "l_w", "l_e", "s_e"):
        setattr(p, k, float(d[k]))
    p.u_inf[0], p.u_inf[1] = (float(v) for v in d["u_inf"])
    for i in range(7):
        p.q[i] = float(d["q"][i])
        p.x_d[i] = float(d["x_d"][i])
    p.precision = int(precision)
    return p


_VP, _I, _D, _F = C.c_void_p, C.c_int, C.c_double, C.c_float
_SIGNATURES = {
    "vpm_last_error": ([], C.c_char_p),
    "vpm_version": ([], C.c_char_p),
    "vpm_state_create": ([C.POINTER(Params), _VP, _I, _I, _VP, C.POINTER(_VP), _VP], _I),
    "vpm_state_destroy": ([_VP], _I),
    "vpm_state_set_history": ([_VP, _VP, _D, _I, _VP], _I),
    "vpm_state_read": ([_VP, _VP, C.POINTER(_I), _VP, _VP, _VP], _I),
    "vpm_state_status": ([_VP, _VP], _I),
    "vpm_state_save": ([_VP, _VP, C.POINTER(C.c_size_t), _VP], _I),
    "vpm_state_load": ([_VP, _VP, C.c_size_t, _VP], _I),
    "vpm_step": ([_VP, _D, _VP, _VP, _VP, _VP, _VP], _I),
    "vpm_rollout_batch": ([_VP, _I, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _I),
    "vpm_rollout_scratch_bytes": ([_VP, _I, _I, C.POINTER(C.c_size_t)], _I),
    "vpm_rollout_scratch_bytes_cap": ([_I, _I, _I, C.POINTER(C.c_size_t)], _I),
    "vpm_rollout_scratch_slot": ([_I, _I, _I, _I, C.POINTER(C.c_longlong)], _I),
    "vpm_rollout_batch_x0": ([_VP, _I, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _I),
    "vpm_state_set_glider": ([_VP, _VP, _VP], _I),
    "vpm_state_inject_pair": ([_VP, _VP, _VP], _I),
    "vpm_state_disturbance": ([_VP, C.POINTER(_I), _VP], _I),
    "vpm_state_get_glider": ([_VP, _VP, _VP], _I),
    "vpm_state_copy": ([_VP, _VP, _VP], _I),
    "vpm_state_advance_policy": ([_VP, _I, _VP, _VP, _VP, _I, _VP], _I),
    "vpm_rollout_batch_policy": ([_VP, _I, _I, _VP, _VP, _VP, _VP, _I, _VP, _VP, _VP, _VP, _VP], _I),
    "vpm_nmpc_create": ([_VP, _VP, _VP, _I, _I, _VP, _VP, _I, _VP, _VP, _VP, C.POINTER(_VP)], _I),
    "vpm_nmpc_control": ([_VP, _I, _VP, C.POINTER(_D)], _I),
    "vpm_nmpc_inject_pair": ([_VP, _VP], _I),
    "vpm_nmpc_policy": ([_VP, C.POINTER(_I), _VP, _VP, _VP], _I),
    "vpm_nmpc_stats": ([_VP, C.POINTER(_I), C.POINTER(_I), C.POINTER(_D), C.POINTER(_D)], _I),
    "vpm_nmpc_destroy": ([_VP], _I),
    "vpm_ls_jacobians": ([_I, _I, _D, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _I),
    "vpm_tvlqr": ([_I, _D, _VP, _VP, _VP, _VP, _D, _VP, _VP, _VP], _I),
    "vpm_rollout_batch_per_launch": ([_VP, _I, _I, _VP, _VP, _VP, _VP], _I),
    "mppi_weights": ([_VP, _I, _F, _VP, _VP], _I),
    "mppi_update": ([_VP, _VP, _I, _I, _VP, _VP], _I),
    "mppi_perturb": ([_VP, _VP, _I, _I, _VP, _VP], _I),
    "vpm_freefield_velocity": ([_VP, _I, _I, _D, _VP, _VP], _I),
    "vpm_freefield_scratch_bytes": ([_I, C.POINTER(C.c_size_t)], _I),
    "vpm_freefield_heun": ([_VP, _I, _I, _D, _D, _I, _VP], _I),
    "vpm_freefield_heun_noalloc": ([_VP, _I, _I, _D, _D, _I, _VP], _I),
    "vpm_fixed_sum": ([_VP, _I, _I, C.POINTER(_D), C.POINTER(_I)], _I),
    "vpm_pool_trim": ([C.POINTER(C.c_size_t)], _I),
    "vpm_fixed_exponent": ([C.c_float, _I, _I, _D, C.POINTER(_I)], _I),
    "vpm_probe_rate": ([_I, _I, C.POINTER(_D)], _I),
    "vpm_batch_create": ([C.POINTER(Params), _I, _VP, _VP, _VP, _I, C.POINTER(_VP), _VP], _I),
    "vpm_batch_destroy": ([_VP], _I),
    "vpm_batch_rollout": ([_VP, _I, _VP, _VP, _VP, _VP, _I, _VP], _I),
    "vpm_batch_tune": ([_VP, _I, _VP, _VP], _I),
    "vpm_batch_set_schedule": ([_VP, _I, _I, _I, _I], _I),
    "vpm_batch_set_ctas": ([_VP, _I, _I, _I], _I),
    "vpm_batch_tuned_modes": ([_VP, C.POINTER(_F), C.POINTER(_F)], _I),
    "vpm_batch_schedule": ([_VP, C.POINTER(_I), _VP, _VP, _VP, _VP, _VP, _VP, C.POINTER(_I)], _I),
    "vpm_batch_status": ([_VP, _VP], _I),
    "vpm_server_create": ([_VP, C.POINTER(_VP)], _I),
    "vpm_server_add_scenario": ([_VP, C.POINTER(Params), _VP, _I, _I, _VP, C.POINTER(_I)], _I),
    "vpm_server_submit": ([_VP, _I, _I, _I, _VP, _VP, _F, _I, _F, C.POINTER(C.c_longlong)], _I),
    "vpm_server_poll": ([_VP, C.c_longlong, _I, _VP, _VP], _I),
    "vpm_server_request_bytes": ([_VP, _I, _I, _I, _I, C.POINTER(C.c_size_t)], _I),
    "vpm_server_stats": ([_VP, C.POINTER(C.c_longlong), C.POINTER(_I), C.POINTER(_I),
                          C.POINTER(C.c_size_t)], _I),
    "vpm_server_read_scenario": ([_VP, _I, _VP, C.POINTER(_I), _VP], _I),
    "vpm_server_destroy": ([_VP], _I),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded libvpm.so (raises ImportError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libvpm.so is not built (run python -m paper_2509_16079_b300.build)")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def check(status: int):
    """Raises VpmError carrying vpm_last_error() for a non-zero status."""
    if status != VPM_OK:
        raise VpmError(status, lib().vpm_last_error().decode())


def stream_handle(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev_tensor(t, dtype, shape=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor of %s" % dtype)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, tuple(t.shape)))
    return t


class State:
    """A resident model (glider + wake) on the current CUDA device."""

    def __init__(self, params: dict, particles, glider7, capacity: int, precision: int = FP32,
                 stream=None):
        self.params = dict(params)
        self.precision = precision
        self._P = make_params(params, precision)
        parts = np.ascontiguousarray(np.asarray(particles, dtype=np.float64).reshape(-1, 3))
        xg = np.ascontiguousarray(np.asarray(glider7, dtype=np.float64))
        self.capacity = int(capacity)
        h = C.c_void_p()
        check(lib().vpm_state_create(C.byref(self._P), parts.ctypes.data_as(_VP), len(parts),
                                     self.capacity, xg.ctypes.data_as(_VP), C.byref(h),
                                     stream_handle(stream)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().vpm_state_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_history(self, gb_prev, glev_prev: float, has_prev: bool, stream=None):
        gb = np.ascontiguousarray(np.asarray(gb_prev, dtype=np.float64))
        check(lib().vpm_state_set_history(self._h, gb.ctypes.data_as(_VP), float(glev_prev),
                                          int(has_prev), stream_handle(stream)))

    def read(self, stream=None):
        """Returns (particles (n, 3) float64, glider (7,), hist (n_b + 2,))."""
        parts = np.zeros((self.capacity, 3))
        xg = np.zeros(7)
        hist = np.zeros(int(self.params["n_b"]) + 2)
        n = C.c_int()
        check(lib().vpm_state_read(self._h, parts.ctypes.data_as(_VP), C.byref(n),
                                   xg.ctypes.data_as(_VP), hist.ctypes.data_as(_VP),
                                   stream_handle(stream)))
        return parts[:n.value].copy(), xg, hist

    def status(self, stream=None):
        check(lib().vpm_state_status(self._h, stream_handle(stream)))

    def glider(self, stream=None) -> np.ndarray:
        xg = np.zeros(7)
        check(lib().vpm_state_get_glider(self._h, xg.ctypes.data_as(_VP), stream_handle(stream)))
        return xg

    def set_glider(self, x7, stream=None):
        xg = np.ascontiguousarray(np.asarray(x7, dtype=np.float64))
        check(lib().vpm_state_set_glider(self._h, xg.ctypes.data_as(_VP), stream_handle(stream)))

    def inject_pair(self, x1, z1, g1, x2, z2, g2, stream=None):
        """Disturbance pair in front of the wake (see vpm_state_inject_pair)."""
        a = np.array([x1, z1, g1, x2, z2, g2], dtype=np.float64)
        check(lib().vpm_state_inject_pair(self._h, a.ctypes.data_as(_VP), stream_handle(stream)))

    def disturbance(self, stream=None) -> int:
        v = C.c_int()
        check(lib().vpm_state_disturbance(self._h, C.byref(v), stream_handle(stream)))
        return v.value

    def copy_from(self, other: "State", stream=None):
        check(lib().vpm_state_copy(self._h, other._h, stream_handle(stream)))

    def advance_policy(self, steps: int, gains, xbar, ubar, offset: int, stream=None):
        """In-place closed-loop steps under a tracking policy (device tensors, absolute index)."""
        import torch
        gains, xbar = _dev_tensor(gains, torch.float64), _dev_tensor(xbar, torch.float64)
        ubar = _dev_tensor(ubar, torch.float32)
        check(lib().vpm_state_advance_policy(self._h, int(steps), ptr(gains), ptr(xbar), ptr(ubar),
                                             int(offset), stream_handle(stream)))

    def rollout_policy(self, K: int, H: int, gains, xbar, ubar, offset: int = 0, x0=None,
                       controls=None, want_traj: bool = False, stream=None):
        """K closed-loop rollouts under a tracking policy (see vpm_rollout_batch_policy)."""
        import torch
        gains, xbar = _dev_tensor(gains, torch.float64), _dev_tensor(xbar, torch.float64)
        ubar = _dev_tensor(ubar, torch.float32)
        dev = gains.device
        if x0 is not None:
            x0 = _dev_tensor(x0, torch.float64)
        if controls is not None:
            controls = _dev_tensor(controls, torch.float32)
        out = dict(costs=torch.empty(K, dtype=torch.float32, device=dev),
                   final_glider=torch.empty((K, 7), dtype=torch.float64, device=dev))
        if want_traj:
            out["traj"] = torch.empty((K, H, 7), dtype=torch.float64, device=dev)
        check(lib().vpm_rollout_batch_policy(self._h, int(K), int(H), ptr(x0), ptr(gains), ptr(xbar),
                                             ptr(ubar), int(offset), ptr(controls), ptr(out["costs"]),
                                             ptr(out["final_glider"]), ptr(out.get("traj")),
                                             stream_handle(stream)))
        return out

    def save(self, stream=None) -> bytes:
        size = C.c_size_t()
        check(lib().vpm_state_save(self._h, None, C.byref(size), stream_handle(stream)))
        buf = C.create_string_buffer(size.value)
        check(lib().vpm_state_save(self._h, C.cast(buf, _VP), C.byref(size), stream_handle(stream)))
        return buf.raw[:size.value]

    def load(self, blob: bytes, stream=None):
        buf = C.create_string_buffer(blob, len(blob))
        check(lib().vpm_state_load(self._h, C.cast(buf, _VP), len(blob), stream_handle(stream)))

    def step(self, u: float = 0.0, probe: bool = False, stream=None):
        """One committed step; with probe=True returns the step's quantities as tensors."""
        import torch
        out = {}
        if probe:
            nb = int(self.params["n_b"])
            dev = torch.device("cuda", torch.cuda.current_device())
            out = dict(fm=torch.zeros(3, dtype=torch.float64, device=dev),
                       gamma_s=torch.zeros(nb + 2, dtype=torch.float64, device=dev),
                       vel=torch.zeros(2 * self.capacity, dtype=torch.float64, device=dev),
                       vtilde=torch.zeros(2 * (2 * nb + 1), dtype=torch.float64, device=dev))
        check(lib().vpm_step(self._h, float(u), ptr(out.get("fm")), ptr(out.get("gamma_s")),
                             ptr(out.get("vel")), ptr(out.get("vtilde")), stream_handle(stream)))
        return out

    def rollout_batch(self, controls, want_final: bool = True, want_traj: bool = False,
                      want_field: bool = False, costs=None, stream=None, x0=None):
        """K rollouts of H steps under controls (K, H) float32 CUDA tensor; x0 (K, 7) float64
        CUDA tensor gives each rollout its own initial glider state (else the root's)."""
        import torch
        controls = _dev_tensor(controls, torch.float32)
        K, H = controls.shape
        dev = controls.device
        out = dict(costs=costs if costs is not None else torch.empty(K, dtype=torch.float32, device=dev))
        if want_final:
            out["final_glider"] = torch.empty((K, 7), dtype=torch.float64, device=dev)
        if want_traj:
            out["traj"] = torch.empty((K, H, 7), dtype=torch.float64, device=dev)
        if want_field:
            out["field"] = torch.zeros((K, self.capacity, 3), dtype=torch.float64, device=dev)
            out["count"] = torch.zeros(K, dtype=torch.int32, device=dev)
        if x0 is not None:
            x0 = _dev_tensor(x0, torch.float64)
            if tuple(x0.shape) != (K, 7):
                raise ValueError("x0 must be (K, 7)")
            check(lib().vpm_rollout_batch_x0(self._h, K, H, ptr(x0), ptr(controls), ptr(out["costs"]),
                                             ptr(out.get("final_glider")), ptr(out.get("traj")),
                                             ptr(out.get("field")), ptr(out.get("count")),
                                             stream_handle(stream)))
        else:
            check(lib().vpm_rollout_batch(self._h, K, H, ptr(controls), ptr(out["costs"]),
                                          ptr(out.get("final_glider")), ptr(out.get("traj")),
                                          ptr(out.get("field")), ptr(out.get("count")),
                                          stream_handle(stream)))
        return out

    def rollout_scratch_bytes(self, K: int, H: int) -> int:
        """Device bytes of pair-sum scratch a batch of K rollouts of H steps allocates."""
        b = C.c_size_t()
        check(lib().vpm_rollout_scratch_bytes(self._h, int(K), int(H), C.byref(b)))
        return b.value

    def rollout_batch_per_launch(self, controls, stream=None):
        import torch
        controls = _dev_tensor(controls, torch.float32)
        K, H = controls.shape
        costs = torch.empty(K, dtype=torch.float32, device=controls.device)
        fin = torch.empty((K, 7), dtype=torch.float64, device=controls.device)
        check(lib().vpm_rollout_batch_per_launch(self._h, K, H, ptr(controls), ptr(costs),
                                                 ptr(fin), stream_handle(stream)))
        return dict(costs=costs, final_glider=fin)


def pool_trim() -> int:
    """Gives the library pool's reserved, unused device memory back to the device
    (vpm_pool_trim); returns the bytes the pool still holds."""
    b = C.c_size_t()
    check(lib().vpm_pool_trim(C.byref(b)))
    return b.value


class ServerConfig(C.Structure):
    _fields_ = [("max_inflight", C.c_int), ("hbm_budget", C.c_size_t), ("max_rollouts", C.c_int),
                ("max_horizon", C.c_int), ("max_inflight_rollouts", C.c_int), ("policy", C.c_int),
                ("max_wait_ms", C.c_double), ("small_rollouts", C.c_int)]


ADMIT_ARRIVAL, ADMIT_LEAST_WORK = 0, 1


class ServerResult(C.Structure):
    _fields_ = [("status", C.c_int), ("scenario", C.c_int), ("K", C.c_int), ("H", C.c_int),
                ("t_submit_ms", C.c_double), ("t_start_ms", C.c_double), ("t_done_ms", C.c_double),
                ("j_min", C.c_float)]


class Server:
    """Replanning server with resident scenario fields (see vpm_server_* in include/vpm.h)."""

    def __init__(self, max_inflight: int = 8, max_rollouts: int = 4096, max_horizon: int = 100,
                 hbm_budget: int = 0, max_inflight_rollouts: int = 0, policy: int = ADMIT_ARRIVAL,
                 max_wait_ms: float = 0.0, small_rollouts: int = 0):
        cfg = ServerConfig(int(max_inflight), int(hbm_budget), int(max_rollouts), int(max_horizon),
                           int(max_inflight_rollouts), int(policy), float(max_wait_ms), int(small_rollouts))
        h = C.c_void_p()
        check(lib().vpm_server_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self.max_horizon = max_horizon

    def close(self):
        if getattr(self, "_h", None):
            lib().vpm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_scenario(self, params: dict, particles, glider7, capacity: int, precision: int = FP32) -> int:
        P = make_params(params, precision)
        parts = np.ascontiguousarray(np.asarray(particles, dtype=np.float64).reshape(-1, 3))
        xg = np.ascontiguousarray(np.asarray(glider7, dtype=np.float64))
        sid = C.c_int()
        check(lib().vpm_server_add_scenario(self._h, C.byref(P), parts.ctypes.data_as(_VP), len(parts),
                                            int(capacity), xg.ctypes.data_as(_VP), C.byref(sid)))
        return sid.value

    def submit(self, scenario: int, eps, mu=None, lam: float = 10.0, advance_steps: int = 0,
               advance_u: float = 0.0) -> int:
        eps = np.ascontiguousarray(eps, dtype=np.float32)
        K, H = eps.shape
        m = None if mu is None else np.ascontiguousarray(mu, dtype=np.float32)
        t = C.c_longlong()
        check(lib().vpm_server_submit(self._h, int(scenario), K, H,
                                      None if m is None else m.ctypes.data_as(_VP),
                                      eps.ctypes.data_as(_VP), float(lam), int(advance_steps),
                                      float(advance_u), C.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """Returns (result dict, mu) or None when not done within the timeout."""
        r = ServerResult()
        mu = np.zeros(self.max_horizon, np.float32)
        st = lib().vpm_server_poll(self._h, C.c_longlong(ticket), int(timeout_ms), C.byref(r),
                                   mu.ctypes.data_as(_VP))
        if st in (VPM_ERR_BUSY, VPM_ERR_TIMEOUT):
            return None
        check(st)
        res = {k: getattr(r, k) for k, _ in ServerResult._fields_}
        return res, mu[:r.H].copy()

    def request_bytes(self, scenario: int, K: int, H: int, advance_steps: int = 0) -> int:
        """Device bytes admission counts for such a request (buffers plus rollout scratch)."""
        b = C.c_size_t()
        check(lib().vpm_server_request_bytes(self._h, int(scenario), int(K), int(H),
                                             int(advance_steps), C.byref(b)))
        return b.value

    def stats(self):
        done, q, f, b = C.c_longlong(), C.c_int(), C.c_int(), C.c_size_t()
        check(lib().vpm_server_stats(self._h, C.byref(done), C.byref(q), C.byref(f), C.byref(b)))
        return dict(completed_rollouts=done.value, queued=q.value, in_flight=f.value,
                    in_flight_bytes=b.value)

    def read_scenario(self, scenario: int, capacity: int):
        parts = np.zeros((capacity, 3))
        xg = np.zeros(7)
        n = C.c_int()
        check(lib().vpm_server_read_scenario(self._h, int(scenario), parts.ctypes.data_as(_VP),
                                             C.byref(n), xg.ctypes.data_as(_VP)))
        return parts[:n.value].copy(), xg


class Batch:
    """Rollouts from R roots with uneven particle counts (one rollout per root)."""

    def __init__(self, params: dict, fields, gliders, max_horizon: int, precision: int = FP32,
                 stream=None):
        self.params = dict(params)
        self._P = make_params(params, precision)
        counts = np.ascontiguousarray([len(f) for f in fields], dtype=np.int32)
        parts = np.ascontiguousarray(np.concatenate([np.asarray(f, np.float64).reshape(-1, 3) for f in fields])
                                     if len(fields) else np.zeros((0, 3)))
        xg = np.ascontiguousarray(np.asarray(gliders, dtype=np.float64).reshape(-1, 7))
        self.R = len(counts)
        self.counts = counts
        h = C.c_void_p()
        check(lib().vpm_batch_create(C.byref(self._P), self.R, counts.ctypes.data_as(_VP),
                                     parts.ctypes.data_as(_VP), xg.ctypes.data_as(_VP),
                                     int(max_horizon), C.byref(h), stream_handle(stream)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().vpm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rollout(self, controls, use_graph: bool = False, out=None, stream=None):
        import torch
        controls = _dev_tensor(controls, torch.float32)
        R, H = controls.shape
        dev = controls.device
        o = out or dict(costs=torch.empty(R, dtype=torch.float32, device=dev),
                        count=torch.empty(R, dtype=torch.int32, device=dev),
                        final_glider=torch.empty((R, 7), dtype=torch.float64, device=dev))
        check(lib().vpm_batch_rollout(self._h, H, ptr(controls), ptr(o["costs"]), ptr(o["count"]),
                                      ptr(o["final_glider"]), int(use_graph), stream_handle(stream)))
        return o

    def tune(self, controls, stream=None):
        import torch
        controls = _dev_tensor(controls, torch.float32)
        check(lib().vpm_batch_tune(self._h, controls.shape[1], ptr(controls), stream_handle(stream)))

    def schedule(self):
        """Per launch of the current schedule: capacity, threads, rollouts, tuned ms, diagonal
        targets per lane, CTAs per rollout, and whether all rollouts run in one launch."""
        n = C.c_int()
        cap, nt, items, dt, ctas = (np.zeros(6, np.int32) for _ in range(5))
        ms = np.zeros(6, np.float32)
        merged = C.c_int()
        check(lib().vpm_batch_schedule(self._h, C.byref(n), cap.ctypes.data_as(_VP), nt.ctypes.data_as(_VP),
                                       items.ctypes.data_as(_VP), ms.ctypes.data_as(_VP),
                                       dt.ctypes.data_as(_VP), ctas.ctypes.data_as(_VP), C.byref(merged)))
        return [dict(cap=int(cap[i]), threads=int(nt[i]), rollouts=int(items[i]), tuned_ms=float(ms[i]),
                     diag_t=int(dt[i]), ctas=int(ctas[i]), merged=bool(merged.value))
                for i in range(n.value)]

    def tuned_modes(self):
        """The tuner's whole-batch times (ms): class launches side by side, one merged launch."""
        a, m = C.c_float(), C.c_float()
        check(lib().vpm_batch_tuned_modes(self._h, C.byref(a), C.byref(m)))
        return dict(class_launches_ms=a.value, one_launch_ms=m.value)

    def set_schedule(self, merged: bool, cls: int, threads: int, diag_t: int):
        check(lib().vpm_batch_set_schedule(self._h, int(bool(merged)), int(cls), int(threads), int(diag_t)))

    def set_ctas(self, merged: bool, cls: int, ctas: int):
        check(lib().vpm_batch_set_ctas(self._h, int(bool(merged)), int(cls), int(ctas)))

    def status(self, stream=None):
        check(lib().vpm_batch_status(self._h, stream_handle(stream)))


def mppi_weights(costs, lam: float, out=None, stream=None):
    import torch
    costs = _dev_tensor(costs, torch.float32)
    w = out if out is not None else torch.empty_like(costs)
    check(lib().mppi_weights(ptr(costs), costs.numel(), float(lam), ptr(w), stream_handle(stream)))
    return w


def mppi_update(weights, controls, out=None, stream=None):
    import torch
    weights = _dev_tensor(weights, torch.float32)
    controls = _dev_tensor(controls, torch.float32)
    K, H = controls.shape
    mu = out if out is not None else torch.empty(H, dtype=torch.float32, device=controls.device)
    check(lib().mppi_update(ptr(weights), ptr(controls), K, H, ptr(mu), stream_handle(stream)))
    return mu


def mppi_perturb(mu, eps, out=None, stream=None):
    import torch
    mu = _dev_tensor(mu, torch.float32)
    eps = _dev_tensor(eps, torch.float32)
    K, H = eps.shape
    c = out if out is not None else torch.empty_like(eps)
    check(lib().mppi_perturb(ptr(mu), ptr(eps), K, H, ptr(c), stream_handle(stream)))
    return c


class NmpcConfig(C.Structure):
    _fields_ = [("horizon", C.c_int), ("replan_every", C.c_int), ("latency", C.c_int),
                ("rollouts", C.c_int), ("iterations", C.c_int), ("lam", C.c_float),
                ("qc", C.c_double * 7), ("qf", C.c_double * 7), ("rc", C.c_double),
                ("threaded", C.c_int)]


class NMPC:
    """Feedback NMPC of §IV-C (see vpm_nmpc_* in include/vpm.h). noise: list over plans of
    (eps (iterations, K, N) float32, xi (K, 7) float64, zeta (K, N) float32)."""

    def __init__(self, params: dict, particles, capacity: int, x0, mu0, noise, horizon: int,
                 replan_every: int, latency: int, rollouts: int, iterations: int, lam: float,
                 qc, qf, rc: float, threaded: bool = False, precision: int = FP32):
        cfg = NmpcConfig()
        cfg.horizon, cfg.replan_every, cfg.latency = int(horizon), int(replan_every), int(latency)
        cfg.rollouts, cfg.iterations, cfg.lam = int(rollouts), int(iterations), float(lam)
        for i in range(7):
            cfg.qc[i], cfg.qf[i] = float(qc[i]), float(qf[i])
        cfg.rc, cfg.threaded = float(rc), int(bool(threaded))
        self._P = make_params(params, precision)
        parts = np.ascontiguousarray(np.asarray(particles, dtype=np.float64).reshape(-1, 3))
        xg = np.ascontiguousarray(np.asarray(x0, dtype=np.float64))
        mu = np.ascontiguousarray(np.asarray(mu0, dtype=np.float32))
        eps = np.ascontiguousarray(np.stack([z[0] for z in noise]).astype(np.float32))
        xi = np.ascontiguousarray(np.stack([z[1] for z in noise]).astype(np.float64))
        zeta = np.ascontiguousarray(np.stack([z[2] for z in noise]).astype(np.float32))
        self.horizon = int(horizon)
        h = C.c_void_p()
        check(lib().vpm_nmpc_create(C.byref(cfg), C.byref(self._P), parts.ctypes.data_as(_VP),
                                    len(parts), int(capacity), xg.ctypes.data_as(_VP),
                                    mu.ctypes.data_as(_VP), len(noise), eps.ctypes.data_as(_VP),
                                    xi.ctypes.data_as(_VP), zeta.ctypes.data_as(_VP), C.byref(h)))
        self._h = h

    def control(self, t: int, x_obs) -> float:
        x = np.ascontiguousarray(np.asarray(x_obs, dtype=np.float64))
        u = C.c_double()
        check(lib().vpm_nmpc_control(self._h, int(t), x.ctypes.data_as(_VP), C.byref(u)))
        return u.value

    def inject_pair(self, x1, z1, g1, x2, z2, g2):
        a = np.array([x1, z1, g1, x2, z2, g2], dtype=np.float64)
        check(lib().vpm_nmpc_inject_pair(self._h, a.ctypes.data_as(_VP)))

    def policy(self):
        t0 = C.c_int()
        N = self.horizon
        g, xb, ub = np.zeros((N, 7)), np.zeros((N + 1, 7)), np.zeros(N, np.float32)
        check(lib().vpm_nmpc_policy(self._h, C.byref(t0), g.ctypes.data_as(_VP),
                                    xb.ctypes.data_as(_VP), ub.ctypes.data_as(_VP)))
        return t0.value, g, xb, ub

    def stats(self):
        d, s_, a, b = C.c_int(), C.c_int(), C.c_double(), C.c_double()
        check(lib().vpm_nmpc_stats(self._h, C.byref(d), C.byref(s_), C.byref(a), C.byref(b)))
        return dict(plans_done=d.value, plans_skipped=s_.value, last_plan_ms=a.value, max_plan_ms=b.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().vpm_nmpc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ls_jacobians(x0, traj, controls, xbar, ubar, dt: float, stream=None):
    """Least-squares Jacobian blocks of §IV-B (see vpm_ls_jacobians). x0 (K, 7), traj (K, H, 7),
    xbar (H + 1, 7) float64 and controls (K, H), ubar (H,) float32 CUDA tensors.
    Returns A_hat (H, 3, 5), B_hat (H, 3) float64 and info (H,) int32 (1: singular step)."""
    import torch
    x0 = _dev_tensor(x0, torch.float64)
    traj = _dev_tensor(traj, torch.float64)
    controls = _dev_tensor(controls, torch.float32)
    xbar = _dev_tensor(xbar, torch.float64)
    ubar = _dev_tensor(ubar, torch.float32)
    K, H = controls.shape
    dev = controls.device
    ahat = torch.empty((H, 3, 5), dtype=torch.float64, device=dev)
    bhat = torch.empty((H, 3), dtype=torch.float64, device=dev)
    info = torch.empty(H, dtype=torch.int32, device=dev)
    check(lib().vpm_ls_jacobians(K, H, float(dt), ptr(x0), ptr(traj), ptr(controls), ptr(xbar),
                                 ptr(ubar), ptr(ahat), ptr(bhat), ptr(info), stream_handle(stream)))
    return ahat, bhat, info


def tvlqr(ahat, bhat, dt: float, qc, qf, rc: float, stream=None):
    """TVLQR gains of §IV-B (see vpm_tvlqr). Returns gains (H, 7) and S_0 (7, 7) float64."""
    import torch
    ahat = _dev_tensor(ahat, torch.float64)
    bhat = _dev_tensor(bhat, torch.float64)
    H = ahat.shape[0]
    qc = np.ascontiguousarray(qc, np.float64)
    qf = np.ascontiguousarray(qf, np.float64)
    gains = torch.empty((H, 7), dtype=torch.float64, device=ahat.device)
    s0 = torch.empty((7, 7), dtype=torch.float64, device=ahat.device)
    check(lib().vpm_tvlqr(H, float(dt), ptr(ahat), ptr(bhat), qc.ctypes.data_as(C.c_void_p),
                          qf.ctypes.data_as(C.c_void_p), float(rc), ptr(gains), ptr(s0),
                          stream_handle(stream)))
    return gains, s0


PROBE_FFMA, PROBE_RSQRT, PROBE_EX2, PROBE_PAIRS_T1, PROBE_PAIRS_T2, PROBE_PAIRS_T4, PROBE_PAIRS_SYM = range(7)


def probe_rate(probe: int, blocks_per_sm: int = 7) -> float:
    """Measured device rate of one probe (see vpm_probe_rate): FP32 FMAs/s, MUFU results/s or
    pair interactions/s of the rollout kernel's pair loop. Synchronises the device."""
    r = C.c_double(0.0)
    check(lib().vpm_probe_rate(int(probe), int(blocks_per_sm), C.byref(r)))
    return r.value


def freefield_velocity(particles, kernel: int, r_core: float, out=None, stream=None):
    """particles: (n, 4) float32 CUDA tensor (x, z, Gamma, unused) -> (n, 2) velocities."""
    import torch
    particles = _dev_tensor(particles, torch.float32)
    n = particles.shape[0]
    v = out if out is not None else torch.empty((n, 2), dtype=torch.float32, device=particles.device)
    check(lib().vpm_freefield_velocity(ptr(particles), n, int(kernel), float(r_core), ptr(v),
                                       stream_handle(stream)))
    return v


def freefield_scratch_bytes(n: int) -> int:
    """Device bytes of pair-sum scratch one free-field velocity evaluation of n particles uses."""
    b = C.c_size_t()
    check(lib().vpm_freefield_scratch_bytes(int(n), C.byref(b)))
    return b.value


def freefield_heun(particles, kernel: int, r_core: float, dt: float, steps: int, stream=None):
    """In-place Heun steps of a free field (n, 4) float32 CUDA tensor."""
    import torch
    particles = _dev_tensor(particles, torch.float32)
    check(lib().vpm_freefield_heun(ptr(particles), particles.shape[0], int(kernel),
                                   float(r_core), float(dt), int(steps), stream_handle(stream)))
    return particles
