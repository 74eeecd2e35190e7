"""Thin ctypes binding of the C ABI in include/ttsh.h (libttsh.so, built for sm_103a).

Functions carry the C entry points' names and only marshal arguments: every arithmetic
step of the solver runs in the library's CUDA kernels.  There is no CPU fallback: if the
library is missing or cannot be loaded the first call raises.

Host arrays are numpy float64 / uint8, C-contiguous, indexed [y][x].  Device pointers and
streams are plain integers (e.g. ``tensor.data_ptr()``, ``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libttsh.so")

TTSH_OK, TTSH_E_INVALID, TTSH_E_OOM, TTSH_E_CUDA, TTSH_E_TIMEOUT, TTSH_E_NONFINITE, \
    TTSH_E_UNSUPPORTED = range(7)
_STATUS_NAMES = ["OK", "INVALID", "OOM", "CUDA", "TIMEOUT", "NONFINITE", "UNSUPPORTED"]


class TTSHError(RuntimeError):
    def __init__(self, status: int, message: str):
        name = _STATUS_NAMES[status] if 0 <= status < len(_STATUS_NAMES) else str(status)
        super().__init__(f"TTSH_E_{name}: {message}")
        self.status = status


class ttsh_params(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("gamma_v", ctypes.c_double), ("gamma_w", ctypes.c_double),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("n", ctypes.c_int32), ("precision", ctypes.c_int32)]


class ttsh_diag(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("enstrophy", ctypes.c_double),
                ("psi", ctypes.c_double), ("max_div", ctypes.c_double), ("mean_vx", ctypes.c_double),
                ("mean_vy", ctypes.c_double), ("step", ctypes.c_int64),
                ("nonfinite", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ttsh_fno_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("width", ctypes.c_int32), ("modes", ctypes.c_int32),
                ("layers", ctypes.c_int32), ("in_channels", ctypes.c_int32), ("max_batch", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def load_library(path: str = LIB_PATH):
    """Load libttsh.so once; raise if it is absent (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2304_03306_gb300.build.build()")
    lib = ctypes.CDLL(path)
    sigs = {
        "ttsh_default_params": (None, [ctypes.POINTER(ttsh_params)]),
        "ttsh_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(ttsh_params)]),
        "ttsh_create_domain": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ttsh_params),
                                              _P, _P, ctypes.POINTER(_P)]),
        "ttsh_destroy_domain": (None, [_P]),
        "ttsh_set_stream": (ctypes.c_int, [_P, _P]),
        "ttsh_set_velocity": (ctypes.c_int, [_P, _D, _D]),
        "ttsh_set_velocity_device": (ctypes.c_int, [_P, _P, _P]),
        "ttsh_init_noise": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double]),
        "ttsh_step": (ctypes.c_int, [_P, ctypes.c_int64]),
        "ttsh_step_record": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, _P, ctypes.c_int64, _D]),
        "ttsh_get_fields": (ctypes.c_int, [_P, _D, _D, _D]),
        "ttsh_get_mask": (ctypes.c_int, [_P, _D]),
        "ttsh_get_spectral_state": (ctypes.c_int, [_P, _D, _D]),
        "ttsh_set_spectral_state": (ctypes.c_int, [_P, _D, _D]),
        "ttsh_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(ttsh_diag), _D, ctypes.c_int32, _D]),
        "ttsh_synchronize": (ctypes.c_int, [_P]),
        "ttsh_test_bounded_wait": (ctypes.c_int, [_P, ctypes.c_double]),
        "ttsh_time_kernels": (ctypes.c_int, [_P, ctypes.c_int32, _D]),
        "ttsh_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
        "ttsh_get_plan": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
        "ttsh_set_plan": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
        "ttsh_set_launch_mode": (ctypes.c_int, [_P, ctypes.c_int32]),
        "ttsh_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, _P, ctypes.POINTER(_P)]),
        "ttsh_batch_step": (ctypes.c_int, [_P, ctypes.c_int64]),
        "ttsh_batch_synchronize": (ctypes.c_int, [_P]),
        "ttsh_batch_groups": (ctypes.c_int32, [_P]),
        "ttsh_batch_set_persistent": (ctypes.c_int, [_P, ctypes.c_int32]),
        "ttsh_batch_persistent": (ctypes.c_int32, [_P]),
        "ttsh_batch_test_stalled_wait": (ctypes.c_int, [_P, ctypes.c_double]),
        "ttsh_batch_destroy": (None, [_P]),
        "ttsh_restrict": (ctypes.c_int, [_P, _P]),
        "ttsh_psd_begin": (ctypes.c_int, [_P, _D, ctypes.c_int32]),
        "ttsh_psd_accumulate": (ctypes.c_int, [_P, ctypes.c_double]),
        "ttsh_psd_result": (ctypes.c_int, [_P, _D]),
        "ttsh_dumbbell_order": (ctypes.c_int, [_P, _D, ctypes.c_double, _D]),
        "ttsh_fno_create": (ctypes.c_int, [ctypes.POINTER(ttsh_fno_config), ctypes.c_uint64, _P, ctypes.POINTER(_P)]),
        "ttsh_fno_destroy": (None, [_P]),
        "ttsh_fno_num_params": (ctypes.c_int64, [_P]),
        "ttsh_fno_get_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
        "ttsh_fno_set_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
        "ttsh_fno_set_scales": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_float]),
        "ttsh_fno_forward": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32]),
        "ttsh_fno_loss_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_float)]),
        "ttsh_fno_adam_step": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
        "ttsh_fno_features": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32]),
        "ttsh_fno_residual": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32]),
        "ttsh_fno_correct": (ctypes.c_int, [_P, _P, _P]),
        "ttsh_fno_rollout": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, _P]),
        "ttsh_lyap_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, _D, ctypes.POINTER(_P)]),
        "ttsh_lyap_step": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32]),
        "ttsh_lyap_result": (ctypes.c_int, [_P, _D, _D]),
        "ttsh_lyap_directions": (ctypes.c_int, [_P, _D]),
        "ttsh_lyap_destroy": (None, [_P]),
        "ttsh_step_count": (ctypes.c_int64, [_P]),
        "ttsh_fma_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _D]),
        "ttsh_step_noalloc": (ctypes.c_int, [ctypes.POINTER(ttsh_params), _P, _P, _P, ctypes.c_int64, _P]),
        "ttsh_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != TTSH_OK:
        raise TTSHError(status, ttsh_last_error())


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (n, n):
        raise ValueError(f"expected shape {(n, n)}, got {a.shape}")
    return a


def _centre(centre):
    c = np.ascontiguousarray(centre, dtype=np.float64).reshape(-1)
    if c.shape != (2,):
        raise ValueError("centre must hold two coordinates")
    return c


def ttsh_last_error() -> str:
    return load_library().ttsh_last_error().decode()


def ttsh_default_params(n: int = 8192, dx: float = 0.005, precision: int = 32, **kw) -> ttsh_params:
    p = ttsh_params()
    load_library().ttsh_default_params(ctypes.byref(p))
    p.n, p.dx, p.precision = n, dx, precision
    for k, v in kw.items():
        setattr(p, "lambda_" if k in ("lam", "lambda") else k, v)
    return p


def ttsh_workspace_bytes(p: ttsh_params) -> int:
    return int(load_library().ttsh_workspace_bytes(ctypes.byref(p)))


def ttsh_create_domain(mask, p: ttsh_params, workspace: int | None = None, stream: int | None = None):
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if m.shape != (p.n, p.n):
        raise ValueError(f"mask must have shape {(p.n, p.n)}")
    h = _P()
    _check(load_library().ttsh_create_domain(m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                             ctypes.byref(p), workspace, stream, ctypes.byref(h)))
    return h


def ttsh_destroy_domain(h):
    load_library().ttsh_destroy_domain(h)


def ttsh_set_stream(h, stream: int | None):
    _check(load_library().ttsh_set_stream(h, stream))


def ttsh_set_velocity(h, vx, vy, n: int):
    vx, vy = _f64(vx, n), _f64(vy, n)
    _check(load_library().ttsh_set_velocity(h, _dptr(vx), _dptr(vy)))


def ttsh_set_velocity_device(h, vx_ptr: int, vy_ptr: int):
    _check(load_library().ttsh_set_velocity_device(h, vx_ptr, vy_ptr))


def ttsh_init_noise(h, seed: int, amplitude: float):
    _check(load_library().ttsh_init_noise(h, int(seed), float(amplitude)))


def ttsh_step(h, nsteps: int):
    _check(load_library().ttsh_step(h, int(nsteps)))


def ttsh_step_record(h, nsteps: int, every: int, series_ptr: int | None, capacity: int, centre=(0.0, 0.0)):
    """Step and append {step, energy, enstrophy, psi, nonfinite} every `every` steps to the
    device array at series_ptr (5 * capacity doubles).  Asynchronous."""
    c = _centre(centre)
    _check(load_library().ttsh_step_record(h, int(nsteps), int(every), series_ptr, int(capacity), _dptr(c)))


def ttsh_get_fields(h, n: int):
    vx, vy, w = (np.empty((n, n)) for _ in range(3))
    _check(load_library().ttsh_get_fields(h, _dptr(vx), _dptr(vy), _dptr(w)))
    return vx, vy, w


def ttsh_get_mask(h, n: int):
    K = np.empty((n, n))
    _check(load_library().ttsh_get_mask(h, _dptr(K)))
    return K


def ttsh_get_spectral_state(h, n: int):
    M = n // 4
    buf = np.empty((M + 1, 2 * M + 1, 2))
    v0 = np.empty(2)
    _check(load_library().ttsh_get_spectral_state(h, _dptr(buf), _dptr(v0)))
    return buf[..., 0] + 1j * buf[..., 1], v0


def ttsh_set_spectral_state(h, w_hat, v0, n: int):
    M = n // 4
    w_hat = np.asarray(w_hat)
    if w_hat.shape != (M + 1, 2 * M + 1):
        raise ValueError(f"w_hat must have shape {(M + 1, 2 * M + 1)}, got {w_hat.shape}")
    buf = np.ascontiguousarray(np.stack([np.real(w_hat), np.imag(w_hat)], axis=-1), dtype=np.float64)
    v = np.ascontiguousarray(v0, dtype=np.float64).reshape(-1)
    if v.shape != (2,):
        raise ValueError("v0 must hold the two mean-flow components")
    _check(load_library().ttsh_set_spectral_state(h, _dptr(buf), _dptr(v)))


def ttsh_diagnostics(h, nbins: int = 0, centre=(0.0, 0.0)) -> dict:
    d = ttsh_diag()
    spec = np.zeros(max(nbins, 1))
    c = _centre(centre)
    st = load_library().ttsh_diagnostics(h, ctypes.byref(d), _dptr(spec) if nbins else None,
                                         int(nbins), _dptr(c))
    if st not in (TTSH_OK, TTSH_E_NONFINITE):
        _check(st)
    out = {k: getattr(d, k) for k, _ in ttsh_diag._fields_ if k != "reserved"}
    out["status"] = st
    if nbins:
        out["spectrum"] = spec[:nbins]
    return out


def ttsh_time_kernels(h, iters: int):
    ms = np.zeros(2)
    _check(load_library().ttsh_time_kernels(h, int(iters), _dptr(ms)))
    return float(ms[0]), float(ms[1])


_PLAN_KEYS = ("row_variant", "col_variant", "rows_per_block", "row_points_per_thread",
              "col_points_per_thread", "n_row_variants", "n_col_variants", "launch_mode",
              "row_cluster", "row_compact")


def _plan_dict(buf):
    return {k: int(buf[i]) for i, k in enumerate(_PLAN_KEYS)}


def ttsh_autotune(h, iters: int = 200) -> dict:
    buf = (ctypes.c_int32 * len(_PLAN_KEYS))()
    _check(load_library().ttsh_autotune(h, int(iters), buf))
    return _plan_dict(buf)


def ttsh_get_plan(h) -> dict:
    buf = (ctypes.c_int32 * len(_PLAN_KEYS))()
    _check(load_library().ttsh_get_plan(h, buf))
    return _plan_dict(buf)


def ttsh_set_plan(h, row_variant: int, col_variant: int):
    _check(load_library().ttsh_set_plan(h, int(row_variant), int(col_variant)))


def ttsh_set_launch_mode(h, mode: int):
    """mode bit 0: programmatic dependent launch; bit 1: TMA staging of the row pass's tile."""
    _check(load_library().ttsh_set_launch_mode(h, int(mode)))


def ttsh_batch_create(handles, stream: int | None = None):
    arr = (_P * len(handles))(*[h.value if isinstance(h, _P) else h for h in handles])
    b = _P()
    _check(load_library().ttsh_batch_create(arr, len(handles), stream, ctypes.byref(b)))
    return b


def ttsh_batch_step(b, nsteps: int):
    _check(load_library().ttsh_batch_step(b, int(nsteps)))


def ttsh_batch_synchronize(b):
    _check(load_library().ttsh_batch_synchronize(b))


def ttsh_batch_groups(b) -> int:
    return int(load_library().ttsh_batch_groups(b))


def ttsh_batch_destroy(b):
    load_library().ttsh_batch_destroy(b)


class Batch:
    """Lock-step stepping of several Domain objects (they must stay alive)."""

    def __init__(self, domains, stream: int | None = None):
        self.domains = list(domains)
        self.b = ttsh_batch_create([d.h for d in self.domains], stream)

    def step(self, nsteps: int):
        ttsh_batch_step(self.b, nsteps)

    def synchronize(self):
        ttsh_batch_synchronize(self.b)

    @property
    def groups(self) -> int:
        return ttsh_batch_groups(self.b)

    @property
    def persistent(self) -> bool:
        return int(load_library().ttsh_batch_persistent(self.b)) == 1

    def test_stalled_wait(self, seconds: float):
        """Failure-path test hook of the persistent stepper (see ttsh.h)."""
        _check(load_library().ttsh_batch_test_stalled_wait(self.b, float(seconds)))

    def set_persistent(self, on: bool):
        """One launch per step() call for every domain (True, the default where allowed) or
        one launch per pass per group of equal domains (False)."""
        _check(load_library().ttsh_batch_set_persistent(self.b, 1 if on else 0))

    def close(self):
        if self.b:
            ttsh_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ttsh_psd_begin(h, omegas):
    om = np.ascontiguousarray(omegas, dtype=np.float64)
    _check(load_library().ttsh_psd_begin(h, _dptr(om), int(om.size)))


def ttsh_psd_accumulate(h, t: float):
    _check(load_library().ttsh_psd_accumulate(h, float(t)))


def ttsh_psd_result(h, nfreq: int):
    S = np.empty(nfreq)
    _check(load_library().ttsh_psd_result(h, _dptr(S)))
    return S


def ttsh_dumbbell_order(h, centres, radius: float):
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(4)
    out = np.empty(3)
    _check(load_library().ttsh_dumbbell_order(h, _dptr(c), float(radius), _dptr(out)))
    return float(out[0]), float(out[1]), float(out[2])


def ttsh_restrict(fine, coarse):
    _check(load_library().ttsh_restrict(fine, coarse))


_FP = ctypes.POINTER(ctypes.c_float)


class FNO:
    """Learned corrector (Fourier neural operator) run by the library's kernels.

    Device arrays are passed as integer pointers (e.g. torch tensor .data_ptr())."""

    def __init__(self, n=256, width=32, modes=16, layers=4, max_batch=8, seed=0, stream: int | None = None):
        self.cfg = ttsh_fno_config(n, width, modes, layers, 4, max_batch)
        self.n = n
        self.h = _P()
        lib = load_library()
        _check(lib.ttsh_fno_create(ctypes.byref(self.cfg), int(seed), stream, ctypes.byref(self.h)))
        self.nparams = int(lib.ttsh_fno_num_params(self.h))

    def close(self):
        if self.h:
            load_library().ttsh_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        _check(load_library().ttsh_fno_get_params(self.h, out.ctypes.data_as(_FP)))
        return out

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        assert a.size == self.nparams
        _check(load_library().ttsh_fno_set_params(self.h, a.ctypes.data_as(_FP)))

    def set_scales(self, in_scale, out_scale: float):
        a = np.ascontiguousarray(in_scale, dtype=np.float32)
        _check(load_library().ttsh_fno_set_scales(self.h, a.ctypes.data_as(_FP), float(out_scale)))

    def forward(self, x_ptr: int, y_ptr: int, batch: int):
        _check(load_library().ttsh_fno_forward(self.h, x_ptr, y_ptr, int(batch)))

    def loss_grad(self, x_ptr: int, t_ptr: int, batch: int, want_grad: bool = False):
        loss = ctypes.c_double()
        g = np.empty(self.nparams, dtype=np.float32) if want_grad else None
        _check(load_library().ttsh_fno_loss_grad(self.h, x_ptr, t_ptr, int(batch), ctypes.byref(loss),
                                                 g.ctypes.data_as(_FP) if want_grad else None))
        return loss.value, g

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        _check(load_library().ttsh_fno_adam_step(self.h, lr, beta1, beta2, eps))

    def features(self, dom, x_ptr: int, sample: int = 0):
        _check(load_library().ttsh_fno_features(self.h, dom.h, x_ptr, int(sample)))

    def residual(self, truth, base, t_ptr: int, sample: int = 0):
        _check(load_library().ttsh_fno_residual(self.h, truth.h, base.h, t_ptr, int(sample)))

    def correct(self, dom, scratch_ptr: int):
        _check(load_library().ttsh_fno_correct(self.h, dom.h, scratch_ptr))

    def rollout(self, dom, nsteps: int, scratch_ptr: int, correct_every: int = 1):
        _check(load_library().ttsh_fno_rollout(self.h, dom.h, int(nsteps), int(correct_every), scratch_ptr))


def ttsh_synchronize(h):
    _check(load_library().ttsh_synchronize(h))


def ttsh_step_noalloc(p: ttsh_params, K_ptr: int, w_hat_ptr: int, v0_ptr: int, nsteps: int,
                      stream: int | None = None):
    """Advance caller-owned device buffers (mask, half-spectrum state, mean flow) without the
    library allocating device memory; n <= 512.  See include/ttsh.h."""
    _check(load_library().ttsh_step_noalloc(ctypes.byref(p), K_ptr, w_hat_ptr, v0_ptr, int(nsteps), stream))


def ttsh_step_count(h) -> int:
    return int(load_library().ttsh_step_count(h))


class Domain:
    """Convenience owner of one ttsh_domain handle."""

    def __init__(self, mask, n: int, dx: float, precision: int = 32, workspace: int | None = None,
                 stream: int | None = None, **coef):
        self.n = n
        self.params = ttsh_default_params(n=n, dx=dx, precision=precision, **coef)
        self.h = ttsh_create_domain(mask, self.params, workspace, stream)

    def close(self):
        if self.h:
            ttsh_destroy_domain(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_velocity(self, vx, vy):
        ttsh_set_velocity(self.h, vx, vy, self.n)

    def init_noise(self, seed: int, amplitude: float = 0.01):
        ttsh_init_noise(self.h, seed, amplitude)

    def set_velocity_device(self, vx_ptr: int, vy_ptr: int):
        ttsh_set_velocity_device(self.h, vx_ptr, vy_ptr)

    def set_stream(self, stream: int | None):
        ttsh_set_stream(self.h, stream)

    def step(self, nsteps: int):
        ttsh_step(self.h, nsteps)

    def step_record(self, nsteps: int, every: int, series_ptr: int | None, capacity: int, centre=(0.0, 0.0)):
        ttsh_step_record(self.h, nsteps, every, series_ptr, capacity, centre)

    def record(self, nsteps: int, every: int, centre=(0.0, 0.0)):
        """Step nsteps and return the recorded time series as an array of rows
        (step, energy, enstrophy, psi, nonfinite); device memory from PyTorch."""
        import torch
        ns = (int(nsteps) + int(every) - 1) // int(every)
        buf = torch.zeros(max(ns, 1) * 5, dtype=torch.float64, device="cuda")
        self.step_record(nsteps, every, buf.data_ptr(), ns, centre)
        self.synchronize()
        return buf[: ns * 5].cpu().numpy().reshape(ns, 5)

    def fields(self):
        return ttsh_get_fields(self.h, self.n)

    def mask(self):
        return ttsh_get_mask(self.h, self.n)

    def spectral_state(self):
        return ttsh_get_spectral_state(self.h, self.n)

    def set_spectral_state(self, w_hat, v0):
        ttsh_set_spectral_state(self.h, w_hat, v0, self.n)

    def diagnostics(self, nbins: int = 0, centre=(0.0, 0.0)):
        return ttsh_diagnostics(self.h, nbins, centre)

    def synchronize(self):
        ttsh_synchronize(self.h)

    def test_bounded_wait(self, seconds: float):
        """Failure-path test hook: a kernel whose bounded wait cannot complete (see ttsh.h)."""
        _check(load_library().ttsh_test_bounded_wait(self.h, float(seconds)))

    def autotune(self, iters: int = 200) -> dict:
        """Time every tile-shape variant of the step kernels and keep the fastest."""
        return ttsh_autotune(self.h, iters)

    def plan(self) -> dict:
        return ttsh_get_plan(self.h)

    def set_plan(self, row_variant: int, col_variant: int, launch_mode: int | None = None):
        ttsh_set_plan(self.h, row_variant, col_variant)
        if launch_mode is not None:
            ttsh_set_launch_mode(self.h, launch_mode)

    def time_kernels(self, iters: int):
        """Mean (row pass, column pass) launch durations in ms, state restored afterwards."""
        return ttsh_time_kernels(self.h, iters)

    @property
    def steps(self) -> int:
        return ttsh_step_count(self.h)

    def psd_begin(self, omegas):
        self._psd_n = len(omegas)
        ttsh_psd_begin(self.h, omegas)

    def psd_accumulate(self, t: float):
        ttsh_psd_accumulate(self.h, t)

    def psd_result(self):
        return ttsh_psd_result(self.h, self._psd_n)

    def dumbbell_order(self, centres, radius: float):
        """(Psi_2, omega at the left peak, omega at the right peak)."""
        return ttsh_dumbbell_order(self.h, centres, radius)


class Lyapunov:
    """Lyapunov exponents of a Domain's trajectory (ttsh_lyap_*): k perturbed copies stepped
    with it, re-orthonormalised every `interval` steps."""

    def __init__(self, dom: "Domain", q0, eps: float):
        q0 = np.ascontiguousarray(q0, dtype=np.float64)
        if q0.ndim != 2:
            raise ValueError("q0 must be a (k, D) array of directions")
        self.k, self.D = q0.shape
        D = 2 * (dom.n // 4 + 1) * (dom.n // 2 + 1) + 2
        if self.D != D:
            raise ValueError(f"each direction must have D = {D} entries for n = {dom.n}")
        self.h = _P()
        _check(load_library().ttsh_lyap_create(dom.h, self.k, float(eps), _dptr(q0), ctypes.byref(self.h)))

    def step(self, nsteps: int, interval: int):
        _check(load_library().ttsh_lyap_step(self.h, int(nsteps), int(interval)))

    def result(self):
        ex, last = np.empty(self.k), np.empty(self.k)
        _check(load_library().ttsh_lyap_result(self.h, _dptr(ex), _dptr(last)))
        return ex, last

    def directions(self):
        q = np.empty((self.k, self.D))
        _check(load_library().ttsh_lyap_directions(self.h, _dptr(q)))
        return q

    def close(self):
        if self.h:
            load_library().ttsh_lyap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ttsh_fma_peak(precision: int, iters: int) -> float:
    """Measured fused multiply-add throughput of the current GPU in TFLOP/s."""
    out = ctypes.c_double()
    _check(load_library().ttsh_fma_peak(int(precision), int(iters), ctypes.byref(out)))
    return out.value
