"""Thin Python binding of libwhg (include/whg.h): argument marshalling only.

Every function here has the name of the C function it calls and does no
arithmetic of the integration path: all of it runs in the library's CUDA
kernels.  Host-buffer calls take numpy arrays; *_device calls take CUDA torch
tensors (PyTorch is used only for device memory and streams).  The library
must have been built (paper_2307_05683_gb300.build.build()); if it is
missing every call raises, there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

WHG_OK, WHG_EINVAL, WHG_ECUDA, WHG_ENOMEM, WHG_ESTATE = 0, -1, -2, -3, -4
WHG_STATUS_NONFINITE, WHG_STATUS_HYPERBOLIC, WHG_STATUS_INVALID = 1, 2, 4
WHG_STATUS_CLOSE_ENCOUNTER, WHG_STATUS_EJECTED = 8, 16
WHG_MAX_PLANETS = 8


class WhgError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"libwhg error {code}: {message}")
        self.code = code


class whg_options(ctypes.Structure):
    _fields_ = [("gr_mode", ctypes.c_int), ("c_light", ctypes.c_double),
                ("newton_terms", ctypes.c_int), ("lanes_per_system", ctypes.c_int),
                ("block_size", ctypes.c_int), ("steps_per_launch", ctypes.c_longlong),
                ("close_encounter_hill", ctypes.c_double), ("eject_factor", ctypes.c_double),
                ("graph_launches", ctypes.c_int), ("merge_jumps", ctypes.c_int),
                ("halley_fp32", ctypes.c_int), ("repack_frozen", ctypes.c_int),
                ("interaction_schedule", ctypes.c_int), ("queue_steps", ctypes.c_int)]


def library_path() -> str:
    """libwhg.so, or the library named by WHG_LIBRARY (e.g. the debug build)."""
    return os.environ.get("WHG_LIBRARY") or _build.LIB


def load():
    """Load libwhg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libwhg.so not found at {path}: build it with "
                               "paper_2307_05683_gb300.build.build() (there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        P, D, I, L = (ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
        sig = {
            "whg_default_options": (None, [ctypes.POINTER(whg_options)]),
            "whg_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(whg_options), ctypes.c_void_p]),
            "whg_set_stream": (ctypes.c_int, [P, ctypes.c_void_p]),
            "whg_init": (ctypes.c_int, [P, D, D, D, I, D]),
            "whg_init_device": (ctypes.c_int, [P, D, D, D, I, D]),
            "whg_step": (ctypes.c_int, [P, ctypes.c_longlong]),
            "whg_read_state": (ctypes.c_int, [P, D, D, I, D]),
            "whg_read_state_device": (ctypes.c_int, [P, D, D, I, D]),
            "whg_energy": (ctypes.c_int, [P, D]),
            "whg_energy_device": (ctypes.c_int, [P, D]),
            "whg_get_raw": (ctypes.c_int, [P, D, D, L, I]),
            "whg_set_raw": (ctypes.c_int, [P, D, D, L, I]),
            "whg_synchronize": (ctypes.c_int, [P]),
            "whg_launch_count": (ctypes.c_longlong, [P]),
            "whg_last_error": (ctypes.c_char_p, [P]),
            "whg_destroy": (None, [P]),
            "whg_measure_fp64_tflops": (ctypes.c_int, [ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
            "whg_test_special": (ctypes.c_int, [D, ctypes.c_int, D]),
            "whg_probe_fp64_lanes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.POINTER(ctypes.c_float)]),
            "whg_test_queue_timeout": (ctypes.c_int, [P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]),
            "whg_probe_fp64_kind": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_double)]),
            "whg_debug_bounds": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_uint)]),
            "whg_noalloc_debug_bounds": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint)]),
            "whg_kepler_sweep": (ctypes.c_int, [D, D, I, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_longlong, D, D]),
            "whg_adjoint_forward": (ctypes.c_int, [P, ctypes.c_longlong, ctypes.c_int, D, D]),
            "whg_adjoint_backward": (ctypes.c_int, [P, D, D, D, D]),
            "whg_adjoint_schedule": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_longlong]),
            "whg_adjoint_layout": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                  ctypes.POINTER(ctypes.c_int)]),
            "whg_integrate_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int,
                                                     ctypes.POINTER(whg_options), D, D, D, I, D,
                                                     ctypes.c_longlong, D, D, I, D, ctypes.c_void_p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_symbols() -> list[str]:
    """Names of the C functions this binding expects the library to export."""
    return ["whg_default_options", "whg_create", "whg_set_stream", "whg_init", "whg_init_device",
            "whg_step", "whg_read_state", "whg_read_state_device", "whg_energy",
            "whg_energy_device", "whg_get_raw", "whg_set_raw", "whg_synchronize",
            "whg_launch_count", "whg_last_error", "whg_destroy", "whg_measure_fp64_tflops",
            "whg_test_special", "whg_integrate_noalloc", "whg_adjoint_forward",
            "whg_adjoint_backward", "whg_kepler_sweep", "whg_probe_fp64_lanes", "whg_test_queue_timeout",
            "whg_debug_bounds", "whg_noalloc_debug_bounds", "whg_probe_fp64_kind",
            "whg_adjoint_schedule", "whg_adjoint_layout"]


def _check(ctx, rc: int) -> None:
    if rc != WHG_OK:
        msg = load().whg_last_error(ctx)
        raise WhgError(rc, msg.decode() if msg else "")


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _dev(t, dtype_name: str):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != dtype_name:
        raise ValueError(f"expected a contiguous CUDA tensor of {dtype_name}")
    return t.data_ptr()


def current_stream():
    """torch's current CUDA stream handle (or None)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


# ---------------------------------------------------------------- calls --

def whg_default_options() -> whg_options:
    o = whg_options()
    load().whg_default_options(ctypes.byref(o))
    return o


def whg_create(n_systems: int, max_planets: int, options: whg_options | None = None,
               stream=None):
    h = ctypes.c_void_p()
    opt = ctypes.byref(options) if options is not None else None
    rc = load().whg_create(ctypes.byref(h), int(n_systems), int(max_planets), opt,
                           ctypes.c_void_p(stream) if stream else None)
    _check(None, rc)
    return h


def whg_set_stream(ctx, stream) -> None:
    _check(ctx, load().whg_set_stream(ctx, ctypes.c_void_p(stream) if stream else None))


def whg_init(ctx, masses, pos, vel, n_planets, dt) -> None:
    m, pm = _host(masses, np.float64)
    x, px = _host(pos, np.float64)
    u, pu = _host(vel, np.float64)
    d, pd = _host(dt, np.float64)
    if n_planets is not None:
        n, pn = _host(n_planets, np.int32)
    else:
        pn = None
    _check(ctx, load().whg_init(ctx, pm, px, pu, pn, pd))


def whg_init_device(ctx, masses, pos, vel, n_planets, dt) -> None:
    _check(ctx, load().whg_init_device(ctx, _dev(masses, "torch.float64"), _dev(pos, "torch.float64"),
                                       _dev(vel, "torch.float64"), _dev(n_planets, "torch.int32"),
                                       _dev(dt, "torch.float64")))


def whg_step(ctx, n_steps: int) -> None:
    _check(ctx, load().whg_step(ctx, int(n_steps)))


def whg_read_state(ctx, pos: np.ndarray, vel: np.ndarray, status: np.ndarray | None = None,
                   t: np.ndarray | None = None) -> None:
    for a, dt in ((pos, np.float64), (vel, np.float64), (status, np.int32), (t, np.float64)):
        if a is not None and (a.dtype != dt or not a.flags.c_contiguous):
            raise ValueError("output arrays must be C-contiguous with the documented dtypes")
    _check(ctx, load().whg_read_state(ctx, pos.ctypes.data, vel.ctypes.data,
                                      status.ctypes.data if status is not None else None,
                                      t.ctypes.data if t is not None else None))


def whg_read_state_device(ctx, pos, vel, status=None, t=None) -> None:
    _check(ctx, load().whg_read_state_device(ctx, _dev(pos, "torch.float64"), _dev(vel, "torch.float64"),
                                             _dev(status, "torch.int32"), _dev(t, "torch.float64")))


def whg_energy(ctx, E: np.ndarray) -> None:
    if E.dtype != np.float64 or not E.flags.c_contiguous:
        raise ValueError("E must be a contiguous float64 array")
    _check(ctx, load().whg_energy(ctx, E.ctypes.data))


def whg_energy_device(ctx, E) -> None:
    _check(ctx, load().whg_energy_device(ctx, _dev(E, "torch.float64")))


def whg_get_raw(ctx, Q: np.ndarray, v: np.ndarray, nstep: np.ndarray, status: np.ndarray) -> None:
    for a, dt in ((Q, np.float64), (v, np.float64), (nstep, np.int64), (status, np.int32)):
        if a.dtype != dt or not a.flags.c_contiguous:
            raise ValueError("output arrays must be C-contiguous with the documented dtypes")
    _check(ctx, load().whg_get_raw(ctx, Q.ctypes.data, v.ctypes.data, nstep.ctypes.data,
                                   status.ctypes.data))


def whg_set_raw(ctx, Q, v, nstep, status) -> None:
    Q, pq = _host(Q, np.float64)
    v, pv = _host(v, np.float64)
    n, pn = _host(nstep, np.int64)
    s, ps = _host(status, np.int32)
    _check(ctx, load().whg_set_raw(ctx, pq, pv, pn, ps))


def whg_adjoint_forward(ctx, n_steps: int, checkpoint_every: int, target, loss) -> None:
    _check(ctx, load().whg_adjoint_forward(ctx, int(n_steps), int(checkpoint_every),
                                           _dev(target, "torch.float64"), _dev(loss, "torch.float64")))


def whg_adjoint_backward(ctx, loss_weight, grad_pos, grad_vel, grad_mass) -> None:
    _check(ctx, load().whg_adjoint_backward(ctx, _dev(loss_weight, "torch.float64"),
                                            _dev(grad_pos, "torch.float64"), _dev(grad_vel, "torch.float64"),
                                            _dev(grad_mass, "torch.float64")))


def whg_adjoint_schedule(ctx, sm_split: int = -1, tape_bytes: int = 0) -> None:
    _check(ctx, load().whg_adjoint_schedule(ctx, int(sm_split), int(tape_bytes)))


def whg_adjoint_layout(ctx) -> dict:
    a, b, n = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(ctx, load().whg_adjoint_layout(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
    return {"chain_sms": a.value, "tape_sms": b.value, "tape_buffers": n.value}


def whg_synchronize(ctx) -> None:
    _check(ctx, load().whg_synchronize(ctx))


def whg_launch_count(ctx) -> int:
    return int(load().whg_launch_count(ctx))


def whg_last_error(ctx=None) -> str:
    msg = load().whg_last_error(ctx)
    return msg.decode() if msg else ""


def whg_destroy(ctx) -> None:
    load().whg_destroy(ctx)


def whg_measure_fp64_tflops(seconds: float = 0.5) -> float:
    out = ctypes.c_double()
    _check(None, load().whg_measure_fp64_tflops(float(seconds), ctypes.byref(out)))
    return out.value


def whg_kepler_sweep(q, v, cfg, mu: float, h: float, steps: int, q_out, v_out) -> None:
    _check(None, load().whg_kepler_sweep(_dev(q, "torch.float64"), _dev(v, "torch.float64"),
                                         _dev(cfg, "torch.int32"), int(q.shape[0]), float(mu), float(h),
                                         int(steps), _dev(q_out, "torch.float64"),
                                         _dev(v_out, "torch.float64")))


def whg_probe_fp64_lanes(warps_per_sm: int, active_lanes: int, iters: int) -> float:
    """Kernel time in ms of the FP64 lane probe (see whg.h)."""
    ms = ctypes.c_float()
    _check(None, load().whg_probe_fp64_lanes(int(warps_per_sm), int(active_lanes), int(iters),
                                             ctypes.byref(ms)))
    return float(ms.value)


def whg_probe_fp64_kind(kind: int, warps_per_sm: int, iters: int) -> float:
    """FP64 lane-operations per SM clock of one instruction kind (see whg.h)."""
    out = ctypes.c_double()
    _check(None, load().whg_probe_fp64_kind(int(kind), int(warps_per_sm), int(iters), ctypes.byref(out)))
    return float(out.value)


def whg_debug_bounds(ctx) -> int:
    """Index-check flag bits of ctx since the last call (debug build only)."""
    flag = ctypes.c_uint()
    _check(ctx, load().whg_debug_bounds(ctx, ctypes.byref(flag)))
    return int(flag.value)


def whg_noalloc_debug_bounds() -> int:
    """Index-check flag bits of whg_integrate_noalloc calls since the last
    read (debug build only)."""
    flag = ctypes.c_uint()
    _check(None, load().whg_noalloc_debug_bounds(ctypes.byref(flag)))
    return int(flag.value)


def whg_test_queue_timeout(ctx, spin_limit: int) -> int:
    """Error flag (1 = a wait gave up) of the queue failure-path test (see whg.h)."""
    flag = ctypes.c_int()
    _check(ctx, load().whg_test_queue_timeout(ctx, int(spin_limit), ctypes.byref(flag)))
    return int(flag.value)


def whg_test_special(x, out) -> None:
    _check(None, load().whg_test_special(_dev(x, "torch.float64"), int(x.numel()),
                                         _dev(out, "torch.float64")))


WHG_NOALLOC_MAX_LANES = 65536


def whg_integrate_noalloc(n_systems: int, max_planets: int, options: whg_options | None,
                          masses, pos, vel, n_planets, dt, n_steps: int,
                          pos_out, vel_out, status_out=None, t_out=None, stream=None) -> None:
    """Allocation-free init + step + read on CUDA tensors (see include/whg.h)."""
    opt = ctypes.byref(options) if options is not None else None
    rc = load().whg_integrate_noalloc(
        int(n_systems), int(max_planets), opt, _dev(masses, "torch.float64"), _dev(pos, "torch.float64"),
        _dev(vel, "torch.float64"), _dev(n_planets, "torch.int32"), _dev(dt, "torch.float64"),
        int(n_steps), _dev(pos_out, "torch.float64"), _dev(vel_out, "torch.float64"),
        _dev(status_out, "torch.int32"), _dev(t_out, "torch.float64"),
        ctypes.c_void_p(stream) if stream else None)
    _check(None, rc)


# ------------------------------------------------------------ convenience --

class Integrator:
    """One libwhg context: S systems of at most N planets (host-array API)."""

    def __init__(self, n_systems: int, max_planets: int, gr_mode: int = 1, c_light: float | None = None,
                 newton_terms: int = 8, lanes_per_system: int = 0, block_size: int = 0,
                 steps_per_launch: int = 0, close_encounter_hill: float = 0.0,
                 eject_factor: float = 0.0, graph_launches: int = 0, merge_jumps: bool = False,
                 halley_fp32: bool = False, repack_frozen: bool | None = None, interaction_schedule: int = 0,
                 queue_steps: int = 100, stream=None):
        opt = whg_default_options()
        opt.gr_mode = gr_mode
        if c_light is not None:
            opt.c_light = c_light
        opt.newton_terms = newton_terms
        opt.lanes_per_system = lanes_per_system
        opt.block_size = block_size
        opt.steps_per_launch = steps_per_launch
        opt.close_encounter_hill = close_encounter_hill
        opt.eject_factor = eject_factor
        opt.graph_launches = graph_launches
        opt.merge_jumps = int(merge_jumps)
        opt.halley_fp32 = int(halley_fp32)
        opt.repack_frozen = -1 if repack_frozen is None else int(bool(repack_frozen))   # None: auto
        opt.interaction_schedule = int(interaction_schedule)
        opt.queue_steps = int(queue_steps)
        self.S, self.N = int(n_systems), int(max_planets)
        self.stream = stream if stream is not None else current_stream()
        self.ctx = whg_create(self.S, self.N, opt, self.stream)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            whg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check_shapes(self, arrays) -> None:
        """The C calls read S x (...) elements from each host array; refuse
        arrays of any other shape before they are read past their end."""
        for name, a, shape in arrays:
            if np.shape(a) != shape:
                raise ValueError(f"{name} has shape {np.shape(a)}, expected {shape}")

    def init(self, ens) -> None:
        S, B = self.S, 1 + self.N
        self._check_shapes((("masses", ens.masses, (S, B)), ("pos", ens.pos, (S, B, 3)),
                            ("vel", ens.vel, (S, B, 3)), ("n_planets", ens.n_planets, (S,)),
                            ("dt", ens.dt, (S,))))
        whg_init(self.ctx, ens.masses, ens.pos, ens.vel, ens.n_planets, ens.dt)

    def step(self, n: int) -> None:
        whg_step(self.ctx, n)

    def read_state(self):
        pos = np.zeros((self.S, 1 + self.N, 3))
        vel = np.zeros((self.S, 1 + self.N, 3))
        st = np.zeros(self.S, np.int32)
        t = np.zeros(self.S)
        whg_read_state(self.ctx, pos, vel, st, t)
        return pos, vel, st, t

    def energy(self) -> np.ndarray:
        E = np.zeros(self.S)
        whg_energy(self.ctx, E)
        return E

    def get_raw(self):
        Q = np.zeros((self.S, self.N, 3))
        v = np.zeros((self.S, self.N, 3))
        ns = np.zeros(self.S, np.int64)
        st = np.zeros(self.S, np.int32)
        whg_get_raw(self.ctx, Q, v, ns, st)
        return Q, v, ns, st

    def set_raw(self, Q, v, nstep, status) -> None:
        S, N = self.S, self.N
        self._check_shapes((("Q", Q, (S, N, 3)), ("v", v, (S, N, 3)), ("nstep", nstep, (S,)),
                            ("status", status, (S,))))
        whg_set_raw(self.ctx, Q, v, nstep, status)

    def synchronize(self) -> None:
        whg_synchronize(self.ctx)

    @property
    def launches(self) -> int:
        return whg_launch_count(self.ctx)
