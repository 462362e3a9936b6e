"""CPU oracle for the WHFast512 timestep -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It loads a plain-C, scalar FP64 implementation of the
Wisdom-Holman map in democratic heliocentric coordinates (see orc_core.c for
the passages of the paper each function follows) built with gcc
-O2 -ffp-contract=off.  It shares no code with the CUDA library.

Parity status of each function (what pins it) is recorded in the test files
tests/test_oracle_*.py; no oracle function is left unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
# A prebuilt oracle library to load instead of _LIB: the planted-mistake tests
# (tests/test_oracle_mutations.py) point this at a copy built with one change.
_LIB_OVERRIDE = os.environ.get("ORC_LIBRARY")
_TANGENT_OVERRIDE = os.environ.get("ORC_TANGENT_LIBRARY")   # the same for the tangent build
_FLOPS = os.path.join(_BUILD, "orc_flopcount")
_TANGENT = os.path.join(_BUILD, "liborc_tangent.so")
_SOURCES = [os.path.join(_HERE, f) for f in ("orc_core.c", "orc_ensemble.c", "flopcount.cpp",
                                              "tangent.cpp")]
_tlib = None
_lock = threading.Lock()
_lib = None

C_LIGHT_DEFAULT = 173.1446326742403 / 0.01720209895


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in _SOURCES)


def compile_library(source_dir: str, out: str) -> None:
    """gcc the oracle library from orc_ensemble.c (which includes orc_core.c)
    in source_dir into out."""
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-O2",
                           "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-o", tmp, os.path.join(source_dir, "orc_ensemble.c"),
                           "-lpthread", "-lm"])
    os.replace(tmp, out)


def compile_tangent(source_dir: str, out: str) -> None:
    """g++ the dual-number build (tangent.cpp, which includes orc_core.c) in
    source_dir into out."""
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
                           os.path.join(source_dir, "tangent.cpp")])
    os.replace(tmp, out)


def build(force: bool = False) -> None:
    """Compile the oracle library and the flop counter with gcc / g++."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or _stale(_LIB):
        compile_library(_HERE, _LIB)
    if force or _stale(_FLOPS):
        tmp = _FLOPS + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-o", tmp,
                               os.path.join(_HERE, "flopcount.cpp")])
        os.replace(tmp, _FLOPS)
    if force or _stale(_TANGENT):
        compile_tangent(_HERE, _TANGENT)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if _LIB_OVERRIDE:
            lib = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        L = ctypes.POINTER(ctypes.c_longlong)
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.orc_destroy.argtypes = [P]
        lib.orc_init.argtypes = [P, D, D, D, I, D]
        lib.orc_init.restype = ctypes.c_int
        lib.orc_step_all.argtypes = [P, ctypes.c_longlong]
        lib.orc_step_range.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_longlong]
        lib.orc_run_threads.argtypes = [P, ctypes.c_longlong, ctypes.c_int]
        lib.orc_run_threads.restype = ctypes.c_int
        lib.orc_read.argtypes = [P, D, D, I, D]
        lib.orc_energy.argtypes = [P, D]
        lib.orc_get_raw.argtypes = [P, D, D, L, I]
        lib.orc_set_raw.argtypes = [P, D, D, L, I]
        lib.orc_apply_kepler.argtypes = [P, ctypes.c_double, ctypes.c_double, D, D, D]
        lib.orc_apply_substep.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        lib.orc_stumpff.argtypes = [ctypes.c_double, ctypes.c_int, D, D]
        _lib = lib
        return lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _l(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))


class OracleEnsemble:
    """S independent systems stepped by the CPU oracle (same contract as the
    CUDA library: init from inertial arrays, step(n), synchronized read)."""

    SUBSTEP = {"kepler": 0, "jump": 1, "interaction": 2, "gr": 3}

    def __init__(self, n_systems: int, max_planets: int, gr_mode: int = 0,
                 c_light: float = C_LIGHT_DEFAULT, newton_terms: int = 8,
                 halley_terms: int = 4, halley_iters: int = 2, newton_iters: int = 2,
                 encounter_hill: float = 0.0, eject_factor: float = 0.0, merge_jumps: bool = False):
        self._lib = _load()
        self.S, self.N = int(n_systems), int(max_planets)
        self._h = self._lib.orc_create(self.S, self.N, int(gr_mode), float(c_light),
                                       int(halley_iters), int(halley_terms),
                                       int(newton_iters), int(newton_terms),
                                       float(encounter_hill), float(eject_factor), int(merge_jumps))
        if not self._h:
            raise ValueError("orc_create: invalid arguments")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    def init(self, ens) -> None:
        m = np.ascontiguousarray(ens.masses, np.float64)
        x = np.ascontiguousarray(ens.pos, np.float64)
        u = np.ascontiguousarray(ens.vel, np.float64)
        npl = np.ascontiguousarray(ens.n_planets, np.int32)
        dt = np.ascontiguousarray(ens.dt, np.float64)
        assert m.shape == (self.S, 1 + self.N)
        if self._lib.orc_init(self._h, _d(m), _d(x), _d(u), _i(npl), _d(dt)) != 0:
            raise ValueError("orc_init: invalid input")

    def step(self, n: int) -> None:
        self._lib.orc_step_all(self._h, int(n))

    def run_threads(self, n: int, threads: int) -> int:
        return self._lib.orc_run_threads(self._h, int(n), int(threads))

    def read_state(self):
        pos = np.zeros((self.S, 1 + self.N, 3))
        vel = np.zeros((self.S, 1 + self.N, 3))
        st = np.zeros(self.S, np.int32)
        t = np.zeros(self.S)
        self._lib.orc_read(self._h, _d(pos), _d(vel), _i(st), _d(t))
        return pos, vel, st, t

    def energy(self) -> np.ndarray:
        E = np.zeros(self.S)
        self._lib.orc_energy(self._h, _d(E))
        return E

    def get_raw(self):
        Q = np.zeros((self.S, self.N, 3))
        v = np.zeros((self.S, self.N, 3))
        ns = np.zeros(self.S, np.int64)
        st = np.zeros(self.S, np.int32)
        self._lib.orc_get_raw(self._h, _d(Q), _d(v), _l(ns), _i(st))
        return Q, v, ns, st

    def set_raw(self, Q, v, nstep, status) -> None:
        Q = np.ascontiguousarray(Q, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        ns = np.ascontiguousarray(nstep, np.int64)
        st = np.ascontiguousarray(status, np.int32)
        self._lib.orc_set_raw(self._h, _d(Q), _d(v), _l(ns), _i(st))

    def kepler(self, mu: float, h: float, Q, v):
        """One Kepler drift of one planet with this ensemble's solver options."""
        Q = np.array(Q, np.float64).copy()
        v = np.array(v, np.float64).copy()
        beta = np.zeros(1)
        self._lib.orc_apply_kepler(self._h, float(mu), float(h), _d(Q), _d(v), _d(beta))
        return Q, v, float(beta[0])

    def substep(self, system: int, which: str, h: float) -> None:
        self._lib.orc_apply_substep(self._h, int(system), self.SUBSTEP[which], float(h))


def stumpff(z: float, terms: int):
    """Truncated-series c_2(z), c_3(z) as the oracle evaluates them."""
    lib = _load()
    c2 = np.zeros(1)
    c3 = np.zeros(1)
    lib.orc_stumpff(float(z), int(terms), _d(c2), _d(c3))
    return float(c2[0]), float(c3[0])


def _load_tangent():
    global _tlib
    with _lock:
        if _tlib is None:
            if _TANGENT_OVERRIDE:
                lib = ctypes.CDLL(_TANGENT_OVERRIDE)
            else:
                build()
                lib = ctypes.CDLL(_TANGENT)
            D = ctypes.POINTER(ctypes.c_double)
            lib.orc_tangent_loss.argtypes = [ctypes.c_int, D, D, D, ctypes.c_double, D, ctypes.c_longlong,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D]
            lib.orc_tangent_loss.restype = ctypes.c_int
            _tlib = lib
        return _tlib


def tangent_gradient(masses, pos, vel, n_planets, dt, target, n_steps, gr_mode=1,
                     c_light=C_LIGHT_DEFAULT, newton_terms=8, merge_jumps=False):
    """Gradient of L = sum_i |Q_i(T) - target_i|^2 (synchronized heliocentric
    positions after n_steps) for ONE system, by forward-mode derivatives of the
    oracle's map, one input direction per pass.  Returns (L, dL/dpos [1+n][3],
    dL/dvel [1+n][3], dL/dmasses [1+n]) for the system's n bodies."""
    lib = _load_tangent()
    n = int(n_planets)
    m = np.ascontiguousarray(masses[:1 + n], np.float64)
    x = np.ascontiguousarray(pos[:1 + n], np.float64)
    u = np.ascontiguousarray(vel[:1 + n], np.float64)
    T = np.ascontiguousarray(target[:n], np.float64)
    L = np.zeros(1)
    dL = np.zeros(1)
    gx = np.zeros((1 + n, 3))
    gu = np.zeros((1 + n, 3))
    gm = np.zeros(1 + n)
    for kind, out in ((0, gx), (1, gu)):
        for k in range(1 + n):
            for c in range(3):
                rc = lib.orc_tangent_loss(n, _d(m), _d(x), _d(u), float(dt), _d(T), int(n_steps),
                                          int(gr_mode), float(c_light), int(newton_terms),
                                          int(merge_jumps), kind, k, c, _d(L), _d(dL))
                if rc:
                    raise RuntimeError("orc_tangent_loss failed (frozen system?)")
                out[k, c] = dL[0]
    for k in range(1 + n):
        rc = lib.orc_tangent_loss(n, _d(m), _d(x), _d(u), float(dt), _d(T), int(n_steps), int(gr_mode),
                                  float(c_light), int(newton_terms), int(merge_jumps), 2, k, 0, _d(L),
                                  _d(dL))
        if rc:
            raise RuntimeError("orc_tangent_loss failed (frozen system?)")
        gm[k] = dL[0]
    return float(L[0]), gx, gu, gm


def count_flops(n_planets: int, newton_terms: int = 8, gr_mode: int = 0, halley_iters: int = 2) -> dict:
    """Operations of one steady-state step of one system, counted on the oracle;
    start_phase = those of the Kepler solver's initial guess and Halley steps."""
    _load()
    out = subprocess.check_output([_FLOPS, str(n_planets), str(newton_terms), str(gr_mode),
                                   str(halley_iters)], text=True).split()
    adds, muls, divs, sqrts, flops, start = (int(v) for v in out)
    return {"adds": adds, "muls": muls, "divs": divs, "sqrts": sqrts, "flops": flops,
            "start_phase": start}
