"""FP64 CPU oracle for the high-order lattice Boltzmann hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import, call, link or
run anything under ``oracle/``.  The product library never does, and the
oracle never imports the product package: the two share no code.  Inputs
that both sides need (sizes, seeds, Knudsen draws) come from
``paper_0908_4520_gb300.inputs``, which holds no arithmetic of the method.

Contents
--------
quadrature.py  velocity sets: Golub-Welsch Gauss-Hermite rules and products,
               the Table 1 sets from their printed surds, D2Q37 by moment
               matching.
lb_oracle.c    plain FP64 LB stepper (moments, tensor-form Hermite
               equilibrium and body-force term of Sec. 2.1, Eq. 2order
               or Eq. slb collision, exact shift or Lax-Wendroff streaming,
               observables).
dvm_oracle.c   reduced linearised-BGK DVM of Sec. 3.3 (Eqs. ga, gb), free or driven.
linear.py      linear-mode matrix of the scheme and the continuous DVM
               dispersion relation (pins).

Parameter readings (the paper is silent or ambiguous on these; each is
listed in the design notes with its justification):
* dx = 2 pi / nx (wave number 1 in the units of Eq. nondime), dy = dx.
* on-lattice dt = dx / c (xi = c e); off-lattice dt = cfl * dx / max|xi_x|.
* Kn convention "lambda" (default): the mean free path lambda = mu/p
  sqrt(pi R T / 2), so the collision time of Eq. bgk is tau = Kn sqrt(2/pi);
  convention "paper": tau = Kn (Eq. KN).
* omega = dt / (tau + dt/2) (Eq. 2order); omega = dt / tau for the first-order
  scheme of Eq. slb.
"""
from __future__ import annotations

import contextlib
import ctypes
import math
import os
import subprocess
import threading

import numpy as np

from . import linear, quadrature  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = [os.path.join(_HERE, "lb_oracle.c"), os.path.join(_HERE, "dvm_oracle.c")]
_lock = threading.Lock()
_lib = None

INNER_NODES = 6  # inner Gauss-Hermite rule for a_eq integrals (exact to degree 11)


def build(force: bool = False, plant: int = 0) -> str:
    """Compile liboracle.so with gcc (plain C99, -O2, no vendor code).  plant = k > 0 (tests
    only) builds the variant with mistake k planted (see lb_oracle.c)."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _LIB_PATH if plant == 0 else os.path.join(_BUILD, f"liboracle_plant{plant}.so")
    newest = max(os.path.getmtime(s) for s in _SOURCES)
    if force or not os.path.exists(path) or os.path.getmtime(path) < newest:
        tmp = path + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu99", "-shared", "-fPIC", f"-DORACLE_PLANT={plant}", "-o", tmp, *_SOURCES, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return path


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("Q", ctypes.c_int), ("N", ctypes.c_int),
        ("xi", ctypes.POINTER(ctypes.c_double)), ("w", ctypes.POINTER(ctypes.c_double)),
        ("e", ctypes.POINTER(ctypes.c_int)),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double),
        ("rho0", ctypes.c_double), ("isothermal", ctypes.c_int), ("ninner", ctypes.c_int),
        ("zin", ctypes.POINTER(ctypes.c_double)), ("win", ctypes.POINTER(ctypes.c_double)),
        ("force_amp", ctypes.c_double), ("force_freq", ctypes.c_double), ("force_uniform", ctypes.c_int),
        ("scheme", ctypes.c_int), ("streaming", ctypes.c_int),
    ]


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    pp = ctypes.POINTER(_Params)
    lib.oracle_lb_run.argtypes = [pp, dp, ctypes.c_int, dp]
    lib.oracle_lb_run_from.argtypes = [pp, dp, ctypes.c_int, ctypes.c_int, dp]
    lib.oracle_lb_moments.argtypes = [pp, dp, ctypes.c_int, dp, dp, dp, dp, dp]
    lib.oracle_feq.argtypes = [pp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
    lib.oracle_force.argtypes = [pp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, dp]
    lib.oracle_lb_init_shear.argtypes = [pp, ctypes.c_double, ctypes.c_double, dp]
    lib.oracle_dvm_run.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, dp, dp, dp]
    lib.oracle_dvm_run_forced.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp,
                                          dp]
    lib.oracle_dvm_dt.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double]
    lib.oracle_dvm_dt.restype = ctypes.c_double
    return lib


@contextlib.contextmanager
def planted(k: int):
    """Tests only: run the oracle with mistake k planted while the context is open."""
    global _lib
    _load()
    old = _lib
    _lib = _bind(ctypes.CDLL(build(plant=k)))
    try:
        yield
    finally:
        _lib = old


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def collision_time(kn: float, convention: str = "lambda") -> float:
    if convention == "lambda":
        return kn * math.sqrt(2.0 / math.pi)
    if convention == "paper":
        return kn
    raise ValueError(convention)


class Problem:
    """One standing-shear-wave configuration for the oracle.

    force_amp, force_freq: body force g = (0, g_y), g_y = force_amp sin(x_i) cos(force_freq t)
    (force_uniform: g_y = force_amp cos(force_freq t)); force_amp = 0 is the free wave.
    N: Hermite order of the equilibrium, 1..4.
    scheme: "second_order" (Eq. 2order) or "first_order" (the standard LB of Eq. slb,
    omega = dt / tau, no dt/2 corrections of the moments, sigma_xy without 1 - omega/2).
    streaming (off-lattice sets): "lax_wendroff" or "upwind2" (second-order upwind)."""

    def __init__(self, set_name: str, N: int, nx: int, ny: int, kn: float,
                 kn_convention: str = "lambda", cfl: float = 1.0, isothermal: bool = False,
                 force_amp: float = 0.0, force_freq: float = 0.0, force_uniform: bool = False,
                 scheme: str = "second_order", streaming: str = "lax_wendroff"):
        self.vs = quadrature.velocity_set(set_name)
        self.set_name, self.N, self.nx, self.ny, self.kn = set_name, N, nx, ny, kn
        self.isothermal = isothermal
        self.force_amp, self.force_freq = force_amp, force_freq
        self.dx = 2.0 * math.pi / nx
        if self.vs.on_lattice:
            self.dt = self.dx / self.vs.c
        else:
            self.dt = cfl * self.dx / float(np.max(np.abs(self.vs.xi[:, 0])))
        self.tau = collision_time(kn, kn_convention)
        if scheme not in ("second_order", "first_order"):
            raise ValueError(scheme)
        self.scheme = scheme
        if streaming not in ("lax_wendroff", "upwind2"):
            raise ValueError(streaming)
        self.streaming = streaming
        if scheme == "first_order":
            self.omega = self.dt / self.tau  # Eq. slb
        else:
            self.omega = self.dt / (self.tau + 0.5 * self.dt)  # Eq. 2order
        self._xi = np.ascontiguousarray(self.vs.xi, dtype=np.float64)
        self._w = np.ascontiguousarray(self.vs.w, dtype=np.float64)
        self._e = (np.ascontiguousarray(self.vs.e, dtype=np.int32) if self.vs.on_lattice else None)
        z, wz = quadrature.gauss_hermite(INNER_NODES)
        self._z, self._wz = np.ascontiguousarray(z), np.ascontiguousarray(wz)
        self._p = _Params(nx, ny, self.vs.Q, N, _dp(self._xi), _dp(self._w),
                          self._e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if self._e is not None else None,
                          self.dx, self.dt, self.tau, 1.0, int(isothermal), INNER_NODES,
                          _dp(self._z), _dp(self._wz), float(force_amp), float(force_freq),
                          int(force_uniform), int(scheme == "first_order"), int(streaming == "upwind2"))

    @property
    def Q(self):
        return self.vs.Q

    def feq(self, rho, ux, uy, T):
        out = np.empty(self.Q)
        _load().oracle_feq(ctypes.byref(self._p), rho, ux, uy, T, _dp(out))
        return out

    def force(self, rho, ux, uy, T, gy):
        """Hermite force term g_alpha of g = (0, gy) at the Maxwellian (rho, u, T)."""
        out = np.empty(self.Q)
        _load().oracle_force(ctypes.byref(self._p), rho, ux, uy, T, gy, _dp(out))
        return out

    def init_shear(self, u0: float, u1: float = 0.0) -> np.ndarray:
        f = np.empty((self.Q, self.ny, self.nx))
        _load().oracle_lb_init_shear(ctypes.byref(self._p), u0, u1, _dp(f))
        return f

    def run(self, f: np.ndarray, nsteps: int, record: bool = True, n0: int = 0):
        """Advance f (Q, ny, nx) in place from time level n0; returns (nsteps+1, 8)
        records (levels n0..n0+nsteps) or None."""
        assert f.dtype == np.float64 and f.flags.c_contiguous and f.shape == (self.Q, self.ny, self.nx)
        diag = np.empty((nsteps + 1, 8)) if record else None
        rc = _load().oracle_lb_run_from(ctypes.byref(self._p), _dp(f), n0, nsteps, _dp(diag))
        if rc != 0:
            raise RuntimeError("oracle_lb_run failed")
        return diag

    def moments(self, f: np.ndarray, n: int = 0) -> dict:
        """Per-cell rho, u, T, sigma_xy of f~ at time level n (n sets the force phase)."""
        out = {k: np.empty((self.ny, self.nx)) for k in ("rho", "ux", "uy", "T", "sxy")}
        _load().oracle_lb_moments(ctypes.byref(self._p), _dp(f), n, *(_dp(out[k]) for k in
                                                                     ("rho", "ux", "uy", "T", "sxy")))
        return out


def run_dvm(n_nodes: int, nx: int, kn: float, u0: float, nsteps: int, cfl: float = 0.5,
            kn_convention: str = "lambda", force_amp: float = 0.0, force_freq: float = 0.0):
    """Reduced linearised-BGK DVM with an n-point Gauss-Hermite rule, free
    (force_amp = 0) or driven by g = force_amp sin(x_i) cos(force_freq t).

    Returns (t, A, S) arrays of length nsteps + 1.
    """
    g, wg = quadrature.gauss_hermite(n_nodes)
    g, wg = np.ascontiguousarray(g), np.ascontiguousarray(wg)
    tau = collision_time(kn, kn_convention)
    t = np.empty(nsteps + 1)
    A = np.empty(nsteps + 1)
    S = np.empty(nsteps + 1)
    rc = _load().oracle_dvm_run_forced(nx, n_nodes, _dp(g), _dp(wg), tau, cfl, u0, float(force_amp),
                                       float(force_freq), nsteps, _dp(t), _dp(A), _dp(S))
    if rc != 0:
        raise RuntimeError("oracle_dvm_run failed")
    return t, A, S


def dvm_dt(n_nodes: int, nx: int, cfl: float = 0.5) -> float:
    g, _ = quadrature.gauss_hermite(n_nodes)
    g = np.ascontiguousarray(g)
    return float(_load().oracle_dvm_dt(nx, n_nodes, _dp(g), cfl))


def decay_fit(t, A, t_start: float, floor: float = 1e-4):
    """Decay rate: minus the least-squares slope of ln|A| against t over
    t >= t_start while |A| >= floor * |A(0)|."""
    t = np.asarray(t)
    A = np.asarray(A)
    a0 = abs(A[0])
    # stop at the first point below the floor after t_start
    idx = np.nonzero(t >= t_start)[0]
    keep = []
    for i in idx:
        if abs(A[i]) < floor * a0:
            break
        keep.append(i)
    if len(keep) < 3:
        raise ValueError("too few points for a decay fit")
    keep = np.array(keep)
    slope, _ = np.polyfit(t[keep], np.log(np.abs(A[keep])), 1)
    return float(-slope)
