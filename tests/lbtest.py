"""Helpers shared by the GPU tests: run the same seeded problem through the
CUDA path (C-ABI via the ctypes binding) and through the oracle."""
from __future__ import annotations

import numpy as np

import oracle


def lib():
    from paper_0908_4520_gb300 import build

    build()
    from paper_0908_4520_gb300 import Lattice, capi

    return Lattice, capi


def order_map(capi, quad, P):
    """perm such that gpu_pop[k] corresponds to oracle_pop[perm[k]]."""
    g = capi.lb_quadrature_info(quad)["xi"]
    r = P.vs.xi
    perm = np.empty(len(g), dtype=np.int64)
    for k, x in enumerate(g):
        d = np.abs(r - x).sum(axis=1)
        perm[k] = int(np.argmin(d))
        assert d[perm[k]] < 1e-12
    assert len(set(perm.tolist())) == len(g)
    return perm


EPS64 = 2.220446049250313e-16


def f64_tol(steps: int, u0: float) -> float:
    """Parity bound of the FP64 path against the oracle.  The oracle stores the full
    f (O(w)) while the signal is the deviation (O(w u0)); each of its steps rounds
    a few operations at eps * |f|, i.e. ~eps / u0 relative to the signal, and these
    accumulate at most linearly: 10 * (steps + 1) * eps / u0."""
    return max(1e-12, 10.0 * (steps + 1) * EPS64 / u0)


EPS32 = 2.0 ** -24


def f32_tol(steps: int) -> float:
    """Bound for FP32 deviation storage against the oracle, relative to the velocity
    amplitude: every step rounds each stored deviation (relative eps32) and the
    rounding of a smooth field is correlated from step to step, so the error can
    grow linearly: 2 (steps + 1) eps32 (1.2e-7 per step)."""
    return 2.0 * (steps + 1) * EPS32


def random_fields(nx, ny, seed, amp=2e-2):
    """Smooth random rho, u, T fields (periodic Fourier modes), seeded."""
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(nx) / nx
    y = 2 * np.pi * np.arange(ny) / ny
    X, Y = np.meshgrid(x, y)

    def field():
        f = np.zeros((ny, nx))
        for kx in range(3):
            for ky in range(2):
                a, b = rng.uniform(-1, 1, 2)
                f += a * np.cos(kx * X + ky * Y) + b * np.sin(kx * X + ky * Y)
        return f / 6.0

    return 1.0 + amp * field(), amp * field(), amp * field(), 1.0 + amp * field()


def oracle_from_fields(P, rho, ux, uy, T):
    f = np.empty((P.Q, P.ny, P.nx))
    for j in range(P.ny):
        for i in range(P.nx):
            f[:, j, i] = P.feq(rho[j, i], ux[j, i], uy[j, i], T[j, i])
    return f


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_both(quad, N, nx, ny, kn, precision, steps, u0=1e-3, u1=0.0, isothermal=False, **kw):
    """GPU lattice (after `steps`) and oracle state/records for the same problem."""
    Lattice, capi = lib()
    L = Lattice(quad, N, nx, ny, kn, precision=precision, isothermal=isothermal, **kw)
    L.init_shear_wave(u0, u1)
    L.step(steps)
    P = oracle.Problem(quad, N, nx, ny, kn, isothermal=isothermal, cfl=kw.get("cfl", 1.0))
    f = P.init_shear(u0, u1)
    d = P.run(f, steps)
    return L, P, f, d, capi
