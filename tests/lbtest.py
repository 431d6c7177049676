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
