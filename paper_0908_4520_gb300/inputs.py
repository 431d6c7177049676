"""Seeded synthetic workloads of the standing shear wave (no arithmetic of the method).

The paper's benchmark (Sec. 4) is an analytic problem, not a dataset: a
periodic shear wave u_y = U0 sin(x) at rest density and temperature, here
unforced and decaying.  These generators fix the sizes, seeds and parameter
draws of the workloads; both the GPU path and the oracle take their output
as input.
"""
from __future__ import annotations

import numpy as np

GH_SETS = ("D2Q16-GH", "D2Q36-GH", "D2Q64-GH")


def plain_small():
    """Standing shear wave, plain method: 64 x 1 grid, D2Q16-GH, N = 2, FP64, Kn 0.1, 5000 steps."""
    return dict(quadrature="D2Q16-GH", n_eq=2, nx=64, ny=1, kn=0.1, precision="f64", u0=1e-3, u1=0.0,
                steps=5000)


def plain_at_scale(quadrature: str = "D2Q36-GH", kn: float = 0.1):
    """4096^2 periodic grid, third-order equilibrium, FP32, u_y = 1e-3 sin x + 1e-3 sin y sin x,
    Kn in {0.01, 0.1, 1}, 2000 steps; quadratures D2Q36-GH (Lax-Wendroff) and D2Q37 (shift)."""
    return dict(quadrature=quadrature, n_eq=3, nx=4096, ny=4096, kn=kn, precision="f32", u0=1e-3, u1=1e-3,
                steps=2000)


PLAIN_AT_SCALE_KN = (0.01, 0.1, 1.0)


def precision_kn(n: int = 8, seed: int = 9084520):
    """Kn log-uniform over [0.01, 10], seeded."""
    rng = np.random.default_rng(seed)
    return list(10.0 ** rng.uniform(-2.0, 1.0, n))


def precision_config(kn: float, precision: str = "bf16", nx: int = 2048, steps: int = 2000):
    """D2Q64-GH, fourth-order equilibrium, 2048^2, U0 = 1e-4, 16-bit deviation storage."""
    return dict(quadrature="D2Q64-GH", n_eq=4, nx=nx, ny=nx, kn=kn, precision=precision, u0=1e-4, u1=0.0,
                steps=steps)


def batch_instances(n: int = 512, seed: int = 9084521, u0: float = 1e-3, max_steps: int = 20000):
    """Uneven instances: nx in {32..1024} (powers of two), ny in {1, 4}, a GH product set,
    N in {2, 3, 4}, Kn log-uniform over [0.01, 10]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        out.append(dict(
            id=i,
            quadrature=GH_SETS[int(rng.integers(0, 3))],
            n_eq=int(rng.integers(2, 5)),
            nx=int(2 ** rng.integers(5, 11)),
            ny=int((1, 4)[int(rng.integers(0, 2))]),
            kn=float(10.0 ** rng.uniform(-2.0, 1.0)),
            u0=u0,
            max_steps=max_steps,
        ))
    return out


def serving_stream(n: int = 20000, rate: float = 2000.0, seed: int = 9084522, large_fraction: float = 0.1,
                   max_steps: int = 20000):
    """Poisson arrivals of shear-wave solves: batch-instance grids, quadratures and orders with the
    precision workload's Kn range and U0 = 1e-4, FP16 deviation storage; a fraction are
    1024 x 1024 D2Q36-GH."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    reqs = []
    for i in range(n):
        if rng.uniform() < large_fraction:
            q, N, nx, ny = "D2Q36-GH", 3, 1024, 1024
        else:
            q = GH_SETS[int(rng.integers(0, 3))]
            N = int(rng.integers(2, 5))
            nx = int(2 ** rng.integers(5, 11))
            ny = int((1, 4)[int(rng.integers(0, 2))])
        reqs.append(dict(id=i, arrival=float(t[i]), quadrature=q, n_eq=N, nx=nx, ny=ny,
                         kn=float(10.0 ** rng.uniform(-2.0, 1.0)), u0=1e-4, precision="f16",
                         max_steps=max_steps))
    return reqs
