"""The pins catch plausible mistakes: each test builds the oracle with one mistake planted
(ORACLE_PLANT, compiled into a separate library) and checks that at least one pin fails,
while all of them hold for the oracle as it is.

Planted mistakes: 1 sign of the force term; 2 no rho g dt/2 in the momentum; 3 force
relaxed with omega instead of omega tau; 4 Lax-Wendroff streaming against xi; 5 the
highest Hermite order dropped from the equilibrium; 6 sigma_xy without (1 - omega/2);
7 the first-order scheme of Eq. slb relaxing with the second-order omega; 8 the driven
DVM pushed by -g; 9 second-order upwind streaming from the downstream side.
"""
import numpy as np
import pytest

import oracle
from oracle import linear


def _p_c():
    """Equilibrium moments up to order N = 3 equal the Maxwellian's (Sec. 2.1)."""
    P = oracle.Problem("D2Q36-GH", 3, 8, 1, 0.1)
    rho, ux, uy, T = 1.02, 0.03, -0.02, 1.01
    f = P.feq(rho, ux, uy, T)
    x, y = P.vs.xi[:, 0], P.vs.xi[:, 1]
    checks = [
        (f.sum(), rho),
        ((x * f).sum(), rho * ux),
        ((x * x * f).sum(), rho * (ux * ux + T)),
        ((x ** 3 * f).sum(), rho * (ux ** 3 + 3 * ux * T)),
        ((x * x * y * f).sum(), rho * (ux * ux * uy + uy * T)),
    ]
    return all(abs(a - b) < 1e-12 for a, b in checks)


def _p_e():
    """Free-wave history equals the linear-mode propagation (A and S)."""
    P = oracle.Problem("D2Q16-GH", 2, 32, 1, 0.1)
    f = P.init_shear(1e-6)
    d = P.run(f, 200)
    A, S = linear.lb_linear_history(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, 1e-6, 200)
    return (np.max(np.abs(d[:, 4] - A)) < 1e-5 * np.max(np.abs(A)) and
            np.max(np.abs(d[:, 5] - S)) < 1e-5 * np.max(np.abs(S)))


def _p_j1():
    P = oracle.Problem("D2Q36-GH", 3, 8, 1, 0.1)
    F = P.force(1.03, 0.021, -0.017, 1.0, 0.37)
    y = P.vs.xi[:, 1]
    return abs(F.sum()) < 1e-13 and abs((y * F).sum() - 1.03 * 0.37) < 1e-13


def _p_j2():
    amp, phi = 2e-3, 0.7
    P = oracle.Problem("D2Q36-GH", 3, 16, 4, 0.3, force_amp=amp, force_freq=phi, force_uniform=True)
    f = P.init_shear(1e-3, 5e-4)
    d = P.run(f, 20)
    g = amp * np.cos(phi * d[:, 0])
    p = d[:, 3] - 0.5 * P.dt * g * d[:, 1]
    return np.allclose(np.diff(p), P.dt * g[:-1] * d[:-1, 1], rtol=1e-11, atol=1e-15)


def _p_j3():
    amp, phi = 1e-5, 1.3
    P = oracle.Problem("D2Q16-GH", 2, 32, 1, 0.1, force_amp=amp, force_freq=phi)
    f = P.init_shear(0.0)
    d = P.run(f, 200)
    A = linear.lb_linear_forced_history(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, amp, phi, 200)
    return np.max(np.abs(d[:, 4] - A)) < 1e-5 * np.max(np.abs(A))


def _p_k1():
    """N = 1 equilibrium is w rho (1 + xi.u) (Sec. 3.3, Eq. lbm1)."""
    P = oracle.Problem("D2Q36-GH", 1, 8, 1, 0.1)
    xi, w = P.vs.xi, P.vs.w
    ref = w * 1.03 * (1.0 + 0.021 * xi[:, 0] - 0.017 * xi[:, 1])
    return np.max(np.abs(P.feq(1.03, 0.021, -0.017, 1.01) - ref)) < 1e-15


def _p_l1():
    """Eq. slb decays with the viscosity tau - dt/2 (Sec. 2.2)."""
    P = oracle.Problem("D2Q9", 2, 128, 1, 0.02, kn_convention="paper", scheme="first_order")
    f = P.init_shear(1e-4)
    d = P.run(f, int(30 / P.dt))
    return abs(oracle.decay_fit(d[:, 0], d[:, 4], 1.0) / (P.tau - 0.5 * P.dt) - 1) < 1e-3


def _p_m2():
    """The driven DVM reaches the continuous reduced-DVM response (Sec. 3.3)."""
    amp, phi, n, kn, nx = 1e-4, 1.0, 8, 0.5, 64
    g, w = oracle.quadrature.gauss_hermite(n)
    dt = oracle.dvm_dt(n, nx)
    t, A, _ = oracle.run_dvm(n, nx, kn, 0.0, int(30.0 / dt), kn_convention="paper", force_amp=amp, force_freq=phi)
    sel = t >= t[-1] - 4 * np.pi / phi
    X = np.stack([np.cos(phi * t[sel]), np.sin(phi * t[sel])], axis=1)
    (a, b), *_ = np.linalg.lstsq(X, A[sel], rcond=None)
    return abs((a - 1j * b) / amp / linear.dvm_forced_response(g, w, kn, phi) - 1) < 3e-3


def _p_n2():
    """Second-order upwind history equals the linear-mode propagation with its symbol."""
    P = oracle.Problem("D2Q16-GH", 2, 32, 1, 0.1, streaming="upwind2")
    f = P.init_shear(1e-6)
    d = P.run(f, 100)
    A, S = linear.lb_linear_history(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, 1e-6, 100, streaming="upwind2")
    return bool(np.max(np.abs(d[:, 4] - A)) < 1e-5 * np.max(np.abs(A)) and
                np.max(np.abs(d[:, 5] - S)) < 1e-5 * np.max(np.abs(S)))


PINS = {"P-c": _p_c, "P-e": _p_e, "P-j1": _p_j1, "P-j2": _p_j2, "P-j3": _p_j3, "P-k1": _p_k1, "P-l1": _p_l1,
        "P-m2": _p_m2, "P-n2": _p_n2}


def test_all_pins_hold_for_the_oracle():
    assert all(fn() for fn in PINS.values())


@pytest.mark.parametrize("plant,expect_failing", [
    (1, {"P-j1", "P-j2", "P-j3"}),
    (2, {"P-j2", "P-j3"}),
    (3, {"P-j2", "P-j3"}),
    (4, {"P-e"}),
    (5, {"P-c", "P-k1"}),
    (6, {"P-e"}),
    (7, {"P-l1"}),
    (8, {"P-m2"}),
    (9, {"P-n2"}),
])
def test_planted_mistake_is_caught(plant, expect_failing):
    with oracle.planted(plant):
        failing = {name for name, fn in PINS.items() if not fn()}
    assert expect_failing <= failing
