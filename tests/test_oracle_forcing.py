"""Pins of the oracle's driven standing shear wave (body force, Secs. 2.1, 2.2 and 4).

P-j1  force-term moments: the Hermite force term is the source -g.grad_xi f^eq, so its
      moments are fixed by integration by parts; N = 2 equals the printed N = 2 form.
P-j2  uniform force: sum xi_y f~ grows by dt g(t_n) sum rho per step, exactly.
P-j3  small-amplitude forced history equals the linearised scheme (independent numpy).
P-j4  the linearised forced response tends to Navier-Stokes at second order and follows
      R13 beyond it; the printed R13 formula reduces to Navier-Stokes as Kn -> 0.
P-j5  the oracle's periodic steady state equals the linear response.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import linear, quadrature

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.mark.parametrize("name,N", [("D2Q16-GH", 2), ("D2Q36-GH", 3), ("D2Q64-GH", 4), ("D2Q37", 3),
                                    ("D2Q16-GH", 4)])
def test_force_term_moments(name, N):
    P = oracle.Problem(name, N, 8, 1, 0.1)
    xi = P.vs.xi
    rho, ux, uy, T, g = 1.03, 0.021, -0.017, 1.012, 0.37
    F = P.force(rho, ux, uy, T, g)
    sx, sy = xi[:, 0], xi[:, 1]
    tol = 1e-13 * rho * g
    assert abs(F.sum()) < tol
    assert abs(np.sum(sx * F)) < tol
    assert abs(np.sum(sy * F) - rho * g) < tol
    # second moments (degree 2 <= N, quadrature degree >= N + 2)
    assert abs(np.sum(sx * sy * F) - rho * g * ux) < tol
    assert abs(np.sum(sy * sy * F) - 2 * rho * g * uy) < tol
    assert abs(np.sum(sx * sx * F)) < tol


@pytest.mark.parametrize("T", [1.0, 1.07])
def test_force_term_second_order_form(T):
    # Sec. 2.1, N = 2: F = w rho [g.xi + (g.xi)(u.xi) - g.u]
    P = oracle.Problem("D2Q36-GH", 2, 8, 1, 0.1)
    xi, w = P.vs.xi, P.vs.w
    rho, ux, uy, g = 0.98, 0.03, 0.05, -0.4
    F = P.force(rho, ux, uy, T, g)
    gx = g * xi[:, 1]
    ref = w * rho * (gx + gx * (ux * xi[:, 0] + uy * xi[:, 1]) - g * uy)
    np.testing.assert_allclose(F, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("name,N", [("D2Q36-GH", 3), ("D2Q37", 3), ("D2Q9", 2)])
def test_uniform_force_momentum_budget(name, N):
    amp, phi = 2e-3, 0.7
    P = oracle.Problem(name, N, 16, 4, 0.3, force_amp=amp, force_freq=phi, force_uniform=True)
    f = P.init_shear(1e-3, 5e-4)
    d = P.run(f, 30)
    t, mass, mom_y = d[:, 0], d[:, 1], d[:, 3]
    g = amp * np.cos(phi * t)
    # sum xi_y f~ = mom_y - dt/2 g sum rho
    p = mom_y - 0.5 * P.dt * g * mass
    np.testing.assert_allclose(np.diff(p), P.dt * g[:-1] * mass[:-1], rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(mass, mass[0], rtol=1e-13)


@pytest.mark.parametrize("name,N,iso", [("D2Q16-GH", 2, False), ("D2Q36-GH", 3, True), ("D2Q37", 3, False)])
def test_forced_history_matches_linear_scheme(name, N, iso):
    amp, phi = 1e-5, 1.3
    P = oracle.Problem(name, N, 32, 1, 0.1, isothermal=iso, force_amp=amp, force_freq=phi)
    f = P.init_shear(0.0)
    d = P.run(f, 300)
    e = P.vs.e if P.vs.on_lattice else None
    A = linear.lb_linear_forced_history(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, amp, phi, 300, e, iso)
    scale = np.max(np.abs(A))
    assert scale > 1e-7
    assert np.max(np.abs(d[:, 4] - A)) < 1e-5 * scale


def test_linear_response_navier_stokes_and_r13_limits():
    vs = quadrature.velocity_set("D2Q16-GH")
    errs = []
    for nx in (32, 64, 128):
        P = oracle.Problem("D2Q16-GH", 2, nx, 1, 1e-3, kn_convention="paper")
        H = linear.lb_linear_forced_response(vs.xi, vs.w, P.omega, P.dx, P.dt, 1.0)
        errs.append(abs(H / linear.ns_response(1e-3, 1.0) - 1))
    assert errs[-1] < 3e-4
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5  # second order
    # beyond Navier-Stokes: at Kn = 0.1 the response is closer to R13 than to NS
    P = oracle.Problem("D2Q16-GH", 2, 128, 1, 0.1, kn_convention="paper")
    H = linear.lb_linear_forced_response(vs.xi, vs.w, P.omega, P.dx, P.dt, 1.0)
    e_ns = abs(H / linear.ns_response(0.1, 1.0) - 1)
    e_r13 = abs(H / linear.r13_response(0.1, 1.0) - 1)
    assert e_r13 < 1e-3 < 5e-3 < e_ns
    # the printed R13 formula: Navier-Stokes to first order in Kn
    for kn in (1e-5, 1e-4):
        assert abs(linear.r13_response(kn, 0.8) / linear.ns_response(kn, 0.8) - 1) < 5 * kn * kn


def test_periodic_steady_state_equals_linear_response():
    amp, phi = 1e-5, 1.0
    P = oracle.Problem("D2Q16-GH", 2, 16, 1, 0.5, kn_convention="paper", force_amp=amp, force_freq=phi)
    f = P.init_shear(0.0)
    n = int(math.ceil(40.0 / P.dt))
    d = P.run(f, n)
    t, A = d[:, 0], d[:, 4]
    sel = t >= t[-1] - 2 * 2 * math.pi / phi
    X = np.stack([np.cos(phi * t[sel]), np.sin(phi * t[sel])], axis=1)
    (a, b), *_ = np.linalg.lstsq(X, A[sel], rcond=None)
    U = (a - 1j * b) / amp
    H = linear.lb_linear_forced_response(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, phi)
    assert abs(U / H - 1) < 1e-4
