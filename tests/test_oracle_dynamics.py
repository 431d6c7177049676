"""Pins of the oracle's time stepping (Eq. 2order, Sec. 2.3 streaming, Sec. 3.3 DVM).

P-d  mass and momentum are conserved to round-off.
P-e  the amplitude history A(n), S(n) of a small shear wave equals the
     linear-mode propagation M(k)^n of the scheme (independent derivation in
     oracle/linear.py), up to O(U0^2) nonlinear terms.
P-f  at Kn = 0.001 the decay rate tends to the Navier-Stokes value nu k^2,
     nu = tau T (Sec. 2.2: viscosity tau R T), second order in dx.
P-g  the reduced linearised-BGK DVM converges at second order to the exact
     single-mode solution exp(B t) of the velocity-discrete system, whose
     eigenvalues are the roots of the dispersion relation.
P-h  LB with a Gauss-Hermite product set and the DVM with the same 1-D rule
     approach the same solution (Sec. 3.2: same velocity discretisation).
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from oracle import linear
from oracle import quadrature as q

U0 = 1e-3


def _exact_single_mode(n, kn, u0, t):
    g, w = q.gauss_hermite(n)
    tau = oracle.collision_time(kn)
    B = -1j * np.diag(g) + (np.outer(np.ones(n), w) - np.eye(n)) / tau
    G0 = np.full(n, u0 / 2j)
    A = np.array([-2 * (w @ (sl.expm(B * tt) @ G0)).imag for tt in t])
    return A, B


@pytest.mark.parametrize("name,N", [("D2Q9", 2), ("D2Q37", 3), ("D2Q25", 4), ("D2Q16-GH", 2), ("D2Q36-GH", 3)])
def test_conservation(oracle_mod, name, N):
    P = oracle.Problem(name, N, 24, 5, 0.3)
    f = P.init_shear(0.05, 0.03)  # large amplitude: nonlinear, compressive
    d = P.run(f, 150)
    assert np.max(np.abs(d[:, 1] - d[0, 1])) < 1e-13 * d[0, 1]
    assert np.max(np.abs(d[:, 2] - d[0, 2])) < 1e-12
    assert np.max(np.abs(d[:, 3] - d[0, 3])) < 1e-12


@pytest.mark.parametrize("name,N,kn", [("D2Q9", 2, 0.1), ("D2Q17", 3, 0.5), ("D2Q21", 4, 1.0),
                                       ("D2Q37", 3, 0.05), ("D2Q16-GH", 2, 0.1), ("D2Q36-GH", 3, 1.0),
                                       ("D2Q64-GH", 4, 0.3), ("D2Q16-int", 2, 0.2)])
def test_linear_mode_history(oracle_mod, name, N, kn):
    P = oracle.Problem(name, N, 32, 3, kn)
    f = P.init_shear(U0)
    d = P.run(f, 80)
    A, S = linear.lb_linear_history(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, U0, 80, e=P.vs.e)
    assert np.max(np.abs(d[:, 4] - A)) < 1e-5 * U0
    assert np.max(np.abs(d[:, 5] - S)) < 1e-5 * np.max(np.abs(S))
    np.testing.assert_allclose(d[:, 0], P.dt * np.arange(81), rtol=1e-14)


def test_linear_mode_isothermal(oracle_mod):
    P = oracle.Problem("D2Q36-GH", 3, 32, 1, 0.2, isothermal=True)
    f = P.init_shear(U0)
    d = P.run(f, 60)
    A, S = linear.lb_linear_history(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, U0, 60, isothermal=True)
    assert np.max(np.abs(d[:, 4] - A)) < 1e-5 * U0


def _ns_rate(name, N, nx, t_end=40.0):
    P = oracle.Problem(name, N, nx, 1, 0.001)
    nsteps = int(round(t_end / P.dt))
    f = P.init_shear(U0)
    d = P.run(f, nsteps)
    t, A = d[:, 0], d[:, 4]
    sel = t > 0.05
    slope = np.polyfit(t[sel], np.log(A[sel]), 1)[0]
    return -slope, P.tau


@pytest.mark.parametrize("name,N", [("D2Q9", 2), ("D2Q37", 3)])
def test_navier_stokes_decay_on_lattice(oracle_mod, name, N):
    r64, nu = _ns_rate(name, N, 64)
    assert abs(r64 / nu - 1) < 0.01
    r32, _ = _ns_rate(name, N, 32)
    # second-order convergence in dx
    assert abs(r32 / nu - 1) / abs(r64 / nu - 1) > 3.0


def test_navier_stokes_decay_lax_wendroff(oracle_mod):
    errs = []
    for nx in (32, 64, 128):
        r, nu = _ns_rate("D2Q16-GH", 2, nx, t_end=20.0)
        errs.append(abs(r / nu - 1))
    assert errs[2] < 0.01
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


@pytest.mark.parametrize("n", [4, 6, 8])
@pytest.mark.parametrize("kn", [0.1, 1.0])
def test_dispersion_roots_are_mode_eigenvalues(n, kn):
    g, w = q.gauss_hermite(n)
    tau = oracle.collision_time(kn)
    roots = linear.dvm_dispersion_roots(g, w, tau)
    _, B = _exact_single_mode(n, kn, U0, [0.0])
    ev = np.linalg.eigvals(B)
    for r in roots:
        assert np.min(np.abs(ev - r)) < 1e-8 * max(1.0, abs(r))


@pytest.mark.parametrize("n,kn", [(4, 0.1), (6, 1.0)])
def test_dvm_converges_to_exact(oracle_mod, n, kn):
    errs = []
    for nx in (64, 128, 256):
        dt = oracle.dvm_dt(n, nx)
        nsteps = int(6.0 / dt)
        t, A, _ = oracle.run_dvm(n, nx, kn, U0, nsteps)
        idx = np.arange(0, nsteps + 1, max(1, nsteps // 30))
        Ae, _ = _exact_single_mode(n, kn, U0, t[idx])
        errs.append(np.max(np.abs(A[idx] - Ae)) / U0)
    assert errs[2] < 2e-4
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


@pytest.mark.parametrize("n,N,kn", [(4, 2, 0.1), (6, 3, 1.0)])
def test_lb_and_dvm_agree_same_quadrature(oracle_mod, n, N, kn):
    nx = 128
    P = oracle.Problem(f"D2Q{n * n}-GH", N, nx, 1, kn)
    nsteps = int(6.0 / P.dt)
    f = P.init_shear(U0)
    d = P.run(f, nsteps)
    tl, Al = d[:, 0], d[:, 4]
    dtd = oracle.dvm_dt(n, nx)
    td, Ad, _ = oracle.run_dvm(n, nx, kn, U0, int(6.0 / dtd) + 2)
    Ad_at = np.interp(tl, td, Ad)
    # both are second-order schemes for the same velocity-discrete system
    assert np.max(np.abs(Al - Ad_at)) / U0 < 1e-3
    Ae, _ = _exact_single_mode(n, kn, U0, tl[:: max(1, nsteps // 30)])
    assert np.max(np.abs(Al[:: max(1, nsteps // 30)] - Ae)) / U0 < 5e-4
