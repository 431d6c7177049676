"""Pins of the driven reduced DVM (Sec. 3.3, Eqs. LBGK, ga, gb; force of Sec. 4).

P-m1  The continuous reduced DVM's periodic response H(phi) (oracle/linear.py) tends
      to Navier-Stokes, 1 / (i phi + tau), with an error of order tau^2, and to the R13
      closed form printed in Sec. 4 with an error of order tau^3: the kinetic equation's
      response agrees with the 13-moment theory one order beyond Navier-Stokes.
P-m2  The oracle's driven DVM (Strang splitting, exact relaxation and force, Lax-Wendroff)
      reaches that response, converging at second order in dx (cfl fixed).
P-m3  With force_amp = 0 the driven solver is the free one.
"""
import numpy as np
import pytest

import oracle
from oracle import linear, quadrature


@pytest.mark.parametrize("n", [8, 20])
def test_dvm_response_limits(n):
    g, w = quadrature.gauss_hermite(n)
    e_ns, e_r13 = [], []
    for tau in (1e-2, 1e-3):
        H = linear.dvm_forced_response(g, w, tau, 1.0)
        e_ns.append(abs(H * (1j + tau) - 1))
        e_r13.append(abs(H / linear.r13_response(tau, 1.0) - 1))
    assert 80 < e_ns[0] / e_ns[1] < 120          # tau^2
    assert 800 < e_r13[0] / e_r13[1] < 1200      # tau^3
    assert e_r13[0] < 1e-6 and e_r13[1] < 1e-3 * e_ns[1]


def driven_dvm_response(n, nx, kn, amp=1e-4, phi=1.0):
    dt = oracle.dvm_dt(n, nx)
    nsteps = int(max(10.0 / kn, 30.0) / dt)
    t, A, S = oracle.run_dvm(n, nx, kn, 0.0, nsteps, kn_convention="paper", force_amp=amp, force_freq=phi)
    sel = t >= t[-1] - 4 * np.pi / phi
    X = np.stack([np.cos(phi * t[sel]), np.sin(phi * t[sel])], axis=1)
    (a, b), *_ = np.linalg.lstsq(X, A[sel], rcond=None)
    return (a - 1j * b) / amp


@pytest.mark.parametrize("n,kn", [(8, 0.1), (8, 1.5), (20, 0.5)])
def test_driven_dvm_converges_to_response(n, kn):
    g, w = quadrature.gauss_hermite(n)
    H = linear.dvm_forced_response(g, w, kn, 1.0)
    errs = [abs(driven_dvm_response(n, nx, kn) / H - 1) for nx in (64, 128, 256)]
    assert errs[-1] < 2e-4
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 2.5


def test_unforced_driven_solver_is_the_free_one():
    t0, A0, S0 = oracle.run_dvm(8, 64, 0.3, 1e-3, 200)
    t1, A1, S1 = oracle.run_dvm(8, 64, 0.3, 1e-3, 200, force_amp=0.0, force_freq=1.0)
    np.testing.assert_array_equal(A0, A1)
    np.testing.assert_array_equal(S0, S1)
