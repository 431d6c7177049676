"""Pins of the oracle's second-order upwind streaming (off-lattice sets).

P-n1  The 1-D Beam-Warming operator's Fourier symbol (oracle/linear.py) is exact at
      |C| = 1 and C = 0, and second-order accurate: |S - exp(-i C theta)| = O(theta^3).
P-n2  The oracle's shear-wave history equals the linear-mode propagation with that
      symbol (and differs from Lax-Wendroff's), free and driven.
P-n3  Mass and momentum are conserved (the weights sum to one) at large amplitude.
P-n4  The decay rate tends to the Navier-Stokes value tau at Kn = 0.001 (k = 1, T = 1),
      at least at second order in dx.
"""
import numpy as np
import pytest

import oracle
from oracle import linear


def test_upwind_symbol_exact_cases_and_order():
    dx, dt = 0.1, 0.1
    th = dx
    xi = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 0.0]])
    S = linear.stream_symbol(xi, dx, dt, 1.0, None, "upwind2")
    np.testing.assert_allclose(S, [np.exp(-1j * th), np.exp(1j * th), 1.0], atol=1e-15)
    errs = []
    for h in (0.1, 0.05, 0.025):
        xi = np.array([[0.4, 0.0], [-0.7, 0.0]])
        S = linear.stream_symbol(xi, h, h, 1.0, None, "upwind2")
        errs.append(np.max(np.abs(S - np.exp(-1j * xi[:, 0] * h))))
    assert 7 < errs[0] / errs[1] < 9 and 7 < errs[1] / errs[2] < 9


@pytest.mark.parametrize("name,N", [("D2Q16-GH", 2), ("D2Q36-GH", 3), ("D2Q64-GH", 4), ("D2Q36-GH", 1)])
def test_upwind_history_equals_linear_scheme(name, N):
    P = oracle.Problem(name, N, 32, 1, 0.1, streaming="upwind2", isothermal=(N == 1))
    f = P.init_shear(1e-6)
    d = P.run(f, 200)
    A, S = linear.lb_linear_history(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, 1e-6, 200, None, N == 1,
                                    streaming="upwind2")
    assert np.max(np.abs(d[:, 4] - A)) < 1e-5 * np.max(np.abs(A))
    assert np.max(np.abs(d[:, 5] - S)) < 1e-5 * np.max(np.abs(S))
    A_lw, _ = linear.lb_linear_history(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, 1e-6, 200, None, N == 1)
    assert np.max(np.abs(A_lw - A)) > 1e-3 * np.max(np.abs(A))


def test_upwind_forced_history_equals_linear_scheme():
    amp, phi = 1e-5, 1.3
    P = oracle.Problem("D2Q36-GH", 3, 32, 1, 0.1, streaming="upwind2", force_amp=amp, force_freq=phi)
    f = P.init_shear(0.0)
    d = P.run(f, 300)
    M = linear.lb_mode_matrix(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, 1.0, None, False, "upwind2")
    Ssym = linear.stream_symbol(P.vs.xi, P.dx, P.dt, 1.0, None, "upwind2")
    fh = np.zeros(P.Q, dtype=complex)
    A = np.empty(301)
    for n in range(301):
        g = amp * np.cos(phi * n * P.dt) / 2j
        A[n] = -2.0 * (np.sum(P.vs.xi[:, 1] * fh) + 0.5 * P.dt * g).imag
        fh = M @ fh + Ssym * (P.dt * P.vs.w * P.vs.xi[:, 1] * g)
    assert np.max(np.abs(d[:, 4] - A)) < 1e-5 * np.max(np.abs(A))


def test_upwind_conserves_mass_and_momentum():
    P = oracle.Problem("D2Q36-GH", 3, 24, 12, 0.2, streaming="upwind2")
    f = P.init_shear(0.05, 0.03)
    d = P.run(f, 60)
    np.testing.assert_allclose(d[:, 1], d[0, 1], rtol=1e-13)
    assert np.max(np.abs(d[:, 2] - d[0, 2])) < 1e-13 * d[0, 1]
    assert np.max(np.abs(d[:, 3] - d[0, 3])) < 1e-13 * d[0, 1]


def test_upwind_navier_stokes_limit():
    errs = []
    for nx in (32, 64, 128):
        P = oracle.Problem("D2Q16-GH", 2, nx, 1, 1e-3, kn_convention="paper", streaming="upwind2")
        r = linear.lb_decay_rate(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, None, False, "upwind2")
        errs.append(abs(r / P.tau - 1))
    assert errs[-1] < 1e-2
    assert errs[0] / errs[1] > 4 and errs[1] / errs[2] > 4
    # the oracle itself at nx = 64 decays at the linear-mode rate
    P = oracle.Problem("D2Q16-GH", 2, 64, 1, 0.05, kn_convention="paper", streaming="upwind2")
    f = P.init_shear(1e-4)
    d = P.run(f, int(40 / P.dt))
    rate = oracle.decay_fit(d[:, 0], d[:, 4], 1.0)
    lin = linear.lb_decay_rate(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, None, False, "upwind2")
    assert abs(rate / lin - 1) < 1e-3
