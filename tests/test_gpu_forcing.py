"""The body-forced (driven) standing shear wave on the GPU against the FP64 oracle.

Force g_y = A_f sin(x_i) cos(phi t) (Sec. 4, Eq. force, turned so that the flow is
along y), with the Hermite force term of Sec. 2.1 and the force-corrected moments of
Sec. 2.2.  Tolerances as in the free-wave parity tests: FP64 within the oracle's own
rounding (f64_tol), FP32 within 1e-6 relative L2 of u_y on short runs and within the
storage bound f32_tol otherwise.  Random smooth initial fields make u_x, T - 1 and
rho - 1 non-zero, so every force correction (u_y, T, sigma_xy) is exercised.
"""
import math

import numpy as np
import pytest

import oracle
from lbtest import f32_tol, f64_tol, lib, oracle_from_fields, order_map, random_fields, rel_l2
from oracle import linear

pytestmark = pytest.mark.gpu

AMP, PHI = 2e-3, 1.3
SETS_N = [("D2Q16-GH", 2), ("D2Q36-GH", 3), ("D2Q64-GH", 4), ("D2Q37", 3), ("D2Q9", 2), ("D2Q25", 4)]


def forced_pair(quad, N, nx, ny, kn, precision, steps, isothermal=False, amp=AMP, phi=PHI, seed=5):
    Lattice, capi = lib()
    rho, ux, uy, T = random_fields(nx, ny, seed=seed, amp=1e-2)
    L = Lattice(quad, N, nx, ny, kn, precision=precision, isothermal=isothermal, force_amp=amp, force_freq=phi)
    L.init_fields(rho, ux, uy, T)
    L.step(steps)
    P = oracle.Problem(quad, N, nx, ny, kn, isothermal=isothermal, force_amp=amp, force_freq=phi)
    f = oracle_from_fields(P, rho, ux, uy, T)
    d = P.run(f, steps)
    return L, P, f, d, capi


@pytest.mark.parametrize("quad,N", SETS_N)
def test_forced_f64_populations_and_records(quad, N):
    steps = 30
    L, P, f, d, capi = forced_pair(quad, N, 70, 9, 0.2, "f64", steps)
    g = L.populations()
    perm = order_map(capi, quad, P)
    w = P.vs.w[perm][:, None, None]
    tol = f64_tol(steps, 1e-2)
    assert rel_l2(g - w, f[perm] - w) < tol
    m, o = L.moments(), P.moments(f, steps)
    assert rel_l2(m["uy"], o["uy"]) < tol
    assert rel_l2(m["sxy"], o["sxy"]) < 10 * tol
    assert np.max(np.abs(m["T"] - o["T"])) < 1e-12
    rec = L.diagnostics()
    assert np.max(np.abs(rec["amp"] - d[:, 4])) < tol * np.max(np.abs(d[:, 4]))
    assert np.max(np.abs(rec["mom_y"] - d[:, 3])) < tol * np.max(np.abs(d[:, 3])) + 1e-13
    assert np.max(np.abs(rec["shear"] - d[:, 5])) < 10 * tol * np.max(np.abs(d[:, 5]))


@pytest.mark.parametrize("quad,N", SETS_N)
@pytest.mark.parametrize("steps", [10, 40])
def test_forced_f32_moments(quad, N, steps):
    """FP32: 1e-6 relative L2 of u_y on a short run; on a longer one the FP32 storage
    bound f32_tol(steps) (rounding that can accumulate linearly)."""
    L, P, f, d, capi = forced_pair(quad, N, 70, 9, 0.2, "f32", steps, isothermal=True)
    m, o = L.moments(), P.moments(f, steps)
    bound = 1e-6 if steps <= 10 else f32_tol(steps)
    assert rel_l2(m["uy"], o["uy"]) < bound
    unorm = np.linalg.norm(o["uy"])
    assert np.linalg.norm(m["sxy"] - o["sxy"]) / unorm < f32_tol(steps)
    rec = L.diagnostics()
    assert np.max(np.abs(rec["amp"] - d[:, 4])) < bound * np.max(np.abs(d[:, 4]))


def test_forced_run_split_into_calls_equals_one_call():
    Lattice, capi = lib()
    a = Lattice("D2Q36-GH", 3, 130, 17, 0.1, force_amp=AMP, force_freq=PHI).init_shear_wave(1e-3)
    b = Lattice("D2Q36-GH", 3, 130, 17, 0.1, force_amp=AMP, force_freq=PHI).init_shear_wave(1e-3)
    a.step(77)
    for n in (1, 2, 31, 40, 3):
        b.step(n)
    np.testing.assert_array_equal(a.populations(), b.populations())
    np.testing.assert_array_equal(a.diagnostics()["amp"], b.diagnostics()["amp"])


def test_forced_tma_request_is_rejected():
    Lattice, capi = lib()
    with pytest.raises(capi.LBError) as e:
        Lattice("D2Q36-GH", 3, 4096, 64, 0.1, step_kernel="tma", force_amp=1e-3, force_freq=1.0)
    assert e.value.status == capi.LB_ERR_UNSUPPORTED


@pytest.mark.parametrize("precision,tol", [("f64", 1e-6), ("f32", 1e-4)])
def test_driven_response_equals_linear_theory(precision, tol):
    """Periodic steady state of the driven wave (amplitude and phase of u_y against the
    force) equals the linearised scheme's response (oracle/linear.py)."""
    Lattice, capi = lib()
    amp, phi = 1e-4, 1.0
    L = Lattice("D2Q16-GH", 2, 16, 1, 0.5, precision=precision, kn_convention="paper", force_amp=amp,
                force_freq=phi, diag_capacity=4096)
    L.init_shear_wave(0.0)
    n = int(math.ceil(40.0 / L.info["dt"]))
    L.step(n)
    rec = L.diagnostics()
    t, A = rec["t"], rec["amp"]
    sel = t >= t[-1] - 4 * math.pi / phi
    X = np.stack([np.cos(phi * t[sel]), np.sin(phi * t[sel])], axis=1)
    (a, b), *_ = np.linalg.lstsq(X, A[sel], rcond=None)
    U = (a - 1j * b) / amp
    P = oracle.Problem("D2Q16-GH", 2, 16, 1, 0.5, kn_convention="paper")
    H = linear.lb_linear_forced_response(P.vs.xi, P.vs.w, P.omega, P.dx, P.dt, phi)
    assert abs(U / H - 1) < tol
