"""The first-order Hermite expansion (N = 1, Sec. 3.3, Eq. lbm1) and the first-order
"standard LB" scheme (Eq. slb, Sec. 2.2) on the GPU against the FP64 oracle.

Tolerances as in the parity tests: FP64 within the oracle's own rounding
(f64_tol), FP32 within 1e-6 relative L2 of u_y on short runs; the two step
kernels (plain loads, TMA-staged) bitwise equal.
"""
import numpy as np
import pytest

import oracle
from lbtest import f32_tol, f64_tol, lib, order_map, rel_l2

pytestmark = pytest.mark.gpu

N1_SETS = ["D2Q16-GH", "D2Q36-GH", "D2Q64-GH", "D2Q37", "D2Q9", "D2Q25"]
SLB_SETS_N = [("D2Q16-GH", 2), ("D2Q36-GH", 3), ("D2Q64-GH", 4), ("D2Q37", 3), ("D2Q9", 2), ("D2Q25", 4),
              ("D2Q36-GH", 1)]


def pair(quad, N, nx, ny, kn, precision, steps, u0=2e-2, u1=1e-2, scheme="second_order", **kw):
    Lattice, capi = lib()
    L = Lattice(quad, N, nx, ny, kn, precision=precision, scheme=scheme, **kw)
    L.init_shear_wave(u0, u1)
    L.step(steps)
    P = oracle.Problem(quad, N, nx, ny, kn, scheme=scheme, isothermal=kw.get("isothermal", False),
                       kn_convention=kw.get("kn_convention", "lambda"), force_amp=kw.get("force_amp", 0.0),
                       force_freq=kw.get("force_freq", 0.0))
    f = P.init_shear(u0, u1)
    d = P.run(f, steps)
    return L, P, f, d, capi


def check_f64(L, P, f, d, capi, quad, steps):
    perm = order_map(capi, quad, P)
    w = P.vs.w[perm][:, None, None]
    tol = f64_tol(steps, 1e-2)
    assert rel_l2(L.populations() - w, f[perm] - w) < tol
    rec = L.diagnostics()
    assert len(rec) == steps + 1
    assert np.max(np.abs(rec["amp"] - d[:, 4])) < tol * np.max(np.abs(d[:, 4]))
    assert np.max(np.abs(rec["shear"] - d[:, 5])) < 10 * tol * np.max(np.abs(d[:, 5]))
    assert np.max(np.abs(rec["mass"] - d[:, 1])) < 1e-12 * d[0, 1]
    m, o = L.moments(), P.moments(f, steps)
    assert rel_l2(m["uy"], o["uy"]) < tol
    assert rel_l2(m["sxy"], o["sxy"]) < 10 * tol


@pytest.mark.parametrize("quad", N1_SETS)
def test_n1_f64_matches_oracle(quad):
    check_f64(*pair(quad, 1, 100, 11, 0.3, "f64", 25), quad, 25)


@pytest.mark.parametrize("quad", N1_SETS)
def test_n1_f32_moments(quad):
    L, P, f, d, capi = pair(quad, 1, 100, 11, 0.3, "f32", 20, u0=1e-3, u1=1e-3)
    m, o = L.moments(), P.moments(f, 20)
    assert rel_l2(m["uy"], o["uy"]) < 1e-6
    assert np.linalg.norm(m["sxy"] - o["sxy"]) / np.linalg.norm(o["uy"]) < f32_tol(20)
    rec = L.diagnostics()
    assert np.max(np.abs(rec["amp"] - d[:, 4])) < 1e-6 * np.max(np.abs(d[:, 4]))


@pytest.mark.parametrize("quad,N", SLB_SETS_N)
def test_first_order_scheme_f64_matches_oracle(quad, N):
    L, P, f, d, capi = pair(quad, N, 100, 11, 0.3, "f64", 25, scheme="first_order")
    assert abs(L.info["omega"] - P.dt / P.tau) < 1e-15
    check_f64(L, P, f, d, capi, quad, 25)


@pytest.mark.parametrize("quad,N", [("D2Q36-GH", 3), ("D2Q37", 3), ("D2Q16-GH", 1)])
def test_first_order_scheme_forced_f64_matches_oracle(quad, N):
    L, P, f, d, capi = pair(quad, N, 70, 9, 0.3, "f64", 30, scheme="first_order", force_amp=2e-3,
                            force_freq=1.3)
    check_f64(L, P, f, d, capi, quad, 30)
    assert np.max(np.abs(L.diagnostics()["mom_y"] - d[:, 3])) < 1e-12 * np.max(np.abs(d[:, 3])) + 1e-13


@pytest.mark.parametrize("quad,N", [("D2Q36-GH", 3), ("D2Q37", 3), ("D2Q9", 2), ("D2Q36-GH", 1)])
def test_first_order_scheme_f32_moments(quad, N):
    L, P, f, d, capi = pair(quad, N, 100, 11, 0.3, "f32", 20, u0=1e-3, u1=1e-3, scheme="first_order")
    m, o = L.moments(), P.moments(f, 20)
    assert rel_l2(m["uy"], o["uy"]) < 1e-6
    rec = L.diagnostics()
    assert np.max(np.abs(rec["amp"] - d[:, 4])) < 1e-6 * np.max(np.abs(d[:, 4]))


@pytest.mark.parametrize("quad,N,prec,scheme", [("D2Q36-GH", 1, "f32", "second_order"),
                                                ("D2Q37", 1, "f32", "second_order"),
                                                ("D2Q64-GH", 1, "bf16", "second_order"),
                                                ("D2Q36-GH", 3, "f32", "first_order"),
                                                ("D2Q37", 3, "f32", "first_order"),
                                                ("D2Q36-GH", 3, "f16", "first_order")])
def test_tma_and_plain_kernels_are_bitwise_equal(quad, N, prec, scheme):
    Lattice, capi = lib()
    kw = dict(precision=prec, scheme=scheme)
    a = Lattice(quad, N, 200, 23, 0.3, step_kernel="tma", **kw).init_shear_wave(1e-3, 1e-3)
    b = Lattice(quad, N, 200, 23, 0.3, step_kernel="plain", **kw).init_shear_wave(1e-3, 1e-3)
    assert a.info["tma_staged"] == 1 and b.info["tma_staged"] == 0
    a.step(29)
    b.step(29)
    np.testing.assert_array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_n1_16bit_storage_tracks_f32(prec):
    Lattice, capi = lib()
    amp = {}
    for p in ("f32", prec):
        L = Lattice("D2Q36-GH", 1, 128, 16, 0.1, precision=p).init_shear_wave(1e-4)
        L.step(300)
        amp[p] = L.diagnostics()["amp"]
    assert np.max(np.abs(amp[prec] - amp["f32"])) < 1e-3 * np.max(np.abs(amp["f32"]))


def test_first_order_scheme_decays_with_artificial_viscosity():
    """Eq. slb on the GPU: decay rate tau - dt/2 (Sec. 2.2); Eq. 2order: tau."""
    Lattice, capi = lib()
    rates = {}
    for scheme in ("first_order", "second_order"):
        L = Lattice("D2Q9", 2, 128, 4, 0.02, precision="f64", kn_convention="paper", scheme=scheme,
                    diag_capacity=4096)
        L.init_shear_wave(1e-4)
        inf = L.info
        L.step(int(30 / inf["dt"]))
        rec = L.diagnostics()
        rates[scheme] = oracle.decay_fit(rec["t"], rec["amp"], 1.0)
    tau, dt = inf["tau"], inf["dt"]
    assert abs(rates["first_order"] / (tau - 0.5 * dt) - 1) < 1e-3
    assert abs(rates["second_order"] / tau - 1) < 1e-3
