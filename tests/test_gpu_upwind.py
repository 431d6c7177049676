"""Second-order upwind streaming of the Gauss-Hermite product sets on the GPU against the
FP64 oracle (same tolerances as the Lax-Wendroff parity tests).  Grids span several
tiles with ragged tails, and the degenerate shapes (nx = 2, ny = 1) whose upstream
columns and rows are all periodic images.  FP32 storage also runs the TMA-staged kernel
(28-cell tile rows with two halo lanes on each side), bitwise equal to the plain one."""
import numpy as np
import pytest

import oracle
from lbtest import f32_tol, f64_tol, lib, oracle_from_fields, order_map, random_fields, rel_l2

pytestmark = pytest.mark.gpu

SETS_N = [("D2Q16-GH", 2), ("D2Q36-GH", 3), ("D2Q64-GH", 4), ("D2Q16-GH", 4), ("D2Q36-GH", 1)]


def pair(quad, N, nx, ny, kn, precision, steps, u0=2e-2, u1=1e-2, **kw):
    Lattice, capi = lib()
    L = Lattice(quad, N, nx, ny, kn, precision=precision, streaming="upwind2", **kw)
    L.init_shear_wave(u0, u1)
    L.step(steps)
    P = oracle.Problem(quad, N, nx, ny, kn, streaming="upwind2", force_amp=kw.get("force_amp", 0.0),
                       force_freq=kw.get("force_freq", 0.0))
    f = P.init_shear(u0, u1)
    d = P.run(f, steps)
    return L, P, f, d, capi


@pytest.mark.parametrize("quad,N", SETS_N)
def test_upwind_f64_matches_oracle(quad, N):
    steps = 25
    L, P, f, d, capi = pair(quad, N, 100, 11, 0.3, "f64", steps)
    assert L.info["tma_staged"] == 0
    perm = order_map(capi, quad, P)
    w = P.vs.w[perm][:, None, None]
    tol = f64_tol(steps, 1e-2)
    assert rel_l2(L.populations() - w, f[perm] - w) < tol
    rec = L.diagnostics()
    assert np.max(np.abs(rec["amp"] - d[:, 4])) < tol * np.max(np.abs(d[:, 4]))
    assert np.max(np.abs(rec["shear"] - d[:, 5])) < tol * np.max(np.abs(d[:, 5]))
    assert np.max(np.abs(rec["mass"] - d[:, 1])) < 1e-12 * d[0, 1]


@pytest.mark.parametrize("quad,N", SETS_N[:3])
def test_upwind_f32_moments(quad, N):
    L, P, f, d, capi = pair(quad, N, 100, 11, 0.3, "f32", 20, u0=1e-3, u1=1e-3)
    m, o = L.moments(), P.moments(f, 20)
    assert rel_l2(m["uy"], o["uy"]) < 1e-6
    assert np.linalg.norm(m["sxy"] - o["sxy"]) / np.linalg.norm(o["uy"]) < f32_tol(20)


@pytest.mark.parametrize("quad,N,nx,ny", [("D2Q36-GH", 3, 2, 1), ("D2Q16-GH", 2, 6, 3), ("D2Q64-GH", 4, 34, 2),
                                          ("D2Q36-GH", 2, 64, 1), ("D2Q16-GH", 3, 98, 5)])
def test_upwind_f64_edge_shapes(quad, N, nx, ny):
    """Tiny, ragged and degenerate grids from random smooth fields (all modes present)."""
    Lattice, capi = lib()
    steps = 12
    rho, ux, uy, T = random_fields(nx, ny, seed=nx * 131 + ny)
    L = Lattice(quad, N, nx, ny, 0.2, precision="f64", streaming="upwind2").init_fields(rho, ux, uy, T)
    P = oracle.Problem(quad, N, nx, ny, 0.2, streaming="upwind2")
    f = oracle_from_fields(P, rho, ux, uy, T)
    L.step(steps)
    P.run(f, steps, record=False)
    perm = order_map(capi, quad, P)
    w = P.vs.w[perm][:, None, None]
    assert rel_l2(L.populations() - w, f[perm] - w) < f64_tol(steps, 2e-2)


def test_upwind_forced_f64_matches_oracle():
    steps = 30
    L, P, f, d, capi = pair("D2Q36-GH", 3, 70, 9, 0.2, "f64", steps, force_amp=2e-3, force_freq=1.3)
    perm = order_map(capi, "D2Q36-GH", P)
    w = P.vs.w[perm][:, None, None]
    tol = f64_tol(steps, 1e-2)
    assert rel_l2(L.populations() - w, f[perm] - w) < tol
    m, o = L.moments(), P.moments(f, steps)
    assert rel_l2(m["uy"], o["uy"]) < tol


def test_upwind_full_size_conserves_and_differs_from_lax_wendroff():
    Lattice, capi = lib()
    n = 1024
    a = Lattice("D2Q36-GH", 3, n, n, 0.1, streaming="upwind2").init_shear_wave(1e-3, 1e-3)
    b = Lattice("D2Q36-GH", 3, n, n, 0.1).init_shear_wave(1e-3, 1e-3)
    a.step(100)
    b.step(100)
    ra, rb = a.diagnostics(), b.diagnostics()
    assert np.all(ra["flags"] == 0)
    np.testing.assert_allclose(ra["mass"], ra["mass"][0], rtol=1e-6)
    # same physics to O(dx^2): amplitudes agree closely but not bitwise
    assert 0 < np.max(np.abs(ra["amp"] - rb["amp"])) < 1e-3 * abs(rb["amp"][0])


@pytest.mark.parametrize("quad,N,nx,ny", [("D2Q36-GH", 3, 200, 23), ("D2Q16-GH", 2, 90, 7), ("D2Q64-GH", 4, 130, 17),
                                          ("D2Q36-GH", 1, 58, 40)])
def test_upwind_tma_and_plain_kernels_are_bitwise_equal(quad, N, nx, ny):
    Lattice, capi = lib()
    a = Lattice(quad, N, nx, ny, 0.3, streaming="upwind2", step_kernel="tma").init_shear_wave(1e-3, 1e-3)
    b = Lattice(quad, N, nx, ny, 0.3, streaming="upwind2", step_kernel="plain").init_shear_wave(1e-3, 1e-3)
    assert a.info["tma_staged"] == 1 and b.info["tma_staged"] == 0
    a.step(29)
    b.step(29)
    np.testing.assert_array_equal(a.populations(), b.populations())
    np.testing.assert_allclose(a.diagnostics()["amp"], b.diagnostics()["amp"], rtol=1e-6, atol=1e-15)


def test_upwind_tma_f32_matches_oracle():
    Lattice, capi = lib()
    L = Lattice("D2Q36-GH", 3, 100, 11, 0.3, streaming="upwind2", step_kernel="tma").init_shear_wave(1e-3, 1e-3)
    L.step(20)
    P = oracle.Problem("D2Q36-GH", 3, 100, 11, 0.3, streaming="upwind2")
    f = P.init_shear(1e-3, 1e-3)
    P.run(f, 20, record=False)
    m, o = L.moments(), P.moments(f, 20)
    assert rel_l2(m["uy"], o["uy"]) < 1e-6
