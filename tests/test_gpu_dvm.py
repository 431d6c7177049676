"""GPU discrete velocity method (Sec. 3.3, reduced linearised BGK, free and driven) against the
FP64 oracle DVM, and the same-quadrature LB-vs-DVM cross-check of Sec. 3.2 on the GPU."""
import numpy as np
import pytest

import oracle
from lbtest import lib

pytestmark = pytest.mark.gpu

U0 = 1e-3


@pytest.mark.parametrize("n,nx", [(4, 32), (8, 100), (20, 64), (6, 257)])
def test_gpu_dvm_matches_oracle(n, nx):
    Lattice, capi = lib()
    kns = [0.05, 0.3, 1.0, 4.0]
    taus = [oracle.collision_time(k) for k in kns]
    nsteps = 300
    A, S = capi.lb_dvm_run(taus, n, nx, U0, nsteps)
    for i, kn in enumerate(kns):
        _, Ao, So = oracle.run_dvm(n, nx, kn, U0, nsteps)
        # FP64 on both sides; different fused-multiply-add contraction and summation order
        assert np.max(np.abs(A[i] - Ao)) < 1e-12 * U0 * (nsteps + 1)
        assert np.max(np.abs(S[i] - So)) < 1e-12 * U0 * (nsteps + 1)


def test_gpu_dvm_rejects_oversize_and_bad_arguments():
    Lattice, capi = lib()
    with pytest.raises(capi.LBError) as e:
        capi.lb_dvm_run([0.1], 64, 1 << 16, U0, 1)
    assert e.value.status == capi.LB_ERR_UNSUPPORTED
    with pytest.raises(capi.LBError) as e:
        capi.lb_dvm_run([-1.0], 4, 64, U0, 1)
    assert e.value.status == capi.LB_ERR_ARG


@pytest.mark.parametrize("n,N,kn", [(4, 2, 0.1), (6, 3, 1.0), (8, 4, 0.5)])
def test_lb_and_dvm_agree_same_quadrature_on_gpu(n, N, kn):
    """Sec. 3.2: the lattice model and the DVM with the same Gauss-Hermite rule solve the
    same velocity-discrete system; both second order, they agree to 1e-3 U0 at nx = 128."""
    Lattice, capi = lib()
    nx = 128
    L = Lattice(f"D2Q{n * n}-GH", N, nx, 1, kn, precision="f64", diag_capacity=8192).init_shear_wave(U0)
    nsteps = int(6.0 / L.info["dt"])
    L.step(nsteps)
    rec = L.diagnostics()
    dtd = oracle.dvm_dt(n, nx)
    Ad, _ = capi.lb_dvm_run([oracle.collision_time(kn)], n, nx, U0, int(6.0 / dtd) + 2)
    td = dtd * np.arange(Ad.shape[1])
    assert np.max(np.abs(rec["amp"] - np.interp(rec["t"], td, Ad[0]))) / U0 < 1e-3


@pytest.mark.parametrize("n,nx,phi", [(8, 100, 1.0), (20, 64, 0.7), (6, 257, 0.0)])
def test_gpu_driven_dvm_matches_oracle(n, nx, phi):
    Lattice, capi = lib()
    kns = [0.1, 0.5, 1.5]
    taus = [oracle.collision_time(k) for k in kns]
    nsteps, amp = 400, 1e-3
    A, S = capi.lb_dvm_run_forced(taus, n, nx, 0.0, amp, phi, nsteps)
    for i, kn in enumerate(kns):
        _, Ao, So = oracle.run_dvm(n, nx, kn, 0.0, nsteps, force_amp=amp, force_freq=phi)
        scale = max(np.max(np.abs(Ao)), amp)
        assert np.max(np.abs(A[i] - Ao)) < 1e-12 * scale * (nsteps + 1)
        assert np.max(np.abs(S[i] - So)) < 1e-12 * scale * (nsteps + 1)


def test_lb_and_dvm_driven_responses_agree():
    """Sec. 4, Fig. exm: with the same Gauss-Hermite rule the driven lattice model and the
    driven DVM give the same periodic response of u_y (amplitude and phase), here within
    0.1 % at nx = 64 for the 8-point rule (D2Q64-GH, N = 4)."""
    Lattice, capi = lib()
    amp, phi, nx, kn = 1e-4, 1.0, 64, 0.5

    def fit(t, A):
        sel = t >= t[-1] - 4 * np.pi / phi
        X = np.stack([np.cos(phi * t[sel]), np.sin(phi * t[sel])], axis=1)
        (a, b), *_ = np.linalg.lstsq(X, A[sel], rcond=None)
        return (a - 1j * b) / amp

    L = Lattice("D2Q64-GH", 4, nx, 1, kn, precision="f64", kn_convention="paper", isothermal=True,
                force_amp=amp, force_freq=phi, diag_capacity=1 << 14)
    L.init_shear_wave(0.0)
    L.step(int(30.0 / L.info["dt"]))
    rec = L.diagnostics()
    U_lb = fit(rec["t"], rec["amp"])
    dtd = oracle.dvm_dt(8, nx)
    nd = int(30.0 / dtd)
    Ad, _ = capi.lb_dvm_run_forced([kn], 8, nx, 0.0, amp, phi, nd)
    U_dvm = fit(dtd * np.arange(nd + 1), Ad[0])
    assert abs(U_lb / U_dvm - 1) < 1e-3
