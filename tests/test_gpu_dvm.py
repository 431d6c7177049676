"""GPU discrete velocity method (Sec. 3.3, reduced linearised BGK, unforced) against the
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
