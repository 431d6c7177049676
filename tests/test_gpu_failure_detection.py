"""Failure detection without a GPU fault: the TMA-staged step kernel's waits are bounded.

With lb_params.test_withhold_stage the producer of block 0 withholds one stage, so nothing
ever completes that stage's barrier; the consumers' waits run out (about a second), the
kernel records status bit 2 and returns, the next synchronising call reports
LB_ERR_TIMEOUT, and the context stays usable for the next lattice.
"""
import numpy as np
import pytest

from lbtest import lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("quad,N,kernel", [("D2Q36-GH", 3, "tma"), ("D2Q37", 3, "tma"), ("D2Q16-GH", 2, "tma"),
                                           ("D2Q36-GH", 3, "tma_store")])
def test_withheld_stage_times_out_and_context_survives(quad, N, kernel):
    """(tma_store: the consumers' waits run out, then the producer's wait for the tile they
    never finish; no store is issued for it.)"""
    Lattice, capi = lib()
    bad = Lattice(quad, N, 256, 96, 0.1, step_kernel=kernel, test_withhold_stage=1).init_shear_wave(1e-3)
    assert bad.info["tma_staged"] == (2 if kernel == "tma_store" else 1)
    bad.step(1)
    with pytest.raises(capi.LBError) as e:
        bad.synchronize()
    assert e.value.status == capi.LB_ERR_TIMEOUT
    bad.close()
    good = Lattice(quad, N, 256, 96, 0.1, step_kernel=kernel).init_shear_wave(1e-3)
    good.step(3)
    good.synchronize()
    rec = good.diagnostics()
    assert len(rec) == 4 and np.all(np.isfinite(rec["amp"]))
    good.close()
