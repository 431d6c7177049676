"""Slab decomposition on one GPU: the bands of one grid as separate lattices whose ghost rows
are filled between levels by lb_halo_pack / lb_halo_unpack through device buffers (the
exchange code of the multi-GPU split, with the copies local), against the undivided lattice:
populations bit for bit (the per-cell arithmetic does not depend on where a band ends), the
grid sums combined in FP64 equal to the rounding of their partial sums."""
import numpy as np
import pytest

from lbtest import lib
from paper_0908_4520_gb300 import slab

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("quad,N,nx,ny,parts,kernel,prec", [("D2Q36-GH", 3, 96, 24, 2, "plain", "f32"),
                                                            ("D2Q37", 3, 70, 21, 3, "plain", "f32"),
                                                            ("D2Q16-GH", 2, 64, 10, 3, "plain", "f32"),
                                                            ("D2Q36-GH", 3, 240, 60, 2, "tma", "f32"),
                                                            ("D2Q36-GH", 3, 240, 60, 3, "tma_store", "f32"),
                                                            ("D2Q37", 3, 256, 48, 2, "tma", "f32"),
                                                            ("D2Q37", 3, 70, 21, 3, "plain", "f64"),
                                                            ("D2Q36-GH", 3, 96, 24, 2, "plain", "f64"),
                                                            ("D2Q36-GH", 3, 240, 60, 2, "tma", "f16")])
def test_bands_equal_the_undivided_lattice(quad, N, nx, ny, parts, kernel, prec):
    """FP32 and FP64: bit for bit.  16-bit storage (one storage scale for every band and the
    undivided lattice): the stochastic-rounding streams are seeded by each band's own cell
    index, so bands and the undivided lattice carry independent rounding noise of the same
    statistics (std at most 2^-12 of a deviation per store for FP16): after 23 levels the
    fields differ by well under 5e-3 of their norm."""
    import torch

    Lattice, capi = lib()
    stream = torch.cuda.Stream()
    kw = dict(stream=stream.cuda_stream, step_kernel=kernel, diag_capacity=64, precision=prec)
    if prec in ("f16", "bf16"):
        # the halo rows travel as stored values: every band takes the same storage scale
        kw["storage_scale"] = 2.0 * 3e-3
    whole = Lattice(quad, N, nx, ny, 0.2, **kw).init_fields(*slab.shear_wave_band(nx, ny, (0, ny), 1e-3, 2e-3))
    bands = []
    for rows in slab.slab_rows(ny, parts):
        L = Lattice(quad, N, nx, rows[1] - rows[0], 0.2, **kw)
        L.init_fields(*slab.shear_wave_band(nx, ny, rows, 1e-3, 2e-3))
        with torch.cuda.stream(stream):
            bands.append(slab.Band(L, ny, rows, lambda n: torch.empty(n, dtype=torch.uint8, device="cuda")))
    t = slab.LocalTransport()
    t.exchange_all(bands)
    levels = 23
    for _ in range(levels):
        whole.step(1)
        for b in bands:
            b.lattice.step(1)
        t.exchange_all(bands)
    got = np.concatenate([b.lattice.populations() for b in bands], axis=1)
    g = t.allreduce_records([b.weighted_records() for b in bands])
    ref = whole.diagnostics()
    assert g.shape[0] == len(ref) == levels + 1
    if prec in ("f16", "bf16"):
        wp = whole.populations()
        # the deviations from each velocity's grid mean (its w_a rho0 background)
        dref = wp - wp.mean(axis=(1, 2), keepdims=True)
        assert np.linalg.norm(got - wp) / np.linalg.norm(dref) < 5e-3
        np.testing.assert_allclose(g[:, 4], ref["amp"], rtol=5e-3, atol=1e-9)
        for b in bands:
            b.lattice.close()
        whole.close()
        return
    np.testing.assert_array_equal(got, whole.populations())
    np.testing.assert_allclose(g[:, 4], ref["amp"], rtol=1e-6, atol=1e-15)
    np.testing.assert_allclose(g[:, 1], ref["mass"], rtol=1e-12)
    np.testing.assert_allclose(g[:, 6], ref["hnorm"], rtol=1e-6)
    for b in bands:
        b.lattice.close()
    whole.close()


def test_halo_calls_check_their_arguments():
    Lattice, capi = lib()
    L = Lattice("D2Q36-GH", 3, 64, 8, 0.1)
    with pytest.raises(capi.LBError) as e:
        capi.lb_halo_pack(L.h, 0, 0)
    assert e.value.status == capi.LB_ERR_STATE  # before init
    L.init_shear_wave(1e-3)
    # 36 planes x one ghost row (Lax-Wendroff) x a padded row of at least nx + 16 FP32 values
    n = capi.lb_halo_bytes(L.h)
    assert n % (36 * 4) == 0 and n // (36 * 4) >= 64 + 16
    with pytest.raises(capi.LBError) as e:
        capi.lb_halo_pack(L.h, 2, 0)
    assert e.value.status == capi.LB_ERR_ARG
    L.close()
