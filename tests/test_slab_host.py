"""Host logic of the slab decomposition (no GPU): the row split, the neighbours, the FP64
combination of the bands' grid sums, and the exchange schedule on CPU ranks (gloo, world
sizes 2 and 3) with a toy lattice: each band shifts its planes by lattice vectors (exact
periodic streaming, the on-lattice step of Sec. 2.3) using ghost rows that only the
exchange fills; the bands together must reproduce the undivided grid bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_0908_4520_gb300 import slab  # noqa: E402

E = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (2, 1), (-1, -2), (1, 2)]  # plane velocities
GY = 2  # max |e_y|


class ToyLattice:
    """Numpy stand-in with the halo interface of Lattice: planes [a][y + GY][x], exact shift
    by e_a, periodic in x; like the library's kernels it writes its own periodic images into
    its ghost rows, which the exchange must then overwrite."""

    def __init__(self, band):
        self.ny, self.nx = band.shape[1:]
        self.f = np.zeros((len(E), self.ny + 2 * GY, self.nx))
        self.f[:, GY:GY + self.ny] = band
        self._own_images()

    def _own_images(self):
        self.f[:, :GY] = self.f[:, self.ny:self.ny + GY]
        self.f[:, self.ny + GY:] = self.f[:, GY:2 * GY]

    def halo_bytes(self):
        return len(E) * GY * self.nx

    def halo_pack(self, side, buf):
        r0 = GY if side == 0 else self.ny
        buf.copy_(torch.from_numpy(self.f[:, r0:r0 + GY].reshape(-1).copy()))

    def halo_unpack(self, side, buf):
        r0 = 0 if side == 0 else self.ny + GY
        self.f[:, r0:r0 + GY] = buf.numpy().reshape(len(E), GY, self.nx)

    def step(self):
        g = np.empty_like(self.f)
        for a, (ex, ey) in enumerate(E):
            g[a, GY:GY + self.ny] = np.roll(self.f[a, GY - ey:GY - ey + self.ny], ex, axis=1)
        self.f = g
        self._own_images()

    def band(self):
        return self.f[:, GY:GY + self.ny].copy()


def undivided(grid, levels):
    f = grid.copy()
    for _ in range(levels):
        f = np.stack([np.roll(np.roll(f[a], ey, axis=0), ex, axis=1) for a, (ex, ey) in enumerate(E)])
    return f


def test_rows_and_neighbours():
    assert slab.slab_rows(10, 3) == [(0, 3), (3, 6), (6, 10)]
    assert slab.slab_rows(8, 1) == [(0, 8)]
    with pytest.raises(ValueError):
        slab.slab_rows(2, 3)
    assert slab.neighbours(0, 3) == (2, 1) and slab.neighbours(2, 3) == (1, 0)
    assert slab.neighbours(0, 1) == (0, 0)


def test_records_combine_to_the_grid_sums():
    """Bands of 3 and 5 rows of an 8-row grid: mass, momentum and H add; the amplitudes,
    normalised per band, add with weights 3/8 and 5/8; flags take the maximum."""
    a = np.array([[0.5, 10.0, 1.0, 2.0, 0.4, 0.04, 7.0, 0.0]])
    b = np.array([[0.5, 20.0, -1.0, 3.0, 0.8, 0.08, 9.0, 1.0]])
    g = slab.combine_records([slab.weight_record(a, 3, 8), slab.weight_record(b, 5, 8)])
    np.testing.assert_allclose(g[0], [0.5, 30.0, 0.0, 5.0, 0.4 * 3 / 8 + 0.8 * 5 / 8, 0.04 * 3 / 8 + 0.08 * 5 / 8,
                                      16.0, 1.0])


def test_local_transport_reproduces_the_grid():
    rng = np.random.default_rng(7)
    ny, nx, levels = 11, 6, 9
    grid = rng.standard_normal((len(E), ny, nx))
    rows = slab.slab_rows(ny, 3)
    bands = [slab.Band(ToyLattice(grid[:, y0:y1]), ny, (y0, y1), lambda n: torch.zeros(n, dtype=torch.float64))
             for y0, y1 in rows]
    t = slab.LocalTransport()
    t.exchange_all(bands)
    for _ in range(levels):
        for b in bands:
            b.lattice.step()
        t.exchange_all(bands)
    got = np.concatenate([b.lattice.band() for b in bands], axis=1)
    np.testing.assert_array_equal(got, undivided(grid, levels))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(11)
    ny, nx, levels = 9, 5, 7
    grid = rng.standard_normal((len(E), ny, nx))
    rows = slab.slab_rows(ny, world)[rank]
    band = slab.Band(ToyLattice(grid[:, rows[0]:rows[1]]), ny, rows, lambda n: torch.zeros(n, dtype=torch.float64))
    t = slab.DistTransport(dist, rank, world)
    band.exchange(t)
    for _ in range(levels):
        band.lattice.step()
        band.exchange(t)
    # grid sums: each band's (t, mass, mom_x, mom_y, amp, shear, H, flags) of its own rows
    f = band.lattice.band()
    rec = np.array([[0.25, f.sum(), f[1].sum(), f[3].sum(), 2.0 * f[0].mean(), 0.0, (f * f).sum(), float(rank)]])
    g = t.allreduce_records(slab.weight_record(rec, rows[1] - rows[0], ny))
    out[rank] = (rows, f, g)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_exchange_edges_and_reduce_sums(world):
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    rng = np.random.default_rng(11)
    grid = rng.standard_normal((len(E), 9, 5))
    want = undivided(grid, 7)
    got = np.concatenate([out[r][1] for r in range(world)], axis=1)
    np.testing.assert_array_equal(got, want)
    for r in range(world):
        g = out[r][2][0]
        np.testing.assert_allclose(g[1], want.sum(), rtol=1e-14)
        np.testing.assert_allclose(g[4], 2.0 * want[0].mean(), rtol=1e-14)
        np.testing.assert_allclose(g[6], (want * want).sum(), rtol=1e-14)
        assert g[7] == world - 1
