"""Slab decomposition of one periodic grid over several lattices.

The grid's rows are split into bands, one lattice per band (one per GPU under
torch.distributed, or several in one process).  Streaming reads `gy` rows past
a band's edges (Sec. 2.3), so between two levels every band sends its first and
last `gy` rows to its lower and upper neighbours and receives theirs into its
ghost rows (``lb_halo_pack`` / ``lb_halo_unpack``; the rows move as device
buffers).  The grid sums of the diagnostics (mass, momentum, the Fourier
amplitudes of u_y and sigma_xy, the H norm) are combined in FP64 across the
bands.  The rows travel as stored, so with 16-bit storage every band's lattice takes the
same `storage_scale`.  This module only schedules and marshals: the populations are
stepped, packed and unpacked by the library's kernels and copies.
"""
from __future__ import annotations

import math

import numpy as np


def slab_rows(ny: int, parts: int):
    """Rows [y0, y1) of each band of a near-even split of ny rows into `parts` bands."""
    if parts < 1 or parts > ny:
        raise ValueError("need 1 <= parts <= ny")
    edges = [(ny * r) // parts for r in range(parts + 1)]
    return [(edges[r], edges[r + 1]) for r in range(parts)]


def neighbours(rank: int, world: int):
    """(lower, upper) band of a periodic split."""
    return (rank - 1) % world, (rank + 1) % world


# Records are FP64 vectors (t, mass, mom_x, mom_y, amp, shear, hnorm, flags) per level.
_SUMMED = (1, 2, 3, 4, 5, 6)


def weight_record(rec: np.ndarray, rows: int, ny: int) -> np.ndarray:
    """A band's records made additive: amp and shear (normalised by the band's own cell
    count in the kernel) scaled by rows / ny; mass, momentum and H are already sums."""
    out = np.array(rec, dtype=np.float64, copy=True)
    out[..., 4] *= rows / ny
    out[..., 5] *= rows / ny
    return out


def combine_records(weighted) -> np.ndarray:
    """Grid records from the bands' weighted records (sum of the sums; t from the first,
    flags the maximum)."""
    w = [np.asarray(r, dtype=np.float64) for r in weighted]
    out = np.array(w[0], copy=True)
    for i in _SUMMED:
        out[..., i] = sum(r[..., i] for r in w)
    out[..., 7] = np.max([r[..., 7] for r in w], axis=0)
    return out


class LocalTransport:
    """All bands in one process (one GPU or several): the packed rows of band r go
    straight into the ghost rows of its neighbours.  Every band's lattice runs on the same
    stream, so the copies are ordered behind the steps."""

    def exchange_all(self, bands):
        n = len(bands)
        for b in bands:
            b._pack()
        for r, b in enumerate(bands):
            lo, up = bands[(r - 1) % n], bands[(r + 1) % n]
            b._unpack(0, lo.send[1])
            b._unpack(1, up.send[0])

    def allreduce_records(self, weighted):
        return combine_records(weighted)


class DistTransport:
    """One band per rank of a torch.distributed process group (NCCL with device buffers, or
    gloo with host buffers): a batched send/receive with the two neighbours per level and an
    FP64 all-reduce of the grid sums."""

    def __init__(self, dist, rank: int, world: int):
        self.dist, self.rank, self.world = dist, rank, world
        self.lower, self.upper = neighbours(rank, world)

    def exchange(self, send, recv):
        """send[s], recv[s]: buffers of side s (0: lower edge, 1: upper edge)."""
        if self.world == 1:
            recv[0].copy_(send[1])
            recv[1].copy_(send[0])
            return
        d = self.dist
        # messages between one pair of ranks match in order: with two ranks both neighbours
        # are the same rank, and the upper edge arrives first, into the lower ghost rows
        ops = [d.P2POp(d.isend, send[1], self.upper), d.P2POp(d.irecv, recv[0], self.lower),
               d.P2POp(d.isend, send[0], self.lower), d.P2POp(d.irecv, recv[1], self.upper)]
        for req in d.batch_isend_irecv(ops):
            req.wait()

    def allreduce_records(self, weighted_local, device="cpu"):
        import torch

        rec = torch.tensor(np.asarray(weighted_local, dtype=np.float64), device=device)
        summed = rec[..., 1:7].contiguous()
        self.dist.all_reduce(summed, op=self.dist.ReduceOp.SUM)
        flags = rec[..., 7].contiguous()
        self.dist.all_reduce(flags, op=self.dist.ReduceOp.MAX)
        out = rec.clone()
        out[..., 1:7] = summed
        out[..., 7] = flags
        return out.cpu().numpy()


class Band:
    """This process's band of an nx x ny grid: rows [y0, y1) held by `lattice` (anything with
    halo_bytes / halo_pack / halo_unpack / step / diagnostics, e.g. Lattice), and the device
    buffers its edge rows travel in."""

    def __init__(self, lattice, ny: int, rows, buffer_factory):
        self.lattice, self.ny = lattice, ny
        self.y0, self.y1 = rows
        n = lattice.halo_bytes()
        self.send = [buffer_factory(n), buffer_factory(n)]
        self.recv = [buffer_factory(n), buffer_factory(n)]

    def _pack(self):
        self.lattice.halo_pack(0, self.send[0])
        self.lattice.halo_pack(1, self.send[1])

    def _unpack(self, side, buf):
        self.lattice.halo_unpack(side, buf)

    def exchange(self, transport):
        self._pack()
        transport.exchange(self.send, self.recv)
        self._unpack(0, self.recv[0])
        self._unpack(1, self.recv[1])

    def weighted_records(self, max_records=None):
        rec = self.lattice.diagnostics(max_records)
        arr = np.stack([rec[k] for k in ("t", "mass", "mom_x", "mom_y", "amp", "shear", "hnorm", "flags")], axis=-1)
        return weight_record(arr, self.y1 - self.y0, self.ny)


def shear_wave_band(nx: int, ny: int, rows, u0: float, u1: float = 0.0):
    """The initial fields of the standing shear wave on rows [y0, y1) of the whole grid
    (u_y = u0 sin x + u1 sin y sin x, x = 2 pi i / nx, y = 2 pi j / ny; rho = 1, u_x = 0)."""
    y0, y1 = rows
    x = 2.0 * math.pi * np.arange(nx) / nx
    y = 2.0 * math.pi * np.arange(y0, y1) / ny
    uy = u0 * np.sin(x)[None, :] + u1 * np.sin(y)[:, None] * np.sin(x)[None, :]
    return np.ones_like(uy), np.zeros_like(uy), uy
