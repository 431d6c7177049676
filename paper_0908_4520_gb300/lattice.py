"""Object wrapper around one liblb.so handle (marshalling only)."""
from __future__ import annotations

import numpy as np

from . import capi


class Lattice:
    """One periodic nx x ny lattice advanced by the fused collide-stream kernels.

    quadrature: "D2Q16-GH", "D2Q36-GH", "D2Q64-GH" (Lax-Wendroff streaming) or
    "D2Q37", "D2Q9", "D2Q16-int", "D2Q17", "D2Q21", "D2Q25" (exact shift).
    precision: "f32" (default), "f64", "bf16", "f16" (16-bit: GH sets only).
    stream: an integer cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream)
    or None for a stream the handle creates.
    step_kernel: "auto", "plain" (coalesced loads), "tma" (TMA-staged) or "tma_store" (TMA-staged
    with TMA tensor stores; Lax-Wendroff sets, FP32 up to 36 velocities or 16-bit, nx a whole
    number of 16-byte granules); same results.
    force_amp, force_freq: body force g_y = force_amp sin(x_i) cos(force_freq t) driving the
    standing shear wave (0: free decay).
    n_eq: Hermite order N of the equilibrium, 1..4 (1: f^eq = w rho (1 + xi.u)).
    scheme: "second_order" (Eq. 2order, default) or "first_order" (the standard LB of
    Eq. slb: omega = dt / tau, state f, no dt/2 corrections).
    streaming: "lax_wendroff" (default) or "upwind2" (second-order upwind; Gauss-Hermite
    product sets, f32/f64).
    """

    def __init__(self, quadrature: str, n_eq: int, nx: int, ny: int, kn: float, precision: str = "f32",
                 kn_convention: str = "lambda", cfl: float = 1.0, isothermal: bool = False,
                 diag_capacity: int = 65536, storage_scale: float = 0.0, stream: int | None = None,
                 step_kernel: str = "auto", force_amp: float = 0.0, force_freq: float = 0.0,
                 test_withhold_stage: int = 0, scheme: str = "second_order", streaming: str = "lax_wendroff"):
        p = capi.lb_params_default()
        p.quadrature = capi.QUADRATURES[quadrature]
        p.n_eq, p.nx, p.ny, p.kn = n_eq, nx, ny, kn
        p.precision = capi.PRECISIONS[precision]
        p.kn_convention = capi.KN_LAMBDA if kn_convention == "lambda" else capi.KN_PAPER
        p.cfl = cfl
        p.isothermal = int(isothermal)
        p.diag_capacity = diag_capacity
        p.storage_scale = storage_scale
        p.stream = stream
        p.step_kernel = {"auto": 0, "plain": 1, "tma": 2, "tma_store": 3}[step_kernel]
        p.force_amp, p.force_freq = force_amp, force_freq
        p.test_withhold_stage = int(test_withhold_stage)
        p.scheme = capi.SCHEMES[scheme]
        p.streaming = capi.STREAMINGS[streaming]
        self.quadrature, self.n_eq, self.nx, self.ny = quadrature, n_eq, nx, ny
        self.h = capi.lb_create_ex(p)
        inf = capi.lb_get_info(self.h)
        self.Q = inf.q

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None):
            capi.lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls
    def init_shear_wave(self, u0: float, u1: float = 0.0):
        capi.lb_init_shear_wave(self.h, u0, u1)
        return self

    def init_fields(self, rho, ux, uy, T=None):
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        capi.lb_init_fields(self.h, f(rho), f(ux), f(uy), f(T))
        return self

    def step(self, n: int = 1):
        capi.lb_step(self.h, n)
        return self

    def synchronize(self):
        capi.lb_synchronize(self.h)

    def moments(self) -> dict:
        out = {k: np.empty((self.ny, self.nx)) for k in ("rho", "ux", "uy", "T", "sxy")}
        capi.lb_moments(self.h, *(out[k] for k in ("rho", "ux", "uy", "T", "sxy")))
        return out

    def populations(self) -> np.ndarray:
        f = np.empty((self.Q, self.ny, self.nx))
        capi.lb_populations(self.h, f)
        return f

    def diagnostics(self, max_records: int | None = None) -> np.ndarray:
        inf = capi.lb_get_info(self.h)
        n = int(inf.records) if max_records is None else max_records
        return capi.lb_diagnostics(self.h, max(n, 1))

    # -- slab decomposition (see slab.py): buffers are device tensors of halo_bytes() bytes
    def halo_bytes(self) -> int:
        return capi.lb_halo_bytes(self.h)

    def halo_pack(self, side: int, buf):
        capi.lb_halo_pack(self.h, side, buf.data_ptr())

    def halo_unpack(self, side: int, buf):
        capi.lb_halo_unpack(self.h, side, buf.data_ptr())

    def fit_decay(self, t_start: float, floor_rel: float = 1e-4):
        """(rate, npoints, shear/amplitude ratio) from the FP64 fit of the library."""
        return capi.lb_fit_decay(self.h, t_start, floor_rel)

    @property
    def info(self) -> dict:
        inf = capi.lb_get_info(self.h)
        return {k: getattr(inf, k) for k, _ in capi.lb_info_t._fields_}

    @property
    def launches(self) -> int:
        return capi.lb_kernel_launches(self.h)
