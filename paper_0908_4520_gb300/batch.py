"""Object wrapper around an lb_batch (marshalling only)."""
from __future__ import annotations

from . import capi


class Batch:
    """Many uneven shear-wave instances advanced by one persistent launch per run.

    precision: "f32", "f16" or "bf16" deviation storage.  threads / smem_bytes / warp_cells:
    launch shape (0 / -1 / -1 = library defaults; the autotuner picks them): threads per CTA,
    the CTA's on-chip budget, and the largest instance (cells) advanced by a single warp.
    """

    def __init__(self, precision: str = "f32", budget_bytes: int = 1 << 30, max_slots: int = 4096,
                 threads: int = 0, smem_bytes: int = -1, kn_convention: str = "lambda", stream: int | None = None,
                 warp_cells: int = -1):
        p = capi.lb_batch_params_default()
        p.precision = capi.PRECISIONS[precision]
        p.budget_bytes = budget_bytes
        p.max_slots = max_slots
        p.threads = threads
        p.smem_bytes = smem_bytes
        p.kn_convention = capi.KN_LAMBDA if kn_convention == "lambda" else capi.KN_PAPER
        p.stream = stream
        p.warp_cells = warp_cells
        self.b = capi.lb_batch_create(p)

    def add(self, quadrature: str, n_eq: int, nx: int, ny: int, kn: float, u0: float = 1e-3,
            max_steps: int = 20000, stop_ratio: float = 1e-3) -> int:
        d = capi.lb_instance_desc(capi.QUADRATURES[quadrature], n_eq, nx, ny, kn, u0, max_steps, stop_ratio)
        return capi.lb_batch_add(self.b, d)

    def remove(self, slot: int):
        capi.lb_batch_remove(self.b, slot)

    def run(self, chunk: int = 0):
        capi.lb_batch_run(self.b, chunk)
        return self

    def sync(self):
        capi.lb_batch_sync(self.b)
        return self

    def state(self, slot: int) -> dict:
        st = capi.lb_batch_state(self.b, slot)
        return {k: getattr(st, k) for k, _ in capi.lb_instance_state._fields_}

    def history(self, slot: int, max_records: int = 1 << 30):
        n = min(max_records, capi.lb_batch_state(self.b, slot).level)
        return capi.lb_batch_history(self.b, slot, n)

    def fit(self, slot: int, t_start: float, floor_rel: float = 1e-4):
        return capi.lb_batch_fit(self.b, slot, t_start, floor_rel)

    def run_profile(self) -> dict:
        """Span and tail (seconds) of the last completed launch and the CTAs that ran."""
        span, tail, ctas = capi.lb_batch_run_profile(self.b)
        return {"span_s": span, "tail_s": tail, "ctas": ctas}

    @property
    def bytes_in_use(self) -> int:
        return capi.lb_batch_bytes_in_use(self.b)

    @property
    def launches(self) -> int:
        return capi.lb_batch_kernel_launches(self.b)

    def close(self):
        if getattr(self, "b", None):
            capi.lb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
