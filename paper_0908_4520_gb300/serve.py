"""Object wrapper around an lb_server (marshalling only), plus a replay driver."""
from __future__ import annotations

import time

from . import capi


class Server:
    """Request loop over a continuously batched lb_batch (small requests) and
    lattices of their own (large requests)."""

    def __init__(self, precision: str = "f16", chunk: int = 200, budget_bytes: int = 1 << 30,
                 large_cells: int = 65536, large_budget_bytes: int = 8 << 30, max_large: int = 4,
                 threads: int = 0, smem_bytes: int = -1, max_slots: int = 4096):
        p = capi.lb_server_params_default()
        p.batch.precision = capi.PRECISIONS[precision]
        p.batch.budget_bytes = budget_bytes
        p.batch.threads = threads
        p.batch.smem_bytes = smem_bytes
        p.batch.max_slots = max_slots
        p.chunk = chunk
        p.large_cells = large_cells
        p.budget_bytes = large_budget_bytes
        p.max_large = max_large
        self.s = capi.lb_server_create(p)

    def submit(self, rid: int, arrival: float, quadrature: str, n_eq: int, nx: int, ny: int, kn: float,
               u0: float = 1e-4, max_steps: int = 20000, stop_ratio: float = 1e-3):
        d = capi.lb_instance_desc(capi.QUADRATURES[quadrature], n_eq, nx, ny, kn, u0, max_steps, stop_ratio)
        capi.lb_server_submit(self.s, capi.lb_request(rid, arrival, d))

    def step(self, now: float):
        return capi.lb_server_step(self.s, now)

    def poll(self):
        return [{k: getattr(r, k) for k, _ in capi.lb_response._fields_} for r in capi.lb_server_poll(self.s)]

    def history(self, rid: int, max_records: int = 1 << 22):
        return capi.lb_server_history(self.s, rid, max_records)

    def close(self):
        if getattr(self, "s", None):
            capi.lb_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def replay(server: Server, requests, time_scale: float = 1.0, max_wall: float = 1e9):
    """Submit requests at their arrival times (wall clock, scaled) and step the server
    until every submitted request has finished.  Returns the responses (times in seconds
    of the replay clock)."""
    t0 = time.perf_counter()
    i, out = 0, []
    n = len(requests)
    while len(out) < n:
        now = (time.perf_counter() - t0) / time_scale
        while i < n and requests[i]["arrival"] <= now:
            r = requests[i]
            server.submit(r["id"], r["arrival"], r["quadrature"], r["n_eq"], r["nx"], r["ny"], r["kn"], r["u0"],
                          r["max_steps"], r.get("stop_ratio", 1e-3))
            i += 1
        active, queued = server.step(now)
        out.extend(server.poll())
        if active == 0 and queued == 0 and i < n:
            time.sleep(max(0.0, min(0.01, (requests[i]["arrival"] - now) * time_scale)))
        if time.perf_counter() - t0 > max_wall:
            break
    return out
