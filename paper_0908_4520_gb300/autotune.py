"""Autotuner for the multi-instance launch shape.

The batch kernel's launch shape is picked by timed trials: threads per CTA, the
shared-memory budget that decides which instances step on chip, and the tile
shape of an instance - a whole CTA, or a single warp for instances of at most
`warp_cells` cells (cells per thread = cells / 32 there, against cells /
threads on a CTA), so that a CTA advances several small instances at once.  A
stratified sample of the instance mix is run for a short chunk under each
candidate shape, and the fastest (cell updates per second) wins.  The sample
holds the whole mix up to 1024 instances: a trial must fill every SM the way the
real launch does, or it times one instance's latency instead of the launch's
throughput.  Results are
cached in a JSON file keyed by the storage type and a signature of the mix
(quadrature, order and grid-size classes), so later runs reuse them.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

from . import capi
from .batch import Batch

CANDIDATES = [(t, s, w) for t in (64, 128, 256) for s in (0, 48 * 1024, 96 * 1024, 200 * 1024)
              for w in (0, 256, 1024, 4096)]
_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_0908_4520_gb300", "autotune.json")


def _signature(instances, precision):
    classes = sorted({(d["quadrature"], d["n_eq"], d["nx"] * d["ny"]) for d in instances})
    h = hashlib.sha256(json.dumps(["threads/smem/warp_cells", precision, classes]).encode()).hexdigest()[:16]
    return f"{precision}:{h}"


def _sample(instances, k):
    """Up to k instances, one per (quadrature, order, size) class first."""
    seen, out = set(), []
    for d in instances:
        key = (d["quadrature"], d["n_eq"], d["nx"] * d["ny"])
        if key not in seen:
            seen.add(key)
            out.append(d)
    for d in instances:
        if len(out) >= k:
            break
        if d not in out:
            out.append(d)
    return out[:k]


def _trial(sample, precision, threads, smem, warp_cells, chunk):
    import torch

    b = Batch(precision=precision, threads=threads, smem_bytes=smem, warp_cells=warp_cells,
              budget_bytes=max(1 << 28, 4 * sum(2 * 64 * d["nx"] * d["ny"] * 4 + 8 * (chunk + 2) for d in sample)))
    cells = 0
    for d in sample:
        b.add(d["quadrature"], d["n_eq"], d["nx"], d["ny"], d["kn"], d.get("u0", 1e-3), max_steps=2 * chunk + 4,
              stop_ratio=0.0)
        cells += d["nx"] * d["ny"]
    b.run(chunk).sync()  # warm-up chunk (levels 0..chunk-1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(chunk).sync()
    el = time.perf_counter() - t0
    b.close()
    return cells * chunk / el


def tune(instances, precision: str = "f32", sample: int = 1024, chunk: int = 32, use_cache: bool = True) -> dict:
    """Best (threads, smem_bytes, warp_cells) for this mix; cached by mix signature."""
    sig = _signature(instances, precision)
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            with open(_CACHE) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
    if use_cache and sig in cache:
        return cache[sig]
    smp = _sample(instances, sample)
    results = []
    for threads, smem, warp_cells in CANDIDATES:
        try:
            rate = _trial(smp, precision, threads, smem, warp_cells, chunk)
        except capi.LBError:
            continue
        results.append({"threads": threads, "smem_bytes": smem, "warp_cells": warp_cells,
                        "cell_updates_per_s": rate})
    if not results:
        raise RuntimeError("no launch shape could run the sample")
    best = max(results, key=lambda r: r["cell_updates_per_s"])
    entry = {"threads": best["threads"], "smem_bytes": best["smem_bytes"], "warp_cells": best["warp_cells"],
             "trials": results, "searched": {"threads": [64, 128, 256], "smem_bytes": [0, 48 << 10, 96 << 10, 200 << 10],
                                             "warp_cells (one warp per instance up to; cells per thread = cells/32)":
                                                 [0, 256, 1024, 4096]}}
    cache[sig] = entry
    try:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as fh:
            json.dump(cache, fh, indent=1)
    except OSError:
        pass
    return entry
