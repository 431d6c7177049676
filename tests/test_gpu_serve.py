"""The request loop: every served result equals the same request solved alone, admission
waits for memory, and a served FP16 stream matches the FP64 oracle request by request."""
import numpy as np
import pytest

from lbtest import lib

pytestmark = pytest.mark.gpu

REQS = [("D2Q16-GH", 2, 32, 1, 0.05), ("D2Q36-GH", 3, 128, 4, 0.3), ("D2Q64-GH", 4, 64, 1, 2.0),
        ("D2Q36-GH", 2, 256, 1, 1.0), ("D2Q16-GH", 3, 64, 4, 0.5), ("D2Q64-GH", 3, 32, 4, 0.1),
        ("D2Q36-GH", 3, 64, 64, 0.2)]  # the last one is "large" with large_cells = 4096


def classes():
    lib()
    from paper_0908_4520_gb300 import Batch, Lattice
    from paper_0908_4520_gb300.serve import Server

    return Batch, Lattice, Server


def test_served_results_equal_alone():
    Batch, Lattice, Server = classes()
    srv = Server(precision="f16", chunk=50, large_cells=4096)
    for i, (q, N, nx, ny, kn) in enumerate(REQS):
        srv.submit(i, 0.0, q, N, nx, ny, kn, u0=1e-4, max_steps=300, stop_ratio=1e-3)
    done = []
    for it in range(100):
        srv.step(float(it))
        done.extend(srv.poll())
        if len(done) == len(REQS):
            break
    assert len(done) == len(REQS)
    for r in done:
        q, N, nx, ny, kn = REQS[r["id"]]
        amp, shear = srv.history(r["id"])
        assert r["status"] == 0 and len(amp) == r["levels"]
        if nx * ny >= 4096:
            L = Lattice(q, N, nx, ny, kn, precision="f16", diag_capacity=400).init_shear_wave(1e-4)
            L.step(r["levels"] - 1)
            rec = L.diagnostics()
            np.testing.assert_array_equal(amp, rec["amp"])
            L.close()
        else:
            b = Batch("f16")
            s = b.add(q, N, nx, ny, kn, 1e-4, 300, 1e-3)
            b.run(0).sync()
            a1, s1 = b.history(s)
            np.testing.assert_array_equal(amp, a1.astype(np.float64))
            b.close()
    srv.close()


def test_admission_waits_for_memory():
    Batch, Lattice, Server = classes()
    # each D2Q64 1024 x 4 FP32 instance holds 2 x 1 MiB of populations: two fit in 5 MiB, three do not
    srv = Server(precision="f32", chunk=40, budget_bytes=5 << 20, large_cells=1 << 30)
    for i in range(8):
        srv.submit(i, 0.0, "D2Q64-GH", 4, 1024, 4, 1.0, u0=1e-3, max_steps=120, stop_ratio=0.0)
    done, max_active = [], 0
    for it in range(200):
        active, queued = srv.step(float(it))
        max_active = max(max_active, active)
        done.extend(srv.poll())
        if len(done) == 8:
            break
    assert len(done) == 8 and max_active == 2
    assert all(r["levels"] == 121 for r in done)
    srv.close()


# A mixed stream against the FP64 oracle: FP16 deviation storage, U0 = 1e-4, requests
# arriving while others run (continuous batching) and one large request on its own
# lattice.  Grids of >= 1024 cells keep the storage noise of the decay rate below 1e-3
# (see test_gpu_precision_oracle for the bound).
STREAM = [(0, "D2Q36-GH", 3, 256, 4, 0.3), (0, "D2Q64-GH", 4, 512, 2, 0.1), (0, "D2Q16-GH", 2, 1024, 1, 0.5),
          (3, "D2Q64-GH", 3, 256, 4, 1.0), (5, "D2Q36-GH", 3, 64, 64, 0.2), (8, "D2Q16-GH", 4, 128, 8, 0.06)]
MAX_STEPS = 1500


def _oracle_history(q, N, nx, ny, kn, levels):
    import oracle

    P = oracle.Problem(q, N, nx, ny, kn)
    f = P.init_shear(1e-4)
    d = P.run(f, levels - 1)
    return d, P.tau, P.vs.w, P.vs.xi


def test_served_stream_matches_oracle():
    import concurrent.futures as cf
    import math
    import multiprocessing as mp

    import oracle

    Batch, Lattice, Server = classes()
    srv = Server(precision="f16", chunk=100, large_cells=4096)
    done, it, nxt = [], 0, 0
    while len(done) < len(STREAM) and it < 400:
        while nxt < len(STREAM) and STREAM[nxt][0] <= it:
            _, q, N, nx, ny, kn = STREAM[nxt]
            srv.submit(nxt, float(it), q, N, nx, ny, kn, u0=1e-4, max_steps=MAX_STEPS, stop_ratio=1e-3)
            nxt += 1
        srv.step(float(it))
        done.extend(srv.poll())
        it += 1
    assert len(done) == len(STREAM)
    # the later arrivals were admitted while earlier requests were still running
    by_id = {r["id"]: r for r in done}
    assert by_id[3]["admitted"] < by_id[0]["finished"] or by_id[3]["admitted"] < by_id[1]["finished"]
    hist = {r["id"]: srv.history(r["id"]) for r in done}
    srv.close()
    with cf.ProcessPoolExecutor(max_workers=len(STREAM), mp_context=mp.get_context("spawn")) as ex:
        futs = {i: ex.submit(_oracle_history, *STREAM[i][1:], by_id[i]["levels"]) for i in by_id}
        ora = {i: f.result() for i, f in futs.items()}
    for i, r in by_id.items():
        _, q, N, nx, ny, kn = STREAM[i]
        d, tau, w, xi = ora[i]
        amp, shear = hist[i]
        assert r["status"] == 0 and len(amp) == len(d) == r["levels"]
        n = r["levels"]
        # FP16 storage noise (m = 10) of the amplitude, 3 standard deviations, plus the FP32
        # arithmetic allowance n omega 2^-24 (omega < 1 here)
        s = 2.0 ** -11 * math.sqrt(float(np.sum(w * w * xi[:, 1] ** 4)))
        bound = 3.0 * math.sqrt(2.0 * n / (nx * ny)) * s + n * 2.0 ** -24
        assert np.max(np.abs(amp - d[:, 4])) / 1e-4 < bound, (i, np.max(np.abs(amp - d[:, 4])) / 1e-4, bound)
        # the served decay rate (the library's fit from t = 5 tau) against the oracle's rule
        r_ora = oracle.decay_fit(d[:, 0], d[:, 4], 5.0 * tau)
        assert abs(r["decay_rate"] / r_ora - 1.0) < 1e-3, (i, r["decay_rate"], r_ora)
