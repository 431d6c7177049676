"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank runs its own
independent instance, the job's time is the slowest rank's, the value counts every rank's
cell updates; the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [12.5, 20.0][rank]
    ms = bench.reduce_max_ms(ms_local, dist, "cpu")
    out[rank] = (ms, bench.weak_value(1000, world, 10, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_value_counts_all_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 20.0
    # 1000 cells x 2 ranks x 10 steps in 20 ms
    assert out[0][1] == pytest.approx(1000 * 2 * 10 / 0.020 / 1e6)


def test_single_rank_needs_no_collective():
    assert bench.reduce_max_ms(7.0, None, "cpu") == 7.0
    assert bench.weak_value(4096 * 4096, 1, 100, 1000.0) == pytest.approx(4096 * 4096 * 100 / 1e6)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_on_rank_zero():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-rows", "2"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_traffic_record_follows_the_kernel_code_not_its_comments(tmp_path):
    """The DRAM traffic record is reported only while the kernel sources' code matches the
    capture; comments and blank space do not count, any code change does."""
    csrc = tmp_path / "paper_0908_4520_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(bench.ROOT, "paper_0908_4520_gb300", "csrc")
    for f in ("lb_kernels.cuh", "lb_device.h", "velocity_sets.h"):
        with open(os.path.join(src, f)) as fh:
            (csrc / f).write_text(fh.read())
    old_root = bench.ROOT
    try:
        bench.ROOT = str(tmp_path)
        d0 = bench.kernel_digest()
        k = csrc / "lb_kernels.cuh"
        k.write_text("// a comment\n/* and a block\n   comment */\n" + k.read_text() + "\n\n")
        assert bench.kernel_digest() == d0
        k.write_text(k.read_text() + "\nconstexpr int lb_extra_code = 1;\n")
        assert bench.kernel_digest() != d0
    finally:
        bench.ROOT = old_root
