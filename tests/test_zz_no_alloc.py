"""lb_solve_static (fixed device scratch, no allocation) against an lb_batch run of the same instance.

Collected last on purpose: a failure here stops a run only after every other test
has run.  One test starts a fresh process whose first CUDA call is the entry
point itself.
"""
import numpy as np
import pytest

from lbtest import lib

pytestmark = pytest.mark.gpu

# (quadrature, N, nx, ny, kn, max_steps, stop_ratio)
CASES = [("D2Q36-GH", 3, 128, 4, 0.3, 300, 1e-3),
         ("D2Q16-GH", 2, 64, 1, 0.1, 150, 0.0),
         ("D2Q64-GH", 4, 48, 4, 0.7, 120, 0.0)]


def _desc(capi, quad, N, nx, ny, kn, max_steps, stop_ratio, u0=1e-3):
    return capi.lb_instance_desc(capi.QUADRATURES[quad], N, nx, ny, kn, u0, max_steps, stop_ratio)


def _batch_history(case, precision="f32"):
    from paper_0908_4520_gb300 import Batch

    quad, N, nx, ny, kn, max_steps, stop_ratio = case
    b = Batch(precision)
    s = b.add(quad, N, nx, ny, kn, u0=1e-3, max_steps=max_steps, stop_ratio=stop_ratio)
    b.run(0).sync()
    amp, shear = b.history(s)
    state = b.state(s)
    b.close()
    return amp, shear, state


def _close(a, b, rel):
    scale = max(np.max(np.abs(b)), 1e-30)
    return np.max(np.abs(a - b)) <= rel * scale


def test_consecutive_calls_match_the_batch_entry_point():
    Lattice, capi = lib()
    # calls in a row, the first case again last: nothing left in the scratch by one call
    # may change the next one
    for case in CASES + CASES[:1]:
        amp, shear, st = capi.lb_solve_static(_desc(capi, *case))
        ref_amp, ref_shear, ref_st = _batch_history(case)
        assert st.level == ref_st["level"] and st.done == ref_st["done"] == 1 and st.status == 0
        assert len(amp) == len(ref_amp) == st.level
        # FP32 arithmetic on both sides: within 2e-6 of the amplitude scale
        assert _close(amp, ref_amp, 2e-6)
        assert _close(shear, ref_shear, 2e-5)
        assert st.bytes <= capi.LB_STATIC_SCRATCH_BYTES


def test_sixteen_bit_storage_matches_the_batch_entry_point():
    Lattice, capi = lib()
    case = CASES[0]
    for prec in ("f16", "bf16"):
        for _ in range(2):
            amp, shear, st = capi.lb_solve_static(_desc(capi, *case), precision=capi.PRECISIONS[prec])
            ref_amp, ref_shear, ref_st = _batch_history(case, prec)
            assert st.level == ref_st["level"]
            assert _close(amp, ref_amp, 2e-6)
            assert _close(shear, ref_shear, 2e-5)


def test_history_is_truncated_to_max_records():
    Lattice, capi = lib()
    case = CASES[1]
    amp, shear, st = capi.lb_solve_static(_desc(capi, *case), max_records=10)
    full_amp, _, _ = capi.lb_solve_static(_desc(capi, *case))
    assert len(amp) == 10 and st.level == case[5] + 1
    np.testing.assert_array_equal(amp, full_amp[:10])


def test_oversize_solve_is_rejected_before_any_work():
    Lattice, capi = lib()
    # D2Q64 FP32 at 1024 x 64 needs 2 x 64 x 65536 x 4 bytes = 32 MiB of populations
    with pytest.raises(capi.LBError) as e:
        capi.lb_solve_static(_desc(capi, "D2Q64-GH", 4, 1024, 64, 0.1, 10, 0.0))
    assert e.value.status == capi.LB_ERR_BUDGET
    assert "bytes" in str(e.value)
    # and a valid call still works afterwards
    amp, _, st = capi.lb_solve_static(_desc(capi, *CASES[1]))
    assert st.level == CASES[1][5] + 1 and np.all(np.isfinite(amp))


def _free_device_bytes():
    import torch

    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_calls_allocate_no_device_memory():
    """After one call per precision (the first call of a kernel may load its module), further
    calls of other sizes and precisions leave the device's free memory unchanged."""
    Lattice, capi = lib()
    _free_device_bytes()  # the caller's own CUDA set-up comes first
    for prec in ("f32", "f16", "bf16"):
        capi.lb_solve_static(_desc(capi, *CASES[1]), precision=capi.PRECISIONS[prec])
    before = _free_device_bytes()
    for case in CASES:
        for prec in ("f32", "f16", "bf16"):
            amp, _, st = capi.lb_solve_static(_desc(capi, *case), precision=capi.PRECISIONS[prec])
            assert st.status == 0 and np.all(np.isfinite(amp))
    assert _free_device_bytes() == before


def test_first_cuda_action_of_a_fresh_process():
    """A process whose first CUDA call is lb_solve_static (the call that finds the array's
    device address) returns the same history as the batch entry point."""
    import json
    import os
    import subprocess
    import sys

    Lattice, capi = lib()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = (
        "import json, sys\n"
        f"sys.path.insert(0, {root!r})\n"
        "from paper_0908_4520_gb300 import capi\n"
        f"d = capi.lb_instance_desc(capi.QUADRATURES[{CASES[0][0]!r}], {CASES[0][1]}, {CASES[0][2]}, {CASES[0][3]}, "
        f"{CASES[0][4]}, 1e-3, {CASES[0][5]}, {CASES[0][6]})\n"
        "amp, shear, st = capi.lb_solve_static(d)\n"
        "print(json.dumps({'amp': list(map(float, amp)), 'level': st.level, 'status': st.status}))\n")
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    got = json.loads(r.stdout.strip().splitlines()[-1])
    ref_amp, _, ref_st = _batch_history(CASES[0])
    assert got["status"] == 0 and got["level"] == ref_st["level"]
    assert _close(np.array(got["amp"]), ref_amp, 2e-6)
