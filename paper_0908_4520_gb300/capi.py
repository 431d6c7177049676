"""ctypes binding of liblb.so (include/lb.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and does no
arithmetic of the method; all compute runs in the library's CUDA kernels.
Importing this module loads liblb.so and raises if it is missing: there is
no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LB_LIB_PATH") or os.path.join(_PKG, "liblb.so")

# lb_status
LB_OK, LB_ERR_ARG, LB_ERR_UNSUPPORTED, LB_ERR_NOMEM, LB_ERR_CUDA = 0, -1, -2, -3, -4
LB_ERR_UNSTABLE, LB_ERR_TIMEOUT, LB_ERR_BUDGET, LB_ERR_STATE = -5, -6, -7, -8
# device scratch of lb_solve_static (LB_STATIC_SCRATCH_BYTES)
LB_STATIC_SCRATCH_BYTES = 8 << 20

# lb_quadrature
QUADRATURES = {
    "D2Q16-GH": 0, "D2Q36-GH": 1, "D2Q64-GH": 2, "D2Q37": 3, "D2Q9": 4,
    "D2Q16-int": 5, "D2Q17": 6, "D2Q21": 7, "D2Q25": 8,
}
# lb_precision
PRECISIONS = {"f32": 0, "f64": 1, "bf16": 2, "f16": 3}
KN_LAMBDA, KN_PAPER = 0, 1
# lb_scheme
SCHEMES = {"second_order": 0, "first_order": 1}
# lb_streaming
STREAMINGS = {"lax_wendroff": 0, "upwind2": 1}

_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class lb_params(ctypes.Structure):
    _fields_ = [
        ("quadrature", ctypes.c_int), ("n_eq", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("kn", ctypes.c_double), ("precision", ctypes.c_int), ("kn_convention", ctypes.c_int),
        ("cfl", ctypes.c_double), ("isothermal", ctypes.c_int), ("diag_capacity", ctypes.c_int),
        ("storage_scale", ctypes.c_double), ("step_kernel", ctypes.c_int), ("stream", ctypes.c_void_p),
        ("alloc", _ALLOC), ("free", _FREE), ("alloc_ctx", ctypes.c_void_p),
        ("force_amp", ctypes.c_double), ("force_freq", ctypes.c_double),
        ("test_withhold_stage", ctypes.c_int), ("scheme", ctypes.c_int), ("streaming", ctypes.c_int),
    ]


class lb_diag(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("t", "mass", "mom_x", "mom_y", "amp", "shear", "hnorm", "flags")]


DIAG_DTYPE = np.dtype([(k, np.float64) for k in ("t", "mass", "mom_x", "mom_y", "amp", "shear", "hnorm", "flags")])


class lb_info_t(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int), ("degree", ctypes.c_int), ("on_lattice", ctypes.c_int), ("halo", ctypes.c_int),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double), ("omega", ctypes.c_double),
        ("c_lattice", ctypes.c_double), ("time_level", ctypes.c_longlong), ("tma_staged", ctypes.c_int),
        ("records", ctypes.c_longlong),
        ("bytes_per_cell_update", ctypes.c_size_t), ("device_bytes", ctypes.c_size_t),
        ("storage_scale", ctypes.c_double),
    ]


class lb_instance_desc(ctypes.Structure):
    _fields_ = [
        ("quadrature", ctypes.c_int), ("n_eq", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("kn", ctypes.c_double), ("u0", ctypes.c_double), ("max_steps", ctypes.c_int),
        ("stop_ratio", ctypes.c_double),
    ]


class lb_batch_params(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int), ("kn_convention", ctypes.c_int), ("budget_bytes", ctypes.c_size_t),
        ("max_slots", ctypes.c_int), ("threads", ctypes.c_int), ("smem_bytes", ctypes.c_int),
        ("stream", ctypes.c_void_p), ("warp_cells", ctypes.c_int),
    ]


class lb_instance_state(ctypes.Structure):
    _fields_ = [
        ("level", ctypes.c_int), ("done", ctypes.c_int), ("status", ctypes.c_int), ("q", ctypes.c_int),
        ("dt", ctypes.c_double), ("omega", ctypes.c_double), ("tau", ctypes.c_double), ("bytes", ctypes.c_size_t),
    ]


class lb_server_params(ctypes.Structure):
    _fields_ = [("batch", lb_batch_params), ("chunk", ctypes.c_int), ("large_cells", ctypes.c_longlong),
                ("budget_bytes", ctypes.c_size_t), ("max_large", ctypes.c_int)]


class lb_request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("arrival", ctypes.c_double), ("desc", lb_instance_desc)]


class lb_response(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("arrival", ctypes.c_double), ("admitted", ctypes.c_double),
                ("finished", ctypes.c_double), ("levels", ctypes.c_int), ("status", ctypes.c_int),
                ("decay_rate", ctypes.c_double), ("fit_points", ctypes.c_int), ("shear_amp", ctypes.c_double)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"liblb.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "lb_params_default": (None, [ctypes.POINTER(lb_params)]),
        "lb_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(H)]),
        "lb_create_ex": (ctypes.c_int, [ctypes.POINTER(lb_params), ctypes.POINTER(H)]),
        "lb_init_shear_wave": (ctypes.c_int, [H, ctypes.c_double, ctypes.c_double]),
        "lb_init_fields": (ctypes.c_int, [H, dp, dp, dp, dp]),
        "lb_step": (ctypes.c_int, [H, ctypes.c_int]),
        "lb_moments": (ctypes.c_int, [H, dp, dp, dp, dp, dp]),
        "lb_moments_device": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p]),
        "lb_populations": (ctypes.c_int, [H, dp]),
        "lb_diagnostics": (ctypes.c_int, [H, ctypes.POINTER(lb_diag), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "lb_diagnostics_at": (ctypes.c_int, [H, ctypes.c_longlong, ctypes.POINTER(lb_diag)]),
        "lb_synchronize": (ctypes.c_int, [H]),
        "lb_halo_bytes": (ctypes.c_int, [H, ctypes.POINTER(ctypes.c_size_t)]),
        "lb_halo_pack": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_void_p]),
        "lb_halo_unpack": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_void_p]),
        "lb_get_info": (ctypes.c_int, [H, ctypes.POINTER(lb_info_t)]),
        "lb_kernel_launches": (ctypes.c_longlong, [H]),
        "lb_destroy": (ctypes.c_int, [H]),
        "lb_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "lb_last_error": (ctypes.c_char_p, [H]),
        "lb_fit_decay": (ctypes.c_int, [H, ctypes.c_double, ctypes.c_double, dp, ctypes.POINTER(ctypes.c_int), dp]),
        "lb_batch_params_default": (None, [ctypes.POINTER(lb_batch_params)]),
        "lb_batch_create": (ctypes.c_int, [ctypes.POINTER(lb_batch_params), ctypes.POINTER(H)]),
        "lb_batch_add": (ctypes.c_int, [H, ctypes.POINTER(lb_instance_desc), ctypes.POINTER(ctypes.c_int)]),
        "lb_batch_remove": (ctypes.c_int, [H, ctypes.c_int]),
        "lb_batch_run": (ctypes.c_int, [H, ctypes.c_int]),
        "lb_batch_sync": (ctypes.c_int, [H]),
        "lb_batch_state": (ctypes.c_int, [H, ctypes.c_int, ctypes.POINTER(lb_instance_state)]),
        "lb_batch_history": (ctypes.c_int, [H, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "lb_batch_fit": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
                                        ctypes.POINTER(ctypes.c_int)]),
        "lb_batch_bytes_in_use": (ctypes.c_size_t, [H]),
        "lb_batch_kernel_launches": (ctypes.c_longlong, [H]),
        "lb_batch_destroy": (ctypes.c_int, [H]),
        "lb_batch_run_profile": (ctypes.c_int, [H, dp, dp, ctypes.POINTER(ctypes.c_int)]),
        "lb_batch_last_error": (ctypes.c_char_p, [H]),
        "lb_server_params_default": (None, [ctypes.POINTER(lb_server_params)]),
        "lb_server_create": (ctypes.c_int, [ctypes.POINTER(lb_server_params), ctypes.POINTER(H)]),
        "lb_server_submit": (ctypes.c_int, [H, ctypes.POINTER(lb_request)]),
        "lb_server_step": (ctypes.c_int, [H, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
        "lb_server_poll": (ctypes.c_int, [H, ctypes.POINTER(lb_response), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]),
        "lb_server_history": (ctypes.c_int, [H, ctypes.c_longlong, dp, dp, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int)]),
        "lb_server_destroy": (ctypes.c_int, [H]),
        "lb_server_last_error": (ctypes.c_char_p, [H]),
        "lb_dvm_run": (ctypes.c_int, [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, dp, dp, ctypes.c_void_p]),
        "lb_dvm_run_forced": (ctypes.c_int, [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp,
                                             dp, ctypes.c_void_p]),
        "lb_solve_static": (ctypes.c_int, [ctypes.POINTER(lb_instance_desc), ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                           ctypes.POINTER(lb_instance_state), ctypes.c_void_p]),
        "lb_quadrature_info": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int), dp, dp,
                                              ctypes.POINTER(ctypes.c_int)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()

# declared entry points of include/lb.h (checked against the library's exports by the tests)
EXPORTS = [
    "lb_params_default", "lb_create", "lb_create_ex", "lb_init_shear_wave", "lb_init_fields", "lb_step",
    "lb_moments", "lb_moments_device", "lb_populations", "lb_diagnostics", "lb_synchronize", "lb_get_info",
    "lb_kernel_launches", "lb_destroy", "lb_status_string", "lb_last_error", "lb_quadrature_info",
    "lb_fit_decay", "lb_batch_params_default", "lb_batch_create", "lb_batch_add", "lb_batch_remove",
    "lb_batch_run", "lb_batch_sync", "lb_batch_state", "lb_batch_history", "lb_batch_fit",
    "lb_batch_bytes_in_use", "lb_batch_kernel_launches", "lb_batch_destroy", "lb_batch_last_error",
    "lb_server_params_default", "lb_server_create", "lb_server_submit", "lb_server_step", "lb_server_poll",
    "lb_server_history", "lb_server_destroy", "lb_server_last_error", "lb_solve_static", "lb_dvm_run",
    "lb_dvm_run_forced", "lb_diagnostics_at", "lb_halo_bytes", "lb_halo_pack", "lb_halo_unpack",
    "lb_batch_run_profile",
]


class LBError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{lib.lb_status_string(status).decode()} ({status}): {message}")
        self.status = status


def check(status: int, handle=None):
    if status != LB_OK:
        msg = lib.lb_last_error(handle)
        raise LBError(status, msg.decode() if msg else "")
    return status


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- thin wrappers with the C names --------------------------------------------------

def lb_params_default() -> lb_params:
    p = lb_params()
    lib.lb_params_default(ctypes.byref(p))
    return p


def lb_create(quadrature, n_eq: int, nx: int, ny: int, kn: float):
    h = ctypes.c_void_p()
    q = QUADRATURES[quadrature] if isinstance(quadrature, str) else int(quadrature)
    st = lib.lb_create(q, n_eq, nx, ny, kn, ctypes.byref(h))
    check(st)
    return h


def lb_create_ex(p: lb_params):
    h = ctypes.c_void_p()
    check(lib.lb_create_ex(ctypes.byref(p), ctypes.byref(h)))
    return h


def lb_init_shear_wave(h, u0: float, u1: float = 0.0):
    return check(lib.lb_init_shear_wave(h, u0, u1), h)


def lb_init_fields(h, rho, ux, uy, T=None):
    return check(lib.lb_init_fields(h, _dptr(rho), _dptr(ux), _dptr(uy), _dptr(T)), h)


def lb_step(h, n: int):
    return check(lib.lb_step(h, int(n)), h)


def lb_moments(h, rho=None, ux=None, uy=None, T=None, sxy=None):
    return check(lib.lb_moments(h, _dptr(rho), _dptr(ux), _dptr(uy), _dptr(T), _dptr(sxy)), h)


def lb_moments_device(h, rho=0, ux=0, uy=0, T=0, sxy=0):
    """Device pointers as integers (0 = skip), e.g. tensor.data_ptr()."""
    return check(lib.lb_moments_device(h, rho or None, ux or None, uy or None, T or None, sxy or None), h)


def lb_populations(h, f):
    return check(lib.lb_populations(h, _dptr(f)), h)


def lb_diagnostics(h, max_records: int):
    out = (lb_diag * max(1, max_records))()
    n = ctypes.c_int(0)
    check(lib.lb_diagnostics(h, out, max_records, ctypes.byref(n)), h)
    arr = np.frombuffer(out, dtype=DIAG_DTYPE, count=n.value).copy()
    return arr


def lb_diagnostics_at(h, level: int, out: lb_diag | None = None) -> lb_diag:
    """Record of one level, waiting only for the launch that produced it."""
    out = out if out is not None else lb_diag()
    check(lib.lb_diagnostics_at(h, level, ctypes.byref(out)), h)
    return out


def lb_synchronize(h):
    return check(lib.lb_synchronize(h), h)


def lb_halo_bytes(h) -> int:
    n = ctypes.c_size_t()
    check(lib.lb_halo_bytes(h, ctypes.byref(n)), h)
    return n.value


def lb_halo_pack(h, side: int, dst: int):
    """dst: device pointer (int) of lb_halo_bytes bytes."""
    return check(lib.lb_halo_pack(h, side, ctypes.c_void_p(dst)), h)


def lb_halo_unpack(h, side: int, src: int):
    return check(lib.lb_halo_unpack(h, side, ctypes.c_void_p(src)), h)


def lb_get_info(h) -> lb_info_t:
    info = lb_info_t()
    check(lib.lb_get_info(h, ctypes.byref(info)), h)
    return info


def lb_kernel_launches(h) -> int:
    return int(lib.lb_kernel_launches(h))


def lb_fit_decay(h, t_start: float, floor_rel: float = 1e-4):
    rate = ctypes.c_double()
    n = ctypes.c_int()
    sr = ctypes.c_double()
    check(lib.lb_fit_decay(h, t_start, floor_rel, ctypes.byref(rate), ctypes.byref(n), ctypes.byref(sr)), h)
    return rate.value, n.value, sr.value


def lb_destroy(h):
    return check(lib.lb_destroy(h))


def lb_quadrature_info(quadrature):
    q = QUADRATURES[quadrature] if isinstance(quadrature, str) else int(quadrature)
    nq, deg = ctypes.c_int(), ctypes.c_int()
    check(lib.lb_quadrature_info(q, ctypes.byref(nq), ctypes.byref(deg), None, None, None))
    xi = np.empty(2 * nq.value)
    w = np.empty(nq.value)
    check(lib.lb_quadrature_info(q, None, None, _dptr(xi), _dptr(w), None))
    e = None
    if q >= 3:
        e_arr = (ctypes.c_int * (2 * nq.value))()
        check(lib.lb_quadrature_info(q, None, None, None, None, e_arr))
        e = np.array(e_arr, dtype=np.int64).reshape(-1, 2)
    return {"q": nq.value, "degree": deg.value, "xi": xi.reshape(-1, 2), "w": w, "e": e}


# ---- batches -----------------------------------------------------------------------------

def check_batch(status: int, b=None):
    if status != LB_OK:
        msg = lib.lb_batch_last_error(b)
        raise LBError(status, msg.decode() if msg else "")
    return status


def lb_batch_params_default() -> lb_batch_params:
    p = lb_batch_params()
    lib.lb_batch_params_default(ctypes.byref(p))
    return p


def lb_batch_create(p: lb_batch_params):
    b = ctypes.c_void_p()
    check_batch(lib.lb_batch_create(ctypes.byref(p), ctypes.byref(b)))
    return b


def lb_batch_add(b, d: lb_instance_desc) -> int:
    slot = ctypes.c_int()
    check_batch(lib.lb_batch_add(b, ctypes.byref(d), ctypes.byref(slot)), b)
    return slot.value


def lb_dvm_run(taus, n_nodes: int, nx: int, u0: float, nsteps: int, cfl: float = 0.5, stream: int = 0):
    """GPU DVM (Sec. 3.3) for each collision time in taus; returns (A, S) arrays of shape
    (len(taus), nsteps + 1)."""
    tau = np.ascontiguousarray(np.atleast_1d(np.asarray(taus, dtype=np.float64)))
    amp = np.empty((tau.size, nsteps + 1))
    shear = np.empty((tau.size, nsteps + 1))
    check(lib.lb_dvm_run(tau.size, _dptr(tau), n_nodes, nx, cfl, u0, nsteps, _dptr(amp), _dptr(shear),
                         stream or None))
    return amp, shear


def lb_dvm_run_forced(taus, n_nodes: int, nx: int, u0: float, force_amp: float, force_freq: float, nsteps: int,
                      cfl: float = 0.5, stream: int = 0):
    """GPU DVM driven by g = force_amp sin(x) cos(force_freq t); returns (A, S) as lb_dvm_run."""
    tau = np.ascontiguousarray(np.atleast_1d(np.asarray(taus, dtype=np.float64)))
    amp = np.empty((tau.size, nsteps + 1))
    shear = np.empty((tau.size, nsteps + 1))
    check(lib.lb_dvm_run_forced(tau.size, _dptr(tau), n_nodes, nx, cfl, u0, force_amp, force_freq, nsteps,
                                _dptr(amp), _dptr(shear), stream or None))
    return amp, shear


def lb_solve_static(desc: lb_instance_desc, precision: int = 0, kn_convention: int = 0, max_records: int = -1,
                    stream: int = 0):
    """Allocation-free single solve (the library's fixed device scratch).  Returns
    (amp, shear, state); amp/shear are the FP32 history as float64 arrays."""
    if max_records < 0:
        max_records = desc.max_steps + 1
    hist = np.empty(2 * max(1, max_records), dtype=np.float32)
    st = lb_instance_state()
    check(lib.lb_solve_static(ctypes.byref(desc), int(precision), int(kn_convention),
                              hist.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), max_records, ctypes.byref(st),
                              stream or None))
    n = min(st.level, max_records)
    h = hist[: 2 * n].reshape(n, 2).astype(np.float64)
    return h[:, 0].copy(), h[:, 1].copy(), st


def lb_batch_remove(b, slot: int):
    return check_batch(lib.lb_batch_remove(b, slot), b)


def lb_batch_run(b, chunk: int = 0):
    return check_batch(lib.lb_batch_run(b, chunk), b)


def lb_batch_sync(b):
    return check_batch(lib.lb_batch_sync(b), b)


def lb_batch_state(b, slot: int) -> lb_instance_state:
    st = lb_instance_state()
    check_batch(lib.lb_batch_state(b, slot, ctypes.byref(st)), b)
    return st


def lb_batch_history(b, slot: int, max_records: int):
    amp = np.empty(max(1, max_records))
    shear = np.empty(max(1, max_records))
    n = ctypes.c_int()
    check_batch(lib.lb_batch_history(b, slot, _dptr(amp), _dptr(shear), max_records, ctypes.byref(n)), b)
    return amp[: n.value].copy(), shear[: n.value].copy()


def lb_batch_fit(b, slot: int, t_start: float, floor_rel: float = 1e-4):
    rate = ctypes.c_double()
    n = ctypes.c_int()
    check_batch(lib.lb_batch_fit(b, slot, t_start, floor_rel, ctypes.byref(rate), ctypes.byref(n)), b)
    return rate.value, n.value


def lb_batch_run_profile(b):
    """(span_s, tail_s, ctas) of the last completed launch."""
    span, tail, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    check_batch(lib.lb_batch_run_profile(b, ctypes.byref(span), ctypes.byref(tail), ctypes.byref(n)), b)
    return span.value, tail.value, n.value


def lb_batch_bytes_in_use(b) -> int:
    return int(lib.lb_batch_bytes_in_use(b))


def lb_batch_kernel_launches(b) -> int:
    return int(lib.lb_batch_kernel_launches(b))


def lb_batch_destroy(b):
    return check_batch(lib.lb_batch_destroy(b))


# ---- serving -----------------------------------------------------------------------------

def check_server(status: int, s=None):
    if status != LB_OK:
        msg = lib.lb_server_last_error(s)
        raise LBError(status, msg.decode() if msg else "")
    return status


def lb_server_params_default() -> lb_server_params:
    p = lb_server_params()
    lib.lb_server_params_default(ctypes.byref(p))
    return p


def lb_server_create(p: lb_server_params):
    s = ctypes.c_void_p()
    check_server(lib.lb_server_create(ctypes.byref(p), ctypes.byref(s)))
    return s


def lb_server_submit(s, r: lb_request):
    return check_server(lib.lb_server_submit(s, ctypes.byref(r)), s)


def lb_server_step(s, now: float):
    a, q = ctypes.c_int(), ctypes.c_int()
    check_server(lib.lb_server_step(s, now, ctypes.byref(a), ctypes.byref(q)), s)
    return a.value, q.value


def lb_server_poll(s, max_n: int = 4096):
    out = (lb_response * max(1, max_n))()
    n = ctypes.c_int()
    check_server(lib.lb_server_poll(s, out, max_n, ctypes.byref(n)), s)
    return [out[i] for i in range(n.value)]


def lb_server_history(s, rid: int, max_records: int):
    amp = np.empty(max(1, max_records))
    shear = np.empty(max(1, max_records))
    n = ctypes.c_int()
    check_server(lib.lb_server_history(s, rid, _dptr(amp), _dptr(shear), max_records, ctypes.byref(n)), s)
    return amp[: n.value].copy(), shear[: n.value].copy()


def lb_server_destroy(s):
    return check_server(lib.lb_server_destroy(s))
