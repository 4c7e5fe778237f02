"""Thin Python binding of the HMS C ABI (include/hms.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Arrays are NumPy
float64 arrays (host memory, HMS_MEM_HOST) or CUDA torch tensors on the
context's device (HMS_MEM_DEVICE, passed by data_ptr()).  Every step of the
solver runs in the CUDA library; if the library cannot be loaded the import
of this module's functions raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HMS_OK = 0
HMS_ERR_ARG = -1
HMS_ERR_NOT_SPD = -2
HMS_ERR_NO_CONVERGENCE = -3
HMS_ERR_NONFINITE = -4
HMS_ERR_OOM = -5
HMS_ERR_TIMEOUT = -6
HMS_ERR_CUDA = -7
HMS_MEM_HOST = 0
HMS_MEM_DEVICE = 1
HMS_FP64 = 0
HMS_MIXED = 1
HMS_BATCH_AUTO = 0
HMS_BATCH_STREAMS = 1
HMS_BATCH_LOCKSTEP = 2

KERNEL_NAMES = ("update_residual", "relax", "coarse_assemble", "coarse_band", "coarse_factor",
                "coarse_residual", "coarse_solve")

_STATUS_NAMES = {0: "HMS_OK", -1: "HMS_ERR_ARG", -2: "HMS_ERR_NOT_SPD", -3: "HMS_ERR_NO_CONVERGENCE",
                 -4: "HMS_ERR_NONFINITE", -5: "HMS_ERR_OOM", -6: "HMS_ERR_TIMEOUT", -7: "HMS_ERR_CUDA"}


class HmsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class LatticeDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("bar_length", ctypes.c_double),
                ("ea", ctypes.c_void_p), ("ea_uniform", ctypes.c_double), ("fixed", ctypes.c_void_p),
                ("fix_bottom_edge", ctypes.c_int32), ("set_sx", ctypes.c_int32),
                ("set_sy", ctypes.c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("coarse_solves", ctypes.c_int32), ("batch", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("coarse_factor", ctypes.c_int32), ("relax_threads", ctypes.c_int32),
                ("relax_copies", ctypes.c_int32), ("relax_overlap", ctypes.c_int32),
                ("mode_mask", ctypes.c_uint32), ("record_history", ctypes.c_int32),
                ("class_factors", ctypes.c_int32), ("relax_balance", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def lib():
    """Load lib/libhms.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"HMS CUDA library missing at {path}")
    L = ctypes.CDLL(path)
    sig = {
        "hms_context_create": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(_P)]),
        "hms_context_destroy": (None, [_P]),
        "hms_context_stream": (_P, [_P]),
        "hms_last_error": (ctypes.c_char_p, [_P]),
        "hms_problem_create": (ctypes.c_int32, [_P, ctypes.POINTER(LatticeDesc), ctypes.POINTER(Options),
                                                ctypes.POINTER(_P)]),
        "hms_problem_destroy": (None, [_P]),
        "hms_problem_device_bytes": (ctypes.c_size_t, [_P]),
        "hms_problem_setup_ms": (ctypes.c_double, [_P]),
        "hms_problem_relax_threads": (ctypes.c_int32, [_P]),
        "hms_problem_relax_copies": (ctypes.c_int32, [_P]),
        "hms_problem_relax_balanced": (ctypes.c_int32, [_P]),
        "hms_relax_schedule": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, _P, ctypes.c_int32, _P]),
        "hms_set_classes": (ctypes.c_int32, [ctypes.POINTER(LatticeDesc), _P, ctypes.c_int32]),
        "hms_nd_plan": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, _P, ctypes.c_int32]),
        "hms_solve": (ctypes.c_int32, [_P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int32, _P, ctypes.c_int32]),
        "hms_kernel_times": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int32]),
        "hms_residual": (ctypes.c_int32, [_P, _P, _P, _P, _P, ctypes.c_int32]),
        "hms_update_residual": (ctypes.c_int32, [_P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int32]),
        "hms_relax": (ctypes.c_int32, [_P, _P, _P, _P, ctypes.c_int32]),
        "hms_coarse_matrix": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int32]),
        "hms_coarse_solve": (ctypes.c_int32, [_P, _P, _P, _P, _P, ctypes.c_int32]),
        "hms_residual_noalloc": (ctypes.c_int32, [_P, _P, _P, _P, _P]),
        "hms_solve_batch": (ctypes.c_int32, [_P, ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.c_int32]),
        "hms_context_set_batch_mode": (ctypes.c_int32, [_P, ctypes.c_int32]),
        "hms_problem_estimate_bytes": (ctypes.c_size_t, [_P, ctypes.POINTER(LatticeDesc), ctypes.POINTER(Options)]),
        "hms_server_create": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(_P)]),
        "hms_server_destroy": (None, [_P]),
        "hms_server_submit": (ctypes.c_int32, [_P, ctypes.POINTER(LatticeDesc), ctypes.POINTER(Options), ctypes.c_int32,
                                               _P, ctypes.POINTER(ctypes.c_int64)]),
        "hms_server_step": (ctypes.c_int32, [_P, _P, ctypes.c_int32, _P, _P, _P, _P]),
        "hms_server_take": (ctypes.c_int32, [_P, ctypes.c_int64, _P, _P]),
        "hms_problem_clone": (ctypes.c_int32, [_P, ctypes.POINTER(_P)]),
        "hms_reactions": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int32]),
        "hms_problem_refine_cap_hits": (ctypes.c_int64, [_P]),
        "hms_problem_set_relax_wait_limit": (ctypes.c_int32, [_P, ctypes.c_int32]),
        "hms_measure_fp64_rate": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
        "hms_relax_force": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return ["hms_context_create", "hms_context_destroy", "hms_context_stream", "hms_last_error",
            "hms_problem_create", "hms_problem_destroy", "hms_problem_device_bytes",
            "hms_problem_setup_ms", "hms_solve", "hms_kernel_times", "hms_residual",
            "hms_update_residual", "hms_relax", "hms_coarse_matrix", "hms_coarse_solve",
            "hms_residual_noalloc", "hms_solve_batch", "hms_problem_estimate_bytes", "hms_server_create",
            "hms_server_destroy", "hms_server_submit", "hms_server_step", "hms_server_take", "hms_problem_clone",
            "hms_problem_relax_threads", "hms_context_set_batch_mode", "hms_problem_relax_copies",
            "hms_reactions", "hms_problem_refine_cap_hits", "hms_problem_set_relax_wait_limit",
            "hms_measure_fp64_rate", "hms_relax_force", "hms_problem_relax_balanced", "hms_relax_schedule",
            "hms_set_classes", "hms_nd_plan"]


# ---------------------------------------------------------------- marshalling
class _Arg:
    """A pointer argument: NumPy array (host) or CUDA tensor (device)."""

    def __init__(self, x, dtype=np.float64, writable=False):
        self.keep = None
        if x is None:
            self.ptr, self.kind = None, None
        elif hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
            if not x.is_cuda:
                x = x.numpy()
            else:
                if not x.is_contiguous():
                    raise ValueError("device tensors must be contiguous")
                # the library reads and writes on its own stream: work torch has
                # queued on the tensor (on torch's current stream) must finish first
                import torch
                torch.cuda.current_stream(x.device).synchronize()
                self.ptr, self.kind, self.keep = x.data_ptr(), HMS_MEM_DEVICE, x
                return
        if x is not None:
            a = np.asarray(x)
            if a.dtype != dtype or not a.flags.c_contiguous or (writable and not a.flags.writeable):
                if writable:
                    raise ValueError(f"output array must be C-contiguous {np.dtype(dtype)}")
                a = np.ascontiguousarray(a, dtype=dtype)
            self.ptr, self.kind, self.keep = a.ctypes.data, HMS_MEM_HOST, a


def _mem_kind(*args):
    kinds = {a.kind for a in args if a.kind is not None}
    if len(kinds) > 1:
        raise ValueError("mix of host arrays and device tensors in one call")
    return kinds.pop() if kinds else HMS_MEM_HOST


def _check(ctx, st, ok=(HMS_OK,)):
    if st not in ok:
        msg = lib().hms_last_error(ctx)
        raise HmsError(st, msg.decode() if msg else "")
    return st


# ---------------------------------------------------------------- entry points
def hms_context_create(device: int = 0):
    h = _P()
    st = lib().hms_context_create(int(device), ctypes.byref(h))
    if st != HMS_OK:
        m = lib().hms_last_error(None)
        raise HmsError(st, f"cannot create a context on device {device}: {m.decode() if m else ''}")
    return h


def hms_context_destroy(ctx):
    lib().hms_context_destroy(ctx)


def hms_context_stream(ctx) -> int:
    return lib().hms_context_stream(ctx) or 0


def hms_last_error(ctx) -> str:
    m = lib().hms_last_error(ctx)
    return m.decode() if m else ""


def _desc_opts(nx, ny, set_sx, set_sy, bar_length=1.0, ea=None, ea_uniform=1.0, fixed=None, fix_bottom_edge=1,
               precision=HMS_FP64, tol=1e-8, max_iter=1000, coarse_solves=0, batch=0, profile=0, coarse_factor=0,
               relax_threads=0, relax_copies=0, relax_overlap=0, mode_mask=0x1FF, record_history=1, class_factors=0,
               relax_balance=0):
    """LatticeDesc and Options structs (plus the arrays they point to, kept alive by the caller)."""
    ea_a = None if ea is None else np.ascontiguousarray(ea, dtype=np.float64)
    fx_a = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
    if ea_a is not None and ea_a.size != 3 * nx * ny:
        raise ValueError("ea must have 3*nx*ny entries")
    if fx_a is not None and fx_a.size != 2 * nx * ny:
        raise ValueError("fixed must have 2*nx*ny entries")
    d = LatticeDesc(int(nx), int(ny), float(bar_length), None if ea_a is None else ea_a.ctypes.data,
                    float(ea_uniform), None if fx_a is None else fx_a.ctypes.data, int(fix_bottom_edge),
                    int(set_sx), int(set_sy))
    o = Options(int(precision), float(tol), int(max_iter), int(coarse_solves), int(batch), int(profile),
                int(coarse_factor), int(relax_threads), int(relax_copies), int(relax_overlap), int(mode_mask),
                int(record_history), int(class_factors), int(relax_balance))
    return d, o, (ea_a, fx_a)


def hms_problem_create(ctx, nx, ny, set_sx, set_sy, **kw):
    """kw: bar_length, ea (host float64 [3, ny, nx]), ea_uniform, fixed (host uint8
    [ny, nx, 2]), fix_bottom_edge, precision, tol, max_iter, coarse_solves, batch,
    profile, coarse_factor, relax_threads, relax_copies, relax_overlap, mode_mask,
    record_history, class_factors, relax_balance."""
    d, o, keep = _desc_opts(nx, ny, set_sx, set_sy, **kw)
    h = _P()
    _check(ctx, lib().hms_problem_create(ctx, ctypes.byref(d), ctypes.byref(o), ctypes.byref(h)))
    return h


def hms_problem_clone(ctx, pr):
    h = _P()
    _check(ctx, lib().hms_problem_clone(pr, ctypes.byref(h)))
    return h


def hms_problem_estimate_bytes(ctx, nx, ny, set_sx, set_sy, **kw) -> int:
    d, o, keep = _desc_opts(nx, ny, set_sx, set_sy, **kw)
    return int(lib().hms_problem_estimate_bytes(ctx, ctypes.byref(d), ctypes.byref(o)))


def hms_problem_destroy(pr):
    lib().hms_problem_destroy(pr)


def hms_problem_device_bytes(pr) -> int:
    return int(lib().hms_problem_device_bytes(pr))


def hms_problem_setup_ms(pr) -> float:
    return float(lib().hms_problem_setup_ms(pr))


def hms_problem_relax_threads(pr) -> int:
    return int(lib().hms_problem_relax_threads(pr))


def hms_problem_relax_copies(pr) -> int:
    return int(lib().hms_problem_relax_copies(pr))


def hms_problem_relax_balanced(pr) -> int:
    return int(lib().hms_problem_relax_balanced(pr))


def hms_set_classes(nx, ny, set_sx, set_sy, fixed=None, fix_bottom_edge=1):
    """Class of every set (row-major over the set grid) that class_factors = 1
    would share one factor across (host only): (classes [M], class count)."""
    d, _, keep = _desc_opts(nx, ny, set_sx, set_sy, fixed=fixed, fix_bottom_edge=fix_bottom_edge)
    m = (-(-nx // set_sx)) * (-(-ny // set_sy))
    out = np.zeros(m, np.int32)
    n = lib().hms_set_classes(ctypes.byref(d), out.ctypes.data, m)
    if n < 0:
        raise HmsError(HMS_ERR_ARG, "hms_set_classes: bad arguments")
    return out, int(n)


def hms_nd_plan(mx, my):
    """The upper level's nested-dissection plan for mx x my sets (host only):
    a list of nodes, children before parents, each a dict with S (sets it
    eliminates), B (its boundary sets) and children (node indices)."""
    m = mx * my
    cap_n, cap_s = 4 * m + 8, 64 * m + 64
    nodes = np.zeros((cap_n, 6), np.int32)
    sets = np.zeros(cap_s, np.int32)
    n = lib().hms_nd_plan(int(mx), int(my), nodes.ctypes.data, cap_n, sets.ctypes.data, cap_s)
    if n < 0:
        raise HmsError(HMS_ERR_ARG, "hms_nd_plan: bad arguments")
    out = []
    for ns, nb, off, nch, c0, c1 in nodes[:n].tolist():
        out.append({"S": sets[off:off + ns].tolist(), "B": sets[off + ns:off + ns + nb].tolist(),
                    "children": [c for c in (c0, c1)[:nch]]})
    return out


def hms_relax_schedule(nx, ny, set_sx, set_sy, ctas):
    """The balanced relaxation schedule over `ctas` CTAs (host only): (segments
    [k, 3] of (set, first op, end op), CTA offsets [ctas + 1]), or None where
    it does not apply."""
    cap = 4 * (-(-nx // set_sx)) * (-(-ny // set_sy)) + 2 * ctas + 4
    segs = np.zeros((cap, 3), np.int32)
    cta = np.zeros(ctas + 1, np.int32)
    n = lib().hms_relax_schedule(int(nx), int(ny), int(set_sx), int(set_sy), int(ctas), segs.ctypes.data, cap,
                                 cta.ctypes.data)
    if n < 0:
        raise HmsError(HMS_ERR_ARG, "hms_relax_schedule: bad arguments")
    return None if n == 0 else (segs[:n].copy(), cta)


def hms_solve(ctx, pr, loads, u_out, u0=None, hist=None, iters=None, allow_no_convergence=False):
    """loads, u_out (and u0): [nrhs, 2*nx*ny]; hist: [nrhs, cap, 3]; iters: int32 [nrhs]."""
    L = _Arg(loads)
    U = _Arg(u_out, writable=True)
    U0 = _Arg(u0)
    H = _Arg(hist, writable=True)
    It = _Arg(iters, dtype=np.int32, writable=True)
    kind = _mem_kind(L, U, U0, H, It)
    nrhs = int(np.prod(loads.shape[:-1])) if len(loads.shape) > 1 else 1
    cap = 0 if hist is None else int(hist.shape[-2])
    st = lib().hms_solve(pr, nrhs, L.ptr, U0.ptr, U.ptr, H.ptr, cap, It.ptr, kind)
    ok = (HMS_OK, HMS_ERR_NO_CONVERGENCE) if allow_no_convergence else (HMS_OK,)
    return _check(ctx, st, ok)


def hms_context_set_batch_mode(ctx, mode):
    _check(ctx, lib().hms_context_set_batch_mode(ctx, int(mode)))


def hms_solve_batch(ctx, problems, loads, u_out, iters=None, allow_no_convergence=False):
    """problems: list of handles; loads[i], u_out[i]: arrays [nrhs_i, 2*nx_i*ny_i]
    (all NumPy, or all CUDA tensors); iters: int32 array of sum(nrhs_i) or None."""
    n = len(problems)
    L = [_Arg(x) for x in loads]
    U = [_Arg(x, writable=True) for x in u_out]
    I = _Arg(iters, dtype=np.int32, writable=True)
    mk = _mem_kind(*L, *U, I)
    nrhs = (ctypes.c_int32 * max(n, 1))(*[int(x.shape[0]) if len(x.shape) > 1 else 1 for x in loads])
    pp = (_P * max(n, 1))(*[ctypes.cast(pr, _P) for pr in problems])
    lp = (_P * max(n, 1))(*[a.ptr for a in L])
    up = (_P * max(n, 1))(*[a.ptr for a in U])
    ok = (HMS_OK, HMS_ERR_NO_CONVERGENCE) if allow_no_convergence else (HMS_OK,)
    return _check(ctx, lib().hms_solve_batch(ctx, n, pp, nrhs, lp, up, I.ptr, mk), ok=ok)


def hms_server_create(ctx, hbm_budget_bytes, max_active=256):
    h = _P()
    _check(ctx, lib().hms_server_create(ctx, int(hbm_budget_bytes), int(max_active), ctypes.byref(h)))
    return h


def hms_server_destroy(srv):
    lib().hms_server_destroy(srv)


def hms_server_submit(ctx, srv, nx, ny, set_sx, set_sy, loads, **kw) -> int:
    """loads: host float64 [nrhs, 2*nx*ny]; kw as hms_problem_create.  Returns the id."""
    d, o, keep = _desc_opts(nx, ny, set_sx, set_sy, **kw)
    a = np.ascontiguousarray(loads, dtype=np.float64).reshape(-1, 2 * int(nx) * int(ny))
    rid = ctypes.c_int64()
    _check(ctx, lib().hms_server_submit(srv, ctypes.byref(d), ctypes.byref(o), int(a.shape[0]), a.ctypes.data,
                                        ctypes.byref(rid)))
    return int(rid.value)


def hms_server_step(ctx, srv, cap=4096):
    """One round; returns (finished ids, n_active, n_queued, bytes_in_use)."""
    ids = (ctypes.c_int64 * cap)()
    nd, na, nq = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    used = ctypes.c_uint64()
    _check(ctx, lib().hms_server_step(srv, ids, int(cap), ctypes.byref(nd), ctypes.byref(na), ctypes.byref(nq),
                                      ctypes.byref(used)))
    return [int(ids[k]) for k in range(min(nd.value, cap))], na.value, nq.value, int(used.value)


def hms_server_take(ctx, srv, rid, u_out=None, iters=None):
    """Copies the results of a finished request; returns its status code."""
    U = _Arg(u_out, writable=True)
    I = _Arg(iters, dtype=np.int32, writable=True)
    if U.kind == HMS_MEM_DEVICE or I.kind == HMS_MEM_DEVICE:
        raise ValueError("hms_server_take writes host arrays")
    return int(lib().hms_server_take(srv, int(rid), U.ptr, I.ptr))


def hms_kernel_times(pr):
    ms = (ctypes.c_double * 7)()
    n = (ctypes.c_int64 * 7)()
    k = lib().hms_kernel_times(pr, ctypes.cast(ms, _P), ctypes.cast(n, _P), 7)
    return {KERNEL_NAMES[i]: (float(ms[i]), int(n[i])) for i in range(k)}


def hms_residual(ctx, pr, p, u, r_out, norms_out):
    A = [_Arg(p), _Arg(u), _Arg(r_out, writable=True), _Arg(norms_out, writable=True)]
    _check(ctx, lib().hms_residual(pr, *[a.ptr for a in A], _mem_kind(*A)))


def hms_reactions(ctx, pr, u, f_out):
    """f_out = K u at every DOF, constrained ones included (u read as 0 there)."""
    A = [_Arg(u), _Arg(f_out, writable=True)]
    _check(ctx, lib().hms_reactions(pr, A[0].ptr, A[1].ptr, _mem_kind(*A)))


def hms_measure_fp64_rate(device=0) -> float:
    """Measured FP64 GFLOP/s of the device (an FMA-loop kernel)."""
    g = ctypes.c_double()
    st = lib().hms_measure_fp64_rate(int(device), ctypes.byref(g))
    if st != HMS_OK:
        raise HmsError(st, "FP64 rate probe failed")
    return float(g.value)


def hms_problem_refine_cap_hits(pr) -> int:
    return int(lib().hms_problem_refine_cap_hits(pr))


def hms_problem_set_relax_wait_limit(ctx, pr, spins):
    _check(ctx, lib().hms_problem_set_relax_wait_limit(pr, int(spins)))


def hms_residual_noalloc(ctx, pr, p, u, r_out, norms_out=None):
    """CUDA tensors only (float64, contiguous): r_out = p - K u and the three sums
    of hms_residual, with no device allocation inside the call.  Inputs must be
    complete before the call (e.g. torch.cuda.synchronize())."""
    A = [_Arg(p), _Arg(u), _Arg(r_out, writable=True), _Arg(norms_out, writable=True)]
    if any(a.kind != HMS_MEM_DEVICE for a in A if a.ptr is not None):
        raise ValueError("hms_residual_noalloc takes CUDA tensors only")
    _check(ctx, lib().hms_residual_noalloc(pr, *[a.ptr for a in A]))


def hms_update_residual(ctx, pr, p, u, delta, a, u_out, r_out, norms_out):
    A = [_Arg(p), _Arg(u), _Arg(delta), _Arg(a), _Arg(u_out, writable=True), _Arg(r_out, writable=True),
         _Arg(norms_out, writable=True)]
    _check(ctx, lib().hms_update_residual(pr, *[x.ptr for x in A], _mem_kind(*A)))


def hms_relax(ctx, pr, r, delta_out, P_out):
    A = [_Arg(r), _Arg(delta_out, writable=True), _Arg(P_out, writable=True)]
    _check(ctx, lib().hms_relax(pr, *[x.ptr for x in A], _mem_kind(*A)))


def hms_relax_force(ctx, pr, r, delta_rf_out):
    """The force-controlled increment delta^RF of Eq. 17 (problems with mode_mask bits 9-11)."""
    A = [_Arg(r), _Arg(delta_rf_out, writable=True)]
    _check(ctx, lib().hms_relax_force(pr, A[0].ptr, A[1].ptr, _mem_kind(*A)))


def hms_coarse_matrix(ctx, pr, delta, Kaa_out):
    A = [_Arg(delta), _Arg(Kaa_out, writable=True)]
    _check(ctx, lib().hms_coarse_matrix(pr, *[x.ptr for x in A], _mem_kind(*A)))


def hms_coarse_solve(ctx, pr, Kaa, P, a_out, dropped_out=None):
    A = [_Arg(Kaa), _Arg(P), _Arg(a_out, writable=True), _Arg(dropped_out, dtype=np.int32, writable=True)]
    _check(ctx, lib().hms_coarse_solve(pr, *[x.ptr for x in A], _mem_kind(*A)))
