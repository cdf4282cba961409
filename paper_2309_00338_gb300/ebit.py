"""Thin ctypes binding of libebit.so (include/ebit.h), same names as the C ABI.

Argument marshalling only: every step of the EBIT path runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams (``data_ptr()`` and
``torch.cuda.current_stream().cuda_stream``).  Loading fails loudly when the
library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH

EBIT_OK, EBIT_EAGAIN = 0, 1
EBIT_EINVAL, EBIT_ENOMEM, EBIT_ECFL, EBIT_EINVARIANT, EBIT_ECUDA, EBIT_ETIMEOUT, EBIT_EFULL, \
    EBIT_ECANCELLED = -1, -2, -3, -4, -5, -6, -7, -8
EBIT_FP64, EBIT_FP32 = 0, 1
EBIT_FIT_LINE = 1
EBIT_CURV_GHF = 2

# diagnostics indices (include/ebit.h)
D_NH, D_NV, D_CANCELLED, D_ZSET, D_ZCONFLICT, D_FIT_ONLINE, D_FIT_LINE, D_FIT_ONE, D_FIT_TWO, \
    D_WALL_CLAMP, D_INVARIANT, D_HF_INVALID, D_CFL, D_HF_OTHER, D_HF_MIXED, D_HF_MARKERS = range(16)
D_COUNT = 16

_STATUS_NAMES = {0: "EBIT_OK", 1: "EBIT_EAGAIN", -1: "EBIT_EINVAL", -2: "EBIT_ENOMEM",
                 -3: "EBIT_ECFL", -4: "EBIT_EINVARIANT", -5: "EBIT_ECUDA", -6: "EBIT_ETIMEOUT",
                 -7: "EBIT_EFULL", -8: "EBIT_ECANCELLED"}


class EbitError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ebit_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_double),
                ("prec", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class ebit_circle(ctypes.Structure):
    _fields_ = [("xc", ctypes.c_double), ("yc", ctypes.c_double), ("r", ctypes.c_double)]


class ebit_curve(ctypes.Structure):
    _fields_ = [("y0", ctypes.c_double), ("nmodes", ctypes.c_int32),
                ("amp", ctypes.POINTER(ctypes.c_double)), ("phase", ctypes.POINTER(ctypes.c_double))]


class ebit_halfplane(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double)]


class ebit_notch(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double),
                ("y1", ctypes.c_double)]


class ebit_scene(ctypes.Structure):
    _fields_ = [("circles", ctypes.POINTER(ebit_circle)), ("ncircles", ctypes.c_int32),
                ("curve", ctypes.POINTER(ebit_curve)), ("line", ctypes.POINTER(ebit_halfplane)),
                ("notches", ctypes.POINTER(ebit_notch)), ("nnotches", ctypes.c_int32),
                ("nlines", ctypes.c_int32)]


class ebit_fluids(ctypes.Structure):
    _fields_ = [("rho1", ctypes.c_double), ("rho2", ctypes.c_double), ("mu1", ctypes.c_double),
                ("mu2", ctypes.c_double), ("sigma", ctypes.c_double)]


class ebit_state_host(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("K", ctypes.c_void_p), ("Z", ctypes.c_void_p),
                ("sH", ctypes.c_void_p), ("sV", ctypes.c_void_p), ("step_index", ctypes.c_int64)]


class ebit_diag(ctypes.Structure):
    _fields_ = [("c", ctypes.c_int64 * D_COUNT), ("area", ctypes.c_double), ("max_cfl", ctypes.c_double)]


_lib = None

# exported symbols and their signatures: (restype, argtypes)
_P = ctypes.c_void_p
SIGNATURES = {
    "ebit_init": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ebit_grid), ctypes.POINTER(ebit_scene), _P]),
    "ebit_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ebit_grid), _P]),
    "ebit_load_state": (ctypes.c_int, [_P, ctypes.POINTER(ebit_state_host)]),
    "ebit_get_state": (ctypes.c_int, [_P, ctypes.POINTER(ebit_state_host)]),
    "ebit_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_double]),
    "ebit_sweep": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_double]),
    "ebit_fraction": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_double)]),
    "ebit_curvature": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int32)]),
    "ebit_fields": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int64)]),
    "ebit_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(ebit_diag)]),
    "ebit_sync": (ctypes.c_int, [_P]),
    "ebit_destroy": (None, [_P]),
    "ebit_last_error": (ctypes.c_char_p, []),
    "ebit_footprint": (ctypes.c_size_t, [ctypes.POINTER(ebit_grid)]),
    "ebit_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "ebit_timings": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "ebit_fraction_noalloc": (ctypes.c_int, [ctypes.POINTER(ebit_grid), _P, _P, _P, _P, _P, _P, _P, _P]),
    "ebit_coupling": (ctypes.c_int, [_P, ctypes.POINTER(ebit_fluids), _P, _P, _P, _P]),
    "ebit_area_async": (ctypes.c_int, [_P, _P]),
    "ebit_fraction_to_host": (ctypes.c_int, [_P, _P, _P]),
    "ebit_check_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
}

K_SWEEP, K_CENTRE, K_FIELDS, K_AREA, K_COUPLING, K_GHF = range(6)
K_COUNT = 8
# slots 1 and 3 are reserved in the ABI (always 0) and not reported
KERNEL_NAMES = ["sweep", None, "fields", None, "coupling", "ghf"]


def lib(path: str | None = None):
    """Load libebit.so (built by paper_2309_00338_gb300.build); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or os.environ.get("EBIT_LIB") or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libebit.so not built ({p}); run __graft_entry__.build() first")
    L = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = L
    return L


def _check(status, where):
    if status != EBIT_OK:
        raise EbitError(status, where, lib().ebit_last_error().decode())
    return status


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _scene(scene: dict, keep: list):
    sc = ebit_scene()
    circles = np.ascontiguousarray(np.asarray(scene.get("circles", np.zeros((0, 3))), np.float64).reshape(-1, 3))
    keep.append(circles)
    sc.ncircles = circles.shape[0]
    sc.circles = circles.ctypes.data_as(ctypes.POINTER(ebit_circle)) if circles.shape[0] else None
    if scene.get("curve") is not None:
        cv = scene["curve"]
        amp = np.ascontiguousarray(cv["amp"], np.float64)
        ph = np.ascontiguousarray(cv["phase"], np.float64)
        c = ebit_curve(float(cv["y0"]), int(amp.size), amp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       ph.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        keep += [amp, ph, c]
        sc.curve = ctypes.pointer(c)
    lines = list(scene.get("lines", []))
    if scene.get("line") is not None:
        lines = [scene["line"]] + lines
    if lines:
        arr = (ebit_halfplane * len(lines))(*(ebit_halfplane(*(float(t) for t in l)) for l in lines))
        keep.append(arr)
        sc.line = ctypes.cast(arr, ctypes.POINTER(ebit_halfplane))
        sc.nlines = len(lines)
    if scene.get("notches"):
        nb = np.ascontiguousarray(np.asarray(scene["notches"], np.float64).reshape(-1, 4))
        keep.append(nb)
        sc.nnotches = nb.shape[0]
        sc.notches = nb.ctypes.data_as(ctypes.POINTER(ebit_notch))
    return sc


def ebit_footprint(nx, ny, dx, prec=EBIT_FP64, flags=0) -> int:
    g = ebit_grid(nx, ny, dx, prec, flags)
    return int(lib().ebit_footprint(ctypes.byref(g)))


# Grid of every live context (handle value -> (nx, ny, prec)): the binding
# checks the caller's tensors against it before a call that reads or writes
# them, so that a wrongly sized buffer is refused instead of being accessed
# out of range.
_CTX = {}


def _grid_of(ctx):
    return _CTX.get(ctx.value if isinstance(ctx, ctypes.c_void_p) else ctx)


def _check_tensor(ctx, t, name, shape_fn, device):
    """Refuses t unless it has the element count shape_fn(nx, ny) and the
    dtype of the context's precision, on the device (or host) expected."""
    if t is None:
        return
    g = _grid_of(ctx)
    if g is None:
        return  # a handle the binding did not create: the caller vouches for it
    nx, ny, prec = g
    import torch
    want = torch.float32 if prec == EBIT_FP32 else torch.float64
    _expect(t, name, shape_fn(nx, ny), want)
    if bool(t.is_cuda) != device:
        raise ValueError(f"{name}: expected a {'CUDA' if device else 'host'} tensor")


def ebit_init(nx, ny, dx, scene: dict, prec=EBIT_FP64, flags=0, stream=None):
    """ebit_init: returns a context handle (c_void_p)."""
    g = ebit_grid(nx, ny, dx, prec, flags)
    keep = []
    sc = _scene(scene, keep)
    h = ctypes.c_void_p()
    _check(lib().ebit_init(ctypes.byref(h), ctypes.byref(g), ctypes.byref(sc), _stream(stream)), "ebit_init")
    _CTX[h.value] = (int(nx), int(ny), int(prec))
    return h


def ebit_create(nx, ny, dx, prec=EBIT_FP64, flags=0, stream=None):
    g = ebit_grid(nx, ny, dx, prec, flags)
    h = ctypes.c_void_p()
    _check(lib().ebit_create(ctypes.byref(h), ctypes.byref(g), _stream(stream)), "ebit_create")
    _CTX[h.value] = (int(nx), int(ny), int(prec))
    return h


def ebit_load_state(ctx, K, Z, sH, sV, step_index=0):
    K = np.ascontiguousarray(K, np.uint8)
    Z = np.ascontiguousarray(Z, np.uint8)
    sH = np.ascontiguousarray(sH, np.float64)
    sV = np.ascontiguousarray(sV, np.float64)
    ny, nx = Z.shape
    for name, arr, size in (("K", K, (ny + 1) * (nx + 1)), ("sH", sH, (ny + 1) * nx), ("sV", sV, ny * (nx + 1))):
        if arr.size != size:
            raise ValueError(f"{name}: expected {size} elements for a {nx} x {ny} grid, got {arr.size}")
    st = ebit_state_host(nx, ny, K.ctypes.data, Z.ctypes.data, sH.ctypes.data, sV.ctypes.data, int(step_index))
    _check(lib().ebit_load_state(ctx, ctypes.byref(st)), "ebit_load_state")


def ebit_get_state(ctx, nx, ny):
    """Returns dict K, Z, sH, sV (numpy) and step_index."""
    K = np.zeros((ny + 1, nx + 1), np.uint8)
    Z = np.zeros((ny, nx), np.uint8)
    sH = np.zeros((ny + 1, nx), np.float64)
    sV = np.zeros((ny, nx + 1), np.float64)
    st = ebit_state_host(nx, ny, K.ctypes.data, Z.ctypes.data, sH.ctypes.data, sV.ctypes.data, 0)
    _check(lib().ebit_get_state(ctx, ctypes.byref(st)), "ebit_get_state")
    return {"K": K, "Z": Z, "sH": sH, "sV": sV, "step_index": int(st.step_index)}


def _dev_ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def ebit_step(ctx, u, v, dt):
    """u, v: contiguous CUDA tensors (ny+1, nx+1) of the context precision."""
    vertices = lambda nx, ny: (nx + 1) * (ny + 1)  # noqa: E731
    _check_tensor(ctx, u, "u", vertices, True)
    _check_tensor(ctx, v, "v", vertices, True)
    _check(lib().ebit_step(ctx, _dev_ptr(u), _dev_ptr(v), float(dt)), "ebit_step")


def ebit_sweep(ctx, axis, vel, dt):
    _check_tensor(ctx, vel, "vel", lambda nx, ny: (nx + 1) * (ny + 1), True)
    _check(lib().ebit_sweep(ctx, int(axis), _dev_ptr(vel), float(dt)), "ebit_sweep")


def ebit_fraction(ctx, C=None, want_area=True):
    _check_tensor(ctx, C, "C", lambda nx, ny: nx * ny, True)
    a = ctypes.c_double(0.0)
    _check(lib().ebit_fraction(ctx, _dev_ptr(C), ctypes.byref(a) if want_area else None), "ebit_fraction")
    return a.value if want_area else None


def ebit_area_async(ctx, area_host):
    """Queue the copy of the area sum into area_host (a pinned CPU tensor of
    one float64) on the context's stream; valid once the stream gets there."""
    if area_host.is_cuda or area_host.dtype.itemsize != 8:
        raise ValueError("expected a host tensor of one float64")
    _check(lib().ebit_area_async(ctx, ctypes.c_void_p(area_host.data_ptr())), "ebit_area_async")


def ebit_fraction_to_host(ctx, C_host, stream=None):
    """Queue the copy of the current fractions C into C_host (a pinned,
    contiguous CPU tensor of ny*nx elements of the context precision) on
    `stream` (a torch.cuda.Stream; None: the context's stream).  C_host is
    filled once that stream gets there; the context's next fields
    computation waits for the copy on the device."""
    if C_host.is_cuda or not C_host.is_contiguous() or not C_host.is_pinned():
        raise ValueError("expected a pinned, contiguous host tensor")
    _check_tensor(ctx, C_host, "C_host", lambda nx, ny: nx * ny, False)
    st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(lib().ebit_fraction_to_host(ctx, ctypes.c_void_p(C_host.data_ptr()), st), "ebit_fraction_to_host")


def ebit_check_status():
    """Nonzero if a kernel of the checked build met an index outside its
    array (always 0 in the release build)."""
    m = ctypes.c_uint32(0)
    _check(lib().ebit_check_status(ctypes.byref(m)), "ebit_check_status")
    return m.value


def ebit_curvature(ctx, kappa=None, want_invalid=True):
    _check_tensor(ctx, kappa, "kappa", lambda nx, ny: nx * ny, True)
    n = ctypes.c_int32(0)
    _check(lib().ebit_curvature(ctx, _dev_ptr(kappa), ctypes.byref(n) if want_invalid else None),
           "ebit_curvature")
    return n.value if want_invalid else None


def ebit_fields(ctx):
    c, k = ctypes.c_void_p(), ctypes.c_void_p()
    p = ctypes.c_int64()
    _check(lib().ebit_fields(ctx, ctypes.byref(c), ctypes.byref(k), ctypes.byref(p)), "ebit_fields")
    return c.value, k.value, p.value


def ebit_coupling(ctx, rho1, rho2, mu1, mu2, sigma, rho=None, mu=None, fx=None, fy=None):
    """Properties (rho, mu: (ny, nx)) and face surface-tension sources (fx:
    (ny, nx+1), fy: (ny+1, nx)) from the context's current C and kappa, into
    caller-owned contiguous CUDA tensors of the context precision (None:
    skipped).  Asynchronous on the context's stream."""
    _check_tensor(ctx, rho, "rho", lambda nx, ny: nx * ny, True)
    _check_tensor(ctx, mu, "mu", lambda nx, ny: nx * ny, True)
    _check_tensor(ctx, fx, "fx", lambda nx, ny: ny * (nx + 1), True)
    _check_tensor(ctx, fy, "fy", lambda nx, ny: (ny + 1) * nx, True)
    fl = ebit_fluids(rho1, rho2, mu1, mu2, sigma)
    _check(lib().ebit_coupling(ctx, ctypes.byref(fl), _dev_ptr(rho), _dev_ptr(mu), _dev_ptr(fx), _dev_ptr(fy)),
           "ebit_coupling")


def ebit_diagnostics(ctx):
    d = ebit_diag()
    _check(lib().ebit_diagnostics(ctx, ctypes.byref(d)), "ebit_diagnostics")
    return {"counters": np.array(d.c[:], np.int64), "area": d.area, "max_cfl": d.max_cfl}


def ebit_sync(ctx):
    _check(lib().ebit_sync(ctx), "ebit_sync")


def ebit_destroy(ctx):
    if ctx:
        _CTX.pop(ctx.value if isinstance(ctx, ctypes.c_void_p) else ctx, None)
        lib().ebit_destroy(ctx)


def ebit_set_timing(ctx, on=True):
    _check(lib().ebit_set_timing(ctx, int(bool(on))), "ebit_set_timing")


def ebit_timings(ctx):
    """{kernel name: (total ms, launches)} since the last call."""
    ms = (ctypes.c_double * K_COUNT)()
    n = (ctypes.c_int64 * K_COUNT)()
    _check(lib().ebit_timings(ctx, ms, n), "ebit_timings")
    return {name: (ms[k], n[k]) for k, name in enumerate(KERNEL_NAMES) if name is not None}


def _expect(t, name, numel, dtype):
    """Refuses a tensor whose element count or type does not match what the
    kernel will read or write, before anything is launched."""
    if t.numel() != numel or t.dtype != dtype:
        raise ValueError(f"{name}: expected {numel} elements of {dtype}, got {t.numel()} of {t.dtype}")


def ebit_fraction_noalloc(nx, ny, dx, prec, K, Z, sH, sV, C, area, marker_counts=None, stream=None):
    """ebit_fraction_noalloc: fractions of a state in caller-owned device
    tensors (byte colours, fractions of the grid precision) without any
    device allocation; C, area (1 double) and marker_counts (2 int64) are
    caller-owned device tensors.  Sizes and types are checked against nx, ny
    and prec first (K (ny+1)(nx+1) and Z ny nx uint8, sH (ny+1) nx, sV
    ny (nx+1) and C ny nx of the precision)."""
    import torch
    nx, ny = int(nx), int(ny)
    if nx < 1 or ny < 1:
        raise ValueError("nx and ny must be positive")
    ft = torch.float64 if prec == EBIT_FP64 else torch.float32
    _expect(K, "K", (ny + 1) * (nx + 1), torch.uint8)
    _expect(Z, "Z", ny * nx, torch.uint8)
    _expect(sH, "sH", (ny + 1) * nx, ft)
    _expect(sV, "sV", ny * (nx + 1), ft)
    _expect(C, "C", ny * nx, ft)
    _expect(area, "area", 1, torch.float64)
    if marker_counts is not None:
        _expect(marker_counts, "marker_counts", 2, torch.int64)
    g = ebit_grid(nx, ny, dx, prec, 0)
    _check(lib().ebit_fraction_noalloc(ctypes.byref(g), _dev_ptr(K), _dev_ptr(Z), _dev_ptr(sH), _dev_ptr(sV),
                                       _dev_ptr(C), _dev_ptr(area), _dev_ptr(marker_counts), _stream(stream)),
           "ebit_fraction_noalloc")


# ---------------------------------------------------------------------------
# batched steps and serving
# ---------------------------------------------------------------------------
EBIT_FIELD_VORTEX, EBIT_FIELD_CELLULAR, EBIT_FIELD_ROTATION = 0, 1, 2


class ebit_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("prec", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("circles", ctypes.POINTER(ebit_circle)), ("ncircles", ctypes.c_int32),
                ("field", ctypes.c_int32), ("period", ctypes.c_double),
                ("omega", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("drift_u", ctypes.c_double), ("drift_v", ctypes.c_double),
                ("steps", ctypes.c_int32), ("cfl", ctypes.c_double), ("C_out", ctypes.c_void_p),
                ("fault_after", ctypes.c_int32), ("fault_dt_factor", ctypes.c_double),
                ("fault_wait", ctypes.c_int32)]


class ebit_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_int64),
                ("area0", ctypes.c_double), ("area", ctypes.c_double), ("e_area", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("step_p50_ms", ctypes.c_double), ("step_p99_ms", ctypes.c_double),
                ("counters", ctypes.c_int64 * D_COUNT), ("cell_updates", ctypes.c_int64)]


(EBIT_SCHED_LARGEST_FIRST, EBIT_SCHED_INTERLEAVED, EBIT_SCHED_SMALLEST_FIRST,
 EBIT_SCHED_PERSISTENT_LARGEST_FIRST, EBIT_SCHED_PERSISTENT_INTERLEAVED, EBIT_SCHED_PERSISTENT_SMALLEST_FIRST,
 EBIT_SCHED_COUNT) = range(7)


class ebit_server_opts(ctypes.Structure):
    _fields_ = [("max_instances", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("device", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("wait_budget_ms", ctypes.c_int32)]


class ebit_server_stats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("batch_steps", ctypes.c_int64), ("cell_updates", ctypes.c_int64),
                ("busy_ms", ctypes.c_double), ("bytes_in_use", ctypes.c_size_t),
                ("schedule", ctypes.c_int32), ("tuned_sets", ctypes.c_int32),
                ("tune_ms", ctypes.c_double * EBIT_SCHED_COUNT),
                ("plans", ctypes.c_int64), ("plan_ms", ctypes.c_double), ("plan_graph_ms", ctypes.c_double),
                ("admit_idle_ms", ctypes.c_double), ("retire_ms", ctypes.c_double)]


SIGNATURES.update({
    "ebit_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_size_t, ctypes.POINTER(ebit_server_opts)]),
    "ebit_submit": (ctypes.c_int, [_P, ctypes.POINTER(ebit_request), ctypes.POINTER(ctypes.c_uint64)]),
    "ebit_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(ebit_result)]),
    "ebit_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "ebit_server_stats_get": (ctypes.c_int, [_P, ctypes.POINTER(ebit_server_stats)]),
    "ebit_server_destroy": (None, [_P]),
})
if _lib is not None:  # signatures added after an earlier load
    for _n in ("ebit_server_create", "ebit_submit", "ebit_poll", "ebit_cancel", "ebit_server_stats_get",
               "ebit_server_destroy"):
        _f = getattr(_lib, _n)
        _f.restype, _f.argtypes = SIGNATURES[_n]


def ebit_server_create(hbm_budget, max_instances=0, use_graphs=True, device=0, autotune=True,
                       schedule=EBIT_SCHED_LARGEST_FIRST, wait_budget_ms=0):
    o = ebit_server_opts(int(max_instances), int(bool(use_graphs)), int(device), int(bool(autotune)),
                         int(schedule), int(wait_budget_ms))
    h = ctypes.c_void_p()
    _check(lib().ebit_server_create(ctypes.byref(h), int(hbm_budget), ctypes.byref(o)), "ebit_server_create")
    return h


def make_request(n, circles, field=EBIT_FIELD_CELLULAR, steps=10, cfl=0.5, prec=EBIT_FP64, period=1.0,
                 omega=0.0, centre=(0.5, 0.5), drift=(0.0, 0.0), C_out=None, flags=0, fault_after=0,
                 fault_dt_factor=0.0, fault_wait=False):
    """Build an ebit_request; returns (request, keep-alive list).
    fault_after / fault_dt_factor: fault injection for tests of the server's
    failure isolation (dt times the factor from that step on; 0 = off);
    fault_wait: from step fault_after on, the persistent schedules' wait for
    this grid's first sweep cannot be met (it runs out: EBIT_ETIMEOUT)."""
    circ = np.ascontiguousarray(np.asarray(circles, np.float64).reshape(-1, 3))
    keep = [circ]
    r = ebit_request()
    r.n, r.prec, r.flags = int(n), int(prec), int(flags)
    r.circles = circ.ctypes.data_as(ctypes.POINTER(ebit_circle)) if circ.shape[0] else None
    r.ncircles = circ.shape[0]
    r.field, r.period, r.omega = int(field), float(period), float(omega)
    r.cx, r.cy = (float(t) for t in centre)
    r.drift_u, r.drift_v = (float(t) for t in drift)
    r.steps, r.cfl = int(steps), float(cfl)
    r.fault_after, r.fault_dt_factor = int(fault_after), float(fault_dt_factor)
    r.fault_wait = 1 if fault_wait else 0
    if C_out is not None:
        assert C_out.flags["C_CONTIGUOUS"] and C_out.size == n * n
        r.C_out = C_out.ctypes.data
        keep.append(C_out)
    return r, keep


def ebit_submit(server, request):
    """Returns the ticket, or raises EbitError (EBIT_EINVAL / EBIT_EFULL)."""
    t = ctypes.c_uint64()
    _check(lib().ebit_submit(server, ctypes.byref(request), ctypes.byref(t)), "ebit_submit")
    return t.value


def ebit_poll(server, ticket):
    """The result dict once done, None while queued or running."""
    r = ebit_result()
    st = lib().ebit_poll(server, ctypes.c_uint64(ticket), ctypes.byref(r))
    if st == EBIT_EAGAIN:
        return None
    _check(st, "ebit_poll")
    return {"status": r.status, "steps": r.steps, "area0": r.area0, "area": r.area, "e_area": r.e_area,
            "queue_ms": r.queue_ms, "run_ms": r.run_ms, "step_p50_ms": r.step_p50_ms,
            "step_p99_ms": r.step_p99_ms, "counters": np.array(r.counters[:], np.int64),
            "cell_updates": r.cell_updates}


def ebit_cancel(server, ticket):
    """Cancels a queued or running request (its result then reports
    EBIT_ECANCELLED); raises EbitError for an unknown or finished ticket."""
    _check(lib().ebit_cancel(server, ctypes.c_uint64(ticket)), "ebit_cancel")


def ebit_server_stats_get(server):
    s = ebit_server_stats()
    _check(lib().ebit_server_stats_get(server, ctypes.byref(s)), "ebit_server_stats_get")
    return {"queued": s.queued, "running": s.running, "batch_steps": s.batch_steps,
            "cell_updates": s.cell_updates, "busy_ms": s.busy_ms, "bytes_in_use": s.bytes_in_use,
            "schedule": s.schedule, "tuned_sets": s.tuned_sets, "tune_ms": list(s.tune_ms),
            "plans": s.plans, "plan_ms": s.plan_ms, "plan_graph_ms": s.plan_graph_ms,
            "admit_idle_ms": s.admit_idle_ms,
            "retire_ms": s.retire_ms}


def ebit_server_destroy(server):
    if server:
        lib().ebit_server_destroy(server)


def wait_all(server, tickets, timeout_s=600.0, poll_s=0.002):
    """Poll until every ticket has a result; returns {ticket: result}."""
    import time
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = ebit_poll(server, t)
                if r is not None:
                    out[t] = r
        if time.time() - t0 > timeout_s:
            raise TimeoutError(f"{len(tickets) - len(out)} requests still running")
        time.sleep(poll_s)
    return out
