"""EBIT oracle: plain single-threaded FP64 (and FP32-state) CPU restatement of
one EBIT interface step (Pan et al., Sec. 2.1-2.5), for tests only.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
package.  The product library never does, and the two share no code.

``build()`` compiles ``ebit_oracle.cpp`` with ``-ffp-contract=off`` into
``oracle/_build/liboracle.so``; the functions below marshal numpy arrays to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ebit_oracle.cpp")
_HDR = os.path.join(_HERE, "ebit_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# counter indices (must follow the enum in ebit_oracle.h)
N_H, N_V, CANCELLED, ZSET, ZCONFLICT, FIT_ONLINE, FIT_LINE, FIT_ONE, FIT_TWO, \
    WALL_CLAMP, INVARIANT, HF_INVALID, CFL = range(13)
NCOUNTERS = 16

FP64, FP32 = 0, 1
LINE_ONLY = 2  # flag: straight-line fit (EBIT-SL)
GHF = 4        # flag: generalised height-function fallbacks for curvature


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Scene(ctypes.Structure):
    _fields_ = [
        ("ncircles", ctypes.c_int32),
        ("xc", ctypes.c_void_p), ("yc", ctypes.c_void_p), ("r", ctypes.c_void_p),
        ("has_curve", ctypes.c_int32), ("y0", ctypes.c_double), ("nmodes", ctypes.c_int32),
        ("amp", ctypes.c_void_p), ("phase", ctypes.c_void_p),
        ("nlines", ctypes.c_int32), ("la", ctypes.c_double * 4), ("lb", ctypes.c_double * 4),
        ("lc", ctypes.c_double * 4),
        ("nnotches", ctypes.c_int32), ("notch", ctypes.c_void_p),
    ]


class use_library:
    """Context manager that points every function of this module at another
    build of the oracle (used by the mutant tests, which compile copies of the
    oracle with one planted mistake each)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        self._saved = _lib
        L = ctypes.CDLL(self.path)
        _set_signatures(L)
        _lib = L
        return L

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source to out_path."""
    d = os.path.dirname(out_path)
    os.makedirs(d, exist_ok=True)
    src = os.path.join(d, "ebit_oracle.cpp")
    with open(src, "w") as f:
        f.write(src_text)
    import shutil
    shutil.copy(_HDR, os.path.join(d, "ebit_oracle.h"))
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared",
                    src, "-o", out_path], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _set_signatures(L):
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.orc_init.argtypes = [i32, i32, f64, i32, ctypes.POINTER(_Scene), P, P, P, P]
    L.orc_sweep.argtypes = [i32, i32, i32, i32, P, P, P, P, P, f64, P, P]
    L.orc_step.argtypes = [i32, i32, f64, i32, i64, P, P, P, P, P, P, f64, P, P, P, P]
    L.orc_fraction.argtypes = [i32, i32, f64, i32, P, P, P, P, P, P]
    L.orc_curvature.argtypes = [i32, i32, f64, i32, P, P, P, P, P, P, P]
    L.orc_fit.argtypes = [P, P, P, i32, P, i32, P]
    L.orc_coupling.argtypes = [i32, i32, f64, i32, P, P, f64, f64, f64, f64, f64, P, P, P, P]
    L.orc_parabola_kappa.argtypes = [i32, P, P, P, f64, f64, f64, f64, f64, P]
    L.orc_loops.argtypes = [i32, i32, f64, i32, P, P, P, P, P, P, P, i64, P]
    L.orc_loops.restype = i64
    L.orc_shape_error.argtypes = [i32, i32, f64, P, P, P, f64, f64, f64]
    L.orc_shape_error.restype = f64
    L.orc_sym_diff.argtypes = [i32, i32, f64, i32, P, P, P, P, P, P, P, P]
    L.orc_sym_diff.restype = f64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            _set_signatures(L)
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class State:
    """Host state of one grid: colour vertices K (corners), Z (centres) and
    edge-local marker fractions sH, sV (float64 arrays; FP32 form values are
    exactly representable in float32)."""

    def __init__(self, nx, ny, dx, prec=FP64):
        self.nx, self.ny, self.dx, self.prec = int(nx), int(ny), float(dx), int(prec)
        self.K = np.zeros((ny + 1, nx + 1), np.uint8)
        self.Z = np.zeros((ny, nx), np.uint8)
        self.sH = np.zeros((ny + 1, nx), np.float64)
        self.sV = np.zeros((ny, nx + 1), np.float64)
        self.step_index = 0

    def copy(self):
        s = State(self.nx, self.ny, self.dx, self.prec)
        s.K[...] = self.K
        s.Z[...] = self.Z
        s.sH[...] = self.sH
        s.sV[...] = self.sV
        s.step_index = self.step_index
        return s

    @property
    def hasH(self):
        return self.K[:, :-1] != self.K[:, 1:]

    @property
    def hasV(self):
        return self.K[:-1, :] != self.K[1:, :]

    @property
    def four(self):
        """Cells with a marker on all four edges."""
        K = self.K
        a, b, c, d = K[:-1, :-1], K[:-1, 1:], K[1:, 1:], K[1:, :-1]
        return (a != b) & (b != c) & (c != d) & (d != a)


def _scene_struct(scene, keep):
    sc = _Scene()
    circles = np.ascontiguousarray(np.asarray(scene.get("circles", np.zeros((0, 3))), np.float64).reshape(-1, 3))
    xc = np.ascontiguousarray(circles[:, 0]); yc = np.ascontiguousarray(circles[:, 1])
    r = np.ascontiguousarray(circles[:, 2])
    keep += [xc, yc, r]
    sc.ncircles = circles.shape[0]
    sc.xc, sc.yc, sc.r = xc.ctypes.data, yc.ctypes.data, r.ctypes.data
    curve = scene.get("curve")
    if curve is not None:
        amp = np.ascontiguousarray(np.asarray(curve["amp"], np.float64))
        ph = np.ascontiguousarray(np.asarray(curve["phase"], np.float64))
        keep += [amp, ph]
        sc.has_curve, sc.y0, sc.nmodes = 1, float(curve["y0"]), int(amp.size)
        sc.amp, sc.phase = amp.ctypes.data, ph.ctypes.data
    lines = list(scene.get("lines", []))
    if scene.get("line") is not None:
        lines = [scene["line"]] + lines
    if len(lines) > 4:
        raise ValueError("at most 4 half-planes")
    sc.nlines = len(lines)
    for l, (a, b, c) in enumerate(lines):
        sc.la[l], sc.lb[l], sc.lc[l] = float(a), float(b), float(c)
    notches = scene.get("notches")
    if notches:
        nb = np.ascontiguousarray(np.asarray(notches, np.float64).reshape(-1, 4))
        keep.append(nb)
        sc.nnotches, sc.notch = nb.shape[0], nb.ctypes.data
    return sc


def init(nx, ny, dx, scene, prec=FP64) -> State:
    """Colour vertices and markers of a scene (Sec. 3.2 initialisation).

    scene: dict with optional "circles" (n,3) [xc, yc, r], "curve"
    {"y0", "amp", "phase"} (reference phase below y = h(x)), "line"
    (a, b, c) and "lines" [(a, b, c), ...] (each toggles where
    a x + b y <= c; four at most) and "notches"."""
    S = State(nx, ny, dx, prec)
    keep = []
    sc = _scene_struct(scene, keep)
    rc = lib().orc_init(nx, ny, dx, prec & 1, ctypes.byref(sc), _p(S.K), _p(S.Z), _p(S.sH), _p(S.sV))
    if rc != 0:
        raise ValueError("orc_init failed")
    return S


def _vel(a, S):
    a = np.ascontiguousarray(a, np.float64)
    assert a.shape == (S.ny + 1, S.nx + 1)
    return a


def sweep(S: State, axis: int, vel, lam: float, line_only=False):
    """One split sweep in place; returns (counters, max |d|)."""
    ctr = np.zeros(NCOUNTERS, np.int64)
    mc = np.zeros(1, np.float64)
    w = _vel(vel, S)
    lib().orc_sweep(S.nx, S.ny, S.prec | (LINE_ONLY if line_only else 0), axis,
                    _p(S.K), _p(S.Z), _p(S.sH), _p(S.sV), _p(w), float(lam), _p(ctr), _p(mc))
    return ctr, float(mc[0])


def step(S: State, u, v, dt: float, line_only=False, ghf=False):
    """One full EBIT step in place.  Returns dict with C, kappa, counters,
    area and max_cfl; the state's step_index advances by one."""
    C = np.zeros((S.ny, S.nx), np.float64)
    kap = np.zeros((S.ny, S.nx), np.float64)
    ctr = np.zeros(NCOUNTERS, np.int64)
    stats = np.zeros(2, np.float64)
    uu, vv = _vel(u, S), _vel(v, S)
    rc = lib().orc_step(S.nx, S.ny, S.dx, S.prec | (LINE_ONLY if line_only else 0) | (GHF if ghf else 0),
                        S.step_index,
                        _p(S.K), _p(S.Z), _p(S.sH), _p(S.sV), _p(uu), _p(vv), float(dt),
                        _p(C), _p(kap), _p(ctr), _p(stats))
    S.step_index += 1
    return {"C": C, "kappa": kap, "counters": ctr, "area": float(stats[0]),
            "max_cfl": float(stats[1]), "status": int(rc)}


def fraction(S: State):
    C = np.zeros((S.ny, S.nx), np.float64)
    a = np.zeros(1, np.float64)
    lib().orc_fraction(S.nx, S.ny, S.dx, S.prec, _p(S.K), _p(S.Z), _p(S.sH), _p(S.sV), _p(C), _p(a))
    return C, float(a[0])


def curvature(S: State, C, ghf=False):
    """kappa (NaN where none) and the number of interface cells without a
    valid 7x3 stencil; with ghf=True also the counts resolved by the other
    direction, mixed heights and the markers of the 3x3 block."""
    C = np.ascontiguousarray(C, np.float64)
    kap = np.zeros((S.ny, S.nx), np.float64)
    n = np.zeros(4, np.int64)
    lib().orc_curvature(S.nx, S.ny, S.dx, S.prec | (GHF if ghf else 0), _p(S.K), _p(S.Z), _p(S.sH),
                        _p(S.sV), _p(C), _p(kap), _p(n))
    if ghf:
        return kap, int(n[0]), {"other": int(n[1]), "mixed": int(n[2]), "markers": int(n[3])}
    return kap, int(n[0])


def parabola_kappa(X, Y, W, origin, normal, dx=1.0):
    """Test hook: the least-squares parabola fit of the generalised
    fallbacks; returns kappa or None when the fit is singular."""
    X = np.ascontiguousarray(X, np.float64); Y = np.ascontiguousarray(Y, np.float64)
    W = np.ascontiguousarray(W, np.float64)
    k = np.zeros(1, np.float64)
    ok = lib().orc_parabola_kappa(len(X), _p(X), _p(Y), _p(W), float(origin[0]), float(origin[1]),
                                  float(normal[0]), float(normal[1]), float(dx), _p(k))
    return float(k[0]) if ok else None


def coupling(S: State, C, kappa, rho1, rho2, mu1, mu2, sigma):
    """Properties and face surface-tension source from C and kappa; returns
    (rho, mu, fx, fy) with shapes (ny, nx), (ny, nx), (ny, nx+1), (ny+1, nx)."""
    C = np.ascontiguousarray(C, np.float64)
    kappa = np.ascontiguousarray(kappa, np.float64)
    rho = np.zeros((S.ny, S.nx)); mu = np.zeros((S.ny, S.nx))
    fx = np.zeros((S.ny, S.nx + 1)); fy = np.zeros((S.ny + 1, S.nx))
    lib().orc_coupling(S.nx, S.ny, S.dx, S.prec, _p(C), _p(kappa), rho1, rho2, mu1, mu2, sigma,
                       _p(rho), _p(mu), _p(fx), _p(fy))
    return rho, mu, fx, fy


def fit(A, B, P1=None, P4=None):
    """Vertex-local circle fit of one crossing; returns (kind, y)."""
    a = np.asarray(A, np.float64); b = np.asarray(B, np.float64)
    p1 = np.asarray(P1 if P1 is not None else (0, 0), np.float64)
    p4 = np.asarray(P4 if P4 is not None else (0, 0), np.float64)
    y = np.zeros(1, np.float64)
    kind = lib().orc_fit(_p(a), _p(b), _p(p1), int(P1 is not None), _p(p4), int(P4 is not None), _p(y))
    return int(kind), float(y[0])


def loops(S: State, with_points=False):
    """(closed loops, open chains, shoelace area[, list of (n,2) polylines])."""
    n_open = np.zeros(1, np.int64)
    area = np.zeros(1, np.float64)
    nw = np.zeros(1, np.int64)
    L = lib()
    if not with_points:
        c = L.orc_loops(S.nx, S.ny, S.dx, S.prec, _p(S.K), _p(S.Z), _p(S.sH), _p(S.sV),
                        _p(n_open), _p(area), None, 0, _p(nw))
        return int(c), int(n_open[0]), float(area[0])
    L.orc_loops(S.nx, S.ny, S.dx, S.prec, _p(S.K), _p(S.Z), _p(S.sH), _p(S.sV),
                _p(n_open), _p(area), None, 0, _p(nw))
    cap = int(nw[0])
    xy = np.zeros((cap, 2), np.float64)
    c = L.orc_loops(S.nx, S.ny, S.dx, S.prec, _p(S.K), _p(S.Z), _p(S.sH), _p(S.sV),
                    _p(n_open), _p(area), _p(xy), cap, _p(nw))
    polys, cur = [], []
    for p in xy:
        if np.isnan(p[0]):
            polys.append(np.array(cur))
            cur = []
        else:
            cur.append(p)
    return int(c), int(n_open[0]), float(area[0]), polys


def shape_error(S: State, xc, yc, R):
    """E_shape of Eq. 14 against the circle (xc, yc, R)."""
    return float(lib().orc_shape_error(S.nx, S.ny, S.dx, _p(S.K), _p(S.sH), _p(S.sV),
                                       float(xc), float(yc), float(R)))


def sym_diff(A: State, B: State):
    """E_sym of Eqs. 15-16: area of the symmetric difference of the two
    states' reference-phase regions (domain units)."""
    assert (A.nx, A.ny, A.prec & 1) == (B.nx, B.ny, B.prec & 1)
    return float(lib().orc_sym_diff(A.nx, A.ny, A.dx, A.prec, _p(A.K), _p(A.Z), _p(A.sH), _p(A.sV),
                                    _p(B.K), _p(B.Z), _p(B.sH), _p(B.sV)))


def markers(S: State):
    """All marker positions (domain units) as an (n,2) array."""
    jH, iH = np.nonzero(S.hasH)
    jV, iV = np.nonzero(S.hasV)
    xh = (iH + S.sH[jH, iH]) * S.dx
    yh = jH * S.dx
    xv = iV * S.dx
    yv = (jV + S.sV[jV, iV]) * S.dx
    return np.concatenate([np.stack([xh, yh], 1), np.stack([xv, yv], 1)])
