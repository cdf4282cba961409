"""Seeded synthetic inputs: scenes (circles, Fourier curve, half-planes) and
velocity fields sampled at grid vertices.

This module holds none of the EBIT arithmetic.  It only produces inputs, and it
is the one piece shared by the CUDA path's tests/benchmarks and by the oracle.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based stream:
draw n is the SplitMix64 output for state seed + (n+1)*0x9E3779B97F4A7C15,
written here from that definition and evaluated vectorised with numpy.  A
uniform double is (x >> 11) * 2^-53.  No library distribution is used, so the
streams are the same on every machine.

The workloads stand in for the paper's analytic tests (translation, single
vortex, solid rotation; Sec. 3.2-3.4); no dataset is involved.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state):
    """SplitMix64 output function of a uint64 array of states."""
    z = np.asarray(state, np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """Counter-based SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & ((1 << 64) - 1))
        self.n = 0

    def u64(self, size: int) -> np.ndarray:
        k = np.arange(self.n + 1, self.n + 1 + size, dtype=np.uint64)
        self.n += size
        with np.errstate(over="ignore"):
            return splitmix64(self.seed + k * _GAMMA)

    def uniform(self, lo=0.0, hi=1.0, size=None):
        m = 1 if size is None else int(size)
        u = (self.u64(m) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        out = lo + (hi - lo) * u
        return float(out[0]) if size is None else out

    def integer(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)


# ---------------------------------------------------------------------------
# exact-at-the-walls trigonometry for vertex fields: sin(pi x) and cos(pi x)
# with the argument reduced first, so that integers and half-integers give
# exact zeros
# ---------------------------------------------------------------------------
def sinpi(x):
    x = np.asarray(x, np.float64)
    r = x - 2.0 * np.round(x * 0.5)          # r in [-1, 1]
    a = np.where(r > 0.5, 1.0 - r, np.where(r < -0.5, -1.0 - r, r))
    out = np.sin(math.pi * a)
    return np.where(a == 0.0, 0.0, out)


def cospi(x):
    return sinpi(np.asarray(x, np.float64) + 0.5)


# ---------------------------------------------------------------------------
# velocity fields at vertices: arrays (ny+1, nx+1), x = i*dx, y = j*dx
# ---------------------------------------------------------------------------
@dataclass
class Field:
    """A velocity field u(x,y) g(t), v(x,y) g(t) sampled at the vertices.

    The time factor g is applied by scaling the step's dt (u g dt = u (g dt)),
    so a step takes the fixed spatial arrays and dt_eff = dt * g(t_n)."""
    name: str
    u: np.ndarray
    v: np.ndarray
    period: float = 0.0          # T for the reversing fields, 0 = steady
    kind: str = "steady"         # "steady" | "cos" | "reverse_half"
    umax: float = 1.0

    def factor(self, t: float) -> float:
        if self.kind == "cos":
            return math.cos(math.pi * t / self.period)
        if self.kind == "reverse_half":
            return 1.0 if t < 0.5 * self.period - 1e-12 else -1.0
        return 1.0

    def dt_eff(self, n: int, dt: float) -> float:
        return dt * self.factor(n * dt)


def _xy(nx, ny, dx):
    x = np.arange(nx + 1, dtype=np.float64) * dx
    y = np.arange(ny + 1, dtype=np.float64) * dx
    return np.meshgrid(x, y)  # shapes (ny+1, nx+1)


def uniform_field(nx, ny, dx, u0, v0, period=0.0, reverse=False):
    U = np.full((ny + 1, nx + 1), float(u0))
    V = np.full((ny + 1, nx + 1), float(v0))
    return Field("uniform", U, V, period, "reverse_half" if reverse else "steady",
                 max(abs(u0), abs(v0)))


def vortex_field(nx, ny, dx, period, paper_sign=False):
    """Single vortex.  paper_sign: stream function pi^-1 sin^2(pi x) sin^2(pi y)
    cos(pi t/T) with u = d phi/dy, v = -d phi/dx (Sec. 3.3); otherwise the
    mirrored field u = -sin^2(pi x) sin(2 pi y), v = sin^2(pi y) sin(2 pi x)."""
    X, Y = _xy(nx, ny, dx)
    sx, sy = sinpi(X), sinpi(Y)
    U = sx * sx * sinpi(2.0 * Y)
    V = -(sy * sy) * sinpi(2.0 * X)
    if not paper_sign:
        U, V = -U, -V
    return Field("vortex", U, V, period, "cos", 1.0)


def cellular_field(nx, ny, dx):
    """Steady cellular flow u = sin(pi x) cos(pi y), v = -cos(pi x) sin(pi y)."""
    X, Y = _xy(nx, ny, dx)
    U = sinpi(X) * cospi(Y)
    V = -cospi(X) * sinpi(Y)
    return Field("cellular", U, V, 0.0, "steady", 1.0)


def rotation_field(nx, ny, dx, omega=2.0 * math.pi, centre=(0.5, 0.5), drift=(0.0, 0.0)):
    """Solid rotation u = -omega (y - yc) + du, v = omega (x - xc) + dv."""
    X, Y = _xy(nx, ny, dx)
    U = -omega * (Y - centre[1]) + drift[0]
    V = omega * (X - centre[0]) + drift[1]
    umax = float(max(np.abs(U).max(), np.abs(V).max()))
    return Field("rotation", U, V, 0.0, "steady", umax)


def linear_field(nx, ny, dx, a=(0.0, 0.0, 0.0), b=(0.0, 0.0, 0.0)):
    """u = a0 + a1 x + a2 y, v = b0 + b1 x + b2 y (exact under linear
    interpolation along an edge)."""
    X, Y = _xy(nx, ny, dx)
    U = a[0] + a[1] * X + a[2] * Y
    V = b[0] + b[1] * X + b[2] * Y
    return Field("linear", U, V, 0.0, "steady", float(max(np.abs(U).max(), np.abs(V).max())))


# ---------------------------------------------------------------------------
# scenes
# ---------------------------------------------------------------------------
def circle_scene(circles):
    return {"circles": np.asarray(circles, np.float64).reshape(-1, 3)}


def fourier_curve(rng: Rng, y0=0.5, nmodes=16, amp0=0.01):
    amp = np.array([amp0 / (k * k) for k in range(1, nmodes + 1)])
    phase = np.array([rng.uniform(0.0, 2.0 * math.pi) for _ in range(nmodes)])
    return {"y0": y0, "amp": amp, "phase": phase}


def curve_height(curve, x):
    x = np.asarray(x, np.float64)
    h = np.full_like(x, curve["y0"])
    for k, (a, p) in enumerate(zip(curve["amp"], curve["phase"]), start=1):
        h = h + a * np.cos(2.0 * math.pi * k * x + p)
    return h


class _Bins:
    """Uniform hash grid of placed circles for the gap test."""

    def __init__(self, cell):
        self.cell = cell
        self.b = {}

    def near(self, x, y):
        ci, cj = int(x // self.cell), int(y // self.cell)
        for a in (ci - 1, ci, ci + 1):
            for b in (cj - 1, cj, cj + 1):
                yield from self.b.get((a, b), ())

    def add(self, c):
        key = (int(c[0] // self.cell), int(c[1] // self.cell))
        self.b.setdefault(key, []).append(c)


def place_circles(rng: Rng, count, rmin, rmax, gap, region, curve=None, max_tries=1000,
                  wall_gap=None):
    """Seeded random sequential placement of `count` attempted circles.  Each
    attempt draws its radius once, then up to max_tries centres (drawn as one
    batch); the first centre whose gap to every placed circle (and to the
    curve, if any) is at least `gap` and for which region(x, y, r) holds is
    accepted, otherwise the attempt is dropped.  Returns an (n, 3) array
    [xc, yc, r] (domain units), n <= count."""
    wall_gap = gap if wall_gap is None else wall_gap
    bins = _Bins(2.0 * rmax + gap)
    out = []
    for _ in range(count):
        r = rng.uniform(rmin, rmax)
        xs = rng.uniform(r + wall_gap, 1.0 - r - wall_gap, max_tries)
        ys = rng.uniform(r + wall_gap, 1.0 - r - wall_gap, max_tries)
        for x, y in zip(xs.tolist(), ys.tolist()):
            if not region(x, y, r):
                continue
            ok = True
            for (px, py, pr) in bins.near(x, y):
                if (x - px) ** 2 + (y - py) ** 2 < (r + pr + gap) ** 2:
                    ok = False
                    break
            if ok and curve is not None:
                cx = np.linspace(x - r - gap, x + r + gap, 64)
                hs = curve_height(curve, cx)
                if np.min((cx - x) ** 2 + (hs - y) ** 2) < (r + gap) ** 2:
                    ok = False
            if ok:
                c = (x, y, r)
                out.append(c)
                bins.add(c)
                break
    return np.array(out, np.float64).reshape(-1, 3)


# ---------------------------------------------------------------------------
# the named workloads
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    n: int
    dx: float
    scene: dict
    field: Field
    dt: float
    steps: int
    meta: dict = field(default_factory=dict)


def vortex_workload(n=64, period=2.0, cfl=0.5, paper_sign=False):
    """Plain FP64 vortex: circle R=0.15 at (0.5,0.75), single vortex with
    period T, dt from CFL with u_max = 1, run to t = T."""
    dx = 1.0 / n
    dt = cfl * dx
    steps = int(round(period / dt))
    f = vortex_field(n, n, dx, period, paper_sign)
    return Workload(f"vortex_T{period:g}_n{n}", n, dx, circle_scene([(0.5, 0.75, 0.15)]), f, dt,
                    steps, {"circle": (0.5, 0.75, 0.15)})


def translation_workload(n=32, cfl=0.125):
    """Translation with uniform velocity (Sec. 3.2): R=0.15 at (0.25,0.75),
    (u,v) = (1,-1), reversed at T/2, T = 1."""
    dx = 1.0 / n
    dt = cfl * dx
    steps = int(round(1.0 / dt))
    f = uniform_field(n, n, dx, 1.0, -1.0, period=1.0, reverse=True)
    return Workload(f"translation_n{n}", n, dx, circle_scene([(0.25, 0.75, 0.15)]), f, dt, steps,
                    {"circle": (0.25, 0.75, 0.15)})


def zalesak_workload(n=64, cfl=math.pi / 16):
    """Zalesak's disk (Sec. 3.4): a disk R=0.15 at (0.5,0.75) with a notch 0.05
    wide reaching 0.25 up from its bottom, in solid rotation (u, v) =
    (2 pi (0.5 - y), 2 pi (x - 0.5)) for one turn, T = 1; dt from the CFL with
    the largest velocity component at t = 0 (pi)."""
    dx = 1.0 / n
    f = rotation_field(n, n, dx, 2.0 * math.pi, (0.5, 0.5))
    dt = cfl * dx / f.umax
    steps = int(round(1.0 / dt))
    scene = {"circles": [(0.5, 0.75, 0.15)], "notches": [(0.475, 0.525, 0.55, 0.85)]}
    return Workload(f"zalesak_n{n}", n, dx, scene, f, dt, steps, {"circle": (0.5, 0.75, 0.15)})


def stagnation_workload(n=8, pad=None, D=0.2, dt=1.0 / 64, T=1.0):
    """Stagnation flow (Sec. 3.1): a film of thickness D between two parallel
    lines at 45 degrees, x + y = 1 -/+ D/sqrt(2), in the unit square of n x n
    cells, drained by (u, v) = (0.5 - y, 0.5 - x) about the stagnation point
    (0.5, 0.5); dt = 1/64 (CFL 0.0625 at n = 8) up to t = T.

    The flow leaves and enters the window through its sides, so the grid
    extends the window by `pad` cells on every side (default 2n): the grid
    origin is at (-pad dx, -pad dx), and the scene and field are given in
    grid coordinates.  The film is the band between the two half-planes
    (each toggles the phase)."""
    pad = 2 * n if pad is None else int(pad)
    N = n + 2 * pad
    dx = 1.0 / n
    off = pad * dx
    h = D / math.sqrt(2.0)
    lines = [(1.0, 1.0, 1.0 + h + 2.0 * off), (1.0, 1.0, 1.0 - h + 2.0 * off)]
    f = linear_field(N, N, dx, a=(0.5 + off, 0.0, -1.0), b=(0.5 + off, -1.0, 0.0))
    steps = int(round(T / dt))
    return Workload(f"stagnation_n{n}_pad{pad}", N, dx, {"lines": lines}, f, dt, steps,
                    {"window": (pad, n), "offset": off, "D": D, "c": (1.0 - h, 1.0 + h)})


ROT_CENTRE = (0.4841, 0.5477)


def rotation_disks_workload(n=1024, count=4096, seed=230900338, cfl=0.5, steps=500,
                            rmin_cells=2.0, rmax_cells=20.0):
    """Disks of radius U[2,20] cells placed by seeded rejection inside
    |c - c'| + r <= 0.45, moved by solid rotation (omega = 2 pi) about
    c' = (0.4841, 0.5477), i.e. u = -2 pi (y - 0.5) + 0.3, v = 2 pi (x - 0.5) + 0.1."""
    dx = 1.0 / n
    rng = Rng(seed)
    cx, cy = ROT_CENTRE

    def region(x, y, r):
        return math.hypot(x - cx, y - cy) + r <= 0.45

    circles = place_circles(rng, count, rmin_cells * dx, rmax_cells * dx, 2.0 * dx, region)
    f = rotation_field(n, n, dx, 2.0 * math.pi, (0.5, 0.5), (0.3, 0.1))
    dt = cfl * dx / f.umax
    return Workload(f"rotation_disks_n{n}", n, dx, circle_scene(circles), f, dt, steps,
                    {"attempted": count, "placed": int(circles.shape[0])})


def cellular_curve_workload(n=4096, count=20000, seed=230900339, cfl=0.5, steps=2000,
                            rmin_cells=3.0, rmax_cells=12.0):
    """Fourier-perturbed interface y = 0.5 + sum_k (0.01/k^2) cos(2 pi k x + phi_k)
    plus seeded circles of radius U[3,12] cells (gap >= 2 cells to each other,
    to the curve and to the walls), in the steady cellular flow, dt = 0.5 dx."""
    dx = 1.0 / n
    rng = Rng(seed)
    curve = fourier_curve(rng)
    circles = place_circles(rng, count, rmin_cells * dx, rmax_cells * dx, 2.0 * dx,
                            lambda x, y, r: True, curve=curve)
    f = cellular_field(n, n, dx)
    dt = cfl * dx / f.umax
    scene = {"circles": circles, "curve": curve}
    return Workload(f"cellular_curve_n{n}", n, dx, scene, f, dt, steps,
                    {"attempted": count, "placed": int(circles.shape[0])})


def random_instance(rng: Rng, nmin=32, nmax=512, cmin=1, cmax=64, smin=200, smax=1000,
                    cfl=0.5, rmin=0.05, rmax=0.15, rmin_cells=3.0):
    """One instance of the batched workload: side n log-uniform, 1-64 circles
    with r ~ U[0.05, 0.15] (at least 3 cells), a coin flip between the
    time-reversed vortex with T = steps * dt and the cellular flow."""
    n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
    dx = 1.0 / n
    count = rng.integer(cmin, cmax)
    steps = rng.integer(smin, smax)
    lo = max(rmin, rmin_cells * dx)
    hi = max(rmax, lo)
    circles = place_circles(rng, count, lo, hi, 2.0 * dx, lambda x, y, r: True, max_tries=50)
    dt = cfl * dx
    if rng.uniform() < 0.5:
        f = vortex_field(n, n, dx, steps * dt)
    else:
        f = cellular_field(n, n, dx)
    return Workload(f"instance_n{n}", n, dx, circle_scene(circles), f, dt, steps,
                    {"placed": int(circles.shape[0])})
