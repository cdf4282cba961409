"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Both sides start from the same loaded state and take their decisions in the
same precision, so colour vertices, marker presence and all counters must be
bit-exact and the FP64 form must agree to 1e-12 (the tolerance the FP64 path
is held to); the FP32 form stores floats computed by the same sequence of
operations and must agree exactly.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2309_00338_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2309_00338_gb300 import ebit  # noqa: E402

TOL64 = 1e-12
COMPARED = [oracle.CANCELLED, oracle.ZSET, oracle.ZCONFLICT, oracle.FIT_ONLINE, oracle.FIT_LINE,
            oracle.FIT_ONE, oracle.FIT_TWO, oracle.WALL_CLAMP, oracle.INVARIANT, oracle.CFL]


def dev(a, prec):
    return torch.from_numpy(np.ascontiguousarray(a, np.float64 if prec == 0 else np.float32)).cuda()


def gpu_from(S):
    ctx = ebit.ebit_create(S.nx, S.ny, S.dx, S.prec)
    ebit.ebit_load_state(ctx, S.K, S.Z, S.sH, S.sV, S.step_index)
    return ctx


def assert_same_state(g, S, prec):
    assert np.array_equal(g["K"], S.K), f"corner colours differ at {np.argwhere(g['K'] != S.K)[:8]}"
    four = S.four
    assert np.array_equal(g["Z"][four], S.Z[four]), "centre colours of four-marker cells differ"
    for name, mask in (("sH", S.hasH), ("sV", S.hasV)):
        a, b = g[name][mask], getattr(S, name)[mask]
        if prec == oracle.FP32:
            assert np.array_equal(a, b), f"{name}: {np.max(np.abs(a - b))}"
        else:
            assert np.max(np.abs(a - b), initial=0.0) <= TOL64, f"{name}: {np.max(np.abs(a - b))}"


def assert_same_fields(ctx, S, r, prec):
    n = S.nx * S.ny
    dt = torch.float64 if prec == 0 else torch.float32
    C = torch.empty((S.ny, S.nx), dtype=dt, device="cuda")
    kap = torch.empty((S.ny, S.nx), dtype=dt, device="cuda")
    area = ebit.ebit_fraction(ctx, C)
    ninv = ebit.ebit_curvature(ctx, kap)
    C = C.double().cpu().numpy()
    kap = kap.double().cpu().numpy()
    if prec == oracle.FP32:
        assert np.array_equal(C, r["C"])
    else:
        assert np.max(np.abs(C - r["C"])) <= TOL64
    assert abs(area - r["area"]) <= TOL64 * max(1.0, abs(r["area"]))
    nan_g, nan_o = np.isnan(kap), np.isnan(r["kappa"])
    assert np.array_equal(nan_g, nan_o)
    d = np.abs(kap[~nan_g] - r["kappa"][~nan_o]) * S.dx
    if prec == oracle.FP32:
        assert np.array_equal(kap[~nan_g], r["kappa"][~nan_o])
    else:
        assert np.max(d, initial=0.0) <= TOL64
    assert ninv == r["counters"][oracle.HF_INVALID]
    assert n > 0


# ---------------------------------------------------------------------------
# scenes: (nx, ny, dx, scene, field) -- ragged sizes spanning several tiles
# ---------------------------------------------------------------------------
def scene_disks(prec):
    nx, ny = 97, 83
    dx = 1.0 / 97
    rng = W.Rng(41)
    circles = W.place_circles(rng, 40, 2 * dx, 9 * dx, 2 * dx, lambda x, y, r: y + r < ny * dx)
    f = W.rotation_field(nx, ny, dx, 2 * math.pi, (0.5, 0.43), (0.3, 0.1))
    dt = 0.5 * dx / f.umax
    return oracle.init(nx, ny, dx, W.circle_scene(circles), prec), f, dt


def scene_curve(prec):
    nx, ny = 130, 70
    dx = 1.0 / 130
    rng = W.Rng(7)
    curve = W.fourier_curve(rng, y0=0.27, amp0=0.02)
    circles = W.place_circles(rng, 30, 2 * dx, 7 * dx, 2 * dx, lambda x, y, r: y + r < ny * dx - 2 * dx,
                              curve=curve)
    f = W.cellular_field(nx, ny, dx)
    return oracle.init(nx, ny, dx, {"circles": circles, "curve": curve}, prec), f, 0.7 * dx


def scene_vortex(prec):
    n = 64
    wl = W.vortex_workload(n, period=2.0, cfl=0.5)
    S = oracle.init(n, n, wl.dx, wl.scene, prec)
    for k in range(90):   # a stretched, strongly curved interface
        oracle.step(S, wl.field.u, wl.field.v, wl.field.dt_eff(k, wl.dt))
    return S, wl.field, wl.dt


def scene_saddle(prec):
    """Two drops approaching along the diagonal until a saddle cell forms."""
    n = 40
    dx = 1.0 / n
    d = 0.5 / math.sqrt(2) * 0.62
    S = oracle.init(n, n, dx, W.circle_scene([(0.5 - d, 0.5 - d, 0.12), (0.5 + d, 0.5 + d, 0.12)]), prec)
    X, Y = np.meshgrid(np.arange(n + 1) * dx, np.arange(n + 1) * dx)
    s = np.sign((X - 0.5) + (Y - 0.5))
    f = W.Field("converge", -0.5 * s, -0.5 * s, 0.0, "steady", 0.5)
    dt = 0.2 * dx / 0.5
    for k in range(400):
        oracle.step(S, f.u, f.v, dt)
        if S.four.any():
            break
    assert S.four.any()
    return S, f, dt


def scene_packed(prec):
    """Disks of radius about 2 cells on a 5.2-cell lattice, rotating: more
    crossing candidates than a tile's list holds (255) in most tiles, so the
    edges beyond it take the in-place path of the sweep."""
    nx, ny = 130, 70
    dx = 1.0 / 130
    rng = W.Rng(43)
    circles = []
    L = 5.2
    for a in range(int(nx / L)):
        for b in range(int(ny / L)):
            x = (a + 0.5) * L + (rng.uniform() - 0.5) * 0.8
            y = (b + 0.5) * L + (rng.uniform() - 0.5) * 0.8
            circles.append((x * dx, y * dx, (1.9 + 0.4 * rng.uniform()) * dx))
    f = W.rotation_field(nx, ny, dx, 2 * math.pi, (0.5, 0.27), (0.3, 0.1))
    dt = 0.5 * dx / f.umax
    return oracle.init(nx, ny, dx, W.circle_scene(circles), prec), f, dt


SCENES = {"disks": scene_disks, "curve": scene_curve, "vortex": scene_vortex, "saddle": scene_saddle,
          "packed": scene_packed}


def test_packed_scene_overflows_the_candidate_list():
    """Every new unaligned marker of an x sweep comes from a crossing
    candidate of the tile that owns its edge (64 x 32 edges), so a tile that
    owns more than 255 of them had more candidates than its list holds."""
    S, f, dt = scene_packed(oracle.FP32)
    oracle.sweep(S, 0, f.u, dt / S.dx)
    per_tile = [int(S.hasV[32 * ty:32 * ty + 32, 64 * tx:64 * tx + 64].sum())
                for ty in range((S.ny + 31) // 32) for tx in range((S.nx + 1 + 63) // 64)]
    assert sum(c > 255 for c in per_tile) >= 4, per_tile


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("axis", [0, 1])
def test_sweep_parity(name, prec, axis):
    S, f, dt = SCENES[name](prec)
    ctx = gpu_from(S)
    try:
        vel = f.u if axis == 0 else f.v
        ebit.ebit_sweep(ctx, axis, dev(vel, prec), dt)
        d = ebit.ebit_diagnostics(ctx)
        ctr, _ = oracle.sweep(S, axis, vel, dt / S.dx)
        g = ebit.ebit_get_state(ctx, S.nx, S.ny)
        assert_same_state(g, S, prec)
        assert np.array_equal(d["counters"][COMPARED], ctr[COMPARED]), (d["counters"][:13], ctr[:13])
    finally:
        ebit.ebit_destroy(ctx)


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name", list(SCENES))
def test_step_parity(name, prec):
    S, f, dt = SCENES[name](prec)
    ctx = gpu_from(S)
    try:
        u, v = dev(f.u, prec), dev(f.v, prec)
        for k in range(2):  # both split orders
            ebit.ebit_step(ctx, u, v, dt)
            r = oracle.step(S, f.u, f.v, dt)
            d = ebit.ebit_diagnostics(ctx)
            assert np.array_equal(d["counters"][:13], r["counters"][:13]), (d["counters"][:13], r["counters"][:13])
            assert d["max_cfl"] == pytest.approx(r["max_cfl"], rel=1e-6)
            g = ebit.ebit_get_state(ctx, S.nx, S.ny)
            assert g["step_index"] == S.step_index
            assert_same_state(g, S, prec)
            assert_same_fields(ctx, S, r, prec)
    finally:
        ebit.ebit_destroy(ctx)


def test_vortex_64_fp64_trajectory():
    """The plain FP64 64x64 vortex workload (256 steps, CFL 0.5, alternating
    split order): GPU and oracle stay identical along the whole trajectory."""
    wl = W.vortex_workload(64, period=2.0, cfl=0.5)
    S = oracle.init(64, 64, wl.dx, wl.scene)
    ctx = ebit.ebit_init(64, 64, wl.dx, wl.scene)
    try:
        g = ebit.ebit_get_state(ctx, 64, 64)
        assert_same_state(g, S, 0)
        u, v = dev(wl.field.u, 0), dev(wl.field.v, 0)
        _, A0 = oracle.fraction(S)
        for k in range(wl.steps):
            dt = wl.field.dt_eff(k, wl.dt)
            ebit.ebit_step(ctx, u, v, dt)
            r = oracle.step(S, wl.field.u, wl.field.v, dt)
            if k % 32 == 31:
                assert_same_state(ebit.ebit_get_state(ctx, 64, 64), S, 0)
                assert_same_fields(ctx, S, r, 0)
        ebit.ebit_sync(ctx)
        area = ebit.ebit_fraction(ctx)
        assert abs(area - r["area"]) <= 1e-12
        e_area = abs(area - A0) / A0
        assert e_area < 5e-2
    finally:
        ebit.ebit_destroy(ctx)


def test_init_parity_circles_bit_exact():
    rng = W.Rng(13)
    nx, ny = 150, 110
    dx = 1.0 / 150
    circles = W.place_circles(rng, 60, 2 * dx, 12 * dx, 2 * dx, lambda x, y, r: y + r < ny * dx)
    scene = {"circles": circles, "line": (0.2, 1.0, 0.66)}
    for prec in (0, 1):
        S = oracle.init(nx, ny, dx, scene, prec)
        ctx = ebit.ebit_init(nx, ny, dx, scene, prec)
        try:
            g = ebit.ebit_get_state(ctx, nx, ny)
            assert np.array_equal(g["Z"], S.Z)
            assert_same_state(g, S, 1)  # exact, in both forms
        finally:
            ebit.ebit_destroy(ctx)


def test_init_parity_curve():
    """The Fourier curve uses cos on both sides (1-2 ulp apart): colours match
    except at vertices within 1e-12 of the curve, fractions to 1e-11."""
    rng = W.Rng(17)
    n = 256
    dx = 1.0 / n
    curve = W.fourier_curve(rng)
    S = oracle.init(n, n, dx, {"curve": curve})
    ctx = ebit.ebit_init(n, n, dx, {"curve": curve})
    try:
        g = ebit.ebit_get_state(ctx, n, n)
        X, Y = np.meshgrid(np.arange(n + 1) * dx, np.arange(n + 1) * dx)
        near = np.abs(Y - W.curve_height(curve, X)) < 1e-12
        assert np.array_equal(g["K"][~near], S.K[~near])
        if not near.any():
            for name, mask in (("sH", S.hasH), ("sV", S.hasV)):
                assert np.max(np.abs(g[name][mask] - getattr(S, name)[mask])) < 1e-11
    finally:
        ebit.ebit_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_full_size_rotating_disks_step(prec):
    """1024^2 rotating disks (the workload's own size and launch shape), one
    step from the same state, every output compared."""
    wl = W.rotation_disks_workload()
    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, prec)
    ctx = ebit.ebit_init(wl.n, wl.n, wl.dx, wl.scene, prec)
    try:
        assert_same_state(ebit.ebit_get_state(ctx, wl.n, wl.n), S, 1)
        ebit.ebit_step(ctx, dev(wl.field.u, prec), dev(wl.field.v, prec), wl.dt)
        r = oracle.step(S, wl.field.u, wl.field.v, wl.dt)
        d = ebit.ebit_diagnostics(ctx)
        assert np.array_equal(d["counters"][:13], r["counters"][:13])
        assert_same_state(ebit.ebit_get_state(ctx, wl.n, wl.n), S, prec)
        assert_same_fields(ctx, S, r, prec)
    finally:
        ebit.ebit_destroy(ctx)


def test_full_size_cellular_curve_fp32_step():
    """4096^2 cellular flow with the Fourier curve and 20000 circles in the
    FP32 form: one step from the same loaded state, every output compared."""
    wl = W.cellular_curve_workload()
    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, oracle.FP32)
    ctx = gpu_from(S)
    try:
        ebit.ebit_step(ctx, dev(wl.field.u, 1), dev(wl.field.v, 1), wl.dt)
        r = oracle.step(S, wl.field.u, wl.field.v, wl.dt)
        d = ebit.ebit_diagnostics(ctx)
        assert np.array_equal(d["counters"][:13], r["counters"][:13])
        assert_same_state(ebit.ebit_get_state(ctx, wl.n, wl.n), S, 1)
        assert_same_fields(ctx, S, r, 1)
    finally:
        ebit.ebit_destroy(ctx)


def test_full_size_cellular_curve_fp64_step():
    """The same 4096^2 workload in the plain FP64 form, one step, every output
    compared at 1e-12."""
    wl = W.cellular_curve_workload()
    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, oracle.FP64)
    ctx = gpu_from(S)
    try:
        ebit.ebit_step(ctx, dev(wl.field.u, 0), dev(wl.field.v, 0), wl.dt)
        r = oracle.step(S, wl.field.u, wl.field.v, wl.dt)
        d = ebit.ebit_diagnostics(ctx)
        assert np.array_equal(d["counters"][:13], r["counters"][:13])
        assert_same_state(ebit.ebit_get_state(ctx, wl.n, wl.n), S, 0)
        assert_same_fields(ctx, S, r, 0)
    finally:
        ebit.ebit_destroy(ctx)


def _merging_workload(n):
    """Workloads whose disks merge and break: at 4096^2 the benchmark's
    cellular flow with the Fourier curve and 20000 disks (gap 2 cells), which
    shears disks into each other and into the curve (pairs of markers cancel
    along grid lines; saddle cells do not form there); at 1024^2, 1250 disks
    of 3-12 cells in the single vortex of period 8, which stretches them into
    filaments that also meet along diagonals, so the centre rule sets new
    saddle colours as well (Sec. 2.3-2.4)."""
    if n == 4096:
        return W.cellular_curve_workload()
    dx = 1.0 / n
    circles = W.place_circles(W.Rng(230900343), 1250, 3 * dx, 12 * dx, 2 * dx, lambda x, y, r: True)
    f = W.vortex_field(n, n, dx, 8.0)
    return W.Workload(f"vortex_disks_n{n}", n, dx, W.circle_scene(circles), f, 0.5 * dx / f.umax, 0)


@pytest.mark.parametrize("n,prec,steps", [(4096, 1, 1000), (1024, 0, 500), (1024, 1, 500)],
                         ids=["4096_fp32_1000", "1024_fp64_500", "1024_fp32_500"])
def test_step_after_topology_changes(n, prec, steps):
    """One step compared from the GPU's own state after `steps` steps, well
    past the first merges and break-ups: the state the GPU reached is loaded
    into the oracle, both take the next step, and every output is compared
    (the kept markers' positions, colours, counters, C and kappa)."""
    wl = _merging_workload(n)
    ctx = ebit.ebit_init(wl.n, wl.n, wl.dx, wl.scene, prec)
    try:
        u, v = dev(wl.field.u, prec), dev(wl.field.v, prec)
        seen = np.zeros(16, np.int64)
        for k in range(steps):
            ebit.ebit_step(ctx, u, v, wl.dt)
            seen += ebit.ebit_diagnostics(ctx)["counters"]
        assert seen[oracle.CANCELLED] > 0
        if n == 1024:
            assert seen[oracle.ZSET] > 0
        assert seen[oracle.INVARIANT] == 0 and seen[oracle.CFL] == 0
        g = ebit.ebit_get_state(ctx, wl.n, wl.n)
        S = oracle.State(wl.n, wl.n, wl.dx, prec)
        S.K[...], S.Z[...], S.sH[...], S.sV[...] = g["K"], g["Z"], g["sH"], g["sV"]
        S.step_index = g["step_index"]
        assert S.step_index == steps
        ebit.ebit_step(ctx, u, v, wl.dt)
        r = oracle.step(S, wl.field.u, wl.field.v, wl.dt)
        d = ebit.ebit_diagnostics(ctx)
        assert np.array_equal(d["counters"][:13], r["counters"][:13]), (d["counters"][:13], r["counters"][:13])
        assert_same_state(ebit.ebit_get_state(ctx, wl.n, wl.n), S, prec)
        assert_same_fields(ctx, S, r, prec)
    finally:
        ebit.ebit_destroy(ctx)


def _fp32_error(wl, steps):
    """The FP32 form on the GPU against the plain FP64 oracle after `steps`
    steps of a workload: marker positions (cells) on edges both keep, C,
    kappa (1/cells) where both have one, and both forms' E_area."""
    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, oracle.FP64)
    _, A0 = oracle.fraction(S)
    ctx = ebit.ebit_init(wl.n, wl.n, wl.dx, wl.scene, ebit.EBIT_FP32)
    try:
        a0 = ebit.ebit_fraction(ctx)
        u, v = dev(wl.field.u, 1), dev(wl.field.v, 1)
        for k in range(steps):
            dt = wl.field.dt_eff(k, wl.dt)
            ebit.ebit_step(ctx, u, v, dt)
            r = oracle.step(S, wl.field.u, wl.field.v, dt)
        g = ebit.ebit_get_state(ctx, wl.n, wl.n)
        C = torch.empty((wl.n, wl.n), dtype=torch.float32, device="cuda")
        kap = torch.empty((wl.n, wl.n), dtype=torch.float32, device="cuda")
        a1 = ebit.ebit_fraction(ctx, C)
        ebit.ebit_curvature(ctx, kap)
        C, kap = C.double().cpu().numpy(), kap.double().cpu().numpy()
    finally:
        ebit.ebit_destroy(ctx)
    hH = S.hasH & (g["K"][:, :-1] != g["K"][:, 1:])
    hV = S.hasV & (g["K"][:-1, :] != g["K"][1:, :])
    dpos = np.concatenate([np.abs(g["sH"][hH] - S.sH[hH]), np.abs(g["sV"][hV] - S.sV[hV])])
    both = ~np.isnan(kap) & ~np.isnan(r["kappa"])
    return {"K_mismatch": int((g["K"] != S.K).sum()), "pos": dpos, "C": np.abs(C - r["C"]),
            "kappa": np.abs(kap[both] - r["kappa"][both]) * wl.dx,
            "kappa_rel": np.abs(kap[both] - r["kappa"][both]) / np.abs(r["kappa"][both]),
            "e32": abs(a1 - a0) / a0, "e64": abs(r["area"] - A0) / A0, "A64": r["area"], "A32": a1}


@pytest.mark.parametrize("name,steps", [("rotating_disks_1024", 50), ("cellular_curve_4096", 10)])
def test_fp32_form_error_against_fp64_oracle(name, steps):
    """Each output of the FP32 form against the plain FP64 oracle (the
    precision pattern: FP32 edge fractions, FP64 circle fit and area sums).
    Positions differ by the float rounding of the state and of the advection
    carried through the steps (1024^2 disks after 50 steps: median 4.7e-7
    cell, 99% below 3.5e-6, largest 3.1e-5), the fractions likewise (median
    2.4e-7 on interface cells, largest 2.3e-6), curvature by the float
    heights (median 1.4e-6 relative, 99% below 9.2e-6) and the area sum by
    7e-11 relative, so E_area is the same in both forms (7.1e-5); colours can
    differ only where a float and a double position fall on either side of
    a grid line.  Bounds: 5x those figures."""
    wl = W.rotation_disks_workload() if name.startswith("rotating") else W.cellular_curve_workload()
    e = _fp32_error(wl, steps)
    assert e["K_mismatch"] <= 1e-6 * wl.n * wl.n
    assert np.median(e["pos"]) < 2.5e-6 and np.percentile(e["pos"], 99) < 2e-5 and e["pos"].max() < 2e-4
    assert np.median(e["C"][e["C"] > 0]) < 1.5e-6 and np.percentile(e["C"], 99.99) < 1.2e-5
    assert np.median(e["kappa_rel"]) < 7e-6 and np.percentile(e["kappa_rel"], 99) < 5e-5
    assert abs(e["A32"] - e["A64"]) / e["A64"] < 5e-10
    assert abs(e["e32"] - e["e64"]) < 5e-10


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 3), (33, 1), (1, 40), (64, 9)])
def test_tiny_and_degenerate_grids(nx, ny):
    dx = 1.0 / max(nx, ny)
    scene = {"line": (1.0, 0.3, 0.41 * nx * dx)}
    for prec in (0, 1):
        S = oracle.init(nx, ny, dx, scene, prec)
        ctx = gpu_from(S)
        try:
            f = W.linear_field(nx, ny, dx, a=(0.2, 0.1, -0.1), b=(-0.1, 0.05, 0.1))
            for k in range(3):
                ebit.ebit_step(ctx, dev(f.u, prec), dev(f.v, prec), 0.9 * dx / 0.4)
                r = oracle.step(S, f.u, f.v, 0.9 * dx / 0.4)
            assert_same_state(ebit.ebit_get_state(ctx, nx, ny), S, prec)
            assert_same_fields(ctx, S, r, prec)
        finally:
            ebit.ebit_destroy(ctx)


def test_empty_and_full_domains():
    for scene, val in (({}, 0.0), ({"line": (0.0, 0.0, 1.0)}, 1.0)):
        ctx = ebit.ebit_init(50, 37, 0.02, scene)
        try:
            f = W.cellular_field(50, 37, 0.02)
            ebit.ebit_step(ctx, dev(f.u, 0), dev(f.v, 0), 0.01)
            C = torch.empty((37, 50), dtype=torch.float64, device="cuda")
            area = ebit.ebit_fraction(ctx, C)
            assert torch.all(C == val) and area == pytest.approx(val * 50 * 37 * 0.02 ** 2)
            assert ebit.ebit_curvature(ctx) == 0
            d = ebit.ebit_diagnostics(ctx)
            assert d["counters"][ebit.D_NH] == 0 and d["counters"][ebit.D_NV] == 0
        finally:
            ebit.ebit_destroy(ctx)


def test_cfl_violation_reported_and_context_survives():
    n = 32
    dx = 1.0 / n
    S = oracle.init(n, n, dx, W.circle_scene([(0.5, 0.5, 0.2)]))
    ctx = gpu_from(S)
    try:
        f = W.uniform_field(n, n, dx, 1.0, 0.5)
        ebit.ebit_step(ctx, dev(f.u, 0), dev(f.v, 0), 1.5 * dx)
        with pytest.raises(ebit.EbitError) as e:
            ebit.ebit_sync(ctx)
        assert e.value.status == ebit.EBIT_ECFL
        r = oracle.step(S, f.u, f.v, 1.5 * dx)
        assert r["status"] == 3
        ebit.ebit_sync(ctx)  # the error was reported once and cleared
        assert_same_state(ebit.ebit_get_state(ctx, n, n), S, 0)
    finally:
        ebit.ebit_destroy(ctx)


def test_fp32_form_mass_error_on_translation():
    """Stated mass-conservation error of the FP32 form: translation (Sec. 3.2)
    at 64^2; FP64 stays at roundoff, FP32 within the storage-rounding bound."""
    wl = W.translation_workload(64)
    out = {}
    for prec in (0, 1):
        ctx = ebit.ebit_init(wl.n, wl.n, wl.dx, wl.scene, prec)
        try:
            a0 = ebit.ebit_fraction(ctx)
            u, v = dev(wl.field.u, prec), dev(wl.field.v, prec)
            for k in range(wl.steps):
                ebit.ebit_step(ctx, u, v, wl.field.dt_eff(k, wl.dt))
            out[prec] = abs(ebit.ebit_fraction(ctx) - a0) / a0
        finally:
            ebit.ebit_destroy(ctx)
    assert out[0] < 1e-12
    bound = wl.steps * 2 * math.pi * 0.15 * 2.0 ** -24 * wl.dx / (math.pi * 0.15 ** 2)
    assert out[1] <= bound


# ---------------------------------------------------------------------------
# EBIT-SL mode (EBIT_FIT_LINE): the straight chord instead of the circle fit
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name", list(SCENES))
def test_step_parity_line_only(name, prec):
    S, f, dt = SCENES[name](prec)
    ctx = ebit.ebit_create(S.nx, S.ny, S.dx, S.prec, flags=ebit.EBIT_FIT_LINE)
    ebit.ebit_load_state(ctx, S.K, S.Z, S.sH, S.sV, S.step_index)
    try:
        u, v = dev(f.u, prec), dev(f.v, prec)
        for k in range(2):
            ebit.ebit_step(ctx, u, v, dt)
            r = oracle.step(S, f.u, f.v, dt, line_only=True)
            d = ebit.ebit_diagnostics(ctx)
            assert np.array_equal(d["counters"][:13], r["counters"][:13]), (d["counters"][:13], r["counters"][:13])
            assert d["counters"][oracle.FIT_ONE] == 0 and d["counters"][oracle.FIT_TWO] == 0
            assert_same_state(ebit.ebit_get_state(ctx, S.nx, S.ny), S, prec)
            assert_same_fields(ctx, S, r, prec)
    finally:
        ebit.ebit_destroy(ctx)


def test_line_only_translation_matches_table1_sl_row():
    """The whole EBIT-SL translation at 64^2 on the GPU: the area loss the
    paper prints for EBIT-SL (Table 1), and the oracle's value to 1e-12."""
    wl = W.translation_workload(64)
    ctx = ebit.ebit_init(wl.n, wl.n, wl.dx, wl.scene, flags=ebit.EBIT_FIT_LINE)
    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene)
    try:
        a0 = ebit.ebit_fraction(ctx)
        u, v = dev(wl.field.u, 0), dev(wl.field.v, 0)
        for k in range(wl.steps):
            dt = wl.field.dt_eff(k, wl.dt)
            ebit.ebit_step(ctx, u, v, dt)
            oracle.step(S, wl.field.u, wl.field.v, dt, line_only=True)
        e_gpu = abs(ebit.ebit_fraction(ctx) - a0) / a0
        _, a1 = oracle.fraction(S)
        _, a0o = oracle.fraction(oracle.init(wl.n, wl.n, wl.dx, wl.scene))
        e_orc = abs(a1 - a0o) / a0o
        assert abs(e_gpu - e_orc) <= 1e-12
        assert abs(e_gpu / 6.83e-1 - 1) < 0.05  # Table 1, EBIT-SL, N=64
        assert_same_state(ebit.ebit_get_state(ctx, wl.n, wl.n), S, 0)
    finally:
        ebit.ebit_destroy(ctx)


# ---------------------------------------------------------------------------
# Zalesak's disk (Sec. 3.4): a scene with a notch cut out of a disk
# ---------------------------------------------------------------------------
def test_init_parity_notched_disk():
    wl = W.zalesak_workload(96)
    for prec in (0, 1):
        S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, prec)
        ctx = ebit.ebit_init(wl.n, wl.n, wl.dx, wl.scene, prec)
        try:
            g = ebit.ebit_get_state(ctx, wl.n, wl.n)
            assert np.array_equal(g["Z"], S.Z)
            assert_same_state(g, S, 1)  # exact, in both forms
        finally:
            ebit.ebit_destroy(ctx)


@pytest.mark.parametrize("line_only", [False, True], ids=["circle_fit", "straight_line"])
def test_zalesak_64_turn(line_only):
    """One turn of the notched disk at 64^2 (1024 steps, FP64): the GPU state
    equals the oracle's along the way and the area error is the one Table 5
    prints (EBIT within x3, EBIT-SL within 5%)."""
    wl = W.zalesak_workload(64)
    flags = ebit.EBIT_FIT_LINE if line_only else 0
    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene)
    ctx = ebit.ebit_init(wl.n, wl.n, wl.dx, wl.scene, flags=flags)
    try:
        u, v = dev(wl.field.u, 0), dev(wl.field.v, 0)
        a0 = ebit.ebit_fraction(ctx)
        for k in range(wl.steps):
            ebit.ebit_step(ctx, u, v, wl.dt)
            r = oracle.step(S, wl.field.u, wl.field.v, wl.dt, line_only=line_only)
            if k % 256 == 255:
                assert_same_state(ebit.ebit_get_state(ctx, wl.n, wl.n), S, 0)
        ebit.ebit_sync(ctx)
        e_area = abs(ebit.ebit_fraction(ctx) - a0) / a0
        assert abs(ebit.ebit_fraction(ctx) - r["area"]) <= 1e-12
        if line_only:
            assert abs(e_area / 7.33e-1 - 1) < 0.05   # Table 5, EBIT-SL, N=64
        else:
            assert 1.22e-3 / 3 <= e_area <= 3 * 1.22e-3  # Table 5, EBIT, N=64
    finally:
        ebit.ebit_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_stagnation_film_run(prec):
    """Sec. 3.1's stagnation flow (8x8 window in a grid with 16-cell margins,
    a film between two half-planes, 64 steps of dt = 1/64): initial state,
    every 16th state, counters and the final fields equal the oracle's."""
    wl = W.stagnation_workload()
    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, prec)
    ctx = ebit.ebit_init(wl.n, wl.n, wl.dx, wl.scene, prec)
    try:
        g = ebit.ebit_get_state(ctx, wl.n, wl.n)
        assert np.array_equal(g["Z"], S.Z)
        assert_same_state(g, S, 1)
        u, v = dev(wl.field.u, prec), dev(wl.field.v, prec)
        for k in range(wl.steps):
            ebit.ebit_step(ctx, u, v, wl.dt)
            r = oracle.step(S, wl.field.u, wl.field.v, wl.dt)
            if k % 16 == 15:
                assert_same_state(ebit.ebit_get_state(ctx, wl.n, wl.n), S, prec)
                d = ebit.ebit_diagnostics(ctx)
                assert np.array_equal(d["counters"][:13], r["counters"][:13])
        assert_same_fields(ctx, S, r, prec)
        pad, n = wl.meta["window"]
        assert S.four[pad:pad + n, pad:pad + n].sum() > 0   # the sub-cell film is there
    finally:
        ebit.ebit_destroy(ctx)


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32], ids=["fp64", "fp32"])
def test_fraction_to_host_every_step(prec):
    """ebit_fraction_to_host after each of four steps, queued while the GPU
    runs ahead of the host (the first on the context's stream, the others on
    a side stream, each with a second copy on another stream): every host copy
    holds the C of its own step — the next step's fields launch waits for all
    copies still pending — and equals the oracle's."""
    S, f, dt = scene_disks(prec)
    ctx = gpu_from(S)
    side, side2 = torch.cuda.Stream(), torch.cuda.Stream()
    dtype = torch.float64 if prec == oracle.FP64 else torch.float32
    try:
        u, v = dev(f.u, prec), dev(f.v, prec)
        hosts = []
        for k in range(4):
            ebit.ebit_step(ctx, u, v, dt)
            h = torch.full((S.ny, S.nx), -1.0, dtype=dtype).pin_memory()
            ebit.ebit_fraction_to_host(ctx, h, None if k == 0 else side)
            mine = [h]
            if k > 0:  # a second copy of the same step on another stream
                h2 = torch.full((S.ny, S.nx), -1.0, dtype=dtype).pin_memory()
                ebit.ebit_fraction_to_host(ctx, h2, side2)
                mine.append(h2)
            hosts.append(mine)
        refs = [oracle.step(S, f.u, f.v, dt)["C"].copy() for _ in range(4)]
        side.synchronize()
        side2.synchronize()
        ebit.ebit_sync(ctx)
        for hs, r in zip(hosts, refs):
            for h in hs:
                c = h.double().numpy()
                if prec == oracle.FP32:
                    assert np.array_equal(c, r)
                else:
                    assert np.max(np.abs(c - r)) <= TOL64
    finally:
        ebit.ebit_destroy(ctx)


def test_area_async_matches_fraction():
    """ebit_area_async queues the area of the current state; after the stream
    reaches it the value equals ebit_fraction's, step by step."""
    S, f, dt = scene_disks(1)
    ctx = gpu_from(S)
    try:
        host = torch.zeros(3, dtype=torch.float64).pin_memory()
        u, v = dev(f.u, 1), dev(f.v, 1)
        want = []
        for k in range(3):
            ebit.ebit_step(ctx, u, v, dt)
            ebit.ebit_area_async(ctx, host[k:k + 1])
            r = oracle.step(S, f.u, f.v, dt)
            want.append(r["area"])
        ebit.ebit_sync(ctx)
        assert host.tolist() == pytest.approx(want, rel=1e-12)
        assert float(host[2]) == ebit.ebit_fraction(ctx)
        assert ebit.lib().ebit_area_async(ctx, None) == ebit.EBIT_EINVAL
    finally:
        ebit.ebit_destroy(ctx)


def test_max_size_grid_fp32():
    """The largest grid the library accepts (32768^2 cells, FP32 form, ~30 GB
    of state; every offset above 2^32 bytes): a disk of radius 0.3
    initialises to its area, keeps it over two steps of solid rotation
    (properties that hold at any size; the oracle cannot run this grid), and
    its height-function curvature is 1/r."""
    if torch.cuda.get_device_properties(0).total_memory < (80 << 30):
        pytest.skip("needs 80 GB of device memory")
    n = 32768
    dx = 1.0 / n
    r = 0.3
    ctx = ebit.ebit_init(n, n, dx, {"circles": [(0.5 + 0.37 * dx, 0.5 - 0.21 * dx, r)]}, ebit.EBIT_FP32)
    try:
        a0 = ebit.ebit_fraction(ctx)
        assert abs(a0 - math.pi * r * r) < 1e-8
        om = 2.0 * math.pi
        xs = torch.arange(n + 1, device="cuda", dtype=torch.float64) * dx - 0.5
        u = (-om * xs).to(torch.float32)[:, None].expand(n + 1, n + 1).contiguous()  # -omega (y - 0.5)
        v = (om * xs).to(torch.float32)[None, :].expand(n + 1, n + 1).contiguous()  # omega (x - 0.5)
        dt = 0.5 * dx / (0.5 * om)
        for _ in range(2):
            ebit.ebit_step(ctx, u, v, dt)
        del u, v
        a1 = ebit.ebit_fraction(ctx)
        assert abs(a1 - a0) / a0 < 1e-8
        c = ebit.ebit_diagnostics(ctx)["counters"]
        assert c[ebit.D_CFL] == 0 and c[ebit.D_INVARIANT] == 0
        assert c[ebit.D_NH] > 2 * r / dx and c[ebit.D_NV] > 2 * r / dx
        kap = torch.empty((n, n), dtype=torch.float32, device="cuda")
        ebit.ebit_curvature(ctx, kap)
        valid = kap[~torch.isnan(kap)]
        assert valid.numel() > 4 * r / dx
        assert abs(float(valid.median()) * r - 1.0) < 2e-2
        del kap, valid
    finally:
        ebit.ebit_destroy(ctx)
        torch.cuda.empty_cache()
