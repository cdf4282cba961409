"""GPU parity of the generalised height-function fallbacks (EBIT_CURV_GHF;
the generalised height-function method Sec. 2.5 cites) against the oracle,
through the C ABI: the same state stepped on both sides, then every kappa and
the fallback counters compared (exactly in the FP32 form, to 1e-9 relative
in the FP64 form)."""
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
from tests.test_gpu_parity import SCENES, dev  # noqa: E402


def gpu_ghf(S):
    ctx = ebit.ebit_create(S.nx, S.ny, S.dx, S.prec, flags=ebit.EBIT_CURV_GHF)
    ebit.ebit_load_state(ctx, S.K, S.Z, S.sH, S.sV, S.step_index)
    return ctx


def kappa_of(ctx, S):
    dt = torch.float64 if S.prec == 0 else torch.float32
    k = torch.empty((S.ny, S.nx), dtype=dt, device="cuda")
    ebit.ebit_curvature(ctx, k)
    return k.double().cpu().numpy()


def assert_same_kappa(g, o, prec, dx):
    nan_g, nan_o = np.isnan(g), np.isnan(o)
    assert np.array_equal(nan_g, nan_o), f"NaN pattern differs at {np.argwhere(nan_g != nan_o)[:6].tolist()}"
    a, b = g[~nan_g], o[~nan_o]
    if prec == oracle.FP32:
        bad = np.argwhere((g != o) & ~nan_g)
        assert bad.size == 0, f"kappa differs at {bad[:6].tolist()}"
    else:
        assert np.max(np.abs(a - b) * dx, initial=0.0) <= 1e-9


def packed_disks(prec, n=160, seed=5):
    dx = 1.0 / n
    rng = W.Rng(seed)
    circles = W.place_circles(rng, 300, 3 * dx, 8 * dx, 2 * dx, lambda x, y, r: True)
    f = W.rotation_field(n, n, dx, 2 * math.pi, (0.5, 0.5), (0.2, -0.1))
    return oracle.init(n, n, dx, W.circle_scene(circles), prec), f, 0.5 * dx / f.umax


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name", ["packed"] + list(SCENES))
def test_ghf_step_parity(name, prec):
    S, f, dt = packed_disks(prec) if name == "packed" else SCENES[name](prec)
    # the initial fields (computed when the state is loaded)
    ctx = gpu_ghf(S)
    try:
        C, _ = oracle.fraction(S)
        k0, n0, res0 = oracle.curvature(S, C, ghf=True)
        assert_same_kappa(kappa_of(ctx, S), k0, prec, S.dx)
        for _ in range(2):
            ebit.ebit_step(ctx, dev(f.u, prec), dev(f.v, prec), dt)
            r = oracle.step(S, f.u, f.v, dt, ghf=True)
        d = ebit.ebit_diagnostics(ctx)
        assert np.array_equal(d["counters"], r["counters"])
        assert_same_kappa(kappa_of(ctx, S), r["kappa"], prec, S.dx)
        if name == "packed":
            c = r["counters"]
            assert c[oracle.NCOUNTERS - 2] > 0 and c[oracle.NCOUNTERS - 1] > 0
    finally:
        ebit.ebit_destroy(ctx)


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 3), (33, 1), (1, 40), (64, 9), (9, 70)])
def test_ghf_tiny_grids(nx, ny):
    """Grids smaller than the 7-cell stencils: every interface cell takes a
    fallback (or none), identically on both sides."""
    dx = 1.0 / max(nx, ny)
    scene = {"circles": [(0.45 * nx * dx, 0.55 * ny * dx, 0.3 * min(nx, ny) * dx + 0.6 * dx)],
             "line": (1.0, 0.3, 0.41 * nx * dx)}
    for prec in (0, 1):
        S = oracle.init(nx, ny, dx, scene, prec)
        ctx = gpu_ghf(S)
        try:
            C, _ = oracle.fraction(S)
            k, n, res = oracle.curvature(S, C, ghf=True)
            assert_same_kappa(kappa_of(ctx, S), k, prec, dx)
        finally:
            ebit.ebit_destroy(ctx)


def test_ghf_off_leaves_standard_path_unchanged():
    S, f, dt = packed_disks(0)
    a = ebit.ebit_create(S.nx, S.ny, S.dx, 0)
    b = gpu_ghf(S)
    try:
        ebit.ebit_load_state(a, S.K, S.Z, S.sH, S.sV, S.step_index)
        ka, kb = kappa_of(a, S), kappa_of(b, S)
        std = ~np.isnan(ka)
        assert np.array_equal(ka[std], kb[std])
        assert (np.isnan(ka) & ~np.isnan(kb)).sum() > 0
        assert ebit.ebit_diagnostics(a)["counters"][ebit.D_HF_OTHER:ebit.D_HF_MARKERS + 1].sum() == 0
    finally:
        ebit.ebit_destroy(a)
        ebit.ebit_destroy(b)


@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP64], ids=["fp32", "fp64"])
def test_ghf_full_size_cellular_curve(prec):
    """4096^2 Fourier curve with 20000 circles, one step with the fallbacks:
    every kappa and counter compared."""
    wl = W.cellular_curve_workload()
    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, prec)
    ctx = gpu_ghf(S)
    try:
        ebit.ebit_step(ctx, dev(wl.field.u, prec), dev(wl.field.v, prec), wl.dt)
        r = oracle.step(S, wl.field.u, wl.field.v, wl.dt, ghf=True)
        d = ebit.ebit_diagnostics(ctx)
        assert np.array_equal(d["counters"], r["counters"])
        assert_same_kappa(kappa_of(ctx, S), r["kappa"], prec, wl.dx)
    finally:
        ebit.ebit_destroy(ctx)


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32], ids=["fp64", "fp32"])
def test_ghf_with_straight_line_fit(prec):
    """The two flags together (EBIT-SL markers, generalised curvature)."""
    S, f, dt = packed_disks(prec, n=96, seed=11)
    ctx = ebit.ebit_create(S.nx, S.ny, S.dx, S.prec, flags=ebit.EBIT_CURV_GHF | ebit.EBIT_FIT_LINE)
    try:
        ebit.ebit_load_state(ctx, S.K, S.Z, S.sH, S.sV, S.step_index)
        for _ in range(3):
            ebit.ebit_step(ctx, dev(f.u, prec), dev(f.v, prec), dt)
            r = oracle.step(S, f.u, f.v, dt, line_only=True, ghf=True)
        d = ebit.ebit_diagnostics(ctx)
        assert np.array_equal(d["counters"], r["counters"])
        assert d["counters"][ebit.D_FIT_LINE] > 0 and d["counters"][ebit.D_FIT_TWO] == 0
        assert_same_kappa(kappa_of(ctx, S), r["kappa"], prec, S.dx)
    finally:
        ebit.ebit_destroy(ctx)
