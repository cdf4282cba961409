"""GPU parity of ebit_coupling (Sec. 2.5: the properties of Eq. 8 and the
face surface-tension source of Eq. 6) against the oracle, through the C ABI.

The oracle evaluates the definitions in double on the GPU's C and kappa; the
library computes them in the context precision (with sigma/dx formed once),
so the outputs agree to the rounding of that arithmetic: a few units in the
last place of float in the FP32 form (16 * 2^-24 of the size of the terms),
1e-12 relative in the FP64 form."""
import numpy as np
import pytest

import oracle
from paper_2309_00338_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2309_00338_gb300 import ebit  # noqa: E402
from tests.test_gpu_parity import SCENES, dev, gpu_from  # noqa: E402

FL = dict(rho1=1000.0, rho2=1.2, mu1=1.0e-3, mu2=1.8e-5, sigma=0.0728)


def gpu_coupling(ctx, S, fl=FL):
    dt = torch.float64 if S.prec == 0 else torch.float32
    out = {"rho": torch.empty((S.ny, S.nx), dtype=dt, device="cuda"),
           "mu": torch.empty((S.ny, S.nx), dtype=dt, device="cuda"),
           "fx": torch.empty((S.ny, S.nx + 1), dtype=dt, device="cuda"),
           "fy": torch.empty((S.ny + 1, S.nx), dtype=dt, device="cuda")}
    ebit.ebit_coupling(ctx, fl["rho1"], fl["rho2"], fl["mu1"], fl["mu2"], fl["sigma"], **out)
    torch.cuda.synchronize()
    return {k: v.double().cpu().numpy() for k, v in out.items()}


def gpu_fields(ctx, S):
    dt = torch.float64 if S.prec == 0 else torch.float32
    C = torch.empty((S.ny, S.nx), dtype=dt, device="cuda")
    kap = torch.empty((S.ny, S.nx), dtype=dt, device="cuda")
    ebit.ebit_fraction(ctx, C)
    ebit.ebit_curvature(ctx, kap)
    return C.double().cpu().numpy(), kap.double().cpu().numpy()


def assert_close(g, o, C, kap, prec, dx, fl=FL):
    """Outputs g of the library against the oracle's o, computed from the
    fields C and kap: each within eps times the size of the terms that form
    it (eps = 16 * 2^-24 for float, 1e-12 for double)."""
    eps = 16 * 2.0 ** -24 if prec == oracle.FP32 else 1e-12
    Ca = np.abs(C)
    scale = {"rho": Ca * abs(fl["rho1"]) + np.abs(1 - C) * abs(fl["rho2"]),
             "mu": Ca * abs(fl["mu1"]) + np.abs(1 - C) * abs(fl["mu2"])}
    ka = np.where(np.isnan(kap), 0.0, np.abs(kap))
    sg = abs(fl["sigma"]) / dx
    fx = np.zeros((C.shape[0], C.shape[1] + 1))
    fx[:, 1:-1] = sg * np.maximum(ka[:, :-1], ka[:, 1:]) * np.maximum(Ca[:, :-1], Ca[:, 1:])
    fy = np.zeros((C.shape[0] + 1, C.shape[1]))
    fy[1:-1, :] = sg * np.maximum(ka[:-1, :], ka[1:, :]) * np.maximum(Ca[:-1, :], Ca[1:, :])
    scale["fx"], scale["fy"] = fx, fy
    for name, ref in zip(("rho", "mu", "fx", "fy"), o):
        assert g[name].shape == ref.shape, name
        bad = np.argwhere(~(np.abs(g[name] - ref) <= eps * scale[name]))
        assert bad.size == 0, f"{name} differs at {bad[:6].tolist()}"


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name", list(SCENES))
def test_coupling_parity_after_step(name, prec):
    S, f, dt = SCENES[name](prec)
    ctx = gpu_from(S)
    try:
        ebit.ebit_step(ctx, dev(f.u, prec), dev(f.v, prec), dt)
        r = oracle.step(S, f.u, f.v, dt)
        g = gpu_coupling(ctx, S)
        C, kap = gpu_fields(ctx, S)
        assert_close(g, oracle.coupling(S, C, kap, **FL), C, kap, prec, S.dx)
        # against the oracle's own chain: in FP32 the fields are bit-exact,
        # so the same bound holds; in FP64 the fields agree to 1e-12 cells
        # and so do these
        o = oracle.coupling(S, r["C"], r["kappa"], **FL)
        if prec == oracle.FP32:
            assert_close(g, o, r["C"], r["kappa"], prec, S.dx)
        else:
            sc = FL["sigma"] / S.dx ** 2
            for name_, ref in zip(("rho", "mu", "fx", "fy"), o):
                scale = {"rho": FL["rho1"], "mu": FL["mu1"]}.get(name_, sc)
                assert np.max(np.abs(g[name_] - ref)) <= 1e-11 * scale, name_
    finally:
        ebit.ebit_destroy(ctx)


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 3), (33, 1), (1, 40), (129, 17), (130, 33), (255, 16)])
def test_coupling_ragged_grids(nx, ny):
    """Sizes around the 128-column and 16-row blocks, and single rows or
    columns where every face is a wall."""
    dx = 1.0 / max(nx, ny)
    c = (0.41 * nx * dx, 0.53 * ny * dx, 0.3 * min(nx, ny) * dx)
    for prec in (0, 1):
        S = oracle.init(nx, ny, dx, {"circles": [c], "line": (1.0, 0.3, 0.37 * nx * dx)}, prec)
        ctx = gpu_from(S)
        try:
            g = gpu_coupling(ctx, S)
            C, kap = gpu_fields(ctx, S)
            assert_close(g, oracle.coupling(S, C, kap, **FL), C, kap, prec, S.dx)
        finally:
            ebit.ebit_destroy(ctx)


def test_coupling_null_outputs_untouched():
    n = 70
    S = oracle.init(n, n, 1.0 / n, W.circle_scene([(0.5, 0.5, 0.2)]), 0)
    ctx = gpu_from(S)
    try:
        fx = torch.full((n, n + 1), 7.0, dtype=torch.float64, device="cuda")
        rho = torch.full((n, n), 7.0, dtype=torch.float64, device="cuda")
        ebit.ebit_coupling(ctx, FL["rho1"], FL["rho2"], FL["mu1"], FL["mu2"], FL["sigma"], fx=fx)
        torch.cuda.synchronize()
        assert torch.all(rho == 7.0)
        C, kap = gpu_fields(ctx, S)
        o = oracle.coupling(S, C, kap, **FL)
        g = {"rho": o[0], "mu": o[1], "fx": fx.cpu().numpy(), "fy": o[3]}
        assert_close(g, o, C, kap, oracle.FP64, S.dx)
        assert ebit.lib().ebit_coupling(ctx, None, None, None, None, None) == ebit.EBIT_EINVAL
        assert ebit.lib().ebit_coupling(None, ebit.ebit_fluids(1, 1, 1, 1, 1), None, None, None,
                                        None) == ebit.EBIT_EINVAL
    finally:
        ebit.ebit_destroy(ctx)


@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP64], ids=["fp32", "fp64"])
def test_coupling_full_size_cellular_curve(prec):
    """4096^2 Fourier curve with 20000 circles: the launch shapes the
    benchmark times (the column-pair float kernel, the queued double kernel),
    every output compared."""
    wl = W.cellular_curve_workload()
    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, prec)
    ctx = gpu_from(S)
    try:
        g = gpu_coupling(ctx, S)
        C, kap = gpu_fields(ctx, S)
        assert_close(g, oracle.coupling(S, C, kap, **FL), C, kap, prec, S.dx)
        # the Laplace balance holds on the GPU output too: from the cell that
        # holds a circle's leftmost point to its centre, along the centre's
        # row, the face forces integrate to a pressure jump of sigma / r
        # (positive for drops above the curve and bubbles below it alike).
        # Circles within three cells of another interface may have no valid
        # 7x3 stencil there (no force); only those with one are checked.
        errs = []
        for xc, yc, r in np.asarray(wl.scene["circles"]):
            j = int(yc / wl.dx)
            i0, i1 = int((xc - r) / wl.dx), int(xc / wl.dx)
            if r < 10 * wl.dx or not np.isfinite(kap[j, i0]):
                continue
            errs.append(g["fx"][j, i0:i1 + 1].sum() * wl.dx / (FL["sigma"] / r) - 1.0)
        errs = np.abs(errs)
        assert errs.size > 1000
        assert np.median(errs) < 1e-2 and np.mean(errs < 5e-2) > 0.85
    finally:
        ebit.ebit_destroy(ctx)
