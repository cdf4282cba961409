"""ebit_fraction_noalloc, the volume-fraction entry point for callers that
cannot allocate device memory (a solver that allocates everything at start-up
and forbids allocation in its time loop, or a host framework that owns all
device buffers).  Its output must equal that of the allocating entry point
ebit_fraction on the same state, on two calls in a row (the second call reuses
the library's scratch array as the first left it).

This file is collected last so that a run stopping at its first failure has
run every other test before it."""
import numpy as np
import pytest

import oracle
from paper_2309_00338_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2309_00338_gb300 import ebit  # noqa: E402


def _states(prec):
    n = 96
    dx = 1.0 / n
    rng = W.Rng(77)
    circles = W.place_circles(rng, 25, 2 * dx, 9 * dx, 2 * dx, lambda x, y, r: True)
    S = oracle.init(n, n, dx, W.circle_scene(circles), prec)
    first = S.copy()
    f = W.vortex_field(n, n, dx, 2.0)
    for k in range(20):
        oracle.step(S, f.u, f.v, 0.5 * dx)
    return [first, S]   # two different states for the two calls


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_noalloc_matches_allocating_fraction_twice(prec):
    dt = torch.float64 if prec == 0 else torch.float32
    for S in _states(prec):
        nx, ny = S.nx, S.ny
        # the allocating path
        ctx = ebit.ebit_create(nx, ny, S.dx, prec)
        try:
            ebit.ebit_load_state(ctx, S.K, S.Z, S.sH, S.sV)
            C_ref = torch.empty((ny, nx), dtype=dt, device="cuda")
            area_ref = ebit.ebit_fraction(ctx, C_ref)
            d = ebit.ebit_diagnostics(ctx)
        finally:
            ebit.ebit_destroy(ctx)
        # the no-allocation path, on the caller's device buffers
        K = torch.from_numpy(S.K).cuda()
        Z = torch.from_numpy(S.Z).cuda()
        sH = torch.from_numpy(S.sH).to(dt).cuda()
        sV = torch.from_numpy(S.sV).to(dt).cuda()
        C = torch.full((ny, nx), float("nan"), dtype=dt, device="cuda")
        area = torch.zeros(1, dtype=torch.float64, device="cuda")
        counts = torch.zeros(2, dtype=torch.int64, device="cuda")
        ebit.ebit_fraction_noalloc(nx, ny, S.dx, prec, K, Z, sH, sV, C, area, counts)
        torch.cuda.synchronize()
        assert torch.equal(C, C_ref)
        assert abs(area.item() - area_ref) <= 1e-12 * max(1.0, abs(area_ref))
        assert counts.tolist() == [int(d["counters"][ebit.D_NH]), int(d["counters"][ebit.D_NV])]
        # and against the oracle's fractions (Sec. 2.5): exact in FP32, where
        # both round the same double area to float; 1e-12 in FP64; the area
        # summed in another order agrees to 1e-12
        C_orc, area_orc = oracle.fraction(S)
        if prec == 1:
            assert np.array_equal(C.double().cpu().numpy(), C_orc)
        else:
            assert np.max(np.abs(C.cpu().numpy() - C_orc)) <= 1e-12
        assert abs(area.item() - area_orc) <= 1e-12 * max(1.0, abs(area_orc))
        assert counts.tolist() == [int(S.hasH.sum()), int(S.hasV.sum())]


def test_noalloc_rejects_grids_beyond_its_scratch():
    """A grid just past the scratch's limit (5800^2 cells: 132858 blocks of
    32x8 vertices against 131072) is refused before any launch; the buffers
    are sized for that grid, so nothing could reach memory outside them."""
    n = 5800
    dt = torch.float32
    K = torch.zeros((n + 1) * (n + 1), dtype=torch.uint8, device="cuda")
    Z = torch.zeros(n * n, dtype=torch.uint8, device="cuda")
    sH = torch.zeros((n + 1) * n, dtype=dt, device="cuda")
    sV = torch.zeros(n * (n + 1), dtype=dt, device="cuda")
    C = torch.zeros(n * n, dtype=dt, device="cuda")
    area = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ebit.EbitError) as e:
        ebit.ebit_fraction_noalloc(n, n, 1.0 / n, 1, K, Z, sH, sV, C, area)
    assert e.value.status == ebit.EBIT_EINVAL and "scratch" in str(e.value)
    # the binding refuses buffers that do not match the grid
    with pytest.raises(ValueError):
        ebit.ebit_fraction_noalloc(n - 1, n, 1.0 / n, 1, K, Z, sH, sV, C, area)
    del K, Z, sH, sV, C
    torch.cuda.empty_cache()
