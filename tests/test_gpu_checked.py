"""The debug build (libebit_check.so, compiled with EBIT_CHECK) on the parity
scenes and a served mix: the step kernels check every global index against its array (the
bounds checking a sanitizer would do, done by the build itself), no index
falls outside, and the results still equal the oracle's."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np
import oracle
from paper_2309_00338_gb300 import ebit, workloads as W
from tests.test_gpu_parity import SCENES, dev, gpu_from, assert_same_state, assert_same_fields
from tests.test_gpu_ghf import packed_disks, gpu_ghf, kappa_of, assert_same_kappa

assert "check" in ebit.lib()._name
for name, make in SCENES.items():
    for prec in (0, 1):
        S, f, dt = make(prec)
        ctx = gpu_from(S)
        for k in range(2):
            ebit.ebit_step(ctx, dev(f.u, prec), dev(f.v, prec), dt)
            r = oracle.step(S, f.u, f.v, dt)
        assert_same_state(ebit.ebit_get_state(ctx, S.nx, S.ny), S, prec)
        assert_same_fields(ctx, S, r, prec)
        ebit.ebit_destroy(ctx)
for nx, ny in ((1, 1), (2, 3), (33, 1), (1, 40), (64, 9), (97, 31)):
    dx = 1.0 / max(nx, ny)
    scene = {"line": (1.0, 0.3, 0.41 * nx * dx), "circles": [(0.5 * nx * dx, 0.5 * ny * dx, 0.3 * min(nx, ny) * dx + dx)]}
    for prec in (0, 1):
        S = oracle.init(nx, ny, dx, scene, prec)
        ctx = gpu_ghf(S)
        f = W.linear_field(nx, ny, dx, a=(0.2, 0.1, -0.1), b=(-0.1, 0.05, 0.1))
        for k in range(2):
            ebit.ebit_step(ctx, dev(f.u, prec), dev(f.v, prec), 0.9 * dx / 0.4)
            r = oracle.step(S, f.u, f.v, 0.9 * dx / 0.4, ghf=True)
        assert_same_kappa(kappa_of(ctx, S), r["kappa"], prec, dx)
        ebit.ebit_destroy(ctx)
S, f, dt = packed_disks(1)
ctx = gpu_ghf(S)
ebit.ebit_step(ctx, dev(f.u, 1), dev(f.v, 1), dt)
r = oracle.step(S, f.u, f.v, dt, ghf=True)
assert_same_kappa(kappa_of(ctx, S), r["kappa"], 1, S.dx)
ebit.ebit_destroy(ctx)

from tests.test_gpu_server import _mix, _run
specs = _mix()[:4]
specs[1]["flags"] = ebit.EBIT_CURV_GHF
res, outs, stats = _run(specs, 8 << 30)
assert all(r["status"] == 0 for r in res)
assert ebit.ebit_check_status() == 0, "an index fell outside its array"
print("checked ok")
'''


def test_checked_build_on_parity_scenes():
    from paper_2309_00338_gb300 import build
    path = build.build_library(checked=True)
    env = dict(os.environ, EBIT_LIB=path)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "checked ok" in r.stdout


def test_release_build_reports_no_checks():
    from paper_2309_00338_gb300 import ebit
    assert ebit.ebit_check_status() == 0
