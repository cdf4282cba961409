"""The library from plain C: a program that includes only include/ebit.h and
the CUDA runtime header, linked against libebit.so, runs the 64² vortex case
(Sec. 3.3's scene: R = 0.15 at (0.5, 0.75), time-reversed single vortex) and
writes its final fractions and area, which must equal the oracle's run of the
same steps on the same inputs (bit for bit in the FP32 form, 1e-12 in FP64)."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import oracle
from paper_2309_00338_gb300 import build as B
from paper_2309_00338_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

SRC = os.path.join(os.path.dirname(__file__), "c_consumer", "ebit_vortex.c")


def _compile(tmp_path):
    lib = B.build_library()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "ebit_vortex")
    subprocess.run([cc, "-O2", "-std=c11", "-I", B.INCLUDE, "-I", os.path.join(cuda, "include"), SRC,
                    "-o", exe, "-L", libdir, "-lebit", f"-Wl,-rpath,{libdir}",
                    "-L", os.path.join(cuda, "lib64"), "-lcudart", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"],
                   check=True)
    return exe


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32], ids=["fp64", "fp32"])
def test_c_program_matches_oracle(tmp_path, prec):
    n, steps = 64, 24
    wl = W.vortex_workload(n, period=2.0, cfl=0.5)
    dts = np.asarray([wl.field.dt_eff(k, wl.dt) for k in range(steps)], np.float64)
    dtype = np.float64 if prec == oracle.FP64 else np.float32
    circles = np.asarray(wl.scene["circles"], np.float64).reshape(-1, 3)
    case = tmp_path / "case.bin"
    with open(case, "wb") as f:
        f.write(struct.pack("<4i", n, prec, steps, circles.shape[0]))
        f.write(circles.tobytes())
        f.write(dts.tobytes())
        f.write(np.ascontiguousarray(wl.field.u, dtype).tobytes())
        f.write(np.ascontiguousarray(wl.field.v, dtype).tobytes())
    exe = _compile(tmp_path)
    out = tmp_path / "out.bin"
    subprocess.run([exe, str(case), str(out)], check=True, timeout=300)
    raw = out.read_bytes()
    area = struct.unpack("<d", raw[:8])[0]
    C = np.frombuffer(raw[8:], dtype).reshape(n, n).astype(np.float64)

    S = oracle.init(n, n, wl.dx, wl.scene, prec)
    for k in range(steps):
        r = oracle.step(S, wl.field.u, wl.field.v, dts[k])
    if prec == oracle.FP32:
        assert np.array_equal(C, r["C"])
    else:
        assert np.max(np.abs(C - r["C"])) <= 1e-12
    assert abs(area - r["area"]) <= 1e-12 * max(1.0, abs(r["area"]))
    assert 0.06 < area < 0.08  # about pi * 0.15^2
