"""The C-ABI library loads and exports every symbol include/*.h declares
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(ebit_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libebit():
    from paper_2309_00338_gb300 import build
    path = build.build_library()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("ebit_init", "ebit_step", "ebit_fraction", "ebit_curvature", "ebit_load_state",
              "ebit_get_state", "ebit_sync", "ebit_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(libebit):
    missing = [n for n in declared_symbols() if not hasattr(libebit, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2309_00338_gb300 import ebit
    assert declared_symbols() <= set(ebit.SIGNATURES)


def test_footprint_and_argument_checks_need_no_gpu(libebit):
    from paper_2309_00338_gb300 import ebit
    ebit.lib()
    fp32 = ebit.ebit_footprint(4096, 4096, 1 / 4096, ebit.EBIT_FP32)
    fp64 = ebit.ebit_footprint(4096, 4096, 1 / 4096, ebit.EBIT_FP64)
    assert 0 < fp32 < fp64 < 2 * 1024 ** 3
    assert ebit.ebit_footprint(0, 16, 0.1) == 0          # invalid grid
    assert ebit.ebit_footprint(16, 16, -1.0) == 0
    # calls that fail argument validation return before touching CUDA
    h = ctypes.c_void_p()
    g = ebit.ebit_grid(0, 4, 0.25, 0, 0)
    st = ebit.lib().ebit_create(ctypes.byref(h), ctypes.byref(g), None)
    assert st == ebit.EBIT_EINVAL and not h.value
    assert ebit.lib().ebit_step(None, None, None, 0.1) == ebit.EBIT_EINVAL
    assert b"NULL" in ebit.lib().ebit_last_error()


def test_product_path_has_no_oracle_dependency():
    """The library sources and the binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2309_00338_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "ebit_oracle" not in text and "orc_" not in text, path


def test_new_entry_points_check_arguments_without_gpu(libebit):
    """ebit_coupling, ebit_area_async, ebit_fraction_to_host and the scene
    checks of ebit_init reject
    bad arguments before any CUDA call; EBIT_CURV_GHF adds its cell list to
    the footprint."""
    from paper_2309_00338_gb300 import ebit
    L = ebit.lib()
    fl = ebit.ebit_fluids(1.0, 1.0, 1.0, 1.0, 1.0)
    assert L.ebit_coupling(None, ctypes.byref(fl), None, None, None, None) == ebit.EBIT_EINVAL
    assert L.ebit_area_async(None, None) == ebit.EBIT_EINVAL
    assert L.ebit_fraction_to_host(None, None, None) == ebit.EBIT_EINVAL
    n = 256
    plain = ebit.ebit_footprint(n, n, 1 / n, ebit.EBIT_FP32)
    ghf = ebit.ebit_footprint(n, n, 1 / n, ebit.EBIT_FP32, ebit.EBIT_CURV_GHF)
    assert ghf - plain >= n * n * 4
    assert ebit.ebit_footprint(n, n, 1 / n, ebit.EBIT_FP32, 4) == 0   # unknown flag
    keep = []
    sc = ebit._scene({"lines": [(1.0, 1.0, 0.5)] * 4}, keep)
    sc.nlines = 5
    h = ctypes.c_void_p()
    g = ebit.ebit_grid(n, n, 1 / n, 0, 0)
    assert L.ebit_init(ctypes.byref(h), ctypes.byref(g), ctypes.byref(sc), None) == ebit.EBIT_EINVAL
    assert not h.value


def test_binding_refuses_wrongly_sized_tensors():
    """The binding checks the caller's tensors against the context's grid
    before any call that reads or writes them (a handle registered by hand
    here: the checks fire before the library is reached)."""
    torch = pytest.importorskip("torch")
    from paper_2309_00338_gb300 import ebit
    fake = ctypes.c_void_p(0x5eed)
    ebit._CTX[fake.value] = (8, 4, ebit.EBIT_FP32)
    try:
        verts = 9 * 5
        with pytest.raises(ValueError, match="u: expected 45"):
            ebit.ebit_step(fake, torch.zeros(44), torch.zeros(verts), 0.1)
        with pytest.raises(ValueError, match="float32"):
            ebit.ebit_step(fake, torch.zeros(verts, dtype=torch.float64), torch.zeros(verts), 0.1)
        with pytest.raises(ValueError, match="CUDA"):
            ebit.ebit_step(fake, torch.zeros(verts), torch.zeros(verts), 0.1)
        with pytest.raises(ValueError, match="vel"):
            ebit.ebit_sweep(fake, 0, torch.zeros(verts + 1), 0.1)
        with pytest.raises(ValueError, match="C: expected 32"):
            ebit.ebit_fraction(fake, torch.zeros(31))
        with pytest.raises(ValueError, match="kappa"):
            ebit.ebit_curvature(fake, torch.zeros(33))
        with pytest.raises(ValueError, match="fx: expected 36"):
            ebit.ebit_coupling(fake, 1, 1, 1, 1, 1, fx=torch.zeros(32))
        with pytest.raises(ValueError, match="fy: expected 40"):
            ebit.ebit_coupling(fake, 1, 1, 1, 1, 1, fy=torch.zeros(36))
        ebit._check_tensor(fake, torch.zeros(32), "C_host", lambda nx, ny: nx * ny, False)  # accepted
        import numpy as np
        with pytest.raises(ValueError, match="sV: expected 36"):
            ebit.ebit_load_state(fake, np.zeros((5, 9)), np.zeros((4, 8)), np.zeros((5, 8)), np.zeros((4, 8)))
    finally:
        ebit._CTX.pop(fake.value, None)
