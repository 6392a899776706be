"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every
function declared in include/*.h (no compute calls: there is no GPU here)."""
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300 import build as B
    if not os.path.exists(L.LIB_PATH):
        B.build()
    return L.load()


def test_library_exports_every_declared_symbol(lib):
    from paper_2411_16392_gb300 import _lib as L
    names = L.declared_symbols()
    assert "render_forward" in names and "render_backward" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_declares_every_symbol():
    from paper_2411_16392_gb300 import _lib as L
    bound = {e[0] for e in L.EXPORTS}
    assert set(L.declared_symbols()) <= bound


def test_config_default_without_gpu(lib):
    from paper_2411_16392_gb300 import _lib as L
    cfg = L.qgs_config()
    lib.qgs_config_default(ctypes.byref(cfg))
    assert abs(cfg.alpha_max - 0.99) < 1e-7 and abs(cfg.alpha_min - 1 / 255) < 1e-9
    assert abs(cfg.T_min - 1e-4) < 1e-10 and cfg.sort_mode == 0


def test_struct_layouts_match_header():
    """The ctypes mirrors have the sizes the C header implies."""
    from paper_2411_16392_gb300 import _lib as L
    assert ctypes.sizeof(L.qgs_camera) == 4 * (2 + 4 + 9 + 3 + 1)
    assert ctypes.sizeof(L.qgs_scene) == 8 * 7
    assert ctypes.sizeof(L.qgs_image) == 8 * 7
    assert ctypes.sizeof(L.qgs_scene_grad) == 8 * 6
    assert ctypes.sizeof(L.qgs_config) == 4 * 7
    assert ctypes.sizeof(L.qgs_frame_stats) == 8 * 13 + 4 * 7 + 4


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2411_16392_gb300 import _lib as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        L.load()


def test_no_oracle_import_on_product_path():
    """The package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2411_16392_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_debug_checks_compiled_out_of_the_normal_build(lib):
    """The normal build reports the bounds checks as absent and touches no device."""
    ci, w = ctypes.c_int32(7), ctypes.c_uint32(9)
    assert lib.qgs_debug_check_word(0, ctypes.byref(ci), ctypes.byref(w)) == 0
    assert ci.value == 0 and w.value == 0
    assert lib.qgs_debug_check_word(0, None, ctypes.byref(w)) == 1   # QGS_EINVAL


def test_debug_check_build_compiles_and_exports():
    """The bounds-checked variant (-DQGS_DEBUG_CHECKS) builds for sm_103a and exports the
    same entry points."""
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300 import build as B
    path = B.build(debug_checks=True)
    assert path.endswith("libqgs_check.so") and os.path.exists(path)
    chk = ctypes.CDLL(path)
    missing = [n for n in L.declared_symbols() if not hasattr(chk, n)]
    assert not missing, missing
