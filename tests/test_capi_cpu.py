"""Host-side checks of the C ABI: the library builds, loads and exports every declared symbol."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rmg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2103_11962_gb300 import build, rmg
    build.build()
    L = rmg.lib()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(rmg.exported_symbols()) == declared


def test_options_defaults_roundtrip():
    from paper_2103_11962_gb300 import rmg
    o = rmg.default_options()
    assert o.levels == 4 and o.smoother == rmg.JACOBI and o.nu1 == 2 and o.nu2 == 2
    assert o.omega == pytest.approx(0.67) and o.cheb_degree == 3
    assert o.eig_ratio == 20.0 and o.boost == pytest.approx(1.1) and o.power_iters == 10
    assert o.use_graph == 1 and o.precision == rmg.FP64


def test_no_device_means_clear_error():
    """Without a GPU the context creation fails with a status, not a crash."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2103_11962_gb300 import rmg
    import ctypes
    h = ctypes.c_void_p()
    st = rmg.lib().rmg_create(ctypes.byref(h), 0, None)
    assert st != rmg.RMG_OK
