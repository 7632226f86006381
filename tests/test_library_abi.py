"""The C ABI library builds, loads without a GPU, and exports every entry
point declared in include/jfnk.h; the oracle never loads it."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "jfnk.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"\b(jfnk_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1512_03662_gb300 import build
    lib_path = build.build()
    import ctypes
    L = ctypes.CDLL(lib_path)
    names = _declared()
    assert "jfnk_create" in names and "jfnk_step" in names
    for n in names:
        assert hasattr(L, n), n
    import paper_1512_03662_gb300 as jf
    assert sorted(jf.EXPORTED) == names


def test_options_defaults_follow_the_paper():
    import paper_1512_03662_gb300 as jf
    o = jf.default_options()
    assert o.theta == 0.5 and o.lambda_ == 1e-7 and o.alpha1 == 1e-5 and o.alpha2 == 1.0
    assert o.eta == 1e-4 and o.newton_min == 2 and o.gmres_max_it == 300


def test_oracle_does_not_touch_the_library():
    code = ("import sys; sys.path.insert(0, %r); import oracle.discretization, oracle.jfnk, oracle.precond; "
            "import workloads; print(any('paper_1512_03662_gb300' in m for m in sys.modules))" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, check=True).stdout.strip()
    assert out == "False"


def test_product_path_fails_loudly_without_the_library(tmp_path, monkeypatch):
    import paper_1512_03662_gb300 as jf
    monkeypatch.setattr(jf, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(jf, "_lib", None)
    with pytest.raises(RuntimeError):
        jf.lib()


def test_probe_library_exports_what_the_bench_and_tests_call():
    """libfp64probe.so (the FP64 peak probe of bench.py and the device
    function checks of the GPU tests) builds and loads without a GPU."""
    from paper_1512_03662_gb300 import build
    build.build()
    import ctypes
    L = ctypes.CDLL(build.PROBE_LIB)
    for n in ("fp64_probe_launch", "fp64_probe_fma_per_thread", "fp64_recip_check", "fp64_conv_check"):
        assert hasattr(L, n), n
