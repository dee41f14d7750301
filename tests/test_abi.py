"""The C-ABI library builds here (nvcc cross-compiles sm_103a without a GPU),
loads without a GPU, and exports exactly the entry points include/gpga.h
declares. No compute call is made."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "gpga.h")).read()
    return sorted(set(re.findall(r"GPGA_API\s+[\w\s\*]+?\b(\w+)\s*\(", hdr)))


def test_library_builds_loads_and_exports_declared_symbols():
    from paper_1403_4099_gb300 import build, gpga
    path = build.build()
    assert os.path.exists(path)
    ctypes.CDLL(path)  # loads with no GPU present
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = sorted(l.split()[-1] for l in out.splitlines() if " T " in l)
    declared = _declared()
    assert declared, "no declarations parsed"
    assert exported == declared, (exported, declared)
    assert sorted(gpga.EXPORTS) == declared


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    from paper_1403_4099_gb300 import gpga
    monkeypatch.setattr(gpga, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gpga, "_lib", None)
    try:
        gpga.lib()
    except RuntimeError as e:
        assert "missing" in str(e)
    else:
        raise AssertionError("binding loaded a missing library")


def test_params_struct_layout_matches_header():
    from paper_1403_4099_gb300 import gpga
    # int32 x4, double x4, int32 x4, double x2, int32 x4 = 16 + 32 + 16 + 16 + 16
    assert ctypes.sizeof(gpga.Params) == 96
