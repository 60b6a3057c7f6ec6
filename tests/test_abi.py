"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/mppi.h (no compute call: this runs without a GPU).  The
oracle library builds and exports its API."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mppi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mppi_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_header_symbols():
    from paper_2409_10469_gb300 import build, _mppi
    path = build.build()
    names = declared_functions()
    assert len(names) >= 12
    lib = ctypes.CDLL(path)
    for n in names:
        assert hasattr(lib, n), "missing export " + n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(r"\bT %s\b" % n, out), n
    assert set(names) == set(_mppi.EXPORTS)


def test_build_targets_sm103a_only():
    from paper_2409_10469_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2409_10469_gb300 import _mppi
    monkeypatch.setattr(_mppi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_mppi, "_lib", None)
    with pytest.raises(ImportError):
        _mppi.lib()


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2409_10469_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "oracle.h" not in txt and "liboracle" not in txt, f


def test_oracle_builds():
    from oracle import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in ("or_aba", "or_rnea", "or_crba", "or_rollout", "or_sample", "or_update", "or_shift",
              "or_mppi_step", "or_philox4x32_10"):
        assert hasattr(lib, n)
