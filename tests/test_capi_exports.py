"""The C-ABI library builds for sm_103a and exports every entry point that
include/fdtd.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(fdtd_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["fdtd_create", "fdtd_set_source", "fdtd_add_probe", "fdtd_set_spectrum", "fdtd_step",
                 "fdtd_probe_spectra", "fdtd_probe_trace", "fdtd_diagnostics", "fdtd_sync", "fdtd_destroy",
                 "fdtd_strerror", "fdtd_batch_create", "fdtd_batch_add", "fdtd_batch_step"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1008_2602_gb300 import build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fdtd_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert getattr(lib, n) is not None


def test_binding_wraps_every_declared_symbol():
    from paper_1008_2602_gb300 import capi
    for n in _declared():
        assert callable(getattr(capi, n)), n
    assert capi.lib.fdtd_strerror(-1) == b"invalid argument"


def test_library_is_built_for_sm_103a():
    from paper_1008_2602_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1008_2602_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import oracle|from oracle)", text, re.M), f
                assert "fdtd_oracle" not in text, f
