"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads, and
exports every entry point include/ss.h declares. No device call is made."""
import ctypes
import os
import subprocess

import pytest

import paper_2604_19890_gb300 as ssg
from paper_2604_19890_gb300 import build


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    declared = ssg.declared_symbols()
    assert len(declared) >= 30
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(path)
    for s in declared:
        assert getattr(lib, s) is not None


def test_binding_covers_the_header():
    assert set(ssg.declared_symbols()) == set(ssg._SIGS)


def test_presets_without_device():
    for i in range(3):
        p = ssg.preset(i)
        assert p.logN in (13, 15, 16) and p.L > 0 and p.h == 120
    with pytest.raises(ssg.SSError):
        ssg.preset(99)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(ssg, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(ssg, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        ssg.lib()


def test_kernels_compiled_for_sm103a():
    objdir = os.path.join(os.path.dirname(build.__file__), "_build")
    objs = [f for f in os.listdir(objdir) if f.endswith(".o")]
    assert objs
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
