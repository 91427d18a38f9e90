"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no GPU needed: nothing is called)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"PT_API\s+[\w\s\*]+?\b(pt_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpt():
    from paper_2305_20061_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for required in ("pt_create", "pt_create_scene", "pt_load_nif", "pt_render", "pt_check", "pt_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(libpt):
    missing = [n for n in _declared() if not hasattr(libpt, n)]
    assert not missing, missing


def test_no_undeclared_exports(libpt):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", libpt._name], capture_output=True, text=True).stdout
    exported = sorted({l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("pt_")})
    assert set(exported) == set(_declared()), (set(exported) ^ set(_declared()))


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2305_20061_gb300 import pt
    monkeypatch.setattr(pt, "_lib", None)
    monkeypatch.setattr(pt, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        pt.lib()
