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


def _declared_arity():
    arity = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"PT_API\s+[\w\s\*]+?\b(pt_\w+)\s*\(([^)]*)\)\s*;", src):
            params = m.group(2).strip()
            arity[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return arity


def test_binding_types_every_entry_point(libpt):
    """The ctypes binding gives every declared entry point its argument
    types, as many as the header declares (no untyped calls)."""
    from paper_2305_20061_gb300 import pt
    L = pt.lib()
    arity = _declared_arity()
    assert set(arity) == set(_declared())
    wrong = {n: (len(getattr(L, n).argtypes or []), k) for n, k in arity.items()
             if getattr(L, n).argtypes is None or len(getattr(L, n).argtypes) != k}
    assert not wrong, wrong


def _decl(name):
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        m = re.search(r"PT_API\s+([\w\s\*]+?)\b" + name + r"\s*\(([^)]*)\)\s*;", src)
        if m:
            return " ".join(m.group(1).split()), [" ".join(p.split()) for p in m.group(2).split(",")]
    raise KeyError(name)


def test_render_and_error_word_signatures():
    """pt_render takes a nullable radiance cache before the configuration;
    pt_device_error_bits returns the word itself; the configuration carries
    the cache vertex."""
    ret, params = _decl("pt_render")
    assert ret == "pt_status"
    assert params[:5] == ["pt_ctx* ctx", "const pt_scene* scene", "const pt_nif* nif", "const pt_cache* cache",
                          "const pt_render_cfg* cfg"]
    assert params[5:] == ["float* d_image", "void* stream"]
    ret, params = _decl("pt_device_error_bits")
    assert ret == "uint32_t" and params == ["pt_ctx* ctx"]
    src = open(os.path.join(ROOT, "include", "pt.h")).read()
    body = src[src.index("typedef struct pt_render_cfg"):src.index("} pt_render_cfg;")]
    assert "int32_t cache_vertex;" in body
    from paper_2305_20061_gb300 import pt
    assert [f for f, _ in pt.RenderCfg._fields_][-1] == "cache_vertex"
