"""The C-ABI library builds for sm_103a, loads, and exports every entry point its header declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(es_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_header_symbols():
    from paper_2407_05568_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared("es_vdw.h")
    assert "es_step" in names and "es_steps" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    """The product path has no fallback: a missing library raises."""
    from paper_2407_05568_gb300 import es
    monkeypatch.setattr(es, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(es, "_lib", None)
    try:
        es.lib()
    except RuntimeError as e:
        assert "missing" in str(e)
    else:
        raise AssertionError("expected a RuntimeError")


def test_params_struct_matches_header():
    """ctypes mirror of es_params has the header's field order."""
    from paper_2407_05568_gb300 import es
    text = open(os.path.join(ROOT, "include", "es_vdw.h")).read()
    body = text[text.index("typedef struct es_params"):text.index("} es_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";")[:-1]:
        decl = decl.split("{")[-1].strip()
        if not decl:
            continue
        names = decl.split(None, 1)[1]
        for nm in names.split(","):
            fields.append(re.sub(r"\[.*\]", "", nm).strip())
    assert fields == [f[0] for f in es.EsParams._fields_]
