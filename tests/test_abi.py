"""Host-side checks of the C-ABI library: it builds, loads without a GPU and
exports every function include/lens.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lens.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lens_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2004_06352_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_2004_06352_gb300 import api
    assert sorted(api.EXPORTS) == declared_functions()


def test_binding_constants_match_the_header():
    from paper_2004_06352_gb300 import api
    src = open(os.path.join(ROOT, "include", "lens.h")).read()
    m = re.search(r"#define LENS_REPAIR_RATIO_DEFAULT ([0-9.]+)", src)
    assert m and float(m.group(1)) == api.LENS_REPAIR_RATIO_DEFAULT


def test_error_strings_without_gpu(libpath):
    from paper_2004_06352_gb300 import api
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert api.strerror(code) and api.strerror(code) != "unknown error code"


def test_oracle_and_library_share_no_source():
    """The oracle and the CUDA path share no file, header or include."""
    csrc = os.path.join(ROOT, "paper_2004_06352_gb300", "csrc")
    for f in os.listdir(csrc):
        if not os.path.isfile(os.path.join(csrc, f)) or f.endswith(".pyc"):
            continue
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower(), f
    otext = open(os.path.join(ROOT, "oracle", "lens_oracle.c")).read()
    assert "#include \"" not in otext
    import ast
    for f in ("api.py", "build.py", "__init__.py"):
        tree = ast.parse(open(os.path.join(ROOT, "paper_2004_06352_gb300", f)).read())
        for node in ast.walk(tree):
            if isinstance(node, (ast.Import, ast.ImportFrom)):
                mod = getattr(node, "module", None) or ""
                names = [a.name for a in node.names]
                assert "oracle" not in mod and not any("oracle" in n for n in names), (f, mod, names)
