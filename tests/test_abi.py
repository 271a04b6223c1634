"""CPU-side checks of the C ABI: the library builds, loads, and exports exactly
the entry points that include/pd.h declares. No compute call runs here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\bint\s+(pd_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("pd_create", "pd_build_neighbors", "pd_force", "pd_step_explicit", "pd_jvp", "pd_vjp",
                 "pd_energy", "pd_destroy", "pd_last_error"):
        assert want in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_1806_06917_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_1806_06917_gb300 import pd
    assert sorted(pd.EXPORTS) == _declared()


def test_binding_rejects_bad_buffers_before_calling_the_library():
    np = pytest.importorskip("numpy")
    from paper_1806_06917_gb300 import pd
    with pytest.raises(ValueError):
        pd._buf(np.zeros(5, np.float32), np.float64, 5, "x")
    with pytest.raises(ValueError):
        pd._buf(np.zeros(4), np.float64, 5, "x")
    with pytest.raises(ValueError):
        pd._buf(np.zeros((5, 2))[:, 0], np.float64, 5, "x")
    assert pd._buf(None, np.float64, 5, "x") is None


def test_oracle_shares_no_code_with_the_cuda_path():
    """The package never imports or includes anything from oracle/."""
    import ast
    pkg = os.path.join(ROOT, "paper_1806_06917_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                tree = ast.parse(open(path).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
                    if isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", path
            if f.endswith((".cu", ".cuh", ".h")):
                for line in open(path):
                    if line.lstrip().startswith("#include"):
                        assert "oracle" not in line, path
