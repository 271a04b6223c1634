"""The C ABI from a plain C program (tests/c/abi_smoke.c): it compiles and links
against libpd with only include/pd.h on any machine; on a GPU it runs and prints
exactly what the same simulation gives through the Python binding."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1806_06917_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "abi_smoke.c")


def _build(tmp_path):
    from paper_1806_06917_gb300 import build as B
    lib = B.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_smoke")
    libdir = os.path.dirname(lib)
    subprocess.run([cc, "-std=c99", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), SRC, "-o", exe,
                    "-L", libdir, "-lpd", "-Wl,-rpath," + libdir, "-lm"], check=True, capture_output=True)
    return exe


def test_c_client_compiles_and_links_against_the_header_alone(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_c_client_matches_the_python_binding(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = _build(tmp_path)
    g = W.Grid(dim=2, n=(24, 17, 1), h=0.02, m=3)
    X = g.positions()
    r2 = ((X - np.array([0.23, 0.17])) ** 2).sum(axis=1)
    u = np.ascontiguousarray(np.stack([1e-5 * np.exp(-r2 / 0.002), 0.5e-5 * np.exp(-r2 / 0.002)], axis=1))
    u0_file = str(tmp_path / "u0.bin")
    u.tofile(u0_file)
    out = subprocess.run([exe, "50", u0_file], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {l.split()[0]: [float(x) for x in l.split()[1:]] for l in out if l.strip()}
    from paper_1806_06917_gb300 import pd
    mat = W.Material(model=W.PMB, E=72e9, rho=2440.0, thickness=1.0)
    gd, md, rd = pd.describe(g, mat, precision=pd.PD_FP64, dt_factor=0.0)
    sim = pd.pd_create(gd, md, rd)
    pd.pd_build_neighbors(sim)
    pd.pd_set_state(sim, u=u, v=np.zeros_like(u))
    e0 = pd.pd_energy(sim)
    pd.pd_step_explicit(sim, 50)
    uo, _ = pd.pd_get_state(sim)
    e1 = pd.pd_energy(sim)
    assert got["bonds"][0] == pd.pd_bond_count(sim)
    assert got["dt"][0] == pd.pd_get_dt(sim)
    assert got["energy0"] == list(e0) and got["energy"] == list(e1)
    n = g.npoints
    assert got["u"] == [uo[0, 0], uo[n // 2, 0], uo[n - 1, 1]]
    sim.close()


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets the
    C compiler gives the struct of the same name in include/pd.h."""
    from paper_1806_06917_gb300 import pd
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [getattr(pd, n) for n in ("pd_grid", "pd_material", "pd_run", "pd_newton_opts", "pd_newton_stats",
                                        "pd_server_opts", "pd_request", "pd_result")]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pd.h"', "int main(void) {"]
    want = []
    for cls in structs:
        name = cls.__name__
        lines.append('printf("%%s %%zu\\n", "%s", sizeof(%s));' % (name, name))
        want.append("%s %d" % (name, ctypes.sizeof(cls)))
        for field, _ in cls._fields_:
            lines.append('printf("%%s %%zu\\n", "%s.%s", offsetof(%s, %s));' % (name, field, name, field))
            want.append("%s.%s %d" % (name, field, getattr(cls, field).offset))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe],
                   check=True, capture_output=True)
    got = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    assert [l for l in got if l] == want
