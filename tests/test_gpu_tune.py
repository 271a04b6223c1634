"""pd_tune_tile: the measured tile choice returns an admissible tile, and a run at
the chosen tile agrees with the default tile to the FP32C tolerance (the tile
changes only the staging's per-tile reference frame)."""
import numpy as np
import pytest

from paper_1806_06917_gb300 import workloads as W
from tests.helpers import gpu_sim, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06917_gb300 import pd as _pd
    return _pd


CASES = [
    ("pmb3", W.Grid(dim=3, n=(24, 22, 20), h=0.01, m=3), W.Material(model=W.PMB, s_c=0.0)),
    ("lps3", W.Grid(dim=3, n=(20, 20, 20), h=0.01, m=3), W.Material(model=W.LPS, K=4e10, mu=3e10)),
    ("np2_wide", W.Grid(dim=2, n=(90, 80, 1), h=0.01, m=12),
     W.Material(model=W.NP, rho=1.0, psi_c=1.0, psi_beta=1.0, thickness=1.0)),
]


@pytest.mark.parametrize("name,grid,mat", CASES, ids=[c[0] for c in CASES])
def test_tuned_tile_is_admissible_and_agrees(pd, name, grid, mat):
    g, m, r = pd.describe(grid, mat, precision=pd.PD_FP32C)
    r.tile_log2 = 7          # ignored by the tuner
    L = pd.pd_tune_tile(g, m, r, steps=3)
    assert 6 <= L <= 9
    rng = np.random.default_rng(4)
    u0 = 1e-4 * grid.h * rng.standard_normal((grid.npoints, grid.dim))
    v0 = 1e-2 * rng.standard_normal((grid.npoints, grid.dim))
    out = []
    for tl in (0, L):
        sim = gpu_sim(pd, grid, mat, pd.PD_FP32C, tile_log2=tl)
        pd.pd_set_state(sim, u=u0, v=v0)
        pd.pd_step_explicit(sim, 10)
        out.append(pd.pd_get_state(sim))
        sim.close()
    assert rel_l2(out[1][0], out[0][0]) < 1e-6
    assert rel_l2(out[1][1], out[0][1]) < 1e-5
