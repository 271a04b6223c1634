"""GPU: body forces b (pd_set_body_force) in the explicit update, a = (f + b) / rho
(Eqs. (7)-(10)), against the oracle's runs with the same b, for every fused
update path: PMB (one pair per thread), LPS (force pass), NP at m = 20 (two
pairs per thread), velocity-Verlet and central difference, FP32C and FP64."""
import numpy as np
import pytest

from oracle import oracle as O
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


def _case(name):
    if name == "pmb3d":
        g = W.Grid(dim=3, n=(19, 18, 17), h=0.05, m=3)
        mat = W.Material(model=W.PMB, E=72e9, rho=2440.0)
        u0 = W.gaussian_ic(g, (2e-5, 0.0, 1e-5), (0.5, 0.45, 0.4), 0.02)
        b = np.zeros((g.npoints, 3))
        b[:, 2] = -2e6
        b += W.random_field(g, 5e5, seed=41)
    elif name == "pmb2d":
        g = W.Grid(dim=2, n=(41, 33, 1), h=0.02, m=3)
        mat = W.Material(model=W.PMB, E=72e9, rho=2440.0, thickness=1.0)
        u0 = W.gaussian_ic(g, (2e-5, 1e-5), (0.4, 0.3), 0.004)
        b = W.random_field(g, 1e6, seed=42)
    elif name == "lps3d":
        g = W.Grid(dim=3, n=(18, 17, 16), h=1.0 / 18, m=3)
        mat = W.Material(model=W.LPS, E=72e9, rho=2440.0, K=40e9, mu=30e9)
        u0 = (1e-4 / 3.0) * g.positions()
        b = W.random_field(g, 2e6, seed=43)
    elif name == "np2d_m20":
        g = W.Grid(dim=2, n=(70, 64, 1), h=0.0025, m=20)
        mat = W.Material(model=W.NP, E=0.0, rho=1.0, psi_c=1.0, psi_beta=1.0, thickness=1.0)
        u0 = W.gaussian_ic(g, (0.001, 0.0005), (0.08, 0.08), 0.003)
        b = W.random_field(g, 4e-4, seed=44)
    else:
        raise KeyError(name)
    return g, mat, u0, b


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("case", ["pmb3d", "pmb2d", "lps3d", "np2d_m20"])
def test_body_force_verlet_matches_oracle(pd, case, precision):
    g, mat, u0, b = _case(case)
    v0 = np.zeros_like(u0)
    steps = 40
    sim = gpu_sim(pd, g, mat, pd.PD_FP32C if precision == "fp32c" else pd.PD_FP64)
    pd.pd_set_state(sim, u=u0, v=v0)
    pd.pd_set_body_force(sim, b)
    pd.pd_step_explicit(sim, steps)
    u_g, v_g = pd.pd_get_state(sim)
    dt = pd.pd_get_dt(sim)
    st = O.ExplicitState(g, mat, O.neighbors(g), u0, v0, b=b)
    st.run(dt, steps)
    ref0 = O.ExplicitState(g, mat, O.neighbors(g), u0, v0)
    ref0.run(dt, steps)
    assert rel_l2(st.u, ref0.u) > 1e-3                   # the body force matters
    tol = 1e-4 if precision == "fp32c" else 1e-10
    assert rel_l2(u_g, st.u) <= tol
    assert rel_l2(v_g, st.v) <= (1e-3 if precision == "fp32c" else 1e-9)
    sim.close()


@pytest.mark.parametrize("case", ["pmb3d", "np2d_m20"])
def test_body_force_central_difference_matches_oracle(pd, case):
    g, mat, u0, b = _case(case)
    v0 = np.zeros_like(u0)
    steps = 40
    sim = gpu_sim(pd, g, mat, pd.PD_FP32C, integrator=pd.PD_INTEGRATOR_CD)
    pd.pd_set_state(sim, u=u0, v=v0)
    pd.pd_set_body_force(sim, b)
    pd.pd_step_explicit(sim, steps)
    u_g, _ = pd.pd_get_state(sim)
    u_o = O.run_central_difference(g, mat, O.neighbors(g), u0, v0, pd.pd_get_dt(sim), steps, b=b)
    assert rel_l2(u_g, u_o) <= 1e-4
    sim.close()
