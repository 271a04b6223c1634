"""GPU: the NP bond law of Algorithm 1 and its linearisation LP through the C
ABI against the FP64 oracle: forces at strains where the NP potential is well
nonlinear (beta |xi| S^2 of order 1), energies, the stable-step bound, and
explicit runs of the paper's 2D convergence setup (Sec. 5.2.2; collar held at
u = 0, Gaussian initial displacement, dt = 1e-5).

Bars as for the other laws: FP32-compensated force within 1e-5 relative L2,
FP64 within 1e-10; displacement within 1e-4 (FP32C) / 1e-10 (FP64).
"""
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


GRIDS = [(2, (70, 37, 1), 3), (2, (45, 33, 1), 4), (3, (20, 17, 11), 3), (3, (12, 13, 9), 2)]


@pytest.mark.parametrize("dim,n,m", GRIDS)
@pytest.mark.parametrize("model", [W.NP, W.LP])
@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_np_lp_force_matches_oracle(pd, dim, n, m, model, precision):
    g = W.Grid(dim=dim, n=n, h=0.5, m=m)
    mat = W.Material(model=model, rho=1.0, psi_c=1.3, psi_beta=1.7)
    rng = np.random.default_rng(31)
    u = rng.normal(0.0, 0.2 * g.h, (g.npoints, dim))        # beta |xi| S^2 of order 1
    u += 0.37                                               # plus a rigid translation
    f_o, _ = O.internal_force(g, mat, O.neighbors(g), u)
    prec = pd.PD_FP32C if precision == "fp32c" else pd.PD_FP64
    sim = gpu_sim(pd, g, mat, prec)
    f_g = pd.pd_force(sim, u=u)
    assert rel_l2(f_g, f_o) <= (1e-5 if precision == "fp32c" else 1e-10)
    sim.close()


@pytest.mark.parametrize("model", [W.NP, W.LP])
def test_np_lp_energy_and_step_bound_match_oracle(pd, model):
    wl = W.np_square(k=4, model=model)
    g = wl.grid
    bonds = O.neighbors(g)
    sim = gpu_sim(pd, g, wl.mat, pd.PD_FP64)
    dt_o = 0.5 * O.stable_dt(g, wl.mat, bonds)
    assert abs(pd.pd_get_dt(sim) - dt_o) <= 1e-12 * dt_o
    rng = np.random.default_rng(32)
    u = rng.normal(0.0, 0.3 * g.h, (g.npoints, 2))
    pd.pd_set_state(sim, u=u, v=np.zeros_like(u))
    _, s_g = pd.pd_energy(sim)
    s_o = O.strain_energy(g, wl.mat, bonds, u)
    assert abs(s_g - s_o) <= 1e-10 * abs(s_o)
    sim.close()


@pytest.mark.parametrize("model", [W.NP, W.LP])
@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_convergence_setup_explicit_run_matches_oracle(pd, model, precision):
    wl = W.np_square(k=4, model=model, ic=2)
    g = wl.grid
    bonds = O.neighbors(g)
    steps = 3000
    prec = pd.PD_FP32C if precision == "fp32c" else pd.PD_FP64
    sim = gpu_sim(pd, g, wl.mat, prec, dt=wl.dt)
    pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
    pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val)
    pd.pd_step_explicit(sim, steps)
    u_g, v_g = pd.pd_get_state(sim)
    st = O.ExplicitState(g, wl.mat, bonds, wl.u0, wl.v0, wl.bc_kind, wl.bc_val)
    st.run(wl.dt, steps)
    assert rel_l2(u_g, st.u) <= (1e-4 if precision == "fp32c" else 1e-10)
    assert np.abs(u_g[wl.bc_kind[:, 0] == W.BC_DISPLACEMENT]).max() == 0.0
    sim.close()


def test_np_lp_refuse_breaking_and_the_tangent(pd):
    g = W.Grid(dim=2, n=(10, 10, 1), h=0.1, m=3)
    gd, md, rd = pd.describe(g, W.Material(model=W.NP, rho=1.0))
    md.s_c = 1e-3
    with pytest.raises(pd.PdError) as e:
        pd.pd_create(gd, md, rd)
    assert e.value.code == pd.PD_EINVAL
    md.s_c, md.psi_beta = 0.0, 0.0
    with pytest.raises(pd.PdError) as e:
        pd.pd_create(gd, md, rd)
    assert e.value.code == pd.PD_EINVAL
    sim = gpu_sim(pd, g, W.Material(model=W.LP, rho=1.0), pd.PD_FP64)
    with pytest.raises(pd.PdError) as e:
        pd.pd_jvp(sim, np.zeros((g.npoints, 2)))
    assert e.value.code == pd.PD_EINVAL
    sim.close()


def test_convergence_rate_to_t02_matches_oracle(pd):
    """The study of Sec. 5.2.2 (NP, IC 1) on its three meshes (h = delta / 2,
    delta / 4, delta / 8) to t = 0.2: each mesh's u against the oracle's run,
    and the rate alpha at t = 0.1 and 0.2 from the GPU's u against the rate
    from the oracle's u (about 80 s of oracle time on 16 host cores)."""
    import bench
    ks = (2, 4, 8)
    wls = [W.np_square(k=k, model=W.NP, ic=1) for k in ks]
    sims = []
    states = []
    for wl in wls:
        sim = gpu_sim(pd, wl.grid, wl.mat, "fp32c", dt=wl.dt)
        pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
        pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val)
        sims.append(sim)
        states.append(O.ExplicitState(wl.grid, wl.mat, O.neighbors(wl.grid), wl.u0, wl.v0, wl.bc_kind, wl.bc_val))
    for _ in range(2):                               # t = 0.1, then t = 0.2
        ug, uo = [], []
        for sim, st, wl in zip(sims, states, wls):
            pd.pd_step_explicit(sim, 10000)
            st.run(wl.dt, 10000)
            u, _ = pd.pd_get_state(sim, want_v=False)
            assert rel_l2(u, st.u) <= 1e-4
            ug.append(u)
            uo.append(st.u.copy())
        a_g = bench.convergence_rate(ug, wls, ks)
        a_o = bench.convergence_rate(uo, wls, ks)
        assert a_g is not None and a_o is not None
        assert abs(a_g - a_o) <= 1e-3, (a_g, a_o)
        assert a_o > 1.0                             # the paper's regime at early times
    for sim in sims:
        sim.close()
