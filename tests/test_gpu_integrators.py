"""The two explicit integrators of Sec. 4.2.4 at the ABI: central difference
(Eq. (10)) against the oracle's central-difference run, and against the
oracle's velocity-Verlet run (Eqs. (7)-(9)) where boundary conditions or
breaking enter (the two schemes give one trajectory in exact arithmetic; the
oracle's pins fix that equality). Plus the restart rules of the CD state.

Bars as in the other parity tests: FP64 within 1e-10 relative L2 of the
oracle's CD run (1e-9 against its Verlet run, a different rounding order),
FP32-compensated within 1e-4 for u and 1e-3 for v; reruns of the same calls
bit-identical.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_06917_gb300 import workloads as W
from tests.helpers import gpu_csr_in_user_numbering, gpu_sim, oracle_setup, rel_l2

pytestmark = pytest.mark.gpu

U_TOL = 1e-4
V_TOL = 1e-3


@pytest.fixture(scope="module")
def pd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06917_gb300 import pd as _pd
    return _pd


def _prec(pd, name):
    return pd.PD_FP32C if name == "fp32c" else pd.PD_FP64


def _free_case(name):
    """Free-boundary cases without breaking: (grid, material, u0, v0)."""
    if name == "pmb2d":
        g = W.Grid(dim=2, n=(41, 37, 1), h=0.02, m=3)
        mat = W.Material(model=W.PMB, E=72e9, rho=2440.0, thickness=1.0)
        u0 = W.gaussian_ic(g, (2e-5, 1e-5), (0.4, 0.35), 0.004)
        v0 = W.random_field(g, 1e-3, seed=21)
    elif name == "pmb3d":
        g = W.Grid(dim=3, n=(20, 19, 18), h=0.05, m=3)
        mat = W.Material(model=W.PMB, E=72e9, rho=2440.0)
        u0 = W.gaussian_ic(g, (3e-5, 0.0, 1e-5), (0.5, 0.45, 0.4), 0.02)
        v0 = W.random_field(g, 1e-3, seed=22)
    elif name == "lps3d":
        g = W.Grid(dim=3, n=(18, 17, 16), h=1.0 / 18, m=3)
        mat = W.Material(model=W.LPS, E=72e9, rho=2440.0, K=40e9, mu=30e9)
        u0 = (1e-4 / 3.0) * g.positions() + W.random_field(g, 1e-5 * g.h, seed=23)
        v0 = W.random_field(g, 1e-3, seed=24)
    elif name in ("np2d", "lp2d"):
        g = W.Grid(dim=2, n=(30, 30, 1), h=0.05, m=2)
        mat = W.Material(model=W.NP if name == "np2d" else W.LP, E=0.0, rho=1.0, psi_c=1.0, psi_beta=1.0,
                         thickness=1.0)
        u0 = W.gaussian_ic(g, (0.001, 0.0005), (0.7, 0.7), 0.05)
        v0 = np.zeros_like(u0)
    else:
        raise KeyError(name)
    return g, mat, u0, v0


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("case", ["pmb2d", "pmb3d", "lps3d", "np2d", "lp2d"])
def test_central_difference_matches_oracle(pd, case, precision):
    g, mat, u0, v0 = _free_case(case)
    steps = 70          # a single step, then graph-replayed chunks, then single steps
    sim = gpu_sim(pd, g, mat, _prec(pd, precision), integrator=pd.PD_INTEGRATOR_CD)
    bonds = O.neighbors(g)
    dt = pd.pd_get_dt(sim)
    assert abs(dt - 0.5 * O.stable_dt(g, mat, bonds)) <= 1e-12 * dt
    pd.pd_set_state(sim, u=u0, v=v0)
    pd.pd_step_explicit(sim, steps)
    u_g, _ = pd.pd_get_state(sim)
    u_o = O.run_central_difference(g, mat, bonds, u0, v0, dt, steps)
    assert np.abs(u_o - u0).max() > 1e-3 * np.abs(u0).max()     # the state moved
    assert rel_l2(u_g, u_o) <= (U_TOL if precision == "fp32c" else 1e-10)
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_central_difference_with_velocity_collars_matches_verlet_oracle(pd, precision):
    """The 50 x 50 plate with prescribed collar velocities, 200 steps."""
    wl = W.plate2d(nside=50, steps=200)
    sim = gpu_sim(pd, wl.grid, wl.mat, _prec(pd, precision), integrator=pd.PD_INTEGRATOR_CD)
    pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
    pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val)
    pd.pd_step_explicit(sim, wl.steps)
    u_g, v_g = pd.pd_get_state(sim)
    st = O.ExplicitState(wl.grid, wl.mat, oracle_setup(wl), wl.u0, wl.v0, wl.bc_kind, wl.bc_val)
    st.run(pd.pd_get_dt(sim), wl.steps)
    assert rel_l2(u_g, st.u) <= (U_TOL if precision == "fp32c" else 1e-9)
    assert rel_l2(v_g, st.v) <= (V_TOL if precision == "fp32c" else 1e-9)
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_central_difference_with_clamped_collar_np_matches_verlet_oracle(pd, precision):
    """NP on the convergence-study square (k = 2) with its collar held at u = 0."""
    wl = W.np_square(k=2, model=W.NP, ic=1, steps=300)
    sim = gpu_sim(pd, wl.grid, wl.mat, _prec(pd, precision), dt=wl.dt, integrator=pd.PD_INTEGRATOR_CD)
    pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
    pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val)
    pd.pd_step_explicit(sim, wl.steps)
    u_g, v_g = pd.pd_get_state(sim)
    st = O.ExplicitState(wl.grid, wl.mat, oracle_setup(wl), wl.u0, wl.v0, wl.bc_kind, wl.bc_val)
    st.run(wl.dt, wl.steps)
    assert np.array_equal(u_g[wl.bc_kind[:, 0] > 0], np.zeros_like(u_g[wl.bc_kind[:, 0] > 0]))
    assert rel_l2(u_g, st.u) <= (U_TOL if precision == "fp32c" else 1e-9)
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_central_difference_with_breaking_matches_verlet_oracle(pd, precision):
    """Pulse + pre-notch + breaking: bond sets equal up to near-threshold bonds."""
    wl = W.block3d_pulse(nside=24, steps=120, s_c=5e-5)
    sim = gpu_sim(pd, wl.grid, wl.mat, _prec(pd, precision), notch=wl.notch, integrator=pd.PD_INTEGRATOR_CD)
    pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
    pd.pd_step_explicit(sim, wl.steps)
    u_g, _ = pd.pd_get_state(sim)
    bonds = oracle_setup(wl)
    st = O.ExplicitState(wl.grid, wl.mat, bonds, wl.u0, wl.v0, wl.bc_kind, wl.bc_val)
    st.run(pd.pd_get_dt(sim), wl.steps)
    _, _, order, _ = gpu_csr_in_user_numbering(pd, sim)
    brk = pd.pd_get_broken(sim)[order].astype(bool)
    ob = bonds.broken.astype(bool)
    assert ob.sum() > oracle_setup(wl).broken.sum()
    assert int((brk != ob).sum()) <= max(2, int(1e-4 * ob.sum()))
    assert rel_l2(u_g, st.u) <= (U_TOL if precision == "fp32c" else 1e-9)
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_central_difference_and_verlet_agree_on_the_gpu(pd, precision):
    g, mat, u0, v0 = _free_case("pmb3d")
    out = []
    for integ in (pd.PD_INTEGRATOR_VERLET, pd.PD_INTEGRATOR_CD):
        sim = gpu_sim(pd, g, mat, _prec(pd, precision), integrator=integ)
        pd.pd_set_state(sim, u=u0, v=v0)
        pd.pd_step_explicit(sim, 50)
        out.append(pd.pd_get_state(sim) + pd.pd_energy(sim))
        sim.close()
    (ua, va, ka, wa), (ub, vb, kb, wb) = out
    assert not np.array_equal(ua, ub)                    # two rounding orders
    tol = 1e-5 if precision == "fp32c" else 1e-12
    assert rel_l2(ub, ua) <= tol and rel_l2(vb, va) <= 10 * tol
    assert abs(kb + wb - ka - wa) <= 10 * tol * (ka + wa)


def test_central_difference_chunks_and_reads_are_bit_identical(pd):
    """One call, single steps, and steps interleaved with full state reads (which
    complete v to the integer step) leave the CD trajectory bit-identical: the
    CD drift never reads v, and the completed half kick is the same addition."""
    g, mat, u0, v0 = _free_case("pmb2d")
    outs = []
    for pattern in ("one", "single", "reads"):
        sim = gpu_sim(pd, g, mat, pd.PD_FP32C, integrator=pd.PD_INTEGRATOR_CD)
        pd.pd_set_state(sim, u=u0, v=v0)
        if pattern == "one":
            pd.pd_step_explicit(sim, 45)
        else:
            for k in range(45):
                pd.pd_step_explicit(sim, 1)
                if pattern == "reads" and k % 6 == 0:
                    pd.pd_get_state(sim)
        outs.append(pd.pd_get_state(sim))
        sim.close()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_central_difference_restarts_from_a_new_state_or_dt(pd, precision):
    """After pd_set_state or pd_set_dt the next step is the Taylor start: the run
    equals a fresh simulation started from the state at that point."""
    g, mat, u0, v0 = _free_case("pmb2d")
    prec = _prec(pd, precision)
    rng = np.random.default_rng(31)
    u_x = u0 + 1e-7 * rng.standard_normal(u0.shape)
    v_x = v0 + 1e-3 * rng.standard_normal(v0.shape)
    a = gpu_sim(pd, g, mat, prec, integrator=pd.PD_INTEGRATOR_CD)
    pd.pd_set_state(a, u=u0, v=v0)
    pd.pd_step_explicit(a, 23)
    pd.pd_set_state(a, u=u_x, v=v_x)
    pd.pd_step_explicit(a, 30)
    b = gpu_sim(pd, g, mat, prec, integrator=pd.PD_INTEGRATOR_CD)
    pd.pd_set_state(b, u=u_x, v=v_x)
    pd.pd_step_explicit(b, 30)
    for x, y in zip(pd.pd_get_state(a), pd.pd_get_state(b)):
        assert np.array_equal(x, y)
    # a new dt: same rule (FP64, where a state read and write is exact)
    if precision == "fp64":
        dt2 = 0.7 * pd.pd_get_dt(a)
        pd.pd_set_dt(a, dt2)
        u_m, v_m = pd.pd_get_state(a)
        pd.pd_step_explicit(a, 25)
        c = gpu_sim(pd, g, mat, prec, dt=dt2, integrator=pd.PD_INTEGRATOR_CD)
        pd.pd_set_state(c, u=u_m, v=v_m)
        pd.pd_step_explicit(c, 25)
        for x, y in zip(pd.pd_get_state(a), pd.pd_get_state(c)):
            assert np.array_equal(x, y)
        c.close()
    a.close()
    b.close()


def test_unknown_integrator_is_rejected(pd):
    g, mat, _, _ = _free_case("pmb2d")
    for bad in (2, -1):
        gd, md, rd = pd.describe(g, mat, integrator=bad)
        with pytest.raises(pd.PdError) as e:
            pd.pd_create(gd, md, rd)
        assert e.value.code == pd.PD_EINVAL
    gd, md, rd = pd.describe(g, mat)
    rd.state = 2
    with pytest.raises(pd.PdError):
        pd.pd_create(gd, md, rd)


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_verlet_with_a_changed_time_step_matches_oracle(pd, precision):
    # pd_set_dt completes the pending half kick first, as the oracle's runs do
    g, mat, u0, v0 = _free_case("pmb3d")
    sim = gpu_sim(pd, g, mat, _prec(pd, precision))
    dt1 = pd.pd_get_dt(sim)
    dt2 = 0.6 * dt1
    pd.pd_set_state(sim, u=u0, v=v0)
    pd.pd_step_explicit(sim, 25)
    pd.pd_set_dt(sim, dt2)
    assert pd.pd_get_dt(sim) == dt2
    pd.pd_step_explicit(sim, 30)
    u_g, v_g = pd.pd_get_state(sim)
    st = O.ExplicitState(g, mat, O.neighbors(g), u0, v0)
    st.run(dt1, 25)
    st.run(dt2, 30)
    assert pd.pd_get_step(sim) == 55
    assert rel_l2(u_g, st.u) <= (U_TOL if precision == "fp32c" else 1e-10)
    assert rel_l2(v_g, st.v) <= (V_TOL if precision == "fp32c" else 1e-9)
    sim.close()
