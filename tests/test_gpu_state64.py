"""The FP32-compensated path's integrator state: FP64 (PD_STATE_F64, the
default) against double-float (PD_STATE_DF) and the oracle, the staging split
of a large FP64 displacement, and the timed stepping entry point."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_06917_gb300 import workloads as W
from tests.helpers import gpu_sim, oracle_setup, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06917_gb300 import pd as _pd
    return _pd


@pytest.mark.parametrize("model", [W.PMB, W.LPS])
def test_large_rigid_offset_is_staged_to_full_precision(pd, model):
    """A 0.37 m rigid offset on top of a strain of order 1e-4: the update splits
    the FP64 u into the FP32 staging pair at every step; with only the high
    FP32 word (2^-24 of 0.37 m against displacement differences of 1e-6 m)
    the stretch would be wrong at the 1e-2 level. The displacement increment
    u - u0 matches the oracle's over 30 steps."""
    if model == W.LPS:
        wl = W.block3d_lps(nside=20, steps=30)
    else:
        wl = W.block3d_pulse(nside=20, steps=30, s_c=0.0)
    u0 = wl.u0 + np.array([0.37, -0.21, 0.55])
    sim = gpu_sim(pd, wl.grid, wl.mat, "fp32c", notch=wl.notch)
    bonds = oracle_setup(wl)
    pd.pd_set_state(sim, u=u0, v=wl.v0)
    pd.pd_step_explicit(sim, wl.steps)
    u_g, v_g = pd.pd_get_state(sim)
    st = O.ExplicitState(wl.grid, wl.mat, bonds, u0, wl.v0)
    st.run(pd.pd_get_dt(sim), wl.steps)
    assert rel_l2(u_g - u0, st.u - u0) <= 1e-4
    assert rel_l2(v_g - wl.v0, st.v - wl.v0) <= 1e-3
    sim.close()


@pytest.mark.parametrize("name", ["pulse", "lps"])
def test_fp64_and_double_float_state_agree(pd, name):
    wl = W.block3d_pulse(nside=24, steps=100) if name == "pulse" else W.block3d_lps(nside=24, steps=100)
    out = []
    for prec in ("fp32c", "fp32c_df"):
        sim = gpu_sim(pd, wl.grid, wl.mat, prec, notch=wl.notch)
        pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
        pd.pd_step_explicit(sim, wl.steps)
        out.append(pd.pd_get_state(sim))
        sim.close()
    (u1, v1), (u2, v2) = out
    assert rel_l2(u2, u1) <= 1e-6
    assert rel_l2(v2 - wl.v0, v1 - wl.v0) <= 1e-5


@pytest.mark.parametrize("name,prec", [("lps", "fp32c"), ("pulse", "fp32c"), ("pulse", "fp32c_df"),
                                       ("pulse", "fp64")])
def test_timed_steps_follow_the_same_trajectory(pd, name, prec):
    """pd_step_explicit_timed: the same trajectory (bit for bit) as
    pd_step_explicit, with positive per-pass device times (two passes for LPS)."""
    wl = W.block3d_pulse(nside=16, steps=20, s_c=5e-5) if name == "pulse" else W.block3d_lps(nside=16, steps=20)
    res = []
    for timed in (False, True):
        sim = gpu_sim(pd, wl.grid, wl.mat, prec, notch=wl.notch)
        pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
        if timed:
            t0, t1 = pd.pd_step_explicit_timed(sim, wl.steps)
            assert t0 > 0 and ((t1 > 0) if name == "lps" else t1 == 0.0)
        else:
            pd.pd_step_explicit(sim, wl.steps)
        assert pd.pd_get_step(sim) == wl.steps
        res.append(pd.pd_get_state(sim) + (pd.pd_get_broken(sim),))
        sim.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)
