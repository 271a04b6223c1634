"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Bars: neighbour lists, permutation and bond states bit-exact; FP64 GPU path
within round-off (1e-10 relative L2); FP32-compensated force within 1e-5
relative L2; displacement within 1e-4 relative L2 after a full run; broken-bond
sets equal except for bonds whose stretch lies within 1e-5 relative of s_c
(checked bond by bond against the oracle's per-bond records), and symmetric:
a bond is broken in both of its rows or in neither. "fp32c" is the FP32
compensated path with FP64 integrator state, "fp32c_df" the same with
double-float state.
Sizes span several tiles (8x8x8 bricks in 3D, 32x16 in 2D) and ragged edges.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_06917_gb300 import workloads as W
from tests.helpers import (assert_broken_match, broken_mates, gpu_csr_in_user_numbering, gpu_sim, oracle_pairs,
                           oracle_setup, rel_l2)

pytestmark = pytest.mark.gpu

FORCE_TOL_FP32C = 1e-5
U_TOL = 1e-4


@pytest.fixture(scope="module")
def pd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06917_gb300 import pd as _pd
    return _pd


GRIDS = [
    (2, (7, 5, 1), 2), (2, (13, 9, 1), 3), (2, (50, 50, 1), 3), (2, (70, 37, 1), 4),
    (3, (9, 7, 8), 3), (3, (10, 9, 9), 4), (3, (20, 20, 20), 3), (3, (37, 29, 11), 3), (3, (17, 9, 26), 2),
    (3, (1, 1, 1), 3), (2, (1, 3, 1), 1),
]


# ----------------------------------------------------------------- neighbours

@pytest.mark.parametrize("dim,n,m", GRIDS)
def test_neighbour_csr_and_morton_order_bit_exact(pd, dim, n, m):
    grid = W.Grid(dim=dim, n=n, h=0.01, m=m)
    mat = W.Material(model=W.PMB)
    sim = gpu_sim(pd, grid, mat, pd.PD_FP32C, dt=1e-7)
    rows_u, cols_u, _, (row_ptr, col, perm) = gpu_csr_in_user_numbering(pd, sim)
    assert np.array_equal(perm, O.morton_perm(grid))
    bonds = O.neighbors(grid, "brute" if grid.npoints <= 4000 else "cells")
    r_o, c_o = oracle_pairs(bonds)
    assert pd.pd_bond_count(sim) == bonds.nbonds
    assert np.array_equal(rows_u, r_o) and np.array_equal(cols_u, c_o)
    for r in range(min(grid.npoints, 2000)):                 # rows ascending in Morton numbering
        seg = col[row_ptr[r]:row_ptr[r + 1]]
        assert np.all(np.diff(seg) > 0)
    assert not pd.pd_get_broken(sim).any()
    sim.close()


def test_notch_bond_states_bit_exact(pd):
    wl = W.block3d_pulse(nside=20, steps=1)
    sim = gpu_sim(pd, wl.grid, wl.mat, pd.PD_FP32C, notch=wl.notch)
    bonds = oracle_setup(wl)
    _, _, order, _ = gpu_csr_in_user_numbering(pd, sim)
    brk = pd.pd_get_broken(sim)[order]
    assert brk.sum() > 0
    assert np.array_equal(brk, bonds.broken)
    sim.close()


# ------------------------------------------------------------------- forces

def _u_random(grid, scale, seed, translate=0.0):
    u = W.random_field(grid, scale * grid.h, seed)
    return u + translate


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("dim,n,m", [(2, (50, 50, 1), 3), (2, (70, 37, 1), 4), (3, (20, 20, 20), 3),
                                     (3, (37, 29, 11), 3), (3, (17, 9, 26), 2), (3, (12, 12, 12), 4)])
def test_pmb_force_matches_oracle(pd, precision, dim, n, m):
    grid = W.Grid(dim=dim, n=n, h=1.0 / 64, m=m)
    mat = W.Material(model=W.PMB, E=72e9)
    prec = pd.PD_FP32C if precision == "fp32c" else pd.PD_FP64
    sim = gpu_sim(pd, grid, mat, prec)
    bonds = O.neighbors(grid)
    # strain ~1e-4 plus a rigid translation of 0.3 m, which FP32 alone could not resolve
    u = _u_random(grid, 1e-4, seed=21, translate=0.3) + 1e-4 * grid.positions()
    f_gpu = pd.pd_force(sim, u=u)
    f_or = O.pmb_force(grid, mat, bonds, u)
    tol = FORCE_TOL_FP32C if precision == "fp32c" else 1e-10
    assert rel_l2(f_gpu, f_or) <= tol
    # the current state path (no u argument) gives the same as passing u
    pd.pd_set_state(sim, u=u)
    assert np.array_equal(pd.pd_force(sim), f_gpu)
    sim.close()


@pytest.mark.parametrize("vol_corr", [0, 1])
def test_pmb_partial_volume_matches_oracle(pd, vol_corr):
    grid = W.Grid(dim=3, n=(19, 18, 17), h=0.01, m=3)
    mat = W.Material(model=W.PMB, E=72e9, vol_corr=vol_corr)
    sim = gpu_sim(pd, grid, mat, pd.PD_FP32C)
    u = _u_random(grid, 3e-4, seed=3)
    assert rel_l2(pd.pd_force(sim, u=u), O.pmb_force(grid, mat, O.neighbors(grid), u)) <= FORCE_TOL_FP32C
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_pmb_breaking_matches_oracle(pd, precision):
    grid = W.Grid(dim=3, n=(18, 17, 16), h=0.01, m=3)
    s_c = 1e-3
    mat = W.Material(model=W.PMB, E=72e9, s_c=s_c)
    sim = gpu_sim(pd, grid, mat, precision)
    bonds = O.neighbors(grid)
    # stretches spread around s_c
    u = _u_random(grid, 1.2e-3, seed=9)
    f_gpu = pd.pd_force(sim, u=u, flags=pd.PD_FORCE_UPDATE_BREAKING)
    f_or = O.pmb_force(grid, mat, bonds, u, update_breaking=True)
    _, _, order, _ = gpu_csr_in_user_numbering(pd, sim)
    brk = pd.pd_get_broken(sim)[order].astype(bool)
    ob = bonds.broken.astype(bool)
    assert 0.05 < ob.mean() < 0.95
    # stretch of every bond (oracle arithmetic) to locate the ones near s_c
    X = grid.positions()
    r, c = oracle_pairs(bonds)
    xi = X[c] - X[r]
    y = xi + (u[c] - u[r])
    s = (np.linalg.norm(y, axis=1) - np.linalg.norm(xi, axis=1)) / np.linalg.norm(xi, axis=1)
    near = np.abs(s - s_c) <= 1e-5 * s_c
    assert np.array_equal(brk[~near], ob[~near])
    assert np.array_equal(brk, brk[broken_mates(bonds.row_ptr, bonds.col)])     # both rows agree
    if not near.any():
        assert rel_l2(f_gpu, f_or) <= (FORCE_TOL_FP32C if precision == "fp32c" else 1e-10)
    # the force is the oracle's with the GPU's bond states, near-s_c bonds included
    b2 = O.neighbors(grid)
    b2.broken[:] = brk
    assert rel_l2(f_gpu, O.pmb_force(grid, mat, b2, u)) <= (FORCE_TOL_FP32C if precision == "fp32c" else 1e-10)
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_break_decision_at_the_threshold_is_the_same_from_both_ends(pd, precision):
    """Displacements that put many bonds exactly at the edge of breaking: a
    rigid translation large against the strain (so that the per-tile staging
    of the two ends rounds differently) plus a uniform stretch of s_c along x.
    Every bond ends up broken in both of its rows or in neither."""
    grid = W.Grid(dim=3, n=(33, 18, 17), h=0.01, m=3)
    s_c = 1e-3
    mat = W.Material(model=W.PMB, E=72e9, s_c=s_c)
    sim = gpu_sim(pd, grid, mat, precision)
    X = grid.positions()
    u = np.zeros_like(X)
    u[:, 0] = s_c * X[:, 0] * (1.0 + 3e-9) + 0.37
    u += W.random_field(grid, 1e-9 * grid.h, seed=2)
    pd.pd_force(sim, u=u, flags=pd.PD_FORCE_UPDATE_BREAKING)
    row_ptr, col, _ = pd.pd_get_neighbors(sim)
    brk = pd.pd_get_broken(sim).astype(bool)
    assert 0 < brk.sum() < brk.size
    assert np.array_equal(brk, brk[broken_mates(row_ptr, col)])
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("n", [(20, 20, 20), (37, 29, 11)])
def test_lps_dilatation_and_force_match_oracle(pd, precision, n):
    grid = W.Grid(dim=3, n=n, h=1.0 / 128, m=3)
    mat = W.Material(model=W.LPS, K=40e9, mu=30e9)
    prec = pd.PD_FP32C if precision == "fp32c" else pd.PD_FP64
    sim = gpu_sim(pd, grid, mat, prec)
    bonds = O.neighbors(grid)
    mv = O.weighted_volume(grid, mat, bonds)
    u = (1e-4 / 3) * grid.positions() + _u_random(grid, 1e-5, seed=3, translate=0.2)
    th_gpu = pd.pd_dilatation(sim, u=u)
    th_or = O.dilatation(grid, mat, bonds, mv, u)
    f_gpu = pd.pd_force(sim, u=u)
    f_or = O.lps_force(grid, mat, bonds, mv, th_or, u)
    tol = FORCE_TOL_FP32C if precision == "fp32c" else 1e-10
    assert rel_l2(th_gpu, th_or) <= tol
    assert rel_l2(f_gpu, f_or) <= tol
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_lps_partial_volume_matches_oracle(pd, precision):
    # V_ij enters the weighted volume, the dilatation and the force pass
    grid = W.Grid(dim=3, n=(21, 19, 18), h=1.0 / 128, m=3)
    mat = W.Material(model=W.LPS, K=40e9, mu=30e9, vol_corr=1)
    sim = gpu_sim(pd, grid, mat, pd.PD_FP32C if precision == "fp32c" else pd.PD_FP64)
    bonds = O.neighbors(grid)
    mv = O.weighted_volume(grid, mat, bonds)
    u = (1e-4 / 3) * grid.positions() + _u_random(grid, 1e-5, seed=4, translate=0.1)
    th_or = O.dilatation(grid, mat, bonds, mv, u)
    tol = FORCE_TOL_FP32C if precision == "fp32c" else 1e-10
    assert rel_l2(pd.pd_dilatation(sim, u=u), th_or) <= tol
    assert rel_l2(pd.pd_force(sim, u=u), O.lps_force(grid, mat, bonds, mv, th_or, u)) <= tol
    sim.close()


# ---------------------------------------------------------------- explicit

def _run_both(pd, wl, precision, steps, dt=None):
    """The workload run on the GPU and by the oracle (with per-bond records)."""
    sim = gpu_sim(pd, wl.grid, wl.mat, precision, notch=wl.notch)
    bonds = oracle_setup(wl)
    dt_o = wl.dt_factor * O.stable_dt(wl.grid, wl.mat, bonds)
    assert abs(pd.pd_get_dt(sim) - dt_o) <= 1e-12 * dt_o
    pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
    if wl.bc_kind is not None and wl.bc_kind.any():
        pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val)
    pd.pd_step_explicit(sim, steps)
    u_g, v_g = pd.pd_get_state(sim)
    st = O.ExplicitState(wl.grid, wl.mat, bonds, wl.u0, wl.v0, wl.bc_kind, wl.bc_val,
                         track=wl.mat.s_c > 0)
    st.run(dt_o, steps)
    return sim, bonds, st, u_g, v_g


def _gpu_broken_user(pd, sim):
    """The GPU's bond states in the oracle's CSR order (user numbering), and
    whether they are symmetric (both rows of every bond agree)."""
    _, _, order, (row_ptr, col, _) = gpu_csr_in_user_numbering(pd, sim)
    raw = pd.pd_get_broken(sim).astype(bool)
    symmetric = bool(np.array_equal(raw, raw[broken_mates(row_ptr, col)]))
    return raw[order], symmetric


@pytest.mark.parametrize("precision", ["fp32c", "fp32c_df", "fp64"])
def test_plate2d_explicit_run_matches_oracle(pd, precision):
    """50 x 50 plate, PMB, collar velocities, 200 steps (the plain-method workload)."""
    wl = W.plate2d(nside=50, steps=200)
    sim, _, st, u_g, v_g = _run_both(pd, wl, precision, wl.steps)
    fp64 = precision == "fp64"
    assert rel_l2(u_g, st.u) <= (1e-10 if fp64 else U_TOL)
    assert rel_l2(v_g, st.v) <= (1e-9 if fp64 else 1e-3)
    assert pd.pd_get_step(sim) == wl.steps
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp32c_df", "fp64"])
def test_block_pulse_with_breaking_matches_oracle(pd, precision):
    """Pulse + pre-notch + breaking (s_c lowered so bonds break within the run)."""
    wl = W.block3d_pulse(nside=24, steps=120, s_c=5e-5)
    sim, bonds, st, u_g, v_g = _run_both(pd, wl, precision, wl.steps)
    brk, symmetric = _gpu_broken_user(pd, sim)
    notch_only = oracle_setup(wl).broken.astype(bool)
    assert bonds.broken.sum() > notch_only.sum() + 100          # bonds broke during the run
    assert symmetric
    assert_broken_match(brk, bonds, st, wl.mat.s_c)
    fp64 = precision == "fp64"
    assert rel_l2(u_g, st.u) <= (1e-9 if fp64 else U_TOL)
    assert rel_l2(v_g, st.v) <= (1e-8 if fp64 else 1e-3)
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp32c_df"])
def test_lps_explicit_run_matches_oracle(pd, precision):
    wl = W.block3d_lps(nside=24, steps=40)
    sim, _, st, u_g, v_g = _run_both(pd, wl, precision, wl.steps)
    assert rel_l2(u_g, st.u) <= U_TOL
    assert rel_l2(v_g - wl.v0, st.v - wl.v0) <= 1e-3
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp32c_df"])
def test_graph_replay_equals_single_steps_and_runs_are_deterministic(pd, precision):
    wl = W.block3d_pulse(nside=16, steps=40, s_c=5e-5)
    outs = []
    for chunks in ([40], [1] * 40, [40]):
        sim = gpu_sim(pd, wl.grid, wl.mat, precision, notch=wl.notch)
        pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
        for c in chunks:
            pd.pd_step_explicit(sim, c)
        outs.append(pd.pd_get_state(sim))
        outs[-1] = (outs[-1][0], outs[-1][1], pd.pd_get_broken(sim))
        sim.close()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp32c", "fp32c_df"])
def test_checkpoint_round_trip_is_bit_identical(pd, precision):
    wl = W.plate2d(nside=40, steps=60)
    ref = gpu_sim(pd, wl.grid, wl.mat, precision)
    pd.pd_set_state(ref, u=wl.u0, v=wl.v0)
    pd.pd_set_bc(ref, wl.bc_kind, wl.bc_val)
    pd.pd_step_explicit(ref, 60)
    u_ref, v_ref = pd.pd_get_state(ref)
    sim = gpu_sim(pd, wl.grid, wl.mat, precision)
    pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
    pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val)
    pd.pd_step_explicit(sim, 30)
    u_mid, v_mid = pd.pd_get_state(sim)
    pd.pd_set_state(sim, u=u_mid, v=v_mid)
    pd.pd_step_explicit(sim, 30)
    u_end, v_end = pd.pd_get_state(sim)
    assert np.array_equal(u_end, u_ref) and np.array_equal(v_end, v_ref)
    ref.close()
    sim.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp32c_df"])
def test_reading_u_alone_leaves_the_trajectory_unchanged(pd, precision):
    # a u-only read skips the completing half kick; steps after it, and the full
    # read at the end, must be bit-identical to a run without intermediate reads
    wl = W.block3d_pulse(nside=16, steps=30, s_c=5e-5)
    outs = []
    for read_every in (0, 1, 7):
        sim = gpu_sim(pd, wl.grid, wl.mat, precision, notch=wl.notch)
        pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
        us = []
        for k in range(30):
            pd.pd_step_explicit(sim, 1)
            if read_every and k % read_every == 0:
                u, v = pd.pd_get_state(sim, want_v=False)
                assert v is None
                us.append((k, u))
        outs.append(pd.pd_get_state(sim))
        outs[-1] = (outs[-1][0], outs[-1][1], pd.pd_get_broken(sim), us)
        sim.close()
    for o in outs[1:]:
        for a, b in zip(outs[0][:3], o[:3]):
            assert np.array_equal(a, b)
    # the intermediate u reads agree between the two read patterns where both read
    k1 = dict(outs[1][3])
    for k, u in outs[2][3]:
        assert np.array_equal(u, k1[k])


def test_replacing_the_state_mid_run_equals_a_fresh_start(pd):
    # pd_set_state(u, v) while v sits at a half step must discard that half step
    wl = W.plate2d(nside=30, steps=20)
    rng = np.random.default_rng(11)
    u_x = wl.u0 + 1e-7 * rng.standard_normal(wl.u0.shape)
    v_x = wl.v0 + 1e-3 * rng.standard_normal(wl.v0.shape)
    a = gpu_sim(pd, wl.grid, wl.mat, pd.PD_FP32C)
    pd.pd_set_state(a, u=wl.u0, v=wl.v0)
    pd.pd_step_explicit(a, 13)
    pd.pd_set_state(a, u=u_x, v=v_x)
    pd.pd_step_explicit(a, 20)
    b = gpu_sim(pd, wl.grid, wl.mat, pd.PD_FP32C)
    pd.pd_set_state(b, u=u_x, v=v_x)
    pd.pd_step_explicit(b, 20)
    for x, y in zip(pd.pd_get_state(a), pd.pd_get_state(b)):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def test_energy_matches_oracle_and_is_conserved(pd):
    grid = W.Grid(dim=2, n=(40, 40, 1), h=0.02, m=3)
    mat = W.Material(model=W.PMB, E=72e9, rho=2440.0)
    u0 = W.gaussian_ic(grid, (1e-5, 0.5e-5), (0.4, 0.35), 0.003)
    sim = gpu_sim(pd, grid, mat, pd.PD_FP64)
    pd.pd_set_state(sim, u=u0, v=np.zeros_like(u0))
    bonds = O.neighbors(grid)
    k0, s0 = pd.pd_energy(sim)
    assert k0 == 0.0
    assert abs(s0 - O.strain_energy(grid, mat, bonds, u0)) <= 1e-10 * s0
    pd.pd_step_explicit(sim, 100)
    u, v = pd.pd_get_state(sim)
    k1, s1 = pd.pd_energy(sim)
    assert abs(k1 - O.kinetic_energy(grid, mat, v)) <= 1e-10 * k1
    assert abs(s1 - O.strain_energy(grid, mat, bonds, u)) <= 1e-9 * s1
    assert abs((k1 + s1) - s0) <= 3e-2 * s0
    assert pd.pd_energy(sim) == (k1, s1)                 # bit-reproducible
    sim.close()


def test_lps_energy_matches_oracle(pd):
    grid = W.Grid(dim=3, n=(14, 13, 12), h=0.01, m=3)
    mat = W.Material(model=W.LPS, K=40e9, mu=30e9)
    sim = gpu_sim(pd, grid, mat, pd.PD_FP64)
    u = _u_random(grid, 2e-4, seed=4)
    pd.pd_set_state(sim, u=u)
    bonds = O.neighbors(grid)
    mv = O.weighted_volume(grid, mat, bonds)
    th = O.dilatation(grid, mat, bonds, mv, u)
    _, s = pd.pd_energy(sim)
    assert abs(s - O.strain_energy(grid, mat, bonds, u, mv, th)) <= 1e-9 * s
    sim.close()


# ------------------------------------------------------------------ tangent

@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_jvp_vjp_match_assembled_tangent(pd, precision):
    """20 x 20 sub-grid: K from Algorithm 3's central differences in the oracle."""
    grid = W.Grid(dim=2, n=(20, 20, 1), h=0.005, m=3)
    mat = W.Material(model=W.PMB, E=72e9)
    prec = pd.PD_FP32C if precision == "fp32c" else pd.PD_FP64
    sim = gpu_sim(pd, grid, mat, prec)
    bonds = O.neighbors(grid)
    u = _u_random(grid, 2e-3, seed=4)
    K = O.tangent_fd(grid, mat, bonds, u, 1e-6 * grid.h)
    w = W.random_field(grid, 1.0, seed=5)
    jv = pd.pd_jvp(sim, w, u_lin=u)
    vj = pd.pd_vjp(sim, w, u_lin=u)
    tol = 1e-6 if precision == "fp64" else 2e-5
    assert rel_l2(jv.ravel(), K @ w.ravel()) <= tol
    assert rel_l2(vj.ravel(), K.T @ w.ravel()) <= tol
    # central differences of the GPU's own force along w
    eps = 1e-6 * grid.h
    fd = O.jvp_fd(grid, mat, bonds, u, w, eps)
    assert rel_l2(jv, fd) <= tol
    sim.close()


def test_jvp_dirichlet_mask_and_rigid_null_space(pd):
    grid = W.Grid(dim=3, n=(12, 11, 10), h=0.01, m=3)
    mat = W.Material(model=W.PMB, E=72e9)
    sim = gpu_sim(pd, grid, mat, pd.PD_FP64)
    X = grid.positions()
    zero = np.zeros((grid.npoints, 3))
    scale = np.abs(pd.pd_jvp(sim, W.random_field(grid, 1.0, seed=1), u_lin=zero)).max()
    for w in (np.tile([1.0, -2.0, 0.5], (grid.npoints, 1)), np.stack([-X[:, 1], X[:, 0], 0 * X[:, 0]], 1)):
        assert np.abs(pd.pd_jvp(sim, w, u_lin=zero)).max() <= 1e-10 * scale * np.abs(w).max() / grid.h
    kind = np.zeros((grid.npoints, 3), np.uint8)
    kind[W.collar_mask(grid, 0, -1)] = pd.PD_BC_DISPLACEMENT
    pd.pd_set_bc(sim, kind, np.zeros((grid.npoints, 3)))
    w = W.random_field(grid, 1.0, seed=2)
    out = pd.pd_jvp(sim, w, u_lin=zero, flags=pd.PD_JVP_MASK_DIRICHLET)
    fixed = kind.astype(bool)
    assert np.array_equal(out[fixed], w[fixed])
    w2 = w.copy()
    w2[fixed] = 0.0
    ref = pd.pd_jvp(sim, w2, u_lin=zero)
    assert np.array_equal(out[~fixed], ref[~fixed])
    sim.close()


# ------------------------------------------------------- full-size sampled

def test_full_size_block64_force_and_short_run(pd):
    """64^3 PMB with breaking at the benchmark's configuration: the force of the
    whole lattice after 5 steps against the oracle, and the broken set."""
    wl = W.block3d_pulse(nside=64, steps=5)
    sim, bonds, st, u_g, v_g = _run_both(pd, wl, pd.PD_FP32C, wl.steps)
    assert rel_l2(u_g, st.u) <= U_TOL
    f_gpu = pd.pd_force(sim, u=st.u)
    f_or = O.pmb_force(wl.grid, wl.mat, bonds, st.u)
    assert rel_l2(f_gpu, f_or) <= FORCE_TOL_FP32C
    sim.close()


def test_full_size_block64_full_run(pd):
    """The 64^3 benchmark workload over its full 1000 fused steps (the pulse
    reaches the faces and reflects) against the oracle's run: u, v and the bond
    states by the near-s_c rule, bond by bond."""
    wl = W.block3d_pulse(nside=64)
    assert wl.steps == 1000
    sim, bonds, st, u_g, v_g = _run_both(pd, wl, "fp32c", wl.steps)
    assert rel_l2(u_g, st.u) <= U_TOL
    assert rel_l2(v_g, st.v) <= 1e-3
    brk, symmetric = _gpu_broken_user(pd, sim)
    assert symmetric
    assert_broken_match(brk, bonds, st, wl.mat.s_c)
    sim.close()


def test_full_size_block128_lps_full_run(pd):
    """The 128^3 LPS workload over its full 500 steps (two launches each)
    against the oracle (about 5 minutes of oracle time on 16 host cores)."""
    wl = W.block3d_lps(nside=128)
    assert wl.steps == 500
    sim, _, st, u_g, v_g = _run_both(pd, wl, "fp32c", wl.steps)
    assert rel_l2(u_g, st.u) <= U_TOL
    assert rel_l2(v_g - wl.v0, st.v - wl.v0) <= 1e-3
    sim.close()


def test_full_size_block128_lps_force_sampled(pd):
    """128^3 LPS: the force at the initial state on the whole lattice."""
    wl = W.block3d_lps(nside=128, steps=1)
    sim = gpu_sim(pd, wl.grid, wl.mat, pd.PD_FP32C)
    bonds = O.neighbors(wl.grid)
    mv = O.weighted_volume(wl.grid, wl.mat, bonds)
    th = O.dilatation(wl.grid, wl.mat, bonds, mv, wl.u0)
    f_or = O.lps_force(wl.grid, wl.mat, bonds, mv, th, wl.u0)
    f_gpu = pd.pd_force(sim, u=wl.u0)
    assert rel_l2(f_gpu, f_or) <= FORCE_TOL_FP32C
    sim.close()


# --------------------------------------------------------------- edge cases

def test_errors_are_reported_not_faulted(pd):
    grid = W.Grid(dim=2, n=(4, 4, 1), h=0.01, m=2)
    g, m, r = pd.describe(grid, W.Material(model=W.LPS, K=1e9, mu=1e9))
    with pytest.raises(pd.PdError) as e:
        pd.pd_create(g, m, r)
    assert e.value.code == pd.PD_EINVAL
    g, m, r = pd.describe(grid, W.Material(model=W.PMB))
    sim = pd.pd_create(g, m, r)
    with pytest.raises(pd.PdError) as e:
        pd.pd_force(sim, u=np.zeros((16, 2)))
    assert e.value.code == pd.PD_ESTATE
    pd.pd_build_neighbors(sim)
    with pytest.raises(pd.PdError):
        pd.pd_set_bc(sim, np.full((16, 2), 7, np.uint8), np.zeros((16, 2)))
    with pytest.raises(pd.PdError):
        pd.pd_step_explicit(sim, -1)
    sim.close()


def test_single_point_and_torch_device_buffers(pd):
    import torch
    grid = W.Grid(dim=3, n=(1, 1, 1), h=0.01, m=3)
    sim = gpu_sim(pd, grid, W.Material(model=W.PMB), pd.PD_FP32C, dt=1e-6)
    assert pd.pd_bond_count(sim) == 0
    assert np.all(pd.pd_force(sim, u=np.ones((1, 3))) == 0)
    sim.close()
    grid = W.Grid(dim=3, n=(16, 16, 16), h=0.01, m=3)
    mat = W.Material(model=W.PMB)
    sim = gpu_sim(pd, grid, mat, pd.PD_FP32C)
    u = _u_random(grid, 1e-4, seed=7)
    ud = torch.from_numpy(u).cuda()
    fd = torch.empty_like(ud)
    pd.pd_force(sim, u=ud, f_out=fd, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(fd.cpu().numpy(), pd.pd_force(sim, u=u))
    sim.close()


@pytest.mark.parametrize("tile_log2,m", [(7, 3), (6, 2), (8, 4)])
def test_lps_small_tiles_match_oracle(pd, tile_log2, m):
    """Tiles other than 2^9 points (the FP32C force pass then runs 2^L threads)."""
    grid = W.Grid(dim=3, n=(21, 18, 17), h=1.0 / 128, m=m)
    mat = W.Material(model=W.LPS, K=40e9, mu=30e9)
    sim = gpu_sim(pd, grid, mat, pd.PD_FP32C, tile_log2=tile_log2)
    bonds = O.neighbors(grid)
    mv = O.weighted_volume(grid, mat, bonds)
    u = (1e-4 / 3) * grid.positions() + _u_random(grid, 1e-5, seed=5)
    th = O.dilatation(grid, mat, bonds, mv, u)
    assert rel_l2(pd.pd_force(sim, u=u), O.lps_force(grid, mat, bonds, mv, th, u)) <= FORCE_TOL_FP32C
    sim.close()


@pytest.mark.parametrize("tile_log2", [6, 7, 8])
def test_pmb_small_tiles_match_oracle(pd, tile_log2):
    grid = W.Grid(dim=3, n=(21, 18, 17), h=0.01, m=3)
    mat = W.Material(model=W.PMB, E=72e9, s_c=1e-3)
    sim = gpu_sim(pd, grid, mat, pd.PD_FP32C, tile_log2=tile_log2)
    u = _u_random(grid, 3e-4, seed=6)
    f = pd.pd_force(sim, u=u)
    assert rel_l2(f, O.pmb_force(grid, mat, O.neighbors(grid), u)) <= FORCE_TOL_FP32C
    sim.close()


LARGE_HORIZONS = [
    (2, (60, 41, 1), 12, W.PMB), (2, (45, 38, 1), 8, W.NP), (3, (14, 13, 12), 6, W.PMB),
    (3, (13, 12, 11), 5, W.LPS), (3, (12, 11, 10), 7, W.PMB),
    (2, (90, 77, 1), 20, W.NP), (2, (83, 70, 1), 20, W.PMB), (2, (75, 71, 1), 20, W.LP),
]


@pytest.mark.parametrize("dim,n,m,model", LARGE_HORIZONS)
@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_large_horizons_match_oracle(pd, dim, n, m, model, precision):
    # wide stencils (up to 1436 offsets, 45 mask words): neighbour build, the
    # automatic tile shrink of the shared-memory halo, and the force kernels
    g = W.Grid(dim=dim, n=n, h=0.01, m=m)
    mat = {W.PMB: W.Material(model=W.PMB), W.NP: W.Material(model=W.NP, rho=1.0, psi_beta=2.0),
           W.LP: W.Material(model=W.LP, rho=1.0, psi_beta=2.0),
           W.LPS: W.Material(model=W.LPS, K=40e9, mu=30e9)}[model]
    bonds = O.neighbors(g)
    rng = np.random.default_rng(m)
    u = rng.normal(0.0, 1e-3 * g.h, (g.npoints, dim))
    if model in (W.NP, W.LP):
        u = rng.normal(0.0, 0.2 * g.h, (g.npoints, dim))
    prec = pd.PD_FP32C if precision == "fp32c" else pd.PD_FP64
    sim = gpu_sim(pd, g, mat, prec)
    assert pd.pd_bond_count(sim) == bonds.nbonds
    f_o, _ = O.internal_force(g, mat, bonds, u, O.weighted_volume(g, mat, bonds) if model == W.LPS else None)
    f_g = pd.pd_force(sim, u=u)
    assert rel_l2(f_g, f_o) <= (FORCE_TOL_FP32C if precision == "fp32c" else 1e-10)
    sim.close()


def test_paper_benchmark_shape_full_size(pd):
    """The explicit benchmark shape of Sec. 6.2 at full size (443^2 nodes, m = 20,
    237,103,580 bonds, NP law, clamped collar): the force at u0 against the
    oracle, then 3 steps, compared by the displacement increment u - u0."""
    wl = W.np_benchmark(steps=3)
    sim = gpu_sim(pd, wl.grid, wl.mat, pd.PD_FP32C, dt=wl.dt)
    bonds = O.neighbors(wl.grid)
    assert pd.pd_bond_count(sim) == bonds.nbonds == 237103580
    f_o, _ = O.internal_force(wl.grid, wl.mat, bonds, wl.u0, None)
    f_g = pd.pd_force(sim, u=wl.u0)
    assert rel_l2(f_g, f_o) <= FORCE_TOL_FP32C
    pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
    pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val)
    pd.pd_step_explicit(sim, wl.steps)
    u_g, _ = pd.pd_get_state(sim)
    st = O.ExplicitState(wl.grid, wl.mat, bonds, wl.u0, wl.v0, wl.bc_kind, wl.bc_val)
    st.run(wl.dt, wl.steps)
    assert np.abs(st.u - wl.u0).max() > 0
    assert rel_l2(u_g - wl.u0, st.u - wl.u0) <= U_TOL
    sim.close()


@pytest.mark.parametrize("m,amp", [(12, 0.3), (20, 0.2)])
def test_wide_horizon_breaking_run_matches_oracle(pd, m, amp):
    """A 2D run with bonds breaking at m = 12 and m = 20, where the fused kernel
    splits each point pair's stencil words over 2 and 4 threads."""
    g = W.Grid(dim=2, n=(70, 61, 1), h=0.01, m=m)
    mat = W.Material(model=W.PMB, E=72e9, rho=2440.0, s_c=2e-5, thickness=1.0)
    X = g.positions()
    r2 = ((X - X.mean(axis=0)) ** 2).sum(axis=1)
    v0 = np.zeros((g.npoints, 2))
    v0[:, 0] = amp * np.exp(-r2 / (0.08 ** 2))       # 0.7 % / 0.2 % of the bonds break
    u0 = np.zeros_like(v0)
    sim = gpu_sim(pd, g, mat, pd.PD_FP32C)
    bonds = O.neighbors(g)
    pd.pd_set_state(sim, u=u0, v=v0)
    steps = 40
    pd.pd_step_explicit(sim, steps)
    u_g, v_g = pd.pd_get_state(sim)
    st = O.ExplicitState(g, mat, bonds, u0, v0, None, None, track=True)
    st.run(pd.pd_get_dt(sim), steps)
    brk, symmetric = _gpu_broken_user(pd, sim)
    assert bonds.broken.sum() > 0
    assert symmetric
    assert_broken_match(brk, bonds, st, mat.s_c)
    assert rel_l2(u_g, st.u) <= U_TOL
    assert rel_l2(v_g, st.v) <= 1e-3
    sim.close()
