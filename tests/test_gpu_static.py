"""GPU: the matrix-free Newton-Krylov static solve (pd_solve_static) and the
autograd bridge, through the C ABI, against the FP64 oracle of the implicit
scheme (Newton with the central-difference stiffness of Eq. (6) / Algorithm 3
and LU) and against properties that hold at any size: the oracle's own
residual at the GPU solution, mirror symmetry, and the uniaxial-stress
continuum solution (CCM) on the roller-loaded plate.

Bars: FP64 solution within 1e-9 relative L2 of the oracle's; FP32-compensated
(FP32 tangent, inexact Newton) within 1e-5; torch.autograd.gradcheck in FP64.
"""
import numpy as np
import pytest

from oracle import implicit as I
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


def _static_sim(pd, L, precision, scale=1.0):
    g = L.grid
    sim = gpu_sim(pd, g, L.mat, precision)
    z = np.zeros((g.npoints, g.dim))
    pd.pd_set_state(sim, u=z, v=z)
    pd.pd_set_bc(sim, L.bc_kind, scale * L.bc_val)
    return sim


@pytest.mark.parametrize("variant,nx,ny", [("roller", 40, 20), ("clamped", 37, 22)])
@pytest.mark.parametrize("krylov", ["gmres", "cg"])
@pytest.mark.parametrize("tangent", ["cached", "jvp"])
def test_fp64_static_solve_matches_oracle_newton(pd, variant, nx, ny, krylov, tangent):
    L = W.plate_static(nx=nx, ny=ny, strain=1e-4, variant=variant)
    g = L.grid
    u_o, _, ok = I.solve_static(g, L.mat, O.neighbors(g), np.zeros((g.npoints, 2)), L.bc_kind, L.bc_val)
    assert ok
    sim = _static_sim(pd, L, pd.PD_FP64)
    kr = pd.PD_KRYLOV_GMRES if krylov == "gmres" else pd.PD_KRYLOV_CG
    tg = pd.PD_TANGENT_CACHED if tangent == "cached" else pd.PD_TANGENT_JVP
    st = pd.pd_solve_static(sim, pd.newton_opts(krylov=kr, linear_rtol=1e-12, newton_rtol=1e-12, tangent=tg))
    assert st["converged"] == 1 and st["linear_failures"] == 0
    u, v = pd.pd_get_state(sim)
    assert rel_l2(u, u_o) <= 1e-9
    assert not v.any()
    sim.close()


@pytest.mark.parametrize("restart", [3, 13, 50])
def test_gmres_restarts_off_the_chunk_size_match_oracle(pd, restart):
    # the device-side Arnoldi runs in chunks of 8 steps: restart lengths below,
    # between and above that, with several restart cycles per solve
    L = W.plate_static(nx=31, ny=17, strain=1e-4, variant="clamped")
    g = L.grid
    u_o, _, ok = I.solve_static(g, L.mat, O.neighbors(g), np.zeros((g.npoints, 2)), L.bc_kind, L.bc_val)
    assert ok
    sim = _static_sim(pd, L, pd.PD_FP64)
    st = pd.pd_solve_static(sim, pd.newton_opts(krylov=pd.PD_KRYLOV_GMRES, restart=restart, max_linear_iters=20000,
                                                linear_rtol=1e-12, newton_rtol=1e-12))
    assert st["converged"] == 1 and st["linear_failures"] == 0
    u, _ = pd.pd_get_state(sim)
    assert rel_l2(u, u_o) <= 1e-9
    sim.close()


@pytest.mark.parametrize("krylov,limit", [("gmres", 37), ("cg", 45)])
def test_linear_iteration_limits_are_exact(pd, krylov, limit):
    # a limit that ends inside a chunk of device-side iterations: each Newton
    # step's linear solve stops after exactly `limit` iterations
    L = W.plate_static(nx=40, ny=20, strain=1e-4, variant="clamped")
    sim = _static_sim(pd, L, pd.PD_FP64)
    kr = pd.PD_KRYLOV_GMRES if krylov == "gmres" else pd.PD_KRYLOV_CG
    st = pd.pd_solve_static(sim, pd.newton_opts(krylov=kr, restart=50, max_linear_iters=limit, max_newton_iters=2,
                                                linear_rtol=1e-14, newton_rtol=1e-14))
    assert st["newton_iters"] == 2
    assert st["linear_iters"] == 2 * limit and st["linear_failures"] == 2
    assert st["converged"] == 0
    sim.close()


@pytest.mark.parametrize("krylov", ["gmres", "cg"])
def test_block_jacobi_preconditioned_solves_match_oracle(pd, krylov):
    # the lattice operator's diagonal blocks are nearly uniform (they change only
    # near the free edges), so block-Jacobi is not expected to cut iterations
    # here; it must give the same root and not cost many more iterations
    L = W.plate_static(nx=60, ny=30, strain=1e-4, variant="roller")
    g = L.grid
    u_o, _, ok = I.solve_static(g, L.mat, O.neighbors(g), np.zeros((g.npoints, 2)), L.bc_kind, L.bc_val)
    assert ok
    kr = pd.PD_KRYLOV_GMRES if krylov == "gmres" else pd.PD_KRYLOV_CG
    iters = {}
    for pc in (pd.PD_PRECOND_NONE, pd.PD_PRECOND_BLOCK_JACOBI):
        sim = _static_sim(pd, L, pd.PD_FP64)
        st = pd.pd_solve_static(sim, pd.newton_opts(krylov=kr, linear_rtol=1e-12, newton_rtol=1e-12, precond=pc))
        assert st["converged"] == 1 and st["linear_failures"] == 0
        u, _ = pd.pd_get_state(sim)
        assert rel_l2(u, u_o) <= 1e-9
        iters[pc] = st["linear_iters"]
        sim.close()
    assert iters[pd.PD_PRECOND_BLOCK_JACOBI] <= 1.2 * iters[pd.PD_PRECOND_NONE]


def test_block_jacobi_needs_the_cached_tangent(pd):
    L = W.plate_static(nx=20, ny=10, variant="clamped")
    sim = _static_sim(pd, L, pd.PD_FP64)
    for bad in (pd.newton_opts(precond=pd.PD_PRECOND_BLOCK_JACOBI, tangent=pd.PD_TANGENT_JVP),
                pd.newton_opts(precond=9)):
        with pytest.raises(pd.PdError) as e:
            pd.pd_solve_static(sim, bad)
        assert e.value.code == pd.PD_EINVAL
    sim.close()


@pytest.mark.parametrize("tangent", ["cached", "jvp"])
def test_fp32c_static_solve_is_an_inexact_newton_to_the_same_root(pd, tangent):
    L = W.plate_static(nx=40, ny=20, strain=1e-4, variant="roller")
    g = L.grid
    u_o, _, _ = I.solve_static(g, L.mat, O.neighbors(g), np.zeros((g.npoints, 2)), L.bc_kind, L.bc_val)
    sim = _static_sim(pd, L, pd.PD_FP32C)
    tg = pd.PD_TANGENT_CACHED if tangent == "cached" else pd.PD_TANGENT_JVP
    st = pd.pd_solve_static(sim, pd.newton_opts(krylov=pd.PD_KRYLOV_CG, linear_rtol=1e-6, newton_rtol=1e-6,
                                                max_newton_iters=12, tangent=tg))
    assert st["converged"] == 1
    u, _ = pd.pd_get_state(sim)
    assert rel_l2(u, u_o) <= 1e-5
    sim.close()


def test_config4_load_path_gmres50_converges_and_satisfies_the_oracle_residual(pd):
    # 200 x 200 plate, left collar clamped, right collar pulled to strain 1e-4
    # in 10 load steps; GMRES(50), linear rtol 1e-8, FP64 tangent
    L = W.plate_static(nx=200, variant="clamped")
    g = L.grid
    sim = _static_sim(pd, L, pd.PD_FP64, scale=0.0)
    opts = pd.newton_opts(krylov=pd.PD_KRYLOV_GMRES, restart=50, linear_rtol=1e-8, newton_rtol=1e-8)
    for s in range(1, L.load_steps + 1):
        pd.pd_set_bc(sim, L.bc_kind, L.bc_val * s / L.load_steps)
        st = pd.pd_solve_static(sim, opts)
        assert st["converged"] == 1 and st["linear_failures"] == 0, (s, st)
    u, _ = pd.pd_get_state(sim)
    # the oracle's force at the GPU solution: the free-DOF residual is tiny next
    # to the residual the final load increment started from
    r = I.residual(g, L.mat, O.neighbors(g), u, L.bc_kind)
    assert np.linalg.norm(r) <= 1e-7 * st["res0"]
    # prescribed DOFs exact, mirror symmetry about the middle row
    fixed = L.bc_kind == W.BC_DISPLACEMENT
    assert np.array_equal(u[fixed], L.bc_val[fixed])
    U = u.reshape(g.n[1], g.n[0], 2)
    sc = np.abs(U).max()
    assert np.abs(U[:, :, 0] - U[::-1, :, 0]).max() <= 1e-7 * sc
    assert np.abs(U[:, :, 1] + U[::-1, :, 1]).max() <= 1e-7 * sc
    sim.close()


def test_roller_plate_200_matches_the_uniaxial_stress_solution(pd):
    L = W.plate_static(nx=200, strain=1e-4, variant="roller")
    g = L.grid
    sim = _static_sim(pd, L, pd.PD_FP64)
    st = pd.pd_solve_static(sim, pd.newton_opts(krylov=pd.PD_KRYLOV_CG, linear_rtol=1e-10, newton_rtol=1e-10))
    assert st["converged"] == 1
    u, _ = pd.pd_get_state(sim)
    X = g.positions()
    c = g.coords()
    k = 2 * g.m
    inner = (c[:, 0] >= k) & (c[:, 0] < g.n[0] - k) & (c[:, 1] >= k) & (c[:, 1] < g.n[1] - k)
    ux = L.strain * X[:, 0]
    uy = -(1.0 / 3.0) * L.strain * (X[:, 1] - X[L.pin, 1])
    assert rel_l2(u[inner, 0], ux[inner]) <= 1e-2
    assert rel_l2(u[inner, 1], uy[inner]) <= 0.1
    sim.close()


def test_autograd_force_passes_gradcheck(pd):
    import torch
    from paper_1806_06917_gb300.autograd import internal_force
    grid = W.Grid(dim=2, n=(11, 7, 1), h=0.01, m=3)
    mat = W.Material(model=W.PMB, E=72e9, rho=2440.0)
    sim = gpu_sim(pd, grid, mat, pd.PD_FP64)
    rng = np.random.default_rng(12)
    u0 = torch.tensor(rng.normal(0.0, 1e-3 * grid.h, (grid.npoints, 2)), device="cuda", requires_grad=True)
    # scale the output so that Jacobian entries are O(1)
    w = np.zeros((grid.npoints, 2))
    w[grid.npoints // 2, 0] = 1.0
    kscale = float(np.abs(pd.pd_jvp(sim, w, u_lin=u0.detach().cpu().numpy())).max())
    fn = lambda u: internal_force(sim, u) / kscale  # noqa: E731
    assert torch.autograd.gradcheck(fn, (u0,), eps=1e-6 * grid.h, atol=1e-6, rtol=1e-5)
    # backward against the oracle's assembled tangent: dL/du = K^T g
    g_out = torch.tensor(rng.normal(size=(grid.npoints, 2)), device="cuda")
    f = internal_force(sim, u0)
    (gu,) = torch.autograd.grad(f, u0, g_out)
    K = O.tangent_fd(grid, mat, O.neighbors(grid), u0.detach().cpu().numpy(), 1e-6 * grid.h)
    ref = K.T @ g_out.cpu().numpy().reshape(-1)
    assert rel_l2(gu.cpu().numpy().reshape(-1), ref) <= 1e-6
    sim.close()


def test_static_solve_argument_errors(pd):
    L = W.plate_static(nx=20, ny=10, variant="clamped")
    sim = _static_sim(pd, L, pd.PD_FP64)
    for bad in (pd.newton_opts(krylov=7), pd.newton_opts(restart=0), pd.newton_opts(linear_rtol=0.0),
                pd.newton_opts(max_newton_iters=0), pd.newton_opts(tangent=5)):
        with pytest.raises(pd.PdError) as e:
            pd.pd_solve_static(sim, bad)
        assert e.value.code == pd.PD_EINVAL
    sim.close()
    grid = W.Grid(dim=3, n=(6, 6, 6), h=0.01, m=2)
    lps = W.Material(model=W.LPS, E=72e9, rho=2440.0, K=40e9, mu=30e9)
    s2 = gpu_sim(pd, grid, lps, pd.PD_FP64)
    with pytest.raises(pd.PdError) as e:
        pd.pd_solve_static(s2)
    assert e.value.code == pd.PD_EINVAL
    s2.close()
