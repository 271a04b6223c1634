"""Pins of the implicit-scheme oracle (Sec. 5: Newton on f(u) + b = 0 with the
central-difference stiffness of Eq. (6) / Algorithm 3) against facts fixed
outside it: a library direct solve, the finite termination of full GMRES, the
classical continuum solution of uniaxial stress (CCM), the symmetry of the
clamped plate, the linear response at small strain, and two independent linear
solver paths."""
import numpy as np
import pytest

from oracle import implicit as I
from oracle import oracle as O
from paper_1806_06917_gb300 import workloads as W


def test_gmres_matches_a_direct_solve():
    # restarted GMRES on a nonsymmetric, well-conditioned system reaches the
    # LAPACK solution; the stopping test is met on the true residual
    rng = np.random.default_rng(40)
    n = 80
    A = np.eye(n) * 4.0 + rng.normal(0.0, 0.3, (n, n))
    b = rng.normal(size=n)
    x_ref = np.linalg.solve(A, b)
    for restart in (10, 80):
        x, it, ok = I.gmres(lambda v: A @ v, b, restart=restart, rtol=1e-12)
        assert ok
        assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b) * 1.0001
        assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_full_gmres_terminates_within_n_iterations():
    # without restarts GMRES minimises over Krylov spaces of growing dimension:
    # at dimension n the residual is zero (up to rounding)
    rng = np.random.default_rng(41)
    n = 25
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = rng.normal(size=n)
    x, it, ok = I.gmres(lambda v: A @ v, b, restart=n, rtol=1e-11)
    assert ok and it <= n


def _interior(grid, layers):
    c = grid.coords()
    nx, ny = grid.n[0], grid.n[1]
    return (c[:, 0] >= layers) & (c[:, 0] < nx - layers) & (c[:, 1] >= layers) & (c[:, 1] < ny - layers)


def test_roller_plate_matches_uniaxial_stress_solution():
    # CCM: u_x = eps X, u_y = -nu eps (Y - Y0), nu = 1/3 for the bond-based model
    # in plane stress; compared on points >= 2 delta from every edge. u_x within
    # 1 %; u_y carries the surface effect of the free edges (a few %)
    L = W.plate_static(nx=40, ny=20, strain=1e-4, variant="roller")
    g = L.grid
    bonds = O.neighbors(g)
    u, hist, ok = I.solve_static(g, L.mat, bonds, np.zeros((g.npoints, 2)), L.bc_kind, L.bc_val)
    assert ok and hist[-1] <= 1e-10 * hist[0]
    X = g.positions()
    inner = _interior(g, 2 * g.m)
    ux = L.strain * X[:, 0]
    uy = -(1.0 / 3.0) * L.strain * (X[:, 1] - X[L.pin, 1])
    ex = np.linalg.norm(u[inner, 0] - ux[inner]) / np.linalg.norm(ux[inner])
    ey = np.linalg.norm(u[inner, 1] - uy[inner]) / np.linalg.norm(uy[inner])
    assert ex <= 1e-2
    assert ey <= 0.1


def test_clamped_plate_is_mirror_symmetric():
    # the clamped plate and its loads are symmetric about the middle row:
    # u_x(x, y) = u_x(x, ny-1-y), u_y(x, y) = -u_y(x, ny-1-y)
    L = W.plate_static(nx=24, ny=14, strain=1e-4, variant="clamped")
    g = L.grid
    bonds = O.neighbors(g)
    u, _, ok = I.solve_static(g, L.mat, bonds, np.zeros((g.npoints, 2)), L.bc_kind, L.bc_val)
    assert ok
    nx, ny = g.n[0], g.n[1]
    U = u.reshape(ny, nx, 2)
    scale = np.abs(U).max()
    assert np.abs(U[:, :, 0] - U[::-1, :, 0]).max() <= 1e-9 * scale
    assert np.abs(U[:, :, 1] + U[::-1, :, 1]).max() <= 1e-9 * scale


def test_small_strain_response_is_linear_and_zero_load_gives_zero():
    L = W.plate_static(nx=20, ny=12, strain=1e-5, variant="clamped")
    g = L.grid
    bonds = O.neighbors(g)
    z = np.zeros((g.npoints, 2))
    u1, _, ok1 = I.solve_static(g, L.mat, bonds, z, L.bc_kind, L.bc_val, newton_rtol=1e-10)
    u2, _, ok2 = I.solve_static(g, L.mat, bonds, z, L.bc_kind, 2.0 * L.bc_val, newton_rtol=1e-10)
    assert ok1 and ok2
    rel = np.linalg.norm(u2 - 2.0 * u1) / np.linalg.norm(u2)
    assert 0.0 < rel <= 1e-3          # geometric nonlinearity of order strain
    u0, hist, ok0 = I.solve_static(g, L.mat, bonds, z, L.bc_kind, 0.0 * L.bc_val)
    assert ok0 and hist[0] == 0.0 and not u0.any()


def test_assembled_and_matrix_free_newton_agree():
    # two independent linear paths: the assembled central-difference stiffness
    # with LU, and inexact Newton with GMRES on directional differences (the
    # restart exceeds the free DOFs); both must reach the same root of f + b
    L = W.plate_static(nx=12, ny=8, strain=1e-4, variant="clamped")
    g = L.grid
    bonds = O.neighbors(g)
    z = np.zeros((g.npoints, 2))
    ua, _, oka = I.solve_static(g, L.mat, bonds, z, L.bc_kind, L.bc_val, linear="lu")
    ub, _, okb = I.solve_static(g, L.mat, bonds, z, L.bc_kind, L.bc_val, linear="gmres", restart=200,
                                linear_rtol=1e-8, linear_maxit=400, newton_rtol=1e-11)
    assert oka and okb
    assert np.linalg.norm(ua - ub) <= 1e-7 * np.linalg.norm(ua)


@pytest.mark.parametrize("variant", ["clamped", "roller"])
def test_load_path_prescribes_only_collar_dofs(variant):
    L = W.plate_static(nx=30, ny=20, variant=variant)
    g = L.grid
    left, right = W.collar_mask(g, 0, -1), W.collar_mask(g, 0, +1)
    fixed = L.bc_kind == W.BC_DISPLACEMENT
    assert fixed[left | right, 0].all()
    assert not fixed[~(left | right), 0].any()
    if variant == "clamped":
        assert fixed[left, 1].all() and not fixed[~left, 1].any()
        assert np.allclose(L.bc_val[right, 0], L.strain * (g.n[0] - 1) * g.h)
    else:
        assert fixed[:, 1].sum() == 1 and fixed[L.pin, 1]


def test_body_force_equilibrium_and_direction():
    # Sec. 5's static problem with a body force: at the solution the internal
    # force balances b on every free DOF, f(u) + b = 0 (checked with the force
    # function itself, not the solver's residual), and a plate clamped on its
    # left collar under a uniform +x body force moves in +x everywhere it is free
    L = W.plate_static(nx=12, ny=8, strain=1e-4, variant="clamped")
    g = L.grid
    bonds = O.neighbors(g)
    left = W.collar_mask(g, 0, -1)
    kind = np.zeros((g.npoints, 2), dtype=np.uint8)
    kind[left, :] = W.BC_DISPLACEMENT
    val = np.zeros((g.npoints, 2))
    b = np.zeros((g.npoints, 2))
    b[:, 0] = 1e6
    u, hist, ok = I.solve_static(g, L.mat, bonds, np.zeros((g.npoints, 2)), kind, val, b=b, newton_rtol=1e-10)
    assert ok and hist[0] > 0.0
    f, _ = O.internal_force(g, L.mat, bonds, u)
    free = kind == 0
    assert np.abs((f + b)[free]).max() <= 1e-9 * 1e6
    assert (u[~left, 0] > 0.0).all()
    assert not u[left].any()
