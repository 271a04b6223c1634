"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: textbook lattice
counts, the paper's statement on horizon membership, closed forms of rigid and
affine motion, continuum (CCM) energy densities, force/energy consistency,
conservation laws, and the structure of the tangent. A plausible slip in the
oracle (a dropped term, a wrong sign or index, a wrong constant) fails one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_06917_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def _grid(dim, n, m, h=0.01):
    nn = (n[0], n[1], n[2] if dim == 3 else 1)
    return W.Grid(dim=dim, n=nn, h=h, m=m)


def _interior(g, width):
    c = g.coords()
    ok = np.ones(g.npoints, dtype=bool)
    for a in range(g.dim):
        ok &= (c[:, a] >= width) & (c[:, a] < g.n[a] - width)
    return ok


# ----------------------------------------------------------------- neighbours

@pytest.mark.parametrize("d,m,count", [tuple(int(x) for x in r) for r in _read_rows("lattice_ball_counts.txt")])
def test_interior_row_length_matches_lattice_ball_count(d, m, count):
    n = 2 * m + 3
    g = _grid(d, (n, n, n), m)
    b = O.neighbors(g, "cells")
    ctr = int(np.flatnonzero(np.all(g.coords()[:, :d] == n // 2, axis=1))[0])
    assert len(b.row(ctr)) == count - 1


def test_paper_horizon_line_count():
    (md, nodes), = _read_rows("paper_horizon_nodes.txt")
    md, nodes = int(md), int(nodes)
    g = _grid(2, (4 * md + 1, 4 * md + 1, 1), md)
    b = O.neighbors(g, "cells")
    ctr = int(np.flatnonzero(np.all(g.coords()[:, :2] == 2 * md, axis=1))[0])
    c = g.coords()
    on_line = [j for j in b.row(ctr) if c[j, 1] == c[ctr, 1]]
    assert len(on_line) + 1 == nodes


def _bond_total_by_offsets(g):
    """Directed bonds counted per lattice offset: sum over offsets of the number of
    ordered pairs (i, i + offset) inside the box, prod_a (n_a - |d_a|)."""
    m = g.m
    rng = range(-m, m + 1)
    total = 0
    for dz in (rng if g.dim == 3 else [0]):
        for dy in rng:
            for dx in rng:
                if (dx, dy, dz) == (0, 0, 0) or dx * dx + dy * dy + dz * dz > m * m:
                    continue
                total += max(g.n[0] - abs(dx), 0) * max(g.n[1] - abs(dy), 0) * max(g.n[2] - abs(dz), 0)
    return total


@pytest.mark.parametrize("dim,n,m", [(2, (7, 5, 1), 2), (2, (13, 9, 1), 3), (2, (11, 11, 1), 4),
                                     (3, (6, 5, 4), 2), (3, (9, 7, 8), 3), (3, (10, 9, 9), 4),
                                     (2, (3, 2, 1), 3), (3, (1, 1, 1), 3)])
def test_brute_force_equals_cell_list_and_offset_count(dim, n, m):
    g = _grid(dim, n, m)
    bb = O.neighbors(g, "brute")
    bc = O.neighbors(g, "cells")
    assert np.array_equal(bb.row_ptr, bc.row_ptr)
    assert np.array_equal(bb.col, bc.col)
    assert bb.nbonds == _bond_total_by_offsets(g)
    for i in range(g.npoints):                          # rows ascending, no self
        r = bb.row(i)
        assert np.all(np.diff(r) > 0) and i not in r


@pytest.mark.parametrize("dim,n,m,expect", [(2, (50, 50, 1), 3, 66436), (3, (64, 64, 64), 3, 30289512)])
def test_workload_bond_totals(dim, n, m, expect):
    g = _grid(dim, n, m)
    assert _bond_total_by_offsets(g) == expect
    if g.npoints <= 5000:
        assert O.neighbors(g).nbonds == expect


def test_morton_order_golden():
    want = np.array(_read_rows("morton_4x4.txt")[0], dtype=np.int64)
    g = _grid(2, (4, 4, 1), 1)
    assert np.array_equal(O.morton_perm(g), want)


def test_morton_order_non_power_of_two_is_sorted_by_interleave():
    g = _grid(3, (5, 3, 6), 1)
    perm = O.morton_perm(g)
    assert sorted(perm.tolist()) == list(range(g.npoints))
    c = g.coords()[perm]
    # consecutive points never go backwards in the most significant differing bit
    for a, b in zip(c[:-1], c[1:]):
        diff = [(int(a[k]) ^ int(b[k])) for k in range(3)]
        hb = [d.bit_length() - 1 for d in diff]
        top = max(range(3), key=lambda k: (hb[k], k))
        assert b[top] > a[top]


def test_notch_full_plane_breaks_exactly_crossing_bonds():
    g = _grid(3, (6, 5, 7), 2)
    b = O.neighbors(g)
    notch = W.Notch(axis=2, pos=2.5, lo=(-1.0, -1.0, 0.0), hi=(10.0, 10.0, 0.0))
    nb = O.break_notch(g, b, notch)
    c = g.coords()
    want = 0
    for i in range(g.npoints):
        for k in range(b.row_ptr[i], b.row_ptr[i + 1]):
            j = b.col[k]
            crosses = (c[i, 2] <= 2) != (c[j, 2] <= 2)
            assert bool(b.broken[k]) == crosses
            want += crosses
    assert nb == want > 0


def test_notch_rectangle_edge_only_cuts_bonds_through_it():
    g = _grid(3, (8, 4, 6), 2)
    b = O.neighbors(g)
    notch = W.Notch(axis=2, pos=2.5, lo=(-0.5, -0.5, 0.0), hi=(3.2, 3.5, 0.0))
    O.break_notch(g, b, notch)
    c = g.coords()
    for i in range(g.npoints):
        for k in range(b.row_ptr[i], b.row_ptr[i + 1]):
            j = b.col[k]
            if b.broken[k]:
                assert (c[i, 2] <= 2) != (c[j, 2] <= 2)
                assert min(c[i, 0], c[j, 0]) <= 3          # segment reaches x <= 3.2
            elif (c[i, 2] <= 2) != (c[j, 2] <= 2):
                # crossing bonds left intact cross the plane beyond x = 3.2
                t = (2.5 - c[i, 2]) / (c[j, 2] - c[i, 2])
                assert c[i, 0] + t * (c[j, 0] - c[i, 0]) > 3.2


# ------------------------------------------------------------------ PMB force

def test_pmb_two_point_closed_form():
    g = _grid(3, (2, 1, 1), 1, h=0.02)
    mat = W.Material(model=W.PMB, E=72e9)
    b = O.neighbors(g)
    c = O.micromodulus(g, mat)
    V = g.h ** 3
    u = np.zeros((2, 3))
    u[1] = (3e-6, 4e-6, 0.0)
    y = np.array([g.h + 3e-6, 4e-6, 0.0])
    s = (np.linalg.norm(y) - g.h) / g.h
    f = O.pmb_force(g, mat, b, u)
    np.testing.assert_allclose(f[0], c * s * V * y / np.linalg.norm(y), rtol=1e-12)
    np.testing.assert_allclose(f[1], -f[0], rtol=1e-15)
    assert f[0, 0] > 0          # stretched bond pulls point 0 towards point 1


@pytest.mark.parametrize("dim", [2, 3])
def test_pmb_energy_density_matches_ccm(dim):
    """Uniform expansion u = eps X stretches every bond by s = eps. The interior
    strain-energy density converges to the continuum value: 9 K eps^2 / 2 = 3 E eps^2
    in 3D (nu = 1/4) and E eps^2 / (1 - nu) = 3/2 E eps^2 in 2D plane stress
    (nu = 1/3). This pins the micromodulus and the energy normalisation."""
    eps = 1e-4
    for m, tol in ((3, 0.15), (6, 0.05)):
        n = 4 * m + 3 if dim == 3 else 6 * m + 5
        g = _grid(dim, (n, n, n), m)
        mat = W.Material(model=W.PMB, E=72e9)
        b = O.neighbors(g)
        _, Wp = O.strain_energy(g, mat, b, eps * g.positions(), per_point=True)
        ctr = np.all(g.coords()[:, :dim] == n // 2, axis=1)
        ccm = (3.0 if dim == 3 else 1.5) * mat.E * eps ** 2
        assert abs(Wp[ctr][0] / ccm - 1.0) < tol


@pytest.mark.parametrize("model", [W.PMB, W.LPS])
def test_force_is_minus_energy_gradient(model):
    """f_i = -(1/V_i) dW_total/du_i (central differences of the oracle's energy)."""
    dim = 3 if model == W.LPS else 2
    g = _grid(dim, (6, 5, 5), 2, h=0.01)
    mat = W.Material(model=model, E=72e9, K=40e9, mu=30e9)
    b = O.neighbors(g)
    mv = O.weighted_volume(g, mat, b) if model == W.LPS else None
    u = W.random_field(g, 2e-4 * g.h, seed=11) + 3e-4 * g.positions()[:, ::-1]
    f, th = O.internal_force(g, mat, b, u, mv)
    V = g.h ** dim
    rng = np.random.default_rng(5)
    for q in rng.choice(g.npoints * dim, size=12, replace=False):
        hstep = 1e-9 * g.h
        up, um = u.copy().ravel(), u.copy().ravel()
        up[q] += hstep
        um[q] -= hstep

        def energy(x):
            x = x.reshape(u.shape)
            _, t = O.internal_force(g, mat, b, x, mv)
            return O.strain_energy(g, mat, b, x, mv, t)
        dW = (energy(up) - energy(um)) / (2 * hstep)
        assert abs(-dW / V - f.ravel()[q]) <= 1e-5 * np.abs(f).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_pmb_rigid_translation_is_force_free_exactly(dim):
    g = _grid(dim, (7, 6, 5), 3)
    mat = W.Material(model=W.PMB)
    b = O.neighbors(g)
    u = np.tile(np.array([1.5e3, -2.25e3, 0.75e3])[:dim], (g.npoints, 1))
    assert np.all(O.pmb_force(g, mat, b, u) == 0.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_pmb_rigid_rotation_is_force_free(dim):
    g = _grid(dim, (8, 7, 6), 3)
    mat = W.Material(model=W.PMB)
    b = O.neighbors(g)
    X = g.positions()
    a = 0.1
    R2 = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    if dim == 2:
        R = R2
    else:
        R = np.eye(3)
        R[:2, :2] = R2
        b2 = 0.07
        Rx = np.array([[1, 0, 0], [0, math.cos(b2), -math.sin(b2)], [0, math.sin(b2), math.cos(b2)]])
        R = Rx @ R
    u = X @ R.T - X
    f = O.pmb_force(g, mat, b, u)
    scale = O.micromodulus(g, mat) * g.h ** dim * g.h * len(b.row(0))
    assert np.abs(f).max() < 1e-12 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_pmb_affine_interior_force_free_and_boundary_not(dim):
    g = _grid(dim, (11, 10, 9), 3)
    mat = W.Material(model=W.PMB)
    b = O.neighbors(g)
    A = np.array([[2e-4, 5e-5, -3e-5], [1e-5, -1e-4, 4e-5], [7e-5, 2e-5, 3e-4]])[:dim, :dim]
    f = O.pmb_force(g, mat, b, g.positions() @ A.T)
    inner = _interior(g, g.m)
    fmax = np.abs(f).max()
    assert fmax > 0
    assert np.abs(f[inner]).max() < 1e-9 * fmax
    assert np.abs(f[~inner]).max() > 1e-3 * fmax      # surface effect at the collar


@pytest.mark.parametrize("model", [W.PMB, W.LPS])
def test_net_internal_force_vanishes(model):
    dim = 3
    g = _grid(dim, (8, 7, 6), 3)
    mat = W.Material(model=model, K=40e9, mu=30e9)
    b = O.neighbors(g)
    mv = O.weighted_volume(g, mat, b) if model == W.LPS else None
    u = W.random_field(g, 1e-3 * g.h, seed=3)
    f, _ = O.internal_force(g, mat, b, u, mv)
    V = g.h ** dim
    net = (f * V).sum(axis=0)
    assert np.abs(net).max() <= 1e-12 * (np.abs(f) * V).sum()


def test_pmb_breaking_is_irreversible():
    g = _grid(3, (2, 1, 1), 1, h=0.02)
    mat = W.Material(model=W.PMB, s_c=1e-3)
    b = O.neighbors(g)
    u = np.zeros((2, 3))
    u[1, 0] = 0.99e-3 * g.h
    f = O.pmb_force(g, mat, b, u, update_breaking=True)
    assert f[0, 0] > 0 and not b.broken.any()
    u[1, 0] = 1.01e-3 * g.h
    f = O.pmb_force(g, mat, b, u, update_breaking=True)
    assert np.all(f == 0) and b.broken.all()
    u[1, 0] = 0.5e-3 * g.h                       # pushed back: stays broken
    f = O.pmb_force(g, mat, b, u, update_breaking=True)
    assert np.all(f == 0) and b.broken.all()


# ---------------------------------------------------------------------- LPS

def test_lps_dilatation_of_uniform_expansion_is_3eps_everywhere():
    g = _grid(3, (9, 8, 7), 3)
    mat = W.Material(model=W.LPS, K=40e9, mu=30e9)
    b = O.neighbors(g)
    mv = O.weighted_volume(g, mat, b)
    eps = 2e-4
    th = O.dilatation(g, mat, b, mv, eps * g.positions())
    np.testing.assert_allclose(th, 3 * eps, rtol=1e-10)
    th0 = O.dilatation(g, mat, b, mv, np.tile([4.0, -1.0, 2.0], (g.npoints, 1)))
    assert np.all(th0 == 0.0)


def test_lps_weighted_volume_interior():
    g = _grid(3, (9, 9, 9), 3)
    mat = W.Material(model=W.LPS, K=40e9, mu=30e9)
    b = O.neighbors(g)
    mv = O.weighted_volume(g, mat, b)
    ctr = np.all(g.coords() == 4, axis=1)
    # sum over the 122 offsets of |d|^2 h^2 * h^3, with |d|^2 summed by shells:
    # 6 at 1, 12 at 2, 8 at 3, 6 at 4, 24 at 5, 24 at 6, 12 at 8, 30 at 9
    shells = {1: 6, 2: 12, 3: 8, 4: 6, 5: 24, 6: 24, 8: 12, 9: 30}
    assert sum(shells.values()) == 122
    want = sum(k * v for k, v in shells.items()) * g.h ** 5
    np.testing.assert_allclose(mv[ctr][0], want, rtol=1e-13)


def test_lps_energy_of_expansion_and_cubic_average_of_shear():
    """Expansion: W = K theta^2 / 2 with theta = 3 eps, exactly. Shear: the cubic
    (Voigt) average (2 W_tetragonal + 3 W_xy) / 5 of the interior energy equals the
    continuum mu eps:eps, because the direction average of (n.eps.n)^2 is
    2 eps:eps / 15 for any traceless eps. Pins K, mu and the 3 and 15 factors."""
    mat = W.Material(model=W.LPS, K=40e9, mu=30e9)
    for m in (3, 4):
        n = 4 * m + 3
        g = _grid(3, (n, n, n), m)
        b = O.neighbors(g)
        mv = O.weighted_volume(g, mat, b)
        X = g.positions()
        ctr = np.all(g.coords() == n // 2, axis=1)
        eps = 1e-5
        u = eps * X
        th = O.dilatation(g, mat, b, mv, u)
        _, Wp = O.strain_energy(g, mat, b, u, mv, th, per_point=True)
        np.testing.assert_allclose(Wp, 0.5 * mat.K * (3 * eps) ** 2, rtol=1e-8)
        gam = 1e-6
        A_xy = np.array([[0, gam / 2, 0], [gam / 2, 0, 0], [0, 0, 0]])
        A_te = np.diag([gam, -gam / 2, -gam / 2])
        res = []
        for A in (A_te, A_xy):
            u = X @ A.T
            th = O.dilatation(g, mat, b, mv, u)
            _, Wp = O.strain_energy(g, mat, b, u, mv, th, per_point=True)
            res.append(Wp[ctr][0] / (mat.mu * np.sum(A * A)))
        assert abs((2 * res[0] + 3 * res[1]) / 5 - 1.0) < 1e-4


def test_lps_gather_equals_scatter_and_affine_interior():
    g = _grid(3, (15, 14, 13), 3)
    mat = W.Material(model=W.LPS, K=40e9, mu=30e9)
    b = O.neighbors(g)
    mv = O.weighted_volume(g, mat, b)
    u = W.random_field(g, 1e-3 * g.h, seed=7)
    th = O.dilatation(g, mat, b, mv, u)
    fg = O.lps_force(g, mat, b, mv, th, u)
    fs = O.lps_force(g, mat, b, mv, th, u, scatter=True)
    assert np.abs(fg - fs).max() <= 1e-12 * np.abs(fg).max()
    A = np.array([[2e-4, 5e-5, -3e-5], [1e-5, -1e-4, 4e-5], [7e-5, 2e-5, 3e-4]])
    u = g.positions() @ A.T
    th = O.dilatation(g, mat, b, mv, u)
    f = O.lps_force(g, mat, b, mv, th, u)
    inner = _interior(g, 2 * g.m)
    assert np.abs(f[inner]).max() < 1e-8 * np.abs(f).max()


# --------------------------------------------------------------- integrator

def _free_plate():
    g = _grid(2, (16, 16, 1), 3, h=0.02)
    mat = W.Material(model=W.PMB, E=72e9, rho=2440.0)
    u0 = W.gaussian_ic(g, (1e-5, 0.5e-5), (0.16, 0.14), 0.003)
    return g, mat, u0


def test_verlet_equals_central_difference():
    g, mat, u0 = _free_plate()
    b = O.neighbors(g)
    dt = 0.5 * O.stable_dt(g, mat, b)
    v0 = W.random_field(g, 1e-3, seed=2)
    st = O.ExplicitState(g, mat, b, u0, v0)
    st.run(dt, 40)
    ucd = O.run_central_difference(g, mat, b, u0, v0, dt, 40)
    assert np.abs(st.u - ucd).max() <= 1e-10 * np.abs(st.u).max()


def test_energy_conservation_second_order_and_momentum():
    g, mat, u0 = _free_plate()
    b = O.neighbors(g)
    dt0 = 0.5 * O.stable_dt(g, mat, b)
    V = g.h ** 2 * mat.thickness
    devs = []
    for k in (1, 2):
        dt = dt0 / k
        v0 = np.zeros_like(u0)
        st = O.ExplicitState(g, mat, b, u0, v0)
        E0 = O.strain_energy(g, mat, b, st.u)
        Es = []
        for _ in range(30):
            st.run(dt, 10 * k)
            Es.append(O.kinetic_energy(g, mat, st.v) + O.strain_energy(g, mat, b, st.u))
        devs.append(np.abs(np.array(Es) - E0).max() / E0)
        p = (mat.rho * V * st.v).sum(axis=0)
        assert np.abs(p).max() < 1e-10 * mat.rho * V * np.abs(st.v).sum()
    assert devs[0] < 3e-2
    assert 3.0 < devs[0] / devs[1] < 5.0


def test_prescribed_velocity_collar_moves_rigidly():
    wl = W.plate2d(nside=20, steps=10)
    g, mat = wl.grid, wl.mat
    b = O.neighbors(g)
    dt = 0.5 * O.stable_dt(g, mat, b)
    st = O.ExplicitState(g, mat, b, wl.u0, wl.v0, wl.bc_kind, wl.bc_val)
    st.run(dt, 10)
    sel = wl.bc_kind[:, 0] == W.BC_VELOCITY
    np.testing.assert_allclose(st.u[sel, 0], wl.u0[sel, 0] + 10 * dt * wl.bc_val[sel, 0], rtol=1e-12)
    assert np.all(st.v[sel, 0] == wl.bc_val[sel, 0])


def test_stable_dt_bound_separates_stable_from_unstable():
    """The Silling-Askari bound is a sufficient stability condition of the explicit
    scheme: at dt_crit a random field stays bounded over 400 steps, at 2.5 dt_crit
    the same run diverges."""
    g = _grid(2, (24, 24, 1), 3, h=0.02)
    mat = W.Material(model=W.PMB, E=72e9, rho=2440.0)
    b = O.neighbors(g)
    dtc = O.stable_dt(g, mat, b)
    u0 = W.random_field(g, 1e-6, seed=1)
    ok = O.ExplicitState(g, mat, b, u0, np.zeros_like(u0))
    ok.run(dtc, 400)
    assert np.isfinite(ok.u).all() and np.abs(ok.u).max() < 1e-5
    bad = O.ExplicitState(g, mat, b, u0, np.zeros_like(u0))
    bad.run(2.5 * dtc, 400)
    assert not (np.isfinite(bad.u).all() and np.abs(bad.u).max() < 1e-3)


@pytest.mark.parametrize("case", ["pmb3", "pmb2", "np2", "lp2"])
def test_stable_dt_is_the_leapfrog_limit_of_a_two_point_body(case):
    """Two points joined by one bond: the relative displacement along the bond is
    one harmonic oscillator, rho w'' = -2 k w with k the bond's linear stiffness
    per unit volume (c V / |xi|), and velocity-Verlet (leapfrog) keeps it bounded
    exactly for omega dt < 2, omega^2 = 2 k / rho. The Silling-Askari sum has the
    one term k here, so the bound sqrt(2 rho / k) is that limit 2 / omega: a run
    at 0.98 dt_crit stays bounded, one at 1.02 dt_crit grows without bound."""
    if case == "pmb3":
        g, mat = _grid(3, (2, 1, 1), 1, h=0.02), W.Material(model=W.PMB, E=72e9, rho=2440.0)
    elif case == "pmb2":
        g, mat = _grid(2, (2, 1, 1), 1, h=0.02), W.Material(model=W.PMB, E=72e9, rho=2440.0, thickness=0.1)
    else:
        # m = 2: the neighbour at distance h lies inside the open horizon ball (J = 1)
        g = _grid(2, (2, 1, 1), 2, h=0.0025)
        mat = W.Material(model=W.NP if case == "np2" else W.LP, rho=1.0, psi_c=1.0, psi_beta=1.0)
    b = O.neighbors(g)
    assert b.nbonds == 2
    dtc = O.stable_dt(g, mat, b)
    a = 1e-9 * g.h                          # small: the NP law stays linear
    u0 = np.zeros((2, g.dim))
    u0[1, 0] = a
    ok = O.ExplicitState(g, mat, b, u0, np.zeros_like(u0))
    ok.run(0.98 * dtc, 3000)
    assert np.isfinite(ok.u).all() and np.abs(ok.u).max() < 20 * a
    bad = O.ExplicitState(g, mat, b, u0, np.zeros_like(u0))
    bad.run(1.02 * dtc, 80)
    assert not (np.isfinite(bad.u).all() and np.abs(bad.u).max() < 1e6 * a)


def test_lps_stable_dt_is_the_pmb_bound_of_the_same_young_modulus():
    """Reading of the LPS step bound: the PMB bound of the material's Young's
    modulus, here formed from K and mu through the Poisson ratio,
    E = 2 mu (1 + nu), nu = (3K - 2mu) / (2 (3K + mu))."""
    g = _grid(3, (9, 8, 7), 3, h=0.01)
    b = O.neighbors(g)
    K, mu, rho = 40e9, 30e9, 2440.0
    nu = (3 * K - 2 * mu) / (2 * (3 * K + mu))
    E = 2 * mu * (1 + nu)
    dt_lps = O.stable_dt(g, W.Material(model=W.LPS, K=K, mu=mu, rho=rho), b)
    dt_pmb = O.stable_dt(g, W.Material(model=W.PMB, E=E, rho=rho), b)
    assert abs(dt_lps - dt_pmb) <= 1e-12 * dt_pmb


def test_2d_pmb_force_density_does_not_depend_on_the_plate_thickness():
    """The 2D micromodulus is calibrated per unit thickness (c t is fixed by E and
    delta), so a plate's force per unit volume is the same for every thickness
    and its strain energy grows in proportion to the thickness."""
    g = _grid(2, (9, 8, 1), 3, h=0.01)
    b = O.neighbors(g)
    u = W.random_field(g, 1e-6, seed=7)
    m1 = W.Material(model=W.PMB, E=72e9, thickness=1.0)
    m2 = W.Material(model=W.PMB, E=72e9, thickness=0.013)
    f1, f2 = O.pmb_force(g, m1, b, u), O.pmb_force(g, m2, b, u)
    np.testing.assert_allclose(f2, f1, rtol=1e-12, atol=1e-12 * np.abs(f1).max())
    e1, e2 = O.strain_energy(g, m1, b, u), O.strain_energy(g, m2, b, u)
    assert abs(e2 / e1 - 0.013) < 1e-12


def test_prescribed_displacement_holds_its_value_with_zero_velocity():
    """A degree of freedom with a prescribed displacement takes its value at every
    step with zero velocity, whatever force acts on it, while the free ones move."""
    g = _grid(2, (12, 10, 1), 3, h=0.01)
    mat = W.Material(model=W.PMB, E=72e9, rho=2440.0)
    b = O.neighbors(g)
    u0 = W.random_field(g, 1e-6, seed=3)
    v0 = W.random_field(g, 1e-3, seed=4)
    c = g.coords()
    kind = np.zeros((g.npoints, 2), dtype=np.uint8)
    val = np.zeros((g.npoints, 2))
    sel = c[:, 0] < 3
    kind[sel] = W.BC_DISPLACEMENT
    val[sel, 0] = 2e-5 * (c[sel, 1] + 1)
    val[sel, 1] = -1e-5
    st = O.ExplicitState(g, mat, b, u0, v0, kind, val)
    st.run(0.5 * O.stable_dt(g, mat, b), 5)
    assert np.all(st.u[sel] == val[sel])
    assert np.all(st.v[sel] == 0.0)
    assert np.all(st.u[~sel] != u0[~sel])


@pytest.mark.parametrize("m,cut", [(1, 0), (2, 2)])
def test_notch_through_a_lattice_point_cuts_only_strict_crossings(m, cut):
    """A bond crosses the notch plane when its ends lie strictly on opposite
    sides of it; an end on the plane is not a crossing. Three points on a line,
    the plane through the middle one: with m = 1 no bond crosses, with m = 2 only
    the bond from the first to the third point, in both directions."""
    g = _grid(2, (3, 1, 1), m, h=0.01)
    b = O.neighbors(g)
    notch = W.Notch(axis=0, pos=1.0, lo=(0.0, -1.0, 0.0), hi=(0.0, 1.0, 0.0))
    assert O.break_notch(g, b, notch) == cut
    c = g.coords()
    for i in range(g.npoints):
        for k in range(b.row_ptr[i], b.row_ptr[i + 1]):
            j = b.col[k]
            assert bool(b.broken[k]) == ({int(c[i, 0]), int(c[j, 0])} == {0, 2})


# ------------------------------------------------------------------ tangent

def test_tangent_structure_and_jvp():
    g = _grid(2, (7, 6, 1), 2, h=0.01)
    mat = W.Material(model=W.PMB)
    b = O.neighbors(g)
    eps = 1e-6 * g.h
    K0 = O.tangent_fd(g, mat, b, np.zeros((g.npoints, 2)), eps)
    np.testing.assert_allclose(K0, K0.T, atol=1e-7 * np.abs(K0).max())
    ev = np.linalg.eigvalsh(-0.5 * (K0 + K0.T))
    assert ev.min() > -1e-7 * ev.max()                  # -K is positive semi-definite
    assert int((ev < 1e-7 * ev.max()).sum()) == 3      # 2 translations + 1 rotation
    X = g.positions()
    modes = [np.tile([1.0, 0.0], (g.npoints, 1)), np.tile([0.0, 1.0], (g.npoints, 1)),
             np.stack([-X[:, 1], X[:, 0]], axis=1)]
    for w in modes:
        assert np.abs(K0 @ w.ravel()).max() < 1e-7 * np.abs(K0).max() * np.abs(w).max()
    u = W.random_field(g, 2e-3 * g.h, seed=4)
    K = O.tangent_fd(g, mat, b, u, eps)
    w = W.random_field(g, 1.0, seed=5)
    jv = O.jvp_fd(g, mat, b, u, w, eps)
    np.testing.assert_allclose(K @ w.ravel(), jv.ravel(), atol=1e-6 * np.abs(jv).max())


# ------------------------------------------------------------ partial volume

def _cell_fraction_in_ball(d, m, samples=48):
    """Fraction of the lattice cell of offset d (a square or cube of side 1 in
    lattice units, centred on d) that lies inside the ball of radius m about the
    origin, by brute-force midpoint sampling: the geometric quantity that the
    partial volume V_ij approximates (the Remark of Sec. 3.1)."""
    q = (np.arange(samples) + 0.5) / samples - 0.5
    pts = np.stack(np.meshgrid(*([q] * len(d)), indexing="ij"), -1).reshape(-1, len(d)) + np.asarray(d, float)
    return float(((pts ** 2).sum(axis=1) <= m * m).mean())


def _two_point_vij(dim, d, m, h=0.01):
    """V_ij of the single bond between the lattice corners 0 and d, read off the
    oracle's PMB force: with only the far point displaced, every other bond of
    point 0 has eta = 0 and carries nothing, so f_0 = c s V V_ij (xi+eta)/|xi+eta|."""
    n = tuple(abs(int(x)) + 1 for x in d) + (1,) * (3 - dim)
    g = _grid(dim, n, m, h=h)
    mat = W.Material(model=W.PMB, E=72e9, vol_corr=1)
    b = O.neighbors(g)
    i0 = int(np.flatnonzero(np.all(g.coords()[:, :dim] == [0 if x >= 0 else abs(x) for x in d], axis=1))[0])
    j = int(np.flatnonzero(np.all(g.coords()[:, :dim] == [abs(x) if x >= 0 else 0 for x in d], axis=1))[0])
    xi = h * np.asarray(d, float)
    eta = 1e-4 * xi                                     # pure stretch along the bond: s = 1e-4
    u = np.zeros((g.npoints, dim))
    u[j] = eta
    f = O.pmb_force(g, mat, b, u)
    s = (np.linalg.norm(xi + eta) - np.linalg.norm(xi)) / np.linalg.norm(xi)
    V = h ** dim * (mat.thickness if dim == 2 else 1.0)
    return float(np.linalg.norm(f[i0]) / (O.micromodulus(g, mat) * s * V))


def test_partial_volume_of_a_bond_at_the_horizon_is_one_half():
    """A neighbour at exactly |xi| = delta: the horizon sphere cuts its cell
    through the centre, so half of V_j lies inside (flat-boundary value,
    hand-computed). A neighbour well inside keeps its full volume."""
    for dim, m in ((2, 3), (3, 3), (2, 5)):
        d = (m,) + (0,) * (dim - 1)
        assert abs(_two_point_vij(dim, d, m) - 0.5) < 1e-9
        d_in = (1,) + (0,) * (dim - 1)
        assert abs(_two_point_vij(dim, d_in, m) - 1.0) < 1e-9


@pytest.mark.parametrize("dim,m", [(2, 3), (2, 4), (2, 6), (3, 3), (3, 4)])
def test_partial_volume_matches_cell_ball_geometry(dim, m):
    """For every bond of the horizon's outer shell (|xi| > delta - h/2), the
    oracle's V_ij is within 0.06 of the fraction of the neighbour's cell inside
    the ball, computed by brute-force sampling; neither leaving the volume
    whole (error ~0.5) nor dropping the h/2 of the cell that reaches past the
    node (V_ij = (delta - |xi|)/h, error ~0.5) passes."""
    offs = set()
    rr = range(0, m + 1)
    for d in (np.array(t) for t in np.stack(np.meshgrid(*([rr] * dim), indexing="ij"), -1).reshape(-1, dim)):
        r = math.sqrt(float((d ** 2).sum()))
        if m - 0.5 < r <= m:
            offs.add(tuple(int(x) for x in sorted(d, reverse=True)))
    assert offs
    for d in sorted(offs):
        got = _two_point_vij(dim, d, m)
        want = _cell_fraction_in_ball(d, m)
        assert abs(got - want) < 0.06, (d, got, want)


# --------------------------------------------------------------- body force

@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_body_force_gives_uniform_acceleration(dim):
    """Eq. (3) with a uniform body force b on a free lattice at rest: every point
    moves together, so eta = 0 and the internal force vanishes, and the motion is
    the closed form u = (b/rho) t^2 / 2, v = (b/rho) t at every step (velocity-
    Verlet and central difference are exact for constant acceleration). Fixes
    the sign of b and its 1/rho."""
    g = _grid(dim, (6, 5, 4), 2, h=0.02)
    mat = W.Material(model=W.PMB, E=72e9, rho=2440.0)
    b = O.neighbors(g)
    bvec = np.array([3.0e5, -1.25e5, 0.5e5])[:dim]
    body = np.tile(bvec, (g.npoints, 1))
    a = bvec / mat.rho
    dt = 1e-4
    z = np.zeros((g.npoints, dim))
    st = O.ExplicitState(g, mat, b, z, z, b=body)
    done = 0
    for k in (1, 7, 20):                                # cumulative step counts
        st.run(dt, k - done)
        done = k
        t = k * dt
        np.testing.assert_allclose(st.u, np.tile(0.5 * a * t * t, (g.npoints, 1)), rtol=1e-12)
        np.testing.assert_allclose(st.v, np.tile(a * t, (g.npoints, 1)), rtol=1e-12)
        assert np.all(st.f == 0.0)
    ucd = O.run_central_difference(g, mat, b, z, z, dt, 20, b=body)
    np.testing.assert_allclose(ucd, np.tile(0.5 * a * (20 * dt) ** 2, (g.npoints, 1)), rtol=1e-12)


# ------------------------------------------------------ bond-state records

def test_run_records_break_steps_and_peak_stretches():
    """The per-bond records of a tracked run (the diagnostics that the GPU
    parity tests use for the near-s_c rule): tracking changes nothing in the
    run; a bond is broken exactly when its record has a break step, its peak
    stretch then exceeds s_c and otherwise does not; re-running an untracked
    state to one step before / at the recorded step finds it intact / broken;
    and the stretch of a bond is the same from both of its ends."""
    wl = W.block3d_pulse(nside=12, steps=30, s_c=5e-5)
    b_t = O.neighbors(wl.grid)
    O.break_notch(wl.grid, b_t, wl.notch)
    b_u = O.neighbors(wl.grid)
    O.break_notch(wl.grid, b_u, wl.notch)
    dt = wl.dt_factor * O.stable_dt(wl.grid, wl.mat, b_t)
    notch = b_t.broken.astype(bool).copy()
    tr = O.ExplicitState(wl.grid, wl.mat, b_t, wl.u0, wl.v0, track=True)
    un = O.ExplicitState(wl.grid, wl.mat, b_u, wl.u0, wl.v0)
    tr.run(dt, 10)
    tr.run(dt, 20)
    un.run(dt, 30)
    assert np.array_equal(tr.u, un.u) and np.array_equal(tr.v, un.v)
    assert np.array_equal(b_t.broken, b_u.broken)
    brk = b_t.broken.astype(bool) & ~notch
    assert brk.sum() > 10
    assert np.array_equal(brk, tr.brk_step >= 0)
    assert np.all(tr.s_max[brk] > wl.mat.s_c)
    assert np.all(tr.s_max[~brk & ~notch] <= wl.mat.s_c)
    assert np.all(tr.brk_step[notch] == -1)            # broken before the run, never evaluated
    rng = np.random.default_rng(0)
    for k in rng.choice(np.flatnonzero(brk), size=5, replace=False):
        step = int(tr.brk_step[k])
        for n, want in ((step - 1, False), (step, True)):
            b = O.neighbors(wl.grid)
            O.break_notch(wl.grid, b, wl.notch)
            O.ExplicitState(wl.grid, wl.mat, b, wl.u0, wl.v0).run(dt, n)   # n = 0: the initial force alone
            assert bool(b.broken[k]) == want
    s = O.bond_stretch(wl.grid, b_t, tr.u)
    rows = np.repeat(np.arange(wl.grid.npoints), np.diff(b_t.row_ptr))
    key = rows * wl.grid.npoints + b_t.col
    rkey = b_t.col.astype(np.int64) * wl.grid.npoints + rows
    order = np.argsort(key)
    mate = order[np.searchsorted(key[order], rkey)]
    assert np.array_equal(s, s[mate])
