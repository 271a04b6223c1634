"""Pins of the oracle's NP law (Algorithm 1: linearised bond strain, potential
psi(r) = C (1 - exp(-beta r)), influence J = 1 inside the open horizon) and its
linearisation LP, against facts fixed outside the force code: the continuum
energy density of a uniform expansion, force = -(1/V) dE/du, exact linearity
of LP, the small-strain limit NP -> LP, cancellation under affine maps, the
softening peak of psi' S, the excluded horizon boundary, and the step bound."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_06917_gb300 import workloads as W


def _mat(model, C=1.0, beta=1.0, rho=1.0):
    return W.Material(model=model, rho=rho, psi_c=C, psi_beta=beta)


def _interior(g, layers):
    c = g.coords()
    ok = np.ones(g.npoints, dtype=bool)
    for a in range(g.dim):
        ok &= (c[:, a] >= layers) & (c[:, a] < g.n[a] - layers)
    return ok


@pytest.mark.parametrize("dim,m,expect", [(2, 10, 2.0 / 3.0), (3, 6, 3.0 / 4.0)])
def test_uniform_expansion_energy_density_approaches_the_continuum_value(dim, m, expect):
    # u = eps X gives S = eps on every bond, so W = C beta eps^2 / (delta |B|) *
    # int_B |xi| dxi = (2/3) C beta eps^2 in 2D, (3/4) C beta eps^2 in 3D. The
    # lattice sum without the boundary shell (J = 0 at |xi| = delta) lies a few
    # per cent below (2D m = 10: -4.3 %; 3D m = 6: -1.4 %)
    n = (2 * m + 3, 2 * m + 3, 2 * m + 3 if dim == 3 else 1)
    g = W.Grid(dim=dim, n=n, h=0.01, m=m)
    eps = 1e-4
    u = eps * g.positions()
    for model in (W.LP, W.NP):
        mat = _mat(model, C=2.0, beta=3.0)
        b = O.neighbors(g)
        _, Wp = O.strain_energy(g, mat, b, u, per_point=True)
        centre = int(np.flatnonzero(_interior(g, m))[0])
        assert abs(Wp[centre] / (2.0 * 3.0 * eps * eps) - expect) <= 0.08 * expect


@pytest.mark.parametrize("model", [W.NP, W.LP])
def test_force_is_minus_the_energy_gradient(model):
    g = W.Grid(dim=2, n=(9, 8, 1), h=0.02, m=3)
    mat = _mat(model, C=1.5, beta=2.0)
    b = O.neighbors(g)
    rng = np.random.default_rng(5)
    u = rng.normal(0.0, 0.2 * g.h, (g.npoints, 2))      # strains of order 0.2: NP is well nonlinear
    f, _ = O.internal_force(g, mat, b, u)
    V = g.h * g.h * mat.thickness
    eps = 1e-6 * g.h
    for i in (0, 17, 40, g.npoints - 1):
        for a in range(2):
            up, um = u.copy(), u.copy()
            up[i, a] += eps
            um[i, a] -= eps
            dE = (O.strain_energy(g, mat, b, up) - O.strain_energy(g, mat, b, um)) / (2 * eps)
            assert abs(f[i, a] + dE / V) <= 1e-6 * np.abs(f).max()


def test_lp_is_exactly_linear_and_np_tends_to_lp_at_small_strain():
    g = W.Grid(dim=2, n=(10, 9, 1), h=0.01, m=3)
    b = O.neighbors(g)
    rng = np.random.default_rng(6)
    u, w = rng.normal(0.0, 1e-3, (2, g.npoints, 2))
    lp, npm = _mat(W.LP), _mat(W.NP)
    fu, _ = O.internal_force(g, lp, b, u)
    fw, _ = O.internal_force(g, lp, b, w)
    fuw, _ = O.internal_force(g, lp, b, u + w)
    f3, _ = O.internal_force(g, lp, b, 3.0 * u)
    sc = np.abs(fuw).max()
    assert np.abs(fuw - fu - fw).max() <= 1e-13 * sc
    assert np.abs(f3 - 3.0 * fu).max() <= 1e-13 * sc
    prev = None
    for amp in (1e-1, 1e-2, 1e-3):                      # relative gap ~ beta |xi| S^2 ~ amp^2
        fn, _ = O.internal_force(g, npm, b, amp * u)
        fl, _ = O.internal_force(g, lp, b, amp * u)
        gap = np.abs(fn - fl).max() / np.abs(fl).max()
        if prev is not None:
            assert gap <= 0.02 * prev
        prev = gap
    assert prev < 1e-6


@pytest.mark.parametrize("model", [W.NP, W.LP])
def test_affine_maps_give_zero_interior_force_and_translation_zero_force(model):
    g = W.Grid(dim=2, n=(14, 13, 1), h=0.01, m=3)
    b = O.neighbors(g)
    A = np.array([[3e-3, -1e-3], [2e-3, 1e-3]])
    u = g.positions() @ A.T
    f, _ = O.internal_force(g, _mat(model), b, u)
    inner = _interior(g, g.m)
    assert np.abs(f[inner]).max() <= 1e-12 * np.abs(f).max()
    assert np.abs(f[~inner]).max() > 0.0
    t, _ = O.internal_force(g, _mat(model), b, np.tile([0.3, -0.7], (g.npoints, 1)))
    assert not t.any()


def test_np_bond_force_softens_past_the_peak_of_psi_prime_s():
    # two points one spacing apart (m = 2, so the bond is inside the open
    # horizon): |f| ~ exp(-beta |xi| S^2) S peaks at |xi| S^2 = 1 / (2 beta)
    g = W.Grid(dim=2, n=(2, 1, 1), h=0.5, m=2)
    beta = 4.0
    mat = _mat(W.NP, beta=beta)
    b = O.neighbors(g)
    S_peak = math.sqrt(1.0 / (2.0 * beta * g.h))
    Ss = S_peak * np.linspace(0.5, 1.5, 41)
    mags = []
    for S in Ss:
        u = np.zeros((2, 2))
        u[1, 0] = S * g.h                                # S = eta . xi / |xi|^2
        f, _ = O.internal_force(g, mat, b, u)
        assert f[0, 1] == 0.0 and f[0, 0] == -f[1, 0]
        mags.append(f[0, 0])
    k = int(np.argmax(mags))
    assert abs(Ss[k] / S_peak - 1.0) <= 0.03
    assert mags[-1] < mags[k] and mags[0] < mags[k]


def test_bonds_on_the_horizon_boundary_carry_no_force():
    # |xi| = delta exactly (m = 1, one spacing): J = 0 for NP and LP, not for PMB
    g = W.Grid(dim=2, n=(2, 1, 1), h=0.5, m=1)
    b = O.neighbors(g)
    assert b.nbonds == 2
    u = np.array([[0.0, 0.0], [0.01, 0.0]])
    for model in (W.NP, W.LP):
        f, _ = O.internal_force(g, _mat(model), b, u)
        assert not f.any()
    fp, _ = O.internal_force(g, W.Material(model=W.PMB), b, u)
    assert fp.any()


def test_lp_step_bound_is_stable_below_and_divergent_above():
    g = W.Grid(dim=2, n=(16, 16, 1), h=1.0 / 16, m=3)
    mat = _mat(W.LP)
    b = O.neighbors(g)
    dtc = O.stable_dt(g, mat, b)
    u0 = W.gaussian_ic(g, (1e-3, 0.0), (0.5, 0.5), 0.01)
    v0 = np.zeros_like(u0)
    u = O.run_central_difference(g, mat, b, u0, v0, dtc, 400)
    assert np.abs(u).max() <= 10 * np.abs(u0).max()
    u = O.run_central_difference(g, mat, b, u0, v0, 2.5 * dtc, 400)
    assert not np.isfinite(u).all() or np.abs(u).max() > 1e3 * np.abs(u0).max()
