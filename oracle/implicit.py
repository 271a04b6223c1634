"""FP64 oracle of the implicit (static) scheme: Newton on the residual of the
equation of motion with the inertia term dropped, f(u) + b = 0 (Eq. (3)), with
the stiffness matrix K = df/du assembled column by column from central
differences of the force (Eq. (6), Algorithm 3) and each linear system solved
densely (LU); or, matrix-free, by a plain restarted GMRES(m) on central
directional differences.

TEST INFRASTRUCTURE. Only the test suite may import this module. The CUDA
library and its Python binding never import it, and it never imports them.

Conventions (the same statement of the problem the library's static solve
takes, written out independently here):
  * a DOF whose kind is BC_DISPLACEMENT is held at its value; every other DOF
    is free;
  * r = f(u) + b on free DOFs; Newton solves (-K_ff) du = r_f, u_f += du;
  * stop when ||r_f|| <= newton_rtol * ||r_f(u_0)|| + newton_atol.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O

BC_DISPLACEMENT = 2


def gmres(matvec, b: np.ndarray, restart: int = 50, rtol: float = 1e-8, maxit: int = 100000):
    """Restarted GMRES(m) from x0 = 0 (Saad, Iterative Methods for Sparse Linear
    Systems, Algorithm 6.9 with Givens rotations, Sec. 6.5.3): Arnoldi by modified
    Gram-Schmidt, least squares by the rotated Hessenberg matrix. Stops when the
    true residual at a restart, or the rotated residual inside a cycle, is at most
    rtol * ||b||. Returns (x, iterations, converged)."""
    n = b.size
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0, True
    it = 0
    while True:
        r = b - matvec(x)
        beta = float(np.linalg.norm(r))
        if beta <= rtol * bnorm:
            return x, it, True
        if it >= maxit:
            return x, it, False
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        V[0] = r / beta
        g[0] = beta
        k = 0
        for j in range(restart):
            w = matvec(V[j])
            for i in range(j + 1):
                H[i, j] = float(np.dot(V[i], w))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / d if d > 0.0 else 1.0
            sn[j] = H[j + 1, j] / d if d > 0.0 else 0.0
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            if abs(g[j + 1]) <= rtol * bnorm or it >= maxit:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - float(np.dot(H[i, i + 1:k], y[i + 1:k]))) / H[i, i]
        x = x + V[:k].T @ y


def residual(grid, mat, bonds, u: np.ndarray, bc_kind: np.ndarray, b=None) -> np.ndarray:
    """r = f(u) + b, zero on prescribed DOFs; (n, dim)."""
    f, _ = O.internal_force(grid, mat, bonds, u)
    r = f + (0.0 if b is None else b)
    r[bc_kind == BC_DISPLACEMENT] = 0.0
    return r


def solve_static(grid, mat, bonds, u0: np.ndarray, bc_kind: np.ndarray, bc_val: np.ndarray, b=None,
                 linear: str = "lu", newton_rtol: float = 1e-12, newton_atol: float = 0.0, maxit: int = 20,
                 restart: int = 50, linear_rtol: float = 1e-12, eps: float | None = None,
                 linear_maxit: int = 2000):
    """Newton iteration of Sec. 5 for f(u) + b = 0 with prescribed displacements.

    linear = "lu": K by central differences of the force, one column per DOF
    (Eq. (6), Algorithm 3), eps = 1e-6 h by default, solved by LU on the free DOFs.
    linear = "gmres": matrix-free GMRES(restart) with the directional difference
    (f(u + e w) - f(u - e w)) / (2 e) as the product K w, e = 1e-5 h / max|w|
    (the oracle's stretch (|y| - |xi|)/|xi| cancels, so the difference needs a
    larger step than a column of the assembly); each solve stops at linear_rtol
    or linear_maxit iterations and Newton continues from there (inexact Newton).
    Returns (u, residual norms per Newton iterate, converged)."""
    n, d = grid.npoints, grid.dim
    eps = 1e-6 * grid.h if eps is None else eps
    kind = np.asarray(bc_kind).reshape(n, d)
    fixed = (kind == BC_DISPLACEMENT).reshape(-1)
    free = ~fixed
    u = np.array(u0, dtype=np.float64).reshape(-1).copy()
    u[fixed] = np.asarray(bc_val, dtype=np.float64).reshape(-1)[fixed]
    hist = []
    for it in range(maxit + 1):
        r = residual(grid, mat, bonds, u.reshape(n, d), kind, b).reshape(-1)
        rn = float(np.linalg.norm(r[free]))
        hist.append(rn)
        if rn <= newton_rtol * hist[0] + newton_atol:
            return u.reshape(n, d), hist, True
        if it == maxit:
            break
        if linear == "lu":
            K = O.tangent_fd(grid, mat, bonds, u.reshape(n, d), eps)
            du = np.linalg.solve(-K[np.ix_(free, free)], r[free])
        elif linear == "gmres":
            ucur = u.reshape(n, d).copy()

            def mv(wf):
                w = np.zeros(n * d)
                w[free] = wf
                wmax = float(np.abs(wf).max())
                if wmax == 0.0:
                    return np.zeros_like(wf)
                e = 1e-5 * grid.h / wmax
                return -O.jvp_fd(grid, mat, bonds, ucur, w.reshape(n, d), e).reshape(-1)[free]

            du, _, _ = gmres(mv, r[free], restart=restart, rtol=linear_rtol, maxit=linear_maxit)
        else:
            raise ValueError("linear must be 'lu' or 'gmres'")
        u[free] += du
    return u.reshape(n, d), hist, False
