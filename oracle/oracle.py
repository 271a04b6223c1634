"""ctypes front end of the FP64 CPU oracle (``pd_oracle.c``).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. The CUDA library and
its Python binding never import it, and it never imports them.

Inputs are the plain descriptions of ``paper_1806_06917_gb300.workloads``
(``Grid``, ``Material``) and numpy arrays in user order; everything is FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction) in-tree."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _OrGrid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("m", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("h", ctypes.c_double), ("ox", ctypes.c_double), ("oy", ctypes.c_double),
                ("oz", ctypes.c_double)]


class _OrMaterial(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("vol_corr", ctypes.c_int32),
                ("E", ctypes.c_double), ("rho", ctypes.c_double), ("K", ctypes.c_double),
                ("mu", ctypes.c_double), ("s_c", ctypes.c_double), ("thickness", ctypes.c_double),
                ("psi_c", ctypes.c_double), ("psi_beta", ctypes.c_double)]


_P = ctypes.c_void_p


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            sig = {
                "or_neighbors_brute": (i64, [_P, _P, _P]),
                "or_neighbors_cells": (i64, [_P, _P, _P]),
                "or_morton_perm": (i32, [_P, _P]),
                "or_break_notch": (i64, [_P, _P, _P, i32, dbl, _P, _P, _P]),
                "or_pmb_micromodulus": (dbl, [_P, _P]),
                "or_pmb_force": (None, [_P, _P, _P, _P, _P, _P, i32, _P]),
                "or_lps_weighted_volume": (None, [_P, _P, _P, _P, _P]),
                "or_lps_dilatation": (None, [_P, _P, _P, _P, _P, _P, _P, _P]),
                "or_lps_force": (None, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
                "or_lps_force_scatter": (None, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
                "or_internal_force": (None, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
                "or_strain_energy": (dbl, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
                "or_kinetic_energy": (dbl, [_P, _P, _P]),
                "or_stable_dt": (dbl, [_P, _P, _P, _P]),
                "or_run_verlet": (i32, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                        dbl, i64, _P, i32, _P]),
                "or_run_verlet_tracked": (i32, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                                dbl, i64, _P, i32, _P, _P, _P, i64]),
                "or_bond_stretch": (None, [_P, _P, _P, _P, _P]),
                "or_run_central_difference": (i32, [_P, _P, _P, _P, _P, _P, _P, _P, _P,
                                                    dbl, i64, _P]),
                "or_tangent_fd": (i32, [_P, _P, _P, _P, _P, _P, _P, dbl, _P]),
                "or_jvp_fd": (i32, [_P, _P, _P, _P, _P, _P, _P, _P, dbl, _P]),
                "or_num_threads": (i32, []),
                "or_set_num_threads": (None, [i32]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _grid(g) -> _OrGrid:
    return _OrGrid(g.dim, g.n[0], g.n[1], g.n[2], g.m, 0, g.h,
                   g.origin[0], g.origin[1], g.origin[2])


def _mat(m) -> _OrMaterial:
    return _OrMaterial(m.model, m.vol_corr, m.E, m.rho, m.K, m.mu, m.s_c, m.thickness, m.psi_c, m.psi_beta)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(_lib_handle().or_num_threads())


def set_num_threads(t: int) -> None:
    _lib_handle().or_set_num_threads(int(t))


class Bonds:
    """CSR neighbour lists in user numbering plus one broken byte per entry."""

    def __init__(self, row_ptr: np.ndarray, col: np.ndarray):
        self.row_ptr = row_ptr
        self.col = col
        self.broken = np.zeros(col.shape[0], dtype=np.uint8)

    @property
    def nbonds(self) -> int:
        return int(self.row_ptr[-1])

    def row(self, i: int) -> np.ndarray:
        return self.col[self.row_ptr[i]:self.row_ptr[i + 1]]


def neighbors(grid, method: str = "cells") -> Bonds:
    """B_delta(X_i) for every point (Sec. 3.1); method 'brute' or 'cells'."""
    lib = _lib_handle()
    g = _grid(grid)
    fn = lib.or_neighbors_brute if method == "brute" else lib.or_neighbors_cells
    row_ptr = np.zeros(grid.npoints + 1, dtype=np.int64)
    nb = fn(ctypes.byref(g), _ptr(row_ptr), None)
    if nb < 0:
        raise MemoryError("oracle neighbour count failed")
    col = np.zeros(int(nb), dtype=np.int32)
    fn(ctypes.byref(g), _ptr(row_ptr), _ptr(col))
    return Bonds(row_ptr, col)


def morton_perm(grid) -> np.ndarray:
    perm = np.zeros(grid.npoints, dtype=np.int64)
    if _lib_handle().or_morton_perm(ctypes.byref(_grid(grid)), _ptr(perm)) != 0:
        raise MemoryError("oracle Morton sort failed")
    return perm


def break_notch(grid, bonds: Bonds, notch) -> int:
    lo = np.asarray(notch.lo, dtype=np.float64)
    hi = np.asarray(notch.hi, dtype=np.float64)
    return int(_lib_handle().or_break_notch(ctypes.byref(_grid(grid)), _ptr(bonds.row_ptr),
                                            _ptr(bonds.col), int(notch.axis), float(notch.pos),
                                            _ptr(lo), _ptr(hi), _ptr(bonds.broken)))


def micromodulus(grid, mat) -> float:
    return float(_lib_handle().or_pmb_micromodulus(ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat))))


def weighted_volume(grid, mat, bonds: Bonds) -> np.ndarray:
    mv = np.zeros(grid.npoints)
    _lib_handle().or_lps_weighted_volume(ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat)),
                                         _ptr(bonds.row_ptr), _ptr(bonds.col), _ptr(mv))
    return mv


def pmb_force(grid, mat, bonds: Bonds, u, update_breaking: bool = False) -> np.ndarray:
    u = _c(u, np.float64)
    f = np.zeros((grid.npoints, grid.dim))
    _lib_handle().or_pmb_force(ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat)),
                               _ptr(bonds.row_ptr), _ptr(bonds.col), _ptr(u),
                               _ptr(bonds.broken), int(update_breaking), _ptr(f))
    return f


def dilatation(grid, mat, bonds: Bonds, mvol, u) -> np.ndarray:
    u = _c(u, np.float64)
    th = np.zeros(grid.npoints)
    _lib_handle().or_lps_dilatation(ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat)),
                                    _ptr(bonds.row_ptr), _ptr(bonds.col), _ptr(bonds.broken),
                                    _ptr(_c(mvol, np.float64)), _ptr(u), _ptr(th))
    return th


def lps_force(grid, mat, bonds: Bonds, mvol, theta, u, scatter: bool = False) -> np.ndarray:
    u = _c(u, np.float64)
    f = np.zeros((grid.npoints, grid.dim))
    fn = _lib_handle().or_lps_force_scatter if scatter else _lib_handle().or_lps_force
    fn(ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat)), _ptr(bonds.row_ptr), _ptr(bonds.col),
       _ptr(bonds.broken), _ptr(_c(mvol, np.float64)), _ptr(_c(theta, np.float64)), _ptr(u), _ptr(f))
    return f


def internal_force(grid, mat, bonds: Bonds, u, mvol=None):
    """Force of either model at u, no breaking update. Returns (f, theta or None)."""
    u = _c(u, np.float64)
    f = np.zeros((grid.npoints, grid.dim))
    th = np.zeros(grid.npoints)
    _lib_handle().or_internal_force(ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat)),
                                    _ptr(bonds.row_ptr), _ptr(bonds.col), _ptr(bonds.broken),
                                    _ptr(_c(mvol, np.float64)), _ptr(th), _ptr(u), _ptr(f))
    return f, (th if mat.model == 1 else None)


def strain_energy(grid, mat, bonds: Bonds, u, mvol=None, theta=None, per_point: bool = False):
    u = _c(u, np.float64)
    W = np.zeros(grid.npoints) if per_point else None
    tot = _lib_handle().or_strain_energy(ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat)),
                                         _ptr(bonds.row_ptr), _ptr(bonds.col), _ptr(bonds.broken),
                                         _ptr(_c(mvol, np.float64)), _ptr(_c(theta, np.float64)),
                                         _ptr(u), _ptr(W))
    return (float(tot), W) if per_point else float(tot)


def kinetic_energy(grid, mat, v) -> float:
    return float(_lib_handle().or_kinetic_energy(ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat)),
                                                 _ptr(_c(v, np.float64))))


def stable_dt(grid, mat, bonds: Bonds) -> float:
    return float(_lib_handle().or_stable_dt(ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat)),
                                            _ptr(bonds.row_ptr), _ptr(bonds.col)))


def bond_stretch(grid, bonds: Bonds, u) -> np.ndarray:
    """Stretch (|xi + eta| - |xi|) / |xi| of every directed bond (CSR order) at u."""
    out = np.zeros(bonds.nbonds)
    _lib_handle().or_bond_stretch(ctypes.byref(_grid(grid)), _ptr(bonds.row_ptr), _ptr(bonds.col),
                                  _ptr(_c(u, np.float64)), _ptr(out))
    return out


class ExplicitState:
    """u, v, the last force and the bond state of a velocity-Verlet run.

    With track=True the run also records, per directed bond (CSR order),
    ``s_max``: the largest stretch at which the bond was evaluated while intact
    (the evaluation that broke it included), and ``brk_step``: the step whose
    force evaluation broke it (0 = the initial force, -1 = never)."""

    def __init__(self, grid, mat, bonds: Bonds, u0, v0, bc_kind=None, bc_val=None, b=None, track=False):
        self.grid, self.mat, self.bonds = grid, mat, bonds
        self.u = np.array(u0, dtype=np.float64, order="C", copy=True)
        self.v = np.array(v0, dtype=np.float64, order="C", copy=True)
        self.bc_kind = _c(bc_kind, np.uint8)
        self.bc_val = _c(bc_val, np.float64)
        self.b = _c(b, np.float64)
        self.f = np.zeros_like(self.u)
        self.f_valid = False
        self.theta = np.zeros(grid.npoints)
        self.mvol = weighted_volume(grid, mat, bonds) if mat.model == 1 else None
        self.steps = 0
        self.s_max = np.full(bonds.nbonds, -np.inf) if track else None
        self.brk_step = np.full(bonds.nbonds, -1, dtype=np.int32) if track else None

    def run(self, dt: float, nsteps: int) -> None:
        rc = _lib_handle().or_run_verlet_tracked(
            ctypes.byref(_grid(self.grid)), ctypes.byref(_mat(self.mat)),
            _ptr(self.bonds.row_ptr), _ptr(self.bonds.col), _ptr(self.bonds.broken),
            _ptr(self.mvol), _ptr(self.u), _ptr(self.v), _ptr(self.b),
            _ptr(self.bc_kind), _ptr(self.bc_val), float(dt), int(nsteps),
            _ptr(self.f), int(self.f_valid), _ptr(self.theta),
            _ptr(self.s_max), _ptr(self.brk_step), int(self.steps))
        if rc != 0:
            raise MemoryError("oracle velocity-Verlet run failed")
        self.f_valid = True
        self.steps += int(nsteps)


def run_central_difference(grid, mat, bonds: Bonds, u0, v0, dt: float, nsteps: int, b=None):
    u = np.array(u0, dtype=np.float64, order="C", copy=True)
    mv = weighted_volume(grid, mat, bonds) if mat.model == 1 else None
    th = np.zeros(grid.npoints)
    rc = _lib_handle().or_run_central_difference(
        ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat)), _ptr(bonds.row_ptr), _ptr(bonds.col),
        _ptr(bonds.broken), _ptr(mv), _ptr(u), _ptr(_c(v0, np.float64)), _ptr(_c(b, np.float64)),
        float(dt), int(nsteps), _ptr(th))
    if rc != 0:
        raise MemoryError("oracle central-difference run failed")
    return u


def tangent_fd(grid, mat, bonds: Bonds, u, eps: float, mvol=None) -> np.ndarray:
    """Dense tangent K = df/du by central differences (Eq. (6), Algorithm 3)."""
    N = grid.npoints * grid.dim
    K = np.zeros((N, N))
    rc = _lib_handle().or_tangent_fd(ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat)),
                                     _ptr(bonds.row_ptr), _ptr(bonds.col), _ptr(bonds.broken),
                                     _ptr(_c(mvol, np.float64)), _ptr(_c(u, np.float64)),
                                     float(eps), _ptr(K))
    if rc != 0:
        raise MemoryError("oracle tangent assembly failed")
    return K


def jvp_fd(grid, mat, bonds: Bonds, u, w, eps: float, mvol=None) -> np.ndarray:
    out = np.zeros((grid.npoints, grid.dim))
    rc = _lib_handle().or_jvp_fd(ctypes.byref(_grid(grid)), ctypes.byref(_mat(mat)),
                                 _ptr(bonds.row_ptr), _ptr(bonds.col), _ptr(bonds.broken),
                                 _ptr(_c(mvol, np.float64)), _ptr(_c(u, np.float64)),
                                 _ptr(_c(w, np.float64)), float(eps), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle directional difference failed")
    return out
