"""Shared helpers of the test suite: run a workload through the CUDA library and
through the oracle, and compare CSR lists across numberings."""
import numpy as np

from oracle import oracle as O
from paper_1806_06917_gb300 import workloads as W


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def gpu_sim(pd, grid, mat, precision, dt=0.0, notch=None, tile_log2=0, integrator=0):
    g, m, r = pd.describe(grid, mat, precision=precision, dt=dt, tile_log2=tile_log2, integrator=integrator)
    sim = pd.pd_create(g, m, r)
    pd.pd_build_neighbors(sim)
    if notch is not None:
        pd.pd_break_bonds(sim, notch.axis, notch.pos, np.asarray(notch.lo), np.asarray(notch.hi))
    return sim


def gpu_csr_in_user_numbering(pd, sim):
    """(rows, cols) of every directed bond in user numbering, sorted, plus the
    raw Morton-numbered CSR and permutation."""
    row_ptr, col, perm = pd.pd_get_neighbors(sim)
    counts = np.diff(row_ptr)
    rows_u = np.repeat(perm, counts)
    cols_u = perm[col]
    order = np.lexsort((cols_u, rows_u))
    return rows_u[order], cols_u[order], order, (row_ptr, col, perm)


def oracle_pairs(bonds):
    counts = np.diff(bonds.row_ptr)
    rows = np.repeat(np.arange(len(counts), dtype=np.int64), counts)
    return rows, bonds.col.astype(np.int64)


def oracle_setup(wl, method="cells"):
    bonds = O.neighbors(wl.grid, method)
    if wl.notch is not None:
        O.break_notch(wl.grid, bonds, wl.notch)
    return bonds
