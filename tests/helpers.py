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


# precision names of the parametrised tests: (pd_run.precision, pd_run.state)
PRECISIONS = {"fp32c": (0, 0), "fp32c_df": (0, 1), "fp64": (1, 0)}


def gpu_sim(pd, grid, mat, precision, dt=0.0, notch=None, tile_log2=0, integrator=0, state=0, pair_threads=0):
    """A built simulation; precision is a PD_* value or a name of PRECISIONS."""
    if isinstance(precision, str):
        precision, state = PRECISIONS[precision]
    g, m, r = pd.describe(grid, mat, precision=precision, dt=dt, tile_log2=tile_log2, integrator=integrator,
                          state=state, pair_threads=pair_threads)
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


def broken_mates(row_ptr, col):
    """For every CSR entry (i, j), the index of the entry (j, i) (rows ascending)."""
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    key = rows * n + col
    order = np.argsort(key, kind="stable")
    return order[np.searchsorted(key[order], col.astype(np.int64) * n + rows)]


def assert_broken_match(brk_gpu, bonds, state, s_c, rel=1e-5):
    """Broken-bond sets (CSR order, user numbering) equal except for bonds whose
    stretch came within rel * s_c of s_c: for a bond that only the oracle broke,
    its stretch at the breaking step; for one that only the GPU broke, the
    largest stretch the oracle evaluated it at (state: a tracked oracle run).
    Returns the number of such mismatches."""
    ob = bonds.broken.astype(bool)
    mism = np.flatnonzero(np.asarray(brk_gpu, dtype=bool) != ob)
    if mism.size:
        smax = state.s_max[mism]
        bad = mism[~(np.abs(smax - s_c) <= rel * s_c)]
        assert bad.size == 0, "broken-bond mismatches away from s_c: %d (stretch %s)" % (
            bad.size, state.s_max[bad[:5]])
    return int(mism.size)
