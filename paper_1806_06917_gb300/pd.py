"""Python binding of libpd (include/pd.h): the same entry points, argument
marshalling only. Every computation runs in the CUDA library; importing this
module raises if ``libpd.so`` has not been built.

Array arguments may be numpy arrays (host memory) or torch CUDA tensors (device
memory of the current device); both are passed to the library as raw pointers.
The binding checks dtype, contiguity and size before each call so that the
library never reads or writes outside the caller's buffers.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PD_LIBRARY may name another build of the same library (e.g. a variant for A/B timing)
LIB_PATH = os.environ.get("PD_LIBRARY") or os.path.join(_HERE, "_build", "libpd.so")

PD_OK, PD_EINVAL, PD_ENOMEM, PD_ECUDA, PD_ETIMEOUT, PD_EBUSY, PD_ENOTREADY, PD_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
PD_MODEL_PMB, PD_MODEL_LPS, PD_MODEL_NP, PD_MODEL_LP = 0, 1, 2, 3
PD_FP32C, PD_FP64 = 0, 1
PD_BC_FREE, PD_BC_VELOCITY, PD_BC_DISPLACEMENT = 0, 1, 2
PD_FORCE_UPDATE_BREAKING = 1
PD_JVP_MASK_DIRICHLET = 1
PD_KRYLOV_GMRES, PD_KRYLOV_CG = 0, 1
PD_TANGENT_CACHED, PD_TANGENT_JVP = 0, 1
PD_PRECOND_NONE, PD_PRECOND_BLOCK_JACOBI = 0, 1
PD_INTEGRATOR_VERLET, PD_INTEGRATOR_CD = 0, 1
PD_STATE_F64, PD_STATE_DF = 0, 1          # pd_run.state of a PD_FP32C simulation
PD_SERVE_PACKED, PD_SERVE_STREAMS = 0, 1   # pd_server_opts.mode
PD_REQ_QUEUED, PD_REQ_RUNNING, PD_REQ_DONE, PD_REQ_CANCELLED, PD_REQ_FAILED = 0, 1, 2, 3, 4

if not os.path.exists(LIB_PATH):
    raise ImportError("libpd.so is not built (%s); run __graft_entry__.build() or "
                      "python paper_1806_06917_gb300/build.py" % LIB_PATH)
_lib = ctypes.CDLL(LIB_PATH)


class pd_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("m", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("h", ctypes.c_double), ("origin", ctypes.c_double * 3)]


class pd_material(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("vol_corr", ctypes.c_int32), ("E", ctypes.c_double),
                ("rho", ctypes.c_double), ("K", ctypes.c_double), ("mu", ctypes.c_double),
                ("s_c", ctypes.c_double), ("thickness", ctypes.c_double), ("psi_c", ctypes.c_double),
                ("psi_beta", ctypes.c_double)]


class pd_run(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("dt_factor", ctypes.c_double), ("precision", ctypes.c_int32),
                ("tile_log2", ctypes.c_int32), ("integrator", ctypes.c_int32), ("state", ctypes.c_int32),
                ("pair_threads", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class pd_newton_opts(ctypes.Structure):
    _fields_ = [("krylov", ctypes.c_int32), ("restart", ctypes.c_int32), ("max_linear_iters", ctypes.c_int32),
                ("max_newton_iters", ctypes.c_int32), ("tangent", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("linear_rtol", ctypes.c_double),
                ("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double)]


class pd_newton_stats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int32), ("linear_iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("linear_failures", ctypes.c_int32), ("res0", ctypes.c_double), ("res", ctypes.c_double)]


class pd_server_opts(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_int64), ("max_active", ctypes.c_int32),
                ("quantum_steps", ctypes.c_int32), ("mode", ctypes.c_int32), ("wait_limit_ms", ctypes.c_int32),
                ("test_stall", ctypes.c_int32), ("pack_max_tiles", ctypes.c_int32),
                ("max_queued", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class pd_request(ctypes.Structure):
    _fields_ = [("grid", pd_grid), ("material", pd_material), ("run", pd_run), ("nsteps", ctypes.c_int64),
                ("u0", ctypes.c_void_p), ("v0", ctypes.c_void_p), ("bc_kind", ctypes.c_void_p),
                ("bc_val", ctypes.c_void_p), ("u_out", ctypes.c_void_p), ("v_out", ctypes.c_void_p)]


class pd_result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("error", ctypes.c_int32), ("tile_log2", ctypes.c_int32),
                ("pair_threads", ctypes.c_int32), ("steps_done", ctypes.c_int64), ("bonds", ctypes.c_int64),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double), ("end_s", ctypes.c_double),
                ("message", ctypes.c_char * 160)]


class PdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libpd error %d: %s" % (code, msg))
        self.code = code


_P = ctypes.c_void_p
_SIGS = {
    "pd_create": [ctypes.POINTER(_P), ctypes.POINTER(pd_grid), ctypes.POINTER(pd_material), ctypes.POINTER(pd_run)],
    "pd_destroy": [_P],
    "pd_last_error": [ctypes.c_char_p, ctypes.c_size_t],
    "pd_build_neighbors": [_P, _P],
    "pd_bond_count": [_P, ctypes.POINTER(ctypes.c_int64)],
    "pd_get_neighbors": [_P, _P, _P, _P, _P],
    "pd_get_broken": [_P, _P, _P],
    "pd_break_bonds": [_P, ctypes.c_int, ctypes.c_double, _P, _P, ctypes.POINTER(ctypes.c_int64), _P],
    "pd_set_state": [_P, _P, _P, _P],
    "pd_get_state": [_P, _P, _P, _P],
    "pd_set_state_async": [_P, _P, _P, _P],
    "pd_get_state_async": [_P, _P, _P, _P],
    "pd_io_sync": [_P],
    "pd_set_bc": [_P, _P, _P, _P],
    "pd_set_body_force": [_P, _P, _P],
    "pd_get_dt": [_P, ctypes.POINTER(ctypes.c_double)],
    "pd_set_dt": [_P, ctypes.c_double],
    "pd_get_step": [_P, ctypes.POINTER(ctypes.c_int64)],
    "pd_force": [_P, _P, _P, ctypes.c_uint, _P],
    "pd_dilatation": [_P, _P, _P, _P],
    "pd_step_explicit": [_P, ctypes.c_int64, _P],
    "pd_step_explicit_timed": [_P, ctypes.c_int64, _P, _P],
    "pd_tune_tile": [ctypes.POINTER(pd_grid), ctypes.POINTER(pd_material), ctypes.POINTER(pd_run), ctypes.c_int32,
                     ctypes.POINTER(ctypes.c_int32), _P],
    "pd_tune": [ctypes.POINTER(pd_grid), ctypes.POINTER(pd_material), ctypes.POINTER(pd_run), ctypes.c_int32,
                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), _P],
    "pd_jvp": [_P, _P, _P, _P, ctypes.c_uint, _P],
    "pd_vjp": [_P, _P, _P, _P, ctypes.c_uint, _P],
    "pd_energy": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _P],
    "pd_solve_static": [_P, ctypes.POINTER(pd_newton_opts), ctypes.POINTER(pd_newton_stats), _P],
    "pd_server_create": [ctypes.POINTER(_P), ctypes.POINTER(pd_server_opts)],
    "pd_server_destroy": [_P],
    "pd_submit": [_P, ctypes.POINTER(pd_request), ctypes.POINTER(ctypes.c_uint64)],
    "pd_poll": [_P, ctypes.c_uint64, ctypes.POINTER(pd_result)],
    "pd_wait": [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(pd_result)],
    "pd_cancel": [_P, ctypes.c_uint64],
    "pd_sum_noalloc": [_P, ctypes.c_int64, ctypes.c_double, _P, _P],
}
for _name, _args in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = ctypes.c_int

EXPORTS = tuple(_SIGS)


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    _lib.pd_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def _check(rc: int) -> None:
    if rc != PD_OK:
        raise PdError(rc, last_error())


CUDA_STREAM_LEGACY = 0x1   # cudaStreamLegacy: the legacy default stream


def _stream(stream):
    """None selects the simulation's own stream. A torch stream object passes its
    handle; torch's default stream has handle 0, which the C ABI would read as
    "own stream", so it is passed as cudaStreamLegacy instead."""
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return _P(stream.cuda_stream or CUDA_STREAM_LEGACY)
    return _P(int(stream))


def _buf(x, dtype, count, name, writable=False):
    """Raw pointer of a numpy array or torch tensor with exactly `count` elements."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):          # torch tensor
        import torch
        tdt = {np.float64: torch.float64, np.uint8: torch.uint8, np.int64: torch.int64,
               np.int32: torch.int32, np.float32: torch.float32}[dtype]
        if x.dtype != tdt or not x.is_contiguous() or x.numel() != count:
            raise ValueError("%s: need a contiguous %s tensor of %d elements" % (name, tdt, count))
        return _P(x.data_ptr())
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous or x.size != count:
        raise ValueError("%s: need a C-contiguous numpy %s array of %d elements" % (name, np.dtype(dtype), count))
    if writable and not x.flags.writeable:
        raise ValueError("%s: array is read-only" % name)
    return x.ctypes.data_as(_P)


class Sim:
    """Owner of one pd_sim handle; every method is the C call of the same name."""

    def __init__(self, grid: pd_grid, mat: pd_material, run: pd_run):
        h = _P()
        _check(_lib.pd_create(ctypes.byref(h), ctypes.byref(grid), ctypes.byref(mat), ctypes.byref(run)))
        self.h = h
        self.grid, self.mat, self.run = grid, mat, run
        self.dim = grid.dim
        self.npoints = grid.n[0] * grid.n[1] * grid.n[2]

    def close(self):
        if getattr(self, "h", None):
            _lib.pd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nvec(self):
        return self.npoints * self.dim


def pd_create(grid: pd_grid, mat: pd_material, run: pd_run) -> Sim:
    return Sim(grid, mat, run)


def pd_destroy(sim: Sim) -> None:
    sim.close()


def pd_build_neighbors(sim: Sim, stream=None) -> None:
    _check(_lib.pd_build_neighbors(sim.h, _stream(stream)))


def pd_bond_count(sim: Sim) -> int:
    v = ctypes.c_int64()
    _check(_lib.pd_bond_count(sim.h, ctypes.byref(v)))
    return v.value


def pd_get_neighbors(sim: Sim, row_ptr=None, col=None, perm=None, stream=None):
    """CSR in Morton numbering and the Morton permutation (allocated if not given)."""
    nb = pd_bond_count(sim)
    row_ptr = np.empty(sim.npoints + 1, np.int64) if row_ptr is None else row_ptr
    col = np.empty(nb, np.int32) if col is None else col
    perm = np.empty(sim.npoints, np.int64) if perm is None else perm
    _check(_lib.pd_get_neighbors(sim.h, _buf(row_ptr, np.int64, sim.npoints + 1, "row_ptr", True),
                                 _buf(col, np.int32, nb, "col", True),
                                 _buf(perm, np.int64, sim.npoints, "perm", True), _stream(stream)))
    return row_ptr, col, perm


def pd_get_broken(sim: Sim, out=None, stream=None):
    nb = pd_bond_count(sim)
    out = np.empty(nb, np.uint8) if out is None else out
    _check(_lib.pd_get_broken(sim.h, _buf(out, np.uint8, nb, "broken", True), _stream(stream)))
    return out


def pd_break_bonds(sim: Sim, axis: int, pos: float, lo, hi, stream=None) -> int:
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    if lo.size != 3 or hi.size != 3:
        raise ValueError("lo and hi need 3 entries")
    n = ctypes.c_int64()
    _check(_lib.pd_break_bonds(sim.h, int(axis), float(pos), _buf(lo, np.float64, 3, "lo"),
                               _buf(hi, np.float64, 3, "hi"), ctypes.byref(n), _stream(stream)))
    return n.value


def pd_set_state(sim: Sim, u=None, v=None, stream=None) -> None:
    _check(_lib.pd_set_state(sim.h, _buf(u, np.float64, sim.nvec, "u"), _buf(v, np.float64, sim.nvec, "v"),
                             _stream(stream)))


def pd_get_state(sim: Sim, u=None, v=None, stream=None, want_v: bool = True):
    """(u, v) at the current step; want_v=False reads u alone (v is None)."""
    u = np.empty((sim.npoints, sim.dim)) if u is None else u
    if v is None and want_v:
        v = np.empty((sim.npoints, sim.dim))
    _check(_lib.pd_get_state(sim.h, _buf(u, np.float64, sim.nvec, "u", True),
                             _buf(v, np.float64, sim.nvec, "v", True), _stream(stream)))
    return u, v


def pd_set_state_async(sim: Sim, u=None, v=None, stream=None) -> None:
    """pd_set_state without waiting for the work queued on the stream: u and v
    (pinned host arrays or device tensors) stay unchanged until pd_io_sync; the
    simulation keeps references to them until then."""
    _check(_lib.pd_set_state_async(sim.h, _buf(u, np.float64, sim.nvec, "u"), _buf(v, np.float64, sim.nvec, "v"),
                                   _stream(stream)))
    sim._io_keep = getattr(sim, "_io_keep", []) + [x for x in (u, v) if x is not None]


def pd_get_state_async(sim: Sim, u=None, v=None, stream=None) -> None:
    """Queue the read of u and/or v into the given arrays and return; they hold
    the result once pd_io_sync has returned."""
    if u is None and v is None:
        raise ValueError("pd_get_state_async needs u or v")
    _check(_lib.pd_get_state_async(sim.h, _buf(u, np.float64, sim.nvec, "u", True),
                                   _buf(v, np.float64, sim.nvec, "v", True), _stream(stream)))
    sim._io_keep = getattr(sim, "_io_keep", []) + [x for x in (u, v) if x is not None]


def pd_io_sync(sim: Sim) -> None:
    """Wait for every host-array copy of the simulation issued so far."""
    _check(_lib.pd_io_sync(sim.h))
    sim._io_keep = []


def pd_set_bc(sim: Sim, kind=None, value=None, stream=None) -> None:
    _check(_lib.pd_set_bc(sim.h, _buf(kind, np.uint8, sim.nvec, "kind"),
                          _buf(value, np.float64, sim.nvec, "value"), _stream(stream)))


def pd_set_body_force(sim: Sim, b=None, stream=None) -> None:
    _check(_lib.pd_set_body_force(sim.h, _buf(b, np.float64, sim.nvec, "b"), _stream(stream)))


def pd_get_dt(sim: Sim) -> float:
    v = ctypes.c_double()
    _check(_lib.pd_get_dt(sim.h, ctypes.byref(v)))
    return v.value


def pd_set_dt(sim: Sim, dt: float) -> None:
    _check(_lib.pd_set_dt(sim.h, float(dt)))


def pd_get_step(sim: Sim) -> int:
    v = ctypes.c_int64()
    _check(_lib.pd_get_step(sim.h, ctypes.byref(v)))
    return v.value


def pd_force(sim: Sim, u=None, f_out=None, flags: int = 0, stream=None):
    f_out = np.empty((sim.npoints, sim.dim)) if f_out is None else f_out
    _check(_lib.pd_force(sim.h, _buf(u, np.float64, sim.nvec, "u"),
                         _buf(f_out, np.float64, sim.nvec, "f_out", True), int(flags), _stream(stream)))
    return f_out


def pd_dilatation(sim: Sim, u=None, theta_out=None, stream=None):
    theta_out = np.empty(sim.npoints) if theta_out is None else theta_out
    _check(_lib.pd_dilatation(sim.h, _buf(u, np.float64, sim.nvec, "u"),
                              _buf(theta_out, np.float64, sim.npoints, "theta", True), _stream(stream)))
    return theta_out


def pd_tune_tile(grid: pd_grid, mat: pd_material, run: pd_run, steps: int = 10, stream=None) -> int:
    """The fastest tile_log2 for this description, measured (the C call of the same name)."""
    out = ctypes.c_int32()
    _check(_lib.pd_tune_tile(ctypes.byref(grid), ctypes.byref(mat), ctypes.byref(run), int(steps),
                             ctypes.byref(out), _stream(stream)))
    return out.value


def pd_tune(grid: pd_grid, mat: pd_material, run: pd_run, steps: int = 10, stream=None):
    """The fastest (tile_log2, pair_threads) for this description, measured."""
    tl, pt = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.pd_tune(ctypes.byref(grid), ctypes.byref(mat), ctypes.byref(run), int(steps), ctypes.byref(tl),
                        ctypes.byref(pt), _stream(stream)))
    return tl.value, pt.value


def pd_step_explicit(sim: Sim, nsteps: int, stream=None) -> None:
    _check(_lib.pd_step_explicit(sim.h, int(nsteps), _stream(stream)))


def pd_step_explicit_timed(sim: Sim, nsteps: int, stream=None):
    """The same steps, one launch at a time with CUDA events around each pass;
    returns the summed device milliseconds of (pass 0, pass 1)."""
    ms = (ctypes.c_double * 2)()
    _check(_lib.pd_step_explicit_timed(sim.h, int(nsteps), ms, _stream(stream)))
    return float(ms[0]), float(ms[1])


def pd_jvp(sim: Sim, w, u_lin=None, out=None, flags: int = 0, stream=None):
    out = np.empty((sim.npoints, sim.dim)) if out is None else out
    _check(_lib.pd_jvp(sim.h, _buf(u_lin, np.float64, sim.nvec, "u_lin"), _buf(w, np.float64, sim.nvec, "w"),
                       _buf(out, np.float64, sim.nvec, "out", True), int(flags), _stream(stream)))
    return out


def pd_vjp(sim: Sim, v, u_lin=None, out=None, flags: int = 0, stream=None):
    out = np.empty((sim.npoints, sim.dim)) if out is None else out
    _check(_lib.pd_vjp(sim.h, _buf(u_lin, np.float64, sim.nvec, "u_lin"), _buf(v, np.float64, sim.nvec, "v"),
                       _buf(out, np.float64, sim.nvec, "out", True), int(flags), _stream(stream)))
    return out


def newton_opts(krylov: int = PD_KRYLOV_GMRES, restart: int = 50, max_linear_iters: int = 20000,
                max_newton_iters: int = 20, linear_rtol: float = 1e-8, newton_rtol: float = 1e-8,
                newton_atol: float = 0.0, tangent: int = PD_TANGENT_CACHED,
                precond: int = PD_PRECOND_NONE) -> pd_newton_opts:
    """pd_newton_opts with the library's defaults."""
    return pd_newton_opts(krylov, restart, max_linear_iters, max_newton_iters, tangent, precond, linear_rtol,
                          newton_rtol, newton_atol)


def pd_solve_static(sim: Sim, opts: pd_newton_opts | None = None, stream=None) -> dict:
    """Newton-Krylov static equilibrium from the current state; returns the stats as a dict."""
    st = pd_newton_stats()
    _check(_lib.pd_solve_static(sim.h, ctypes.byref(opts) if opts is not None else None, ctypes.byref(st),
                                _stream(stream)))
    return {k: getattr(st, k) for k, _ in pd_newton_stats._fields_}


def _result(r: pd_result) -> dict:
    d = {k: getattr(r, k) for k, _ in pd_result._fields_ if k != "message"}
    d["message"] = r.message.decode(errors="replace")
    return d


class Server:
    """Owner of one pd_server handle. Requests keep their host arrays alive
    until the ticket has ended (the library copies the inputs at submit and
    writes the outputs at completion)."""

    def __init__(self, device_bytes: int = 0, max_active: int = 16, quantum_steps: int = 64,
                 mode: int = 0, wait_limit_ms: int = 0, test_stall: int = 0, pack_max_tiles: int = 0,
                 max_queued: int = 0):
        h = _P()
        opts = pd_server_opts(device_bytes, max_active, quantum_steps, mode, wait_limit_ms, test_stall,
                              pack_max_tiles, max_queued, 0)
        _check(_lib.pd_server_create(ctypes.byref(h), ctypes.byref(opts)))
        self.h = h
        self._keep = {}

    def close(self) -> None:
        if self.h:
            _check(_lib.pd_server_destroy(self.h))
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pd_server_create(device_bytes: int = 0, max_active: int = 16, quantum_steps: int = 64) -> Server:
    return Server(device_bytes, max_active, quantum_steps)


def pd_server_destroy(srv: Server) -> None:
    srv.close()


def pd_submit(srv: Server, grid: pd_grid, mat: pd_material, run: pd_run, nsteps: int, u0=None, v0=None,
              bc_kind=None, bc_val=None, u_out=None, v_out=None) -> int:
    """Queue a request; host numpy arrays of npoints x dim (u_out / v_out are
    written when it completes). Returns the ticket."""
    npts = grid.n[0] * grid.n[1] * (grid.n[2] if grid.dim == 3 else 1)
    nvec = npts * grid.dim
    arrs = {"u0": (u0, np.float64, False), "v0": (v0, np.float64, False), "bc_kind": (bc_kind, np.uint8, False),
            "bc_val": (bc_val, np.float64, False), "u_out": (u_out, np.float64, True),
            "v_out": (v_out, np.float64, True)}
    req = pd_request()
    req.grid, req.material, req.run, req.nsteps = grid, mat, run, int(nsteps)
    for name, (a, dt, wr) in arrs.items():
        if a is not None and hasattr(a, "data_ptr"):
            raise ValueError("%s: server requests take host numpy arrays" % name)
        p = _buf(a, dt, nvec, name, wr)
        setattr(req, name, p.value if p is not None else None)
    t = ctypes.c_uint64()
    _check(_lib.pd_submit(srv.h, ctypes.byref(req), ctypes.byref(t)))
    srv._keep[t.value] = (u_out, v_out)
    return t.value


def pd_poll(srv: Server, ticket: int) -> dict:
    r = pd_result()
    _check(_lib.pd_poll(srv.h, int(ticket), ctypes.byref(r)))
    return _result(r)


def pd_wait(srv: Server, ticket: int, timeout_s: float = 60.0) -> dict:
    """Block until the ticket ends (PdError with code PD_ETIMEOUT after timeout_s)."""
    r = pd_result()
    _check(_lib.pd_wait(srv.h, int(ticket), float(timeout_s), ctypes.byref(r)))
    return _result(r)


def pd_cancel(srv: Server, ticket: int) -> None:
    _check(_lib.pd_cancel(srv.h, int(ticket)))


def pd_energy(sim: Sim, stream=None):
    k, s = ctypes.c_double(), ctypes.c_double()
    _check(_lib.pd_energy(sim.h, ctypes.byref(k), ctypes.byref(s), _stream(stream)))
    return k.value, s.value


PD_SUM_NOALLOC_MAX_VALUES = 4194304


def pd_sum_noalloc(x, scale=1.0, out=None, stream=None):
    """scale * sum(x) in FP64 and fixed order, with no device allocation in the
    library. x and out are float64 CUDA tensors on the same device; out has one
    element. stream None means torch's current stream of x's device."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise ValueError("x: need a contiguous float64 CUDA tensor")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=x.device)
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1):
        raise ValueError("out: need a float64 CUDA tensor with one element")
    if out.device != x.device:
        raise ValueError("out must be on x's device (%s), got %s" % (x.device, out.device))
    # the library looks up its scratch array and launches on the current device;
    # the default stream is torch's current stream of x's device, so that the sum
    # is ordered after the work that produced x
    with torch.cuda.device(x.device):
        strm = torch.cuda.current_stream(x.device) if stream is None else stream
        _check(_lib.pd_sum_noalloc(_P(x.data_ptr()) if x.numel() else None, int(x.numel()), float(scale),
                                   _P(out.data_ptr()), _stream(strm)))
    return out


# ------------------------------------------------------------ conveniences

def describe(workload_grid, workload_mat, precision=PD_FP32C, dt=0.0, dt_factor=0.5, tile_log2=0,
             integrator=PD_INTEGRATOR_VERLET, state=0, pair_threads=0):
    """pd_grid / pd_material / pd_run from the plain workload descriptions."""
    g = pd_grid()
    g.dim = workload_grid.dim
    for a in range(3):
        g.n[a] = workload_grid.n[a]
        g.origin[a] = workload_grid.origin[a]
    g.m = workload_grid.m
    g.reserved = 0
    g.h = workload_grid.h
    m = pd_material()
    m.model = workload_mat.model
    m.vol_corr = workload_mat.vol_corr
    m.E, m.rho, m.K, m.mu = workload_mat.E, workload_mat.rho, workload_mat.K, workload_mat.mu
    m.s_c, m.thickness = workload_mat.s_c, workload_mat.thickness
    m.psi_c = getattr(workload_mat, "psi_c", 1.0)
    m.psi_beta = getattr(workload_mat, "psi_beta", 1.0)
    r = pd_run()
    r.dt, r.dt_factor, r.precision, r.tile_log2 = dt, dt_factor, precision, tile_log2
    r.integrator, r.state, r.pair_threads, r.reserved = integrator, state, pair_threads, 0
    return g, m, r
