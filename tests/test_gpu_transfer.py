"""State transfers through the C ABI: pd_set_state / pd_get_state with host
arrays (pageable numpy, pinned torch) go through a chunked pipeline (copies on
a second stream overlapping the per-chunk scatter or gather); device arrays are
used in place. Both routes must give the same staged state, bit for bit, and a
round trip must return the caller's values (exactly in FP64; to the
double-float pair's 2^-48 relative rounding in FP32C)."""
import numpy as np
import pytest

from paper_1806_06917_gb300 import workloads as W
from tests.helpers import gpu_sim

pytestmark = pytest.mark.gpu

# 3D 40^3 (1.5 MB per field: four chunks), 2D 400 x 300 (1.9 MB: four chunks), and
# small grids below 1 MB (one chunk), ragged against the tiles
GRIDS = [(3, (40, 40, 40)), (2, (400, 300, 1)), (3, (13, 11, 9)), (2, (37, 29, 1))]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06917_gb300 import pd as _pd
    return _pd, torch


def _sim(pd, dim, n, precision):
    grid = W.Grid(dim=dim, n=n, h=0.01, m=3)
    mat = W.Material(model=W.PMB, s_c=0.0)
    return gpu_sim(pd, grid, mat, precision), grid


def _fields(grid, seed):
    rng = np.random.default_rng(seed)
    u = 1e-4 * rng.standard_normal((grid.npoints, grid.dim)) + 0.3
    v = rng.standard_normal((grid.npoints, grid.dim))
    return u, v


@pytest.mark.parametrize("dim,n", GRIDS)
@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_host_round_trip(env, dim, n, prec):
    pd, torch = env
    precision = pd.PD_FP32C if prec == "fp32c" else pd.PD_FP64
    sim, grid = _sim(pd, dim, n, precision)
    u, v = _fields(grid, 5)
    pd.pd_set_state(sim, u=u, v=v)
    u2, v2 = pd.pd_get_state(sim)
    if precision == pd.PD_FP64:
        assert np.array_equal(u2, u) and np.array_equal(v2, v)
    else:
        for a, b in ((u2, u), (v2, v)):
            assert np.all(np.abs(a - b) <= 2.0 ** -47 * np.abs(b))
    sim.close()


@pytest.mark.parametrize("dim,n", GRIDS[:2])
@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_host_and_device_routes_agree(env, dim, n, prec):
    # the same state set from pageable host, pinned host, device and a host/device
    # mix, stepped, and read back to host and to device: all bit-identical
    pd, torch = env
    precision = pd.PD_FP32C if prec == "fp32c" else pd.PD_FP64
    outs = []
    for route in ("numpy", "pinned", "device", "mixed"):
        sim, grid = _sim(pd, dim, n, precision)
        u, v = _fields(grid, 9)
        if route == "numpy":
            pd.pd_set_state(sim, u=u, v=v)
        elif route == "pinned":
            pd.pd_set_state(sim, u=torch.from_numpy(u).pin_memory(), v=torch.from_numpy(v).pin_memory())
        elif route == "device":
            ud0, vd0 = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
            torch.cuda.synchronize()
            pd.pd_set_state(sim, u=ud0, v=vd0)
        else:
            vd0 = torch.from_numpy(v).cuda()
            torch.cuda.synchronize()
            pd.pd_set_state(sim, u=torch.from_numpy(u).pin_memory(), v=vd0)
        pd.pd_step_explicit(sim, 5)
        uh, vh = pd.pd_get_state(sim)
        ud = torch.empty((grid.npoints, grid.dim), dtype=torch.float64, device="cuda")
        vd = torch.empty_like(ud)
        torch.cuda.synchronize()
        pd.pd_get_state(sim, u=ud, v=vd)     # synchronous: the tensors are written on return
        up = torch.empty((grid.npoints, grid.dim), dtype=torch.float64).pin_memory()
        pd.pd_get_state(sim, u=up, want_v=False)
        assert np.array_equal(uh, ud.cpu().numpy()) and np.array_equal(vh, vd.cpu().numpy())
        assert np.array_equal(uh, up.numpy())
        outs.append((uh, vh))
        sim.close()
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])


def test_repeated_host_transfers_in_a_loop(env):
    # the bench's end-to-end loop: set (u, v) from pinned host, one step, read u
    # to pinned host, many times over without a host wait between the set and the
    # step; every read must equal a fresh single step from the same state
    pd, torch = env
    sim, grid = _sim(pd, 3, (40, 40, 40), pd.PD_FP32C)
    ref, _ = _sim(pd, 3, (40, 40, 40), pd.PD_FP32C)
    u, v = _fields(grid, 2)
    uh, vh = torch.from_numpy(u).pin_memory(), torch.from_numpy(v).pin_memory()
    uo = torch.empty_like(uh).pin_memory()
    pd.pd_set_state(ref, u=u, v=v)
    pd.pd_step_explicit(ref, 1)
    want, _ = pd.pd_get_state(ref, want_v=False)
    for _ in range(20):
        pd.pd_set_state(sim, u=uh, v=vh)
        pd.pd_step_explicit(sim, 1)
        pd.pd_get_state(sim, u=uo, want_v=False)
        assert np.array_equal(uo.numpy(), want)
    sim.close()
    ref.close()


@pytest.mark.parametrize("dim,n", [GRIDS[0], GRIDS[2]])
@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_pipelined_transfers_equal_the_synchronous_ones(env, dim, n, prec):
    """pd_set_state_async / pd_step_explicit / pd_get_state_async per step, one
    pd_io_sync at the end (the next step's upload overlapping this step's
    compute and download), with a different state every step and a result array
    per step: every result equals the synchronous loop's, bit for bit."""
    pd, torch = env
    precision = pd.PD_FP32C if prec == "fp32c" else pd.PD_FP64
    steps = 5
    ins = [_fields(W.Grid(dim=dim, n=n, h=0.01, m=3), 11 + k) for k in range(steps)]
    want = []
    sim, grid = _sim(pd, dim, n, precision)
    for u, v in ins:
        pd.pd_set_state(sim, u=u, v=v)
        pd.pd_step_explicit(sim, 1)
        want.append(pd.pd_get_state(sim, want_v=True))
    sim.close()
    sim, grid = _sim(pd, dim, n, precision)
    pin = [(torch.from_numpy(u).pin_memory(), torch.from_numpy(v).pin_memory()) for u, v in ins]
    outs = [(torch.empty(u.shape, dtype=torch.float64).pin_memory(),
             torch.empty(v.shape, dtype=torch.float64).pin_memory()) for u, v in ins]
    for (u, v), (uo, vo) in zip(pin, outs):
        pd.pd_set_state_async(sim, u=u, v=v)
        pd.pd_step_explicit(sim, 1)
        pd.pd_get_state_async(sim, u=uo, v=vo)
    pd.pd_io_sync(sim)
    # the last result again into one array written by every step (ordered copies)
    same = torch.empty(ins[0][0].shape, dtype=torch.float64).pin_memory()
    for u, v in pin:
        pd.pd_set_state_async(sim, u=u, v=v)
        pd.pd_step_explicit(sim, 1)
        pd.pd_get_state_async(sim, u=same)
    pd.pd_io_sync(sim)
    sim.close()
    for (uw, vw), (uo, vo) in zip(want, outs):
        assert np.array_equal(uo.numpy(), uw) and np.array_equal(vo.numpy(), vw)
    assert np.array_equal(same.numpy(), want[-1][0])


def test_async_calls_mix_with_synchronous_ones_and_device_arrays(env):
    """pd_get_state_async with v (the half-step velocity completed first), its
    result read after pd_io_sync; a synchronous pd_set_state / pd_get_state
    between asynchronous ones; device tensors through the async calls (used in
    place, stream-ordered): every read equals the synchronous reference."""
    pd, torch = env
    dim, n = GRIDS[0]
    grid = W.Grid(dim=dim, n=n, h=0.01, m=3)
    u0, v0 = _fields(grid, 21)
    u1, v1 = _fields(grid, 22)
    ref, _ = _sim(pd, dim, n, pd.PD_FP32C)
    pd.pd_set_state(ref, u=u0, v=v0)
    pd.pd_step_explicit(ref, 3)
    want0 = pd.pd_get_state(ref)
    pd.pd_set_state(ref, u=u1, v=v1)
    pd.pd_step_explicit(ref, 2)
    want1 = pd.pd_get_state(ref)
    ref.close()
    sim, _ = _sim(pd, dim, n, pd.PD_FP32C)
    pd.pd_set_state_async(sim, u=torch.from_numpy(u0).pin_memory(), v=torch.from_numpy(v0).pin_memory())
    pd.pd_step_explicit(sim, 3)
    uo, vo = (torch.empty(u0.shape, dtype=torch.float64).pin_memory() for _ in range(2))
    pd.pd_get_state_async(sim, u=uo, v=vo)
    pd.pd_io_sync(sim)
    assert np.array_equal(uo.numpy(), want0[0]) and np.array_equal(vo.numpy(), want0[1])
    # synchronous calls in between, then device tensors through the async ones
    pd.pd_set_state(sim, u=u1, v=v1)
    ud, vd = torch.from_numpy(u1).cuda(), torch.from_numpy(v1).cuda()
    pd.pd_set_state_async(sim, u=ud, v=vd, stream=torch.cuda.current_stream())
    pd.pd_step_explicit(sim, 2, torch.cuda.current_stream())
    uo2, vo2 = torch.empty_like(ud), torch.empty_like(vd)
    pd.pd_get_state_async(sim, u=uo2, v=vo2, stream=torch.cuda.current_stream())
    pd.pd_io_sync(sim)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(uo2.cpu().numpy(), want1[0]) and np.array_equal(vo2.cpu().numpy(), want1[1])
    u_s, v_s = pd.pd_get_state(sim)
    assert np.array_equal(u_s, want1[0]) and np.array_equal(v_s, want1[1])
    sim.close()
