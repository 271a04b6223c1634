"""GPU: the request server (pd_server_* / pd_submit / pd_poll / pd_wait /
pd_cancel). A served request's result must equal, bit for bit, the same
simulation run alone through the ordinary entry points with the tile size and
threads per point pair the server reports, whether it ran in the packed kernel
(with whatever else was packed with it) or on its own stream; admission must
respect the memory budget; cancellation and bounded waits (host-side, and the
packed kernel's device-side wait) must work without touching the GPU's state."""
import time

import numpy as np
import pytest

from paper_1806_06917_gb300 import workloads as W
from tests.helpers import gpu_sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06917_gb300 import pd as _pd
    return _pd


def _submit(pd, srv, r, u_out=None, v_out=None, precision=None, tile_log2=0, integrator=0):
    g, m, run = pd.describe(r.grid, r.mat, precision=pd.PD_FP32C if precision is None else precision,
                            tile_log2=tile_log2, integrator=integrator)
    return pd.pd_submit(srv, g, m, run, r.steps, u0=r.u0, v0=np.zeros_like(r.u0), u_out=u_out, v_out=v_out)


def _alone(pd, r, tile_log2, precision=None, integrator=0, pair_threads=0):
    sim = gpu_sim(pd, r.grid, r.mat, pd.PD_FP32C if precision is None else precision, tile_log2=tile_log2,
                  integrator=integrator, pair_threads=pair_threads)
    pd.pd_set_state(sim, u=r.u0, v=np.zeros_like(r.u0))
    pd.pd_step_explicit(sim, r.steps)
    u, v = pd.pd_get_state(sim)
    sim.close()
    return u, v


def _small_mix(count, seed):
    return W.serving_mix(count=count, seed=seed, side_median=14.0, side_sigma=0.4, side_lo=6, side_hi=28,
                         steps_lo=5, steps_hi=70, m_choices=(2, 3))


@pytest.mark.parametrize("mode", ["packed", "streams", "packed_small_only"])
def test_served_results_equal_the_same_runs_alone(pd, mode):
    # packed_small_only: requests of more than 4 tiles run on their own streams
    # beside the packed kernel, which steps the rest
    mix = _small_mix(10, 21)
    assert {r.grid.dim for r in mix} == {2, 3} and {r.mat.model for r in mix} == {W.PMB, W.LPS}
    if mode == "packed_small_only":
        tiles = [(r.grid.npoints + 511) // 512 for r in mix]
        assert min(tiles) <= 4 < max(tiles)
    srv = pd.Server(max_active=3, quantum_steps=7,        # quanta that do not divide the step counts
                    mode=pd.PD_SERVE_STREAMS if mode == "streams" else pd.PD_SERVE_PACKED,
                    pack_max_tiles=4 if mode == "packed_small_only" else 0)
    outs = [(np.full(r.u0.shape, np.nan), np.full(r.u0.shape, np.nan)) for r in mix]
    tickets = [_submit(pd, srv, r, u_out=o[0], v_out=o[1]) for r, o in zip(mix, outs)]
    results = [pd.pd_wait(srv, t, timeout_s=120.0) for t in tickets]
    srv.close()
    for r, res, (u, v) in zip(mix, results, outs):
        assert res["state"] == pd.PD_REQ_DONE and res["error"] == pd.PD_OK, res["message"]
        assert res["steps_done"] == r.steps and res["bonds"] > 0
        assert 0.0 < res["submit_s"] <= res["start_s"] <= res["end_s"]
        if mode == "packed":
            assert res["tile_log2"] == 9 and res["pair_threads"] in (1, 2) or r.mat.model == W.LPS
        ua, va = _alone(pd, r, res["tile_log2"], pair_threads=res["pair_threads"])
        assert np.array_equal(u, ua) and np.array_equal(v, va)


def test_a_request_is_the_same_alone_and_in_a_packed_mix(pd):
    """The same request served alone and among others in the packed kernel:
    bit-identical results (its work items run the same arithmetic whatever is
    packed beside them)."""
    mix = _small_mix(8, 31)
    probe = [r for r in mix if r.mat.model == W.LPS][0]
    res = []
    for others in (False, True):
        srv = pd.Server(max_active=8, quantum_steps=5)
        u = np.full(probe.u0.shape, np.nan)
        t = _submit(pd, srv, probe, u_out=u)
        ts = [_submit(pd, srv, r) for r in mix if r is not probe] if others else []
        rp = pd.pd_wait(srv, t, timeout_s=120.0)
        for x in ts:
            assert pd.pd_wait(srv, x, timeout_s=120.0)["state"] == pd.PD_REQ_DONE
        srv.close()
        assert rp["state"] == pd.PD_REQ_DONE, rp
        res.append(u)
    assert np.array_equal(res[0], res[1])


def test_packed_kernel_wait_runs_out_and_the_server_goes_on(pd):
    """test_stall: the first packed quantum's first LPS force item waits for a
    flag that nothing sets; its bounded wait (200 ms) runs out, the launch ends,
    the quantum's request fails with PD_ETIMEOUT, and the next request is served
    normally (the GPU context is intact)."""
    mix = _small_mix(12, 41)
    lps = [r for r in mix if r.mat.model == W.LPS][:2]
    srv = pd.Server(max_active=1, quantum_steps=4, wait_limit_ms=200, test_stall=1)
    first = pd.pd_wait(srv, _submit(pd, srv, lps[0]), timeout_s=60.0)
    assert first["state"] == pd.PD_REQ_FAILED and first["error"] == pd.PD_ETIMEOUT, first
    assert "wait ran out" in first["message"]
    u = np.full(lps[1].u0.shape, np.nan)
    second = pd.pd_wait(srv, _submit(pd, srv, lps[1], u_out=u), timeout_s=60.0)
    srv.close()
    assert second["state"] == pd.PD_REQ_DONE, second
    ua, _ = _alone(pd, lps[1], second["tile_log2"], pair_threads=second["pair_threads"])
    assert np.array_equal(u, ua)


def test_a_full_queue_refuses_new_requests(pd):
    """max_queued: with the one active slot held by a long request and two more
    waiting, the next submit is refused with PD_EBUSY and nothing is queued; once
    the queue has drained, submits are accepted again."""
    g3 = W.Grid(dim=3, n=(20, 20, 20), h=0.05, m=3)
    held = W.Request(grid=g3, mat=W.Material(model=W.PMB), steps=10 ** 7, arrival=0.0,
                     u0=np.zeros((g3.npoints, 3)), seed=0)
    short = _small_mix(3, 51)
    srv = pd.Server(max_active=1, quantum_steps=16, max_queued=2)
    t0 = _submit(pd, srv, held)
    for _ in range(4000):                                  # admission is asynchronous
        if pd.pd_poll(srv, t0)["state"] == pd.PD_REQ_RUNNING:
            break
        time.sleep(0.005)
    assert pd.pd_poll(srv, t0)["state"] == pd.PD_REQ_RUNNING
    waiting = [_submit(pd, srv, short[0]), _submit(pd, srv, short[1])]
    with pytest.raises(pd.PdError) as e:
        _submit(pd, srv, short[2])
    assert e.value.code == pd.PD_EBUSY
    pd.pd_cancel(srv, t0)
    assert pd.pd_wait(srv, t0, timeout_s=120.0)["state"] == pd.PD_REQ_CANCELLED
    for t in waiting:
        assert pd.pd_wait(srv, t, timeout_s=120.0)["state"] == pd.PD_REQ_DONE
    again = pd.pd_wait(srv, _submit(pd, srv, short[2]), timeout_s=120.0)
    srv.close()
    assert again["state"] == pd.PD_REQ_DONE


def test_central_difference_requests_equal_the_same_runs_alone(pd):
    # the CD state (u^{k-1} in the other staging buffer) carries across quanta
    mix = _small_mix(4, 23)
    srv = pd.Server(max_active=2, quantum_steps=9)
    outs = [np.full(r.u0.shape, np.nan) for r in mix]
    tickets = [_submit(pd, srv, r, u_out=o, integrator=pd.PD_INTEGRATOR_CD) for r, o in zip(mix, outs)]
    results = [pd.pd_wait(srv, t, timeout_s=120.0) for t in tickets]
    srv.close()
    for r, res, u in zip(mix, results, outs):
        assert res["state"] == pd.PD_REQ_DONE, res
        ua, _ = _alone(pd, r, res["tile_log2"], integrator=pd.PD_INTEGRATOR_CD, pair_threads=res["pair_threads"])
        assert np.array_equal(u, ua)


def test_fp64_requests_are_served_too(pd):
    r = _small_mix(1, 22)[0]
    srv = pd.Server(max_active=2, quantum_steps=16)
    u = np.full(r.u0.shape, np.nan)
    t = _submit(pd, srv, r, u_out=u, precision=pd.PD_FP64)
    res = pd.pd_wait(srv, t, timeout_s=120.0)
    srv.close()
    assert res["state"] == pd.PD_REQ_DONE
    ua, _ = _alone(pd, r, res["tile_log2"], precision=pd.PD_FP64, pair_threads=res["pair_threads"])
    assert np.array_equal(u, ua)


def test_admission_respects_the_memory_budget(pd):
    # requests of ~20 MB each under a 50 MB budget: at most two run at once
    reqs = []
    for k in range(5):
        g = W.Grid(dim=2, n=(190, 190, 1), h=1.0 / 190, m=3)
        u0 = np.random.default_rng(100 + k).normal(0.0, 1e-4 * g.h, (g.npoints, 2))
        reqs.append(W.Request(grid=g, mat=W.Material(model=W.PMB), steps=200, arrival=0.0, u0=u0, seed=k))
    srv = pd.Server(device_bytes=50 << 20, max_active=8, quantum_steps=32)
    tickets = [_submit(pd, srv, r) for r in reqs]
    res = [pd.pd_wait(srv, t, timeout_s=120.0) for t in tickets]
    srv.close()
    assert all(x["state"] == pd.PD_REQ_DONE for x in res)
    events = sorted([(x["start_s"], 1) for x in res] + [(x["end_s"], -1) for x in res])
    live = peak = 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak <= 2
    # a request above the whole budget is refused at submission
    tiny = pd.Server(device_bytes=1 << 20)
    with pytest.raises(pd.PdError) as e:
        _submit(pd, tiny, reqs[0])
    assert e.value.code == pd.PD_EINVAL
    tiny.close()


def test_cancel_bounded_wait_and_unknown_tickets(pd):
    g = W.Grid(dim=3, n=(24, 24, 24), h=1.0 / 24, m=3)
    u0 = np.random.default_rng(7).normal(0.0, 1e-4 * g.h, (g.npoints, 3))
    long_req = W.Request(grid=g, mat=W.Material(model=W.PMB), steps=10 ** 7, arrival=0.0, u0=u0, seed=7)
    srv = pd.Server(max_active=1, quantum_steps=64)
    u_a = np.full(u0.shape, np.nan)
    a = _submit(pd, srv, long_req, u_out=u_a)
    b = _submit(pd, srv, long_req)                         # waits behind a (max_active = 1)
    with pytest.raises(pd.PdError) as e:
        pd.pd_wait(srv, a, timeout_s=0.2)
    assert e.value.code == pd.PD_ETIMEOUT
    pd.pd_cancel(srv, b)                                   # queued: ends at once
    rb = pd.pd_wait(srv, b, timeout_s=5.0)
    assert rb["state"] == pd.PD_REQ_CANCELLED and rb["start_s"] == 0.0
    pd.pd_cancel(srv, a)                                   # running: ends after its quantum
    ra = pd.pd_wait(srv, a, timeout_s=30.0)
    assert ra["state"] == pd.PD_REQ_CANCELLED and 0 < ra["steps_done"] < long_req.steps
    assert np.isnan(u_a).all()                             # outputs of a cancelled request are not written
    for bad in (0, 999):
        with pytest.raises(pd.PdError):
            pd.pd_poll(srv, bad)
    srv.close()


def test_invalid_requests_are_refused_and_destroy_cancels_the_rest(pd):
    srv = pd.Server(max_active=1)
    g = W.Grid(dim=2, n=(20, 20, 1), h=0.05, m=3)
    gd, md, rd = pd.describe(g, W.Material(model=W.PMB))
    gd.m = 0
    with pytest.raises(pd.PdError) as e:
        pd.pd_submit(srv, gd, md, rd, 10)
    assert e.value.code == pd.PD_EINVAL
    g3 = W.Grid(dim=3, n=(20, 20, 20), h=0.05, m=3)
    u0 = np.zeros((g3.npoints, 3))
    r = W.Request(grid=g3, mat=W.Material(model=W.PMB), steps=10 ** 7, arrival=0.0, u0=u0, seed=0)
    tickets = [_submit(pd, srv, r) for _ in range(3)]
    srv.close()                                            # returns: the running one stops after a quantum
    assert srv.h is None and len(tickets) == 3
