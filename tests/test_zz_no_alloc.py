"""The allocation-free sum (pd_sum_noalloc) against pd_energy's own reduction.

Some callers of this library may not allocate device memory themselves (a host
framework that owns every allocation, or a loop where cudaMalloc's implicit
synchronisation is not allowed). pd_sum_noalloc serves them with the same
fixed-order FP64 sum that pd_energy uses, its scratch in a static device array.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import numpy as np
import pytest

from paper_1806_06917_gb300 import workloads as W
from tests.helpers import gpu_sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06917_gb300 import pd
    return torch, pd


def test_noalloc_sum_matches_energy_reduction_on_two_calls(env):
    torch, pd = env
    grid = W.Grid(dim=3, n=(40, 37, 33), h=0.01, m=3)
    mat = W.Material(model=W.PMB, E=72e9, rho=2440.0)
    sim = gpu_sim(pd, grid, mat, pd.PD_FP64)
    v = W.random_field(grid, 0.7, seed=12)
    pd.pd_set_state(sim, u=np.zeros_like(v), v=v)
    kinetic, _ = pd.pd_energy(sim)                         # the existing entry point
    x = torch.from_numpy((v * v).sum(axis=1)).cuda()        # |v_i|^2 per point
    scale = 0.5 * mat.rho * grid.h ** 3
    stream = torch.cuda.current_stream()
    for _ in range(2):                                      # two calls in a row
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        pd.pd_sum_noalloc(x, scale, out, stream=stream)
        torch.cuda.synchronize()
        assert abs(out.item() - kinetic) <= 1e-12 * kinetic
    sim.close()


def test_noalloc_sum_limits(env):
    torch, pd = env
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    pd.pd_sum_noalloc(torch.empty(0, dtype=torch.float64, device="cuda"), 1.0, out)
    torch.cuda.synchronize()
    assert out.item() == 0.0
    n = pd.PD_SUM_NOALLOC_MAX_VALUES
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    pd.pd_sum_noalloc(x, 0.5, out)
    torch.cuda.synchronize()
    assert out.item() == 0.5 * n
    with pytest.raises(pd.PdError) as e:
        pd.pd_sum_noalloc(torch.ones(n + 1, dtype=torch.float64, device="cuda"), 1.0, out)
    assert e.value.code == pd.PD_EINVAL and "4194304" in str(e.value)
