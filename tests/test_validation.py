"""CPU-side checks of the descriptions pd_create validates before it touches a
device: every malformed grid, material or run parameter is refused with
PD_EINVAL and a message, and no simulation handle is returned. pd_create
validates first, so these run on a machine without a GPU."""
import pytest

from paper_1806_06917_gb300 import workloads as W


@pytest.fixture(scope="module")
def pd():
    from paper_1806_06917_gb300 import build as B
    B.build()
    from paper_1806_06917_gb300 import pd as _pd
    return _pd


def _good(pd, dim=3, model=W.PMB):
    grid = W.Grid(dim=dim, n=(8, 8, 8 if dim == 3 else 1), h=0.01, m=3)
    mat = {W.PMB: W.Material(model=W.PMB), W.LPS: W.Material(model=W.LPS, K=4e10, mu=3e10),
           W.NP: W.Material(model=W.NP, rho=1.0, psi_c=1.0, psi_beta=1.0, thickness=1.0)}[model]
    return pd.describe(grid, mat)


BAD = {
    "dim 4": lambda g, m, r: setattr(g, "dim", 4),
    "n[0] = 0": lambda g, m, r: g.n.__setitem__(0, 0),
    "2D with n[2] = 2": None,
    "m = 0": lambda g, m, r: setattr(g, "m", 0),
    "m = 25": lambda g, m, r: setattr(g, "m", 25),
    "h = 0": lambda g, m, r: setattr(g, "h", 0.0),
    "h = inf": lambda g, m, r: setattr(g, "h", float("inf")),
    "grid reserved": lambda g, m, r: setattr(g, "reserved", 1),
    "more than 1e9 points": lambda g, m, r: (g.n.__setitem__(0, 2000), g.n.__setitem__(1, 2000),
                                             g.n.__setitem__(2, 300)),
    "unknown model": lambda g, m, r: setattr(m, "model", 9),
    "rho = 0": lambda g, m, r: setattr(m, "rho", 0.0),
    "E = 0": lambda g, m, r: setattr(m, "E", 0.0),
    "s_c < 0": lambda g, m, r: setattr(m, "s_c", -1e-3),
    "unknown precision": lambda g, m, r: setattr(r, "precision", 5),
    "tile_log2 = 5": lambda g, m, r: setattr(r, "tile_log2", 5),
    "tile_log2 = 10": lambda g, m, r: setattr(r, "tile_log2", 10),
    "dt < 0": lambda g, m, r: setattr(r, "dt", -1e-6),
    "dt_factor < 0": lambda g, m, r: setattr(r, "dt_factor", -0.5),
    "unknown integrator": lambda g, m, r: setattr(r, "integrator", 2),
    "unknown state precision": lambda g, m, r: setattr(r, "state", 2),
    "pair_threads = 3": lambda g, m, r: setattr(r, "pair_threads", 3),
    "run reserved": lambda g, m, r: setattr(r, "reserved", 1),
    "FP64 path with double-float state": lambda g, m, r: (setattr(r, "precision", 1), setattr(r, "state", 1)),
}


@pytest.mark.parametrize("case", sorted(k for k, v in BAD.items() if v is not None))
def test_malformed_descriptions_are_refused(pd, case):
    g, m, r = _good(pd)
    BAD[case](g, m, r)
    with pytest.raises(pd.PdError) as e:
        pd.pd_create(g, m, r)
    assert e.value.code == pd.PD_EINVAL
    assert pd.last_error()


def test_2d_grid_needs_one_layer(pd):
    g, m, r = _good(pd, dim=2)
    g.n[2] = 2
    with pytest.raises(pd.PdError) as e:
        pd.pd_create(g, m, r)
    assert e.value.code == pd.PD_EINVAL


@pytest.mark.parametrize("case", ["lps 2D", "lps breaking", "lps K = 0", "np psi_beta = 0", "np breaking",
                                  "2D thickness 0"])
def test_model_specific_rules(pd, case):
    if case == "lps 2D":
        g, m, r = _good(pd, dim=2, model=W.LPS)
    elif case.startswith("lps"):
        g, m, r = _good(pd, model=W.LPS)
        if case == "lps breaking":
            m.s_c = 1e-3
        else:
            m.K = 0.0
    elif case.startswith("np"):
        g, m, r = _good(pd, model=W.NP)
        if case == "np breaking":
            m.s_c = 1e-3
        else:
            m.psi_beta = 0.0
    else:
        g, m, r = _good(pd, dim=2)
        m.thickness = 0.0
    with pytest.raises(pd.PdError) as e:
        pd.pd_create(g, m, r)
    assert e.value.code == pd.PD_EINVAL


def test_tune_tile_refuses_bad_arguments(pd):
    g, m, r = _good(pd)
    for steps in (0, -3):
        with pytest.raises(pd.PdError) as e:
            pd.pd_tune_tile(g, m, r, steps=steps)
        assert e.value.code == pd.PD_EINVAL
    # a malformed description fails the same way for every tile size
    g.m = 0
    with pytest.raises(pd.PdError) as e:
        pd.pd_tune_tile(g, m, r, steps=2)
    assert e.value.code == pd.PD_EINVAL


@pytest.mark.parametrize("opt", [dict(max_active=0), dict(max_active=257), dict(quantum_steps=0), dict(mode=7),
                                 dict(wait_limit_ms=-1), dict(pack_max_tiles=-1), dict(device_bytes=-1),
                                 dict(max_queued=-1)])
def test_server_options_are_refused_before_any_device_call(pd, opt):
    with pytest.raises(pd.PdError) as e:
        pd.Server(**opt)
    assert e.value.code == pd.PD_EINVAL
