"""Host logic of bench.py that needs no GPU: the lookup of recorded ncu traffic
by kernel and tile (null for an unrecorded tile or changed sources), and the
oracle's side rates on tiny samples (positive, labelled as the oracle with the
thread count it used)."""
import pytest

pytest.importorskip("torch")
import bench  # noqa: E402
from paper_1806_06917_gb300 import workloads as W  # noqa: E402


def _sources_sha(files):
    import hashlib
    import os
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(bench.ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def test_traffic_lookup_is_keyed_by_kernel_tile_and_sources(monkeypatch):
    files = ["paper_1806_06917_gb300/csrc/pd_force_lps.cu"] + bench._KERNEL_COMMON
    rec = {"bytes": 123456, "sha": _sources_sha(files), "sources": files, "profile": "profiles/x.md"}
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("lps_force", 9), rec)
    assert bench.ncu_traffic("lps_force", 9) == 123456
    assert bench.ncu_traffic("lps_force", 7) is None           # no capture at that tile
    assert bench.ncu_traffic("no-such-kernel", 9) is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("lps_force", 9), dict(rec, sha="0" * 16))
    assert bench.ncu_traffic("lps_force", 9) is None            # sources changed since the capture
    for key, r in bench.NCU_TRAFFIC.items():
        assert r["bytes"] > 0 and len(r["sha"]) == 16 and r["profile"].startswith("profiles/")


def test_roofline_of_the_lps_step():
    """The dominant launch is the force pass; its bytes are 4 B/bond + 120
    B/point, the step's 8 B/bond + 164 B/point; fractions against the peak."""
    wl = W.block3d_lps(nside=8)
    nb, npts = 10000, wl.grid.npoints
    r = bench.roofline_of("lps", wl, nb, [0.001, 0.002], 0.0031, 9, {"hbm_gbs": 5000.0})
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 5000.0
    want = (4.0 * nb + 120.0 * npts) / 2e-6 / 1e9
    assert abs(r["achieved"] - want) <= 1e-9 * want and abs(r["frac"] - want / 5000.0) <= 1e-12
    assert abs(r["step"]["bytes"] - (8.0 * nb + 164.0 * npts)) < 1e-6
    assert set(r["passes"]) == {"lps_dil", "lps_force"}
    r2 = bench.roofline_of("pmb3", W.block3d_pulse(nside=8), nb, [0.001, 0.0], 0.001, 9, None)
    assert r2["peak"] == bench.FALLBACK_HBM_GBS and "fallback" in r2["peak_source"]


def test_oracle_side_rates_on_tiny_samples():
    pmb = bench.oracle_step_rate(W.block3d_pulse(nside=10), "a 10^3 block", target_s=0.2, max_steps=3)
    lps = bench.oracle_step_rate(W.block3d_lps(nside=8), "an 8^3 LPS block", target_s=0.2, max_steps=3)
    build = bench.oracle_build_rate(W.block3d_pulse(nside=10).grid, "a 10^3 lattice")
    for r in (pmb, lps, build):
        assert r["value"] > 0 and r["kind"] == "oracle" and r["cores"] >= 1 and r["sample"]
    assert pmb["unit"] == "bond-updates/s" and build["unit"] == "bonds/s"
