"""Host logic of bench.py that needs no GPU: the lookup of recorded ncu traffic
by kernel and tile (null for an unrecorded tile or changed sources), and the
oracle's side rates on tiny samples (positive, labelled as the oracle with the
thread count it used)."""
import pytest

pytest.importorskip("torch")
import bench  # noqa: E402
from paper_1806_06917_gb300 import workloads as W  # noqa: E402


def test_traffic_lookup_is_keyed_by_kernel_tile_and_sources(monkeypatch):
    assert bench.ncu_traffic("pmb3", 7) is None              # no capture at that tile
    assert bench.ncu_traffic("no-such-kernel", 9) is None
    rec = dict(bench.NCU_TRAFFIC[("pmb3", 9)])
    rec["sha"] = "0" * 16                                      # sources changed since the capture
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("pmb3", 9), rec)
    assert bench.ncu_traffic("pmb3", 9) is None
    for key, rec in bench.NCU_TRAFFIC.items():
        assert rec["bytes"] > 0 and len(rec["sha"]) == 16 and rec["profile"].startswith("profiles/")


def test_oracle_side_rates_on_tiny_samples():
    pmb = bench.oracle_step_rate(W.block3d_pulse(nside=10), "a 10^3 block", target_s=0.2, max_steps=3)
    lps = bench.oracle_step_rate(W.block3d_lps(nside=8), "an 8^3 LPS block", target_s=0.2, max_steps=3)
    build = bench.oracle_build_rate(W.block3d_pulse(nside=10).grid, "a 10^3 lattice")
    for r in (pmb, lps, build):
        assert r["value"] > 0 and r["kind"] == "oracle" and r["cores"] >= 1 and r["sample"]
    assert pmb["unit"] == "bond-updates/s" and build["unit"] == "bonds/s"
