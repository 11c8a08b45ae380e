"""CPU checks of bench.py's roofline tables: every measured instruction mix names the five pipes,
the pipe bound is the arithmetic of 152 SMs x lanes x clock / instructions, and the headline's
binding pipe and bound match the figures quoted with it (issue, 1209 G/s at 2070 MHz)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_every_mix_names_the_five_pipes():
    for key, mix in bench.PIPE_MIX.items():
        assert set(mix) == {"issue", "fma", "alu", "xu", "lsu"}, key
        assert all(v > 0 for v in mix.values()), key
        # no pipe executes more instructions than are issued
        assert max(mix["fma"], mix["alu"], mix["xu"], mix["lsu"]) <= mix["issue"], key


def test_pipe_bound_arithmetic_and_headline():
    pipe, peak, bounds = bench.pipe_roofline(bench.PIPE_MIX["3d-vz-100k-256cube"], 2070.0)
    assert pipe == "issue"
    assert peak == pytest.approx(152 * 128 * 2070e6 / bench.PIPE_MIX["3d-vz-100k-256cube"]["issue"] / 1e9)
    assert round(peak) == 1209
    assert bounds["xu"] == pytest.approx(152 * 16 * 2070e6 / bench.PIPE_MIX["3d-vz-100k-256cube"]["xu"] / 1e9)
    # the bound scales with the clock
    _, peak_half, _ = bench.pipe_roofline(bench.PIPE_MIX["3d-vz-100k-256cube"], 1035.0)
    assert peak_half == pytest.approx(peak / 2)


def test_traffic_entries_are_measured_kernels():
    for key, nbytes in bench.TRAFFIC.items():
        assert key in bench.PIPE_MIX, key
        assert nbytes > 0


def test_workload_models_match_their_surveys():
    # the mix guard compares a run's (velocity, weight) with the workload's own: they must agree
    wl = bench.workloads()
    for name, (vel, weight) in bench.WORKLOAD_MODEL.items():
        assert name in wl, name
        s = wl[name]()
        assert (s.vel, s.weight) == (vel, weight), name
        assert (getattr(s, "aa_spacing", 0.0) > 0) == ("-aa-" in name), name
    for key in bench.PIPE_MIX:
        base = key.split("-table-")[0].replace("-demigrate", "").replace("-vgrad", "").replace("-f32", "")
        assert base in wl or base.replace("3d-vz", "3d-pstm") in wl or base.startswith("batch"), key
