"""The binning sort (the step before Eq. 1's sum): offset bin (Eq. 1's delta) and midpoint
cell per trace, a stable radix sort over all SMs, and the per-(bin, cell) starts.  Compared
bit for bit with numpy's stable sort of the same keys, where each key's bin comes from the
FP64 oracle; up to 10^7 traces.  Then the migration with the per-tile cell ranges keeps the
same (point, trace) pairs as the whole-bin scan (same image up to FP32 summation order)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, gpu_migrate, rel_l2
from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu


def expected_order(s, grid):
    """Keys from the oracle's offset bins and the documented cell formula; numpy stable sort."""
    b = oracle.bins(s).astype(np.int64)
    ncell = grid["ncx"] * grid["ncy"]
    nkeys = s.n_bins * ncell
    key = np.full(s.ntr, nkeys, dtype=np.int64)
    ok = b >= 0
    if grid["inv_cell"] > 0:
        mx = ((s.sx + s.rx) * np.float32(0.5)).astype(np.float32).astype(np.float64)
        my = ((s.sy + s.ry) * np.float32(0.5)).astype(np.float32).astype(np.float64)
        cx = np.floor((mx - grid["gx0"]) * grid["inv_cell"])
        cy = np.floor((my - grid["gy0"]) * grid["inv_cell"]) if s.dim == 3 else np.zeros_like(cx)
        ok &= (cx >= 0) & (cx < grid["ncx"]) & (cy >= 0) & (cy < grid["ncy"])
        key[ok] = b[ok] * ncell + cy[ok].astype(np.int64) * grid["ncx"] + cx[ok].astype(np.int64)
    else:
        key[ok] = b[ok] * ncell
    order = np.argsort(key, kind="stable")
    nkept = int(ok.sum())
    starts = np.searchsorted(key[order], np.arange(nkeys + 1), side="left")
    return order[:nkept], starts


def random_headers(rng, dim, ntr, extent):
    sx, rx = rng.uniform(-200, extent + 200, ntr), rng.uniform(-200, extent + 200, ntr)
    sy = rng.uniform(-200, extent + 200, ntr) if dim == 3 else np.zeros(ntr)
    ry = rng.uniform(-200, extent + 200, ntr) if dim == 3 else np.zeros(ntr)
    return [np.asarray(a, np.float32) for a in (sx, sy, rx, ry)]


def check_sort(s, spatial=True):
    p = kh.Plan(s)
    p.set_spatial_sort(spatial)
    hdr = kh.Headers.of(s)
    perm, starts, grid = p.bin_sort(hdr)
    want_perm, want_starts = expected_order(s, grid)
    got_starts = starts.cpu().numpy()
    assert np.array_equal(got_starts, want_starts)
    assert np.array_equal(perm.cpu().numpy()[: got_starts[-1]], want_perm)
    return grid


@pytest.mark.parametrize("dim,aperture,spatial", [(3, 150.0, True), (3, 150.0, False), (2, 150.0, True),
                                                  (3, 0.0, True), (2, 0.0, False)])
def test_bin_sort_matches_stable_sort(dim, aperture, spatial):
    rng = np.random.default_rng(40 + dim)
    nx = 64 if dim == 3 else 400
    sx, sy, rx, ry = random_headers(rng, dim, 50_000, nx * 12.5 + 1000.0)
    s = sv.survey_random(np.random.default_rng(1), dim, 1, nx, 48 if dim == 3 else 1, 16, 64,
                         aperture=aperture, n_bins=7, h=12.5).replace(sx=sx, sy=sy, rx=rx, ry=ry,
                                                                      bin_width=150.0)
    grid = check_sort(s, spatial)
    if aperture > 0 and spatial:
        assert grid["ncx"] > 1
    # the traces dropped for their midpoint reach no image column within the aperture
    if aperture > 0:
        want_perm, _ = expected_order(s, grid)
        dropped = np.setdiff1d(np.flatnonzero(oracle.bins(s) >= 0), want_perm)
        assert dropped.size > 0
        assert oracle.count(s.subset(dropped)) == 0


def test_bin_sort_ten_million_traces():
    rng = np.random.default_rng(77)
    ntr = 10_000_000
    sx, sy, rx, ry = random_headers(rng, 3, ntr, 6000.0)
    s = sv.survey_random(np.random.default_rng(2), 3, 1, 256, 256, 16, 64, aperture=500.0,
                         n_bins=16, h=25.0).replace(sx=sx, sy=sy, rx=rx, ry=ry, bin_width=400.0)
    grid = check_sort(s)
    assert grid["ncx"] >= 8 and grid["ncy"] >= 8


@pytest.mark.parametrize("vel,weight", [("linear", "obliq"), ("const", "one")])
def test_cell_ranges_keep_the_same_pairs(vel, weight):
    rng = np.random.default_rng(51)
    s = sv.survey_random(rng, 3, 3000, 64, 56, 32, 300, vel=vel, weight=weight, aperture=90.0,
                         n_bins=3, h=12.5, v0=1700.0, k=0.6 if vel == "linear" else 0.0)
    assert kh.kirchhoff_cell_grid(kh.desc_from(s))["ncx"] > 1
    d = sv.random_traces(s, 5, smooth=5)
    p = kh.Plan(s)
    hdr = kh.Headers.of(s)
    dt = torch.as_tensor(d, device="cuda")
    p.profile(True)
    img_cells = p.migrate(hdr, dt).clone()
    ex_cells, st_cells, n_cells = p.staging_stats()
    p.set_spatial_sort(False)
    img_bins = p.migrate(hdr, dt).clone()
    ex_bins, st_bins, n_bins = p.staging_stats()
    p.sync()
    assert st_cells == st_bins > 0                     # the same traces are staged per tile
    assert n_cells == n_bins > 0
    assert ex_cells < ex_bins                          # fewer are examined
    a, b = img_cells.double().cpu().numpy(), img_bins.double().cpu().numpy()
    assert rel_l2(a, b) < 1e-6                         # only the summation order differs
    assert rel_l2(a, oracle.migrate(s, d)) < FP32_REL_L2
    # deterministic run to run
    p.set_spatial_sort(True)
    assert torch.equal(p.migrate(hdr, dt), img_cells)
