"""Pins of the oracle's operator anti-aliasing (constant velocity, ``aa_spacing`` > 0): the weight
keeps a contribution whose moveout between adjacent traces, L = spacing x max(|p_x|, |p_y|) with p
the midpoint gradient of the two-way time (samples per metre), is at most one sample, removes it
from two samples on, and falls as cos^2(pi (L - 1) / 2) between.

Pinned by: hand values of a zero-offset geometry where p = 2 d / (R v dt) (L = 0.75, 1.5 and 3 give
1, 1/2 and 0); p against central differences of the two-way time over the midpoint; symmetry
(source-receiver reciprocity); Eq. 1 with the weight by brute force on a tiny survey; the
weight off (spacing 0) leaves the image unchanged.  A planted mistake makes a pin fail."""
import math

import numpy as np
import pytest

import oracle
from paper_1204_1225_gb300 import survey as sv


def base(dim=3, spacing=10.0):
    s = sv.survey_random(np.random.default_rng(1), dim, 4, 8, 8, 8, 16, v0=2000.0)
    return s.replace(aa_spacing=spacing, dt=0.004)


def check_hand_values():
    # zero offset at the surface point (0, 0), image point 300 m away at 400 m depth: R = 500 m,
    # p_x = 2 * 300 / (500 * 2000 * 0.004) = 0.15 samples per metre
    for spacing, want in ((5.0, 1.0), (10.0, 0.5), (20.0, 0.0), (6.0, 1.0)):
        for dim in (2, 3):
            w = oracle.aa_weight(base(dim, spacing), [[300.0, 0.0, 400.0, 0.0, 0.0, 0.0, 0.0]])[0]
            assert abs(w - want) < 1e-12, (spacing, dim, w)
    # directly below a zero-offset trace the dip is zero
    assert oracle.aa_weight(base(3, 1000.0), [[50.0, 70.0, 600.0, 50.0, 70.0, 50.0, 70.0]])[0] == 1.0


def tau(p, v, dt, mx=0.0, my=0.0):
    x, y, z, sx, sy, rx, ry = p
    Rs = math.sqrt((x - sx - mx) ** 2 + (y - sy - my) ** 2 + z * z)
    Rr = math.sqrt((x - rx - mx) ** 2 + (y - ry - my) ** 2 + z * z)
    return (Rs + Rr) / (v * dt)


def check_finite_differences():
    rng = np.random.default_rng(5)
    s = base(3, 12.5)
    n = 400
    pts = np.stack([rng.uniform(-600, 600, n), rng.uniform(-600, 600, n), rng.uniform(50, 1200, n),
                    rng.uniform(-800, 800, n), rng.uniform(-800, 800, n), rng.uniform(-800, 800, n),
                    rng.uniform(-800, 800, n)], 1)
    W = oracle.aa_weight(s, pts)
    d = 1e-3
    for p, w in zip(pts, W):
        px = (tau(p, s.v0, s.dt, d, 0) - tau(p, s.v0, s.dt, -d, 0)) / (2 * d)
        py = (tau(p, s.v0, s.dt, 0, d) - tau(p, s.v0, s.dt, 0, -d)) / (2 * d)
        L = s.aa_spacing * max(abs(px), abs(py))
        want = 1.0 if L <= 1 else (0.0 if L >= 2 else math.cos(0.5 * math.pi * (L - 1)) ** 2)
        assert abs(w - want) < 1e-6, (p, w, want, L)
    assert 0.2 < np.mean((W > 0) & (W < 1)) + np.mean(W == 0)   # the sample spans every branch
    assert np.any(W == 1.0) and np.any(W == 0.0) and np.any((W > 0) & (W < 1))


def check_reciprocity():
    rng = np.random.default_rng(6)
    s = base(3, 15.0)
    p = np.stack([rng.uniform(-500, 500, 200), rng.uniform(-500, 500, 200), rng.uniform(50, 900, 200),
                  rng.uniform(-700, 700, 200), rng.uniform(-700, 700, 200), rng.uniform(-700, 700, 200),
                  rng.uniform(-700, 700, 200)], 1)
    assert np.array_equal(oracle.aa_weight(s, p), oracle.aa_weight(s, p[:, [0, 1, 2, 5, 6, 3, 4]]))


def check_brute_force_sum():
    rng = np.random.default_rng(7)
    s = sv.survey_random(rng, 2, 25, 9, 1, 10, 250, n_bins=2, h=20.0, v0=2000.0).replace(aa_spacing=25.0)
    d = sv.random_traces(s, 3, smooth=3).astype(np.float64)
    b = oracle.bins(s)
    pts = np.arange(int(np.prod(s.image_shape)))
    got = oracle.migrate_points(s, d, pts)
    want = np.zeros(pts.size)
    for q in pts:
        iz, ix, bb = q % s.nz, (q // s.nz) % s.nx, q // (s.nz * s.nx)
        x, z = s.ox + ix * s.dx, s.oz + iz * s.dz
        for j in range(s.ntr):
            if b[j] != bb:
                continue
            p = (x, 0.0, z, float(s.sx[j]), 0.0, float(s.rx[j]), 0.0)
            t = tau(p, s.v0, s.dt) - s.t0 / s.dt
            if 0 <= t <= s.nt - 1:
                i = min(int(math.floor(t)), s.nt - 2)
                f = t - i
                w = oracle.aa_weight(s, [p])[0]
                want[q] += w * ((1 - f) * d[j, i] + f * d[j, i + 1])
    assert np.count_nonzero(want) > pts.size // 3
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    off = s.replace(aa_spacing=0.0)
    assert not np.allclose(oracle.migrate_points(off, d, pts), got)   # the weight acts here


def tau_lin(s, p, mx=0.0, my=0.0):
    """Two-way time in samples of v0 + k z from the oracle's own traveltime (pinned elsewhere by
    its closed forms and quadrature), with the trace's midpoint shifted by (mx, my)."""
    x, y, z, sx, sy, rx, ry = p
    Rs = math.sqrt((x - sx - mx) ** 2 + (y - sy - my) ** 2 + z * z)
    Rr = math.sqrt((x - rx - mx) ** 2 + (y - ry - my) ** 2 + z * z)
    return float(np.sum(oracle.traveltime(s, np.array([Rs, Rr]), z))) / s.dt


def check_finite_differences_linear():
    # v(z) = 1500 + 0.8 z: the horizontal slowness of each curved leg against central differences
    # of the two-way time over the midpoint
    rng = np.random.default_rng(8)
    s = base(3, 12.5).replace(vel="linear", v0=1500.0, k=0.8)
    n = 300
    pts = np.stack([rng.uniform(-600, 600, n), rng.uniform(-600, 600, n), rng.uniform(50, 1500, n),
                    rng.uniform(-900, 900, n), rng.uniform(-900, 900, n), rng.uniform(-900, 900, n),
                    rng.uniform(-900, 900, n)], 1)
    W = oracle.aa_weight(s, pts)
    d = 1e-3
    for p, w in zip(pts, W):
        px = (tau_lin(s, p, d, 0) - tau_lin(s, p, -d, 0)) / (2 * d)
        py = (tau_lin(s, p, 0, d) - tau_lin(s, p, 0, -d)) / (2 * d)
        L = s.aa_spacing * max(abs(px), abs(py))
        want = 1.0 if L <= 1 else (0.0 if L >= 2 else math.cos(0.5 * math.pi * (L - 1)) ** 2)
        assert abs(w - want) < 1e-6, (p, w, want, L)
    assert np.any(W == 1.0) and np.any(W == 0.0) and np.any((W > 0) & (W < 1))
    # k -> 0 gives the constant-velocity weight; the curved rays differ from the straight ones
    s0 = s.replace(k=1e-9)
    assert np.max(np.abs(oracle.aa_weight(s0, pts) - oracle.aa_weight(s0.replace(vel="const"), pts))) < 1e-6
    assert not np.allclose(W, oracle.aa_weight(s.replace(vel="const"), pts))


def check_brute_force_sum_linear():
    rng = np.random.default_rng(17)
    s = sv.survey_random(rng, 2, 25, 9, 1, 10, 250, n_bins=2, h=20.0, vel="linear", v0=1600.0,
                         k=0.7).replace(aa_spacing=25.0)
    d = sv.random_traces(s, 4, smooth=3).astype(np.float64)
    b = oracle.bins(s)
    pts = np.arange(int(np.prod(s.image_shape)))
    got = oracle.migrate_points(s, d, pts)
    want = np.zeros(pts.size)
    for q in pts:
        iz, ix, bb = q % s.nz, (q // s.nz) % s.nx, q // (s.nz * s.nx)
        x, z = s.ox + ix * s.dx, s.oz + iz * s.dz
        for j in range(s.ntr):
            if b[j] != bb:
                continue
            p = (x, 0.0, z, float(s.sx[j]), 0.0, float(s.rx[j]), 0.0)
            t = tau_lin(s, p) - s.t0 / s.dt
            if 0 <= t <= s.nt - 1:
                i = min(int(math.floor(t)), s.nt - 2)
                f = t - i
                w = oracle.aa_weight(s, [p])[0]   # W = 1 (the survey's weight "one")
                want[q] += w * ((1 - f) * d[j, i] + f * d[j, i + 1])
    assert np.count_nonzero(want) > pts.size // 3
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    assert not np.allclose(oracle.migrate_points(s.replace(aa_spacing=0.0), d, pts), got)


def test_hand_values():
    check_hand_values()


def test_finite_differences_linear_vz():
    check_finite_differences_linear()


def test_brute_force_sum_linear_vz():
    check_brute_force_sum_linear()


def test_finite_differences():
    check_finite_differences()


def test_reciprocity():
    check_reciprocity()


def test_brute_force_sum():
    check_brute_force_sum()


MUTATIONS = [
    (23, check_finite_differences),   # the receiver leg's dip dropped
    (23, check_hand_values),
    (23, check_finite_differences_linear),
]


@pytest.mark.parametrize("mutation,check", MUTATIONS, ids=[f"m{m}-{c.__name__}" for m, c in MUTATIONS])
def test_aa_pins_catch_planted_mistakes(mutation, check):
    oracle.set_mutation(mutation)
    try:
        with pytest.raises(AssertionError):
            check()
    finally:
        oracle.set_mutation(0)


@pytest.mark.parametrize("vel", ["const", "linear"])
def test_migrate_and_demigrate_stay_transposes(vel):
    # <L d, m> = <d, L^T m> in FP64 with the weight on (it multiplies W in both operators)
    rng = np.random.default_rng(23)
    kw = dict(v0=1800.0) if vel == "const" else dict(vel="linear", v0=1600.0, k=0.6)
    s = sv.survey_random(rng, 3, 40, 9, 8, 12, 200, n_bins=2, h=15.0, aperture=120.0, **kw)
    s = s.replace(aa_spacing=20.0, taper=0.3)
    d = sv.random_traces(s, 5, smooth=3).astype(np.float64)
    m = sv.random_image(s, 6).astype(np.float64)
    lhs = float(np.vdot(oracle.migrate(s, d), m))
    rhs = float(np.vdot(d, oracle.demigrate(s, m.astype(np.float32))))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)) + 1e-14
    assert not np.allclose(oracle.migrate(s.replace(aa_spacing=0.0), d), oracle.migrate(s, d))
