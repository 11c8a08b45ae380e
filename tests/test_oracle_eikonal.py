"""Pins of the oracle's first-arrival traveltime tables for a gridded model v(x, z) (the
"ray-theoretic" single-path times of Sec. 3) and of the migration that reads them.

The factored fast-sweeping solution (T = T0 + tau, T0 the constant-slowness time of the source) is
pinned by:
* a second solver of the same node equations: a Jacobi iteration that updates every node at once
  and solves each node's equation max(t - c_x, 0)^2 + max(t - c_z, 0)^2 = (h s)^2 by bisection
  (no closed form), iterated until nothing changes; the sweeps' fixed point must equal it;
* exact values: constant velocity gives the distance / v at every node (the factorisation is
  exact there); linear v(z) stays within a bound of its closed form that halves with the grid
  spacing (first order), and the source box within the trapezoid rule's error;
* mirror symmetry of a symmetric problem, and positivity.
The interpolation of the tables by the migration is pinned by planar tables T = a + b x + c z (which
bilinear interpolation reproduces exactly) against a brute-force sum of Eq. 1.  Planted mistakes
make a pin fail."""
import math

import numpy as np
import pytest

import oracle
from paper_1204_1225_gb300 import survey as sv


def jacobi(v, ox, h, xs):
    """Fixed point of the factored upwind equations by Jacobi iteration with a bisection solve per
    node; the source box as the oracle reads it (straight ray, trapezoid slowness)."""
    nx, nz = v.shape
    s = 1.0 / v.astype(np.float64)
    X, Z = np.meshgrid(ox + np.arange(nx) * h, np.arange(nz) * h, indexing="ij")
    DX = X - xs
    R = np.hypot(DX, Z)
    u = (xs - ox) / h
    i0 = min(max(int(math.floor(u)), 0), nx - 2)
    s0 = s[i0, 0] + (u - i0) * (s[i0 + 1, 0] - s[i0, 0])
    box = (np.abs(DX) <= 2.0 * h) & (np.arange(nz)[None, :] <= 2)
    tau = np.full((nx, nz), np.inf)
    tau[box] = R[box] * 0.5 * (s[box] - s0)
    with np.errstate(divide="ignore", invalid="ignore"):
        gx = np.where(box, 0.0, h * s0 * DX / R)      # h d(T0)/dx at the node
        gz = np.where(box, 0.0, h * s0 * Z / R)
    F = h * s
    inf_col = np.full((1, nz), np.inf)
    inf_row = np.full((nx, 1), np.inf)
    while True:
        left = np.concatenate([inf_col, tau[:-1]], 0) - gx
        right = np.concatenate([tau[1:], inf_col], 0) + gx
        up = np.concatenate([inf_row, tau[:, :-1]], 1) - gz
        down = np.concatenate([tau[:, 1:], inf_row], 1) + gz
        a, b = np.minimum(left, right), np.minimum(up, down)
        lo = np.minimum(a, b)
        ok = np.isfinite(lo) & ~box
        lo_, hi_ = np.where(ok, lo, 0.0), np.where(ok, lo + F, 1.0)
        aa, bb = np.where(ok, a, 0.0), np.where(ok, b, 0.0)
        for _ in range(200):                           # phi(t) = sum max(t - c, 0)^2 - F^2, monotone
            mid = 0.5 * (lo_ + hi_)
            phi = np.maximum(mid - aa, 0.0) ** 2 + np.maximum(mid - bb, 0.0) ** 2 - F * F
            lo_, hi_ = np.where(phi < 0, mid, lo_), np.where(phi < 0, hi_, mid)
        new = np.where(ok, np.minimum(tau, hi_), tau)
        with np.errstate(invalid="ignore"):
            change = np.where(np.isfinite(tau), tau - new, np.where(np.isfinite(new), 1.0, 0.0))
        if np.max(change) <= 1e-15:
            return s0 * R + new
        tau = new


def models(nx, nz, h, ox):
    x = ox + np.arange(nx) * h
    z = np.arange(nz) * h
    X, Z = np.meshgrid(x, z, indexing="ij")
    xc, zc = x.mean(), z.mean()
    lens = 2000.0 - 900.0 * np.exp(-((X - xc) ** 2 + (Z - zc) ** 2) / (2 * (0.18 * (x[-1] - x[0])) ** 2))
    wavy = 1800.0 + 0.7 * Z + 250.0 * np.sin(X / 60.0) * np.cos(Z / 45.0)
    return {"const": np.full(X.shape, 2100.0), "vz": 1500.0 + 0.8 * Z, "lens": lens, "wavy": wavy,
            "fast-lens": 1500.0 + 2500.0 * np.exp(-((X - xc) ** 2 + (Z - zc) ** 2) / (2 * 60.0 ** 2))}


def check_matches_jacobi():
    nx, nz, h, ox = 15, 11, 20.0, -40.0
    for name, v in models(nx, nz, h, ox).items():
        v = v.astype(np.float32)
        for xs in (ox + 7 * h, ox + 3.3 * h, ox + 0.6 * h, ox + (nx - 1) * h):
            T, r = oracle.eikonal(v, ox, h, xs, tol=0.0)
            assert r > 0, (name, xs)
            ref = jacobi(v, ox, h, xs)
            assert np.max(np.abs(T - ref)) <= 1e-12 * np.max(ref), (name, xs, np.max(np.abs(T - ref)))


def check_constant_velocity():
    # the factorisation is exact for constant slowness: T = |x - x_s| / v at every node, on any grid
    v0 = 2000.0
    for h, xs in ((40.0, 310.0), (10.0, 310.0), (10.0, 0.0), (5.0, 1277.5)):
        nx, nz = int(1280 / h) + 1, int(640 / h) + 1
        v = np.full((nx, nz), v0, np.float32)
        T, r = oracle.eikonal(v, 0.0, h, xs, tol=0.0)   # the converged discrete solution
        assert r > 0
        x = np.arange(nx)[:, None] * h
        z = np.arange(nz)[None, :] * h
        exact = np.hypot(x - xs, z) / v0
        assert np.max(np.abs(T - exact)) <= 1e-12 * np.max(exact)   # rounding accumulated over the sweeps


def check_linear_vz():
    v0, k, xs = 1500.0, 0.8, 400.0
    s = sv.survey_2d_const().replace(vel="linear", v0=v0, k=k)
    errs = []
    for h in (20.0, 10.0, 5.0):
        nx, nz = int(1600 / h) + 1, int(1200 / h) + 1
        z = np.arange(nz) * h
        v = np.broadcast_to(v0 + k * z, (nx, nz)).astype(np.float32)
        T, r = oracle.eikonal(v, 0.0, h, xs)
        assert r > 0
        X, Z = np.meshgrid(np.arange(nx) * h, z, indexing="ij")
        exact = oracle.traveltime(s, np.hypot(X - xs, Z).ravel(), Z.ravel()).reshape(X.shape)
        box = (np.abs(X - xs) <= 2 * h) & (Z <= 2 * h)
        # straight ray with the trapezoid slowness: its error is of third order in the box size
        assert np.max(np.abs(T - exact)[box]) < 6e-7 * (h / 10.0) ** 3
        errs.append(float(np.max(np.abs(T - exact))))
    for a, b in zip(errs, errs[1:]):
        assert b < 0.6 * a                       # first order: the error halves with h
    assert errs[1] < 2e-3                        # 10 m nodes: within 2 ms over 1.6 x 1.2 km


def check_symmetry_and_positivity():
    nx, nz, h = 41, 31, 10.0
    x = np.arange(nx) * h
    z = np.arange(nz) * h
    X, Z = np.meshgrid(x, z, indexing="ij")
    xc = x[nx // 2]
    v = (1700.0 + 0.5 * Z - 500.0 * np.exp(-((X - xc) ** 2 + (Z - 150.0) ** 2) / (2 * 50.0 ** 2))).astype(np.float32)
    T, r = oracle.eikonal(v, 0.0, h, xc, tol=0.0)   # converged: the orderings' asymmetry is gone
    assert r > 0
    assert np.max(np.abs(T - T[::-1])) <= 1e-13 * np.max(T)
    T[nx // 2, 0] = 1.0
    assert np.all(T > 0)


def check_rounds():
    # with the source mid-grid the corrections of later rounds shrink geometrically: several
    # rounds run before one changes no node by more than the tolerance, and too few rounds are
    # reported as not settled
    nx, nz, h = 31, 31, 10.0
    v = models(nx, nz, h, 0.0)["lens"].astype(np.float32)
    T, r = oracle.eikonal(v, 0.0, h, 155.0)
    assert r >= 3
    T0, r0 = oracle.eikonal(v, 0.0, h, 155.0, tol=0.0)
    # stopped once a round moved no node by more than the tolerance: what later rounds would
    # still change is about 1 % of that
    assert r0 >= r and np.max(np.abs(T - T0)) < 0.05 * oracle.TOL
    _, r1 = oracle.eikonal(v, 0.0, h, 155.0, max_rounds=1)
    assert r1 == -1


def plane_survey(weight="one"):
    rng = np.random.default_rng(11)
    s = sv.survey_random(rng, 2, 60, 9, 1, 12, 300, n_bins=3, h=10.0)
    s = s.replace(sx=np.round(s.sx / 5.0).astype(np.float32) * 5.0, rx=np.round(s.rx / 5.0).astype(np.float32) * 5.0,
                  weight=weight)
    loc = oracle.locations(s)
    h, ox = 20.0, -40.0
    nx, nz = 8, 12
    x = ox + np.arange(nx) * h
    z = np.arange(nz) * h
    X, Z = np.meshgrid(x, z, indexing="ij")
    coef = np.stack([rng.uniform(0.0, 0.05, loc.size), rng.uniform(2e-4, 6e-4, loc.size),
                     rng.uniform(3e-4, 9e-4, loc.size)], 1)
    T = coef[:, 0, None, None] + coef[:, 1, None, None] * np.abs(X - 0.0) + coef[:, 2, None, None] * Z
    g = oracle.GridTables(T, loc, ox, h, None)
    s = s.replace(vel="grid", grid_v=np.ones((nx, nz), np.float32), grid_ox=ox, grid_h=h)
    s.oracle_tables = g
    return s, coef, loc


def check_grid_interpolation():
    s, coef, loc = plane_survey()
    d = sv.random_traces(s, 5, smooth=3).astype(np.float64)
    idx = {float(x): i for i, x in enumerate(loc)}
    b = oracle.bins(s)
    pts = np.arange(int(np.prod(s.image_shape)))[::7]
    got = oracle.migrate_points(s, d, pts)
    want = np.zeros(pts.size)
    for p, q in enumerate(pts):
        iz = q % s.nz
        ix = (q // s.nz) % s.nx
        bb = q // (s.nz * s.nx)
        x, zz = s.ox + ix * s.dx, s.oz + iz * s.dz
        for j in range(s.ntr):
            if b[j] != bb:
                continue
            cs, cr = coef[idx[float(s.sx[j])]], coef[idx[float(s.rx[j])]]
            t = (cs[0] + cs[1] * x + cs[2] * zz) + (cr[0] + cr[1] * x + cr[2] * zz)
            tau = (t - s.t0) / s.dt
            if 0 <= tau <= s.nt - 1:
                i = min(int(math.floor(tau)), s.nt - 2)
                f = tau - i
                want[p] += (1 - f) * d[j, i] + f * d[j, i + 1]
    assert np.count_nonzero(want) > pts.size // 3
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def check_unknown_location_contributes_nothing():
    s, _, loc = plane_survey()
    d = sv.random_traces(s, 5, smooth=3).astype(np.float64)
    a = oracle.migrate(s, d)
    s2 = s.replace(sx=s.sx.copy())
    s2.oracle_tables = s.oracle_tables
    s2.sx[0] = np.float32(s2.sx[0] + 1.25)       # no table at that position
    keep = s.subset(np.arange(1, s.ntr))
    keep.oracle_tables = s.oracle_tables
    assert np.array_equal(oracle.migrate(s2, d), oracle.migrate(keep, d[1:]))
    assert not np.array_equal(a, oracle.migrate(keep, d[1:]))


def test_matches_jacobi():
    check_matches_jacobi()


def test_constant_velocity_exact():
    check_constant_velocity()


def test_linear_vz_closed_form():
    check_linear_vz()


def test_symmetry_and_positivity():
    check_symmetry_and_positivity()


def test_rounds_reported():
    check_rounds()


def test_grid_interpolation_planes():
    check_grid_interpolation()


def test_unknown_location_contributes_nothing():
    check_unknown_location_contributes_nothing()


def test_grid_tables_of_a_survey():
    s = sv.vxz_model(sv.survey_2d_const().replace(v0=1800.0, k=0.6), 4)
    g = oracle.grid_tables(s)
    assert g.T.shape == (oracle.locations(s).size,) + s.grid_v.shape
    assert np.all(g.rounds > 0)
    # the table of a location on a node (a shot at 40 + 80 i on 40 m nodes) read at that point is 0
    l = int(np.searchsorted(g.loc, np.float32(120.0)))
    assert g.loc[l] == 120.0 and s.grid_h == 40.0
    t = oracle.grid_traveltime(s, l, np.array([120.0, 160.0]), np.array([0.0, 0.0]))
    i = int(round((120.0 - s.grid_ox) / s.grid_h))
    slow = 1.0 / s.grid_v[i:i + 2, 0].astype(np.float64)
    assert t[0] == 0.0 and abs(t[1] - 40.0 * 0.5 * (slow[0] + slow[1])) < 1e-15


MUTATIONS = [
    (14, check_grid_interpolation),        # x and z node coordinates swapped
    (15, check_grid_interpolation),        # the receiver leg read from the source's table
    (16, check_matches_jacobi),            # the smaller root of the upwind quadratic
    (16, check_constant_velocity),
    (17, check_linear_vz),                 # the source box with the node's slowness only
    (18, check_matches_jacobi),            # one round of passes, settled or not
    (19, check_constant_velocity),         # neighbour shifts of the wrong sign
    (19, check_matches_jacobi),
]


@pytest.mark.parametrize("mutation,check", MUTATIONS, ids=[f"m{m}-{c.__name__}" for m, c in MUTATIONS])
def test_eikonal_pins_catch_planted_mistakes(mutation, check):
    oracle.set_mutation(mutation)
    try:
        with pytest.raises(AssertionError):
            check()
    finally:
        oracle.set_mutation(0)
