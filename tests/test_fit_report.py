"""CPU checks of the host logic behind the linear-v(z) kernels' ln(1 + rho) evaluation, through
the host-only kirchhoff_fit_report (no device work):

* the per-leg bound b covers |k| |T(p) - T(c)| for every point p of the tile and any surface
  position, checked against the linear-gradient closed form of T;
* the per-leg coefficients the kernels receive reproduce C1 ln(1 + rho) within the 2.5e-6-sample
  share of the 5e-6-sample budget over [expm1(-b), expm1(b)], evaluated by FP32 Horner steps as
  the kernels do;
* the fit lengths of the benchmark workloads, and the refusals."""
import math

import numpy as np
import pytest

from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300.survey import survey_25d_lsm, survey_3d_gradient

CASES = [
    ("3d-vz-256cube", lambda: survey_3d_gradient(), (16, 16, 1), 6, 5),
    ("3d-vz-128cube", lambda: survey_3d_gradient(40000, 128), (16, 16, 1), 8, 6),
    ("25d-vz-512x400", lambda: survey_25d_lsm(), (64, 1, 4), 8, 5),
]


def _report(s, tile):
    return kh.kirchhoff_fit_report(kh.desc_from(s), tile)


def _leg_time(px, py, pz, ax, ay, v0, k):
    """One-way time of the linear gradient v0 + k z from the surface point (ax, ay, 0)."""
    r2 = (px - ax) ** 2 + (py - ay) ** 2 + pz ** 2
    vz = v0 + k * pz
    return np.arccosh(1.0 + k * k * r2 / (2.0 * v0 * vz)) / abs(k)


@pytest.mark.parametrize("name,make,tile,two,leg", CASES, ids=[c[0] for c in CASES])
def test_fit_lengths_of_the_workloads(name, make, tile, two, leg):
    r = _report(make(), tile)
    assert (r["two_leg_terms"], r["leg_terms"]) == (two, leg)
    assert r["leg_terms"] > 8 or (r["scale"], r["offset"]) == (1.0, 0.0)   # monomial up to 8 terms
    assert all(c == 0.0 for c in r["coef"][r["leg_terms"]:])


@pytest.mark.parametrize("name,make,tile,two,leg", CASES, ids=[c[0] for c in CASES])
def test_leg_bound_covers_every_point_of_the_tile(name, make, tile, two, leg):
    s = make()
    b = _report(s, tile)["leg_bound"]
    cx, cy, cz = tile
    rng = np.random.default_rng(7)
    ny = s.ny if s.dim == 3 else 1
    for _ in range(4):
        # a tile at a random position of the grid: its points and its centre
        ix0 = int(rng.integers(0, max(1, s.nx - cx + 1)))
        iy0 = int(rng.integers(0, max(1, ny - cy + 1))) if s.dim == 3 else 0
        iz0 = int(rng.integers(0, max(1, s.nz - cz * 16 + 1)))
        ix = ix0 + np.arange(cx)
        iy = iy0 + np.arange(cy)
        iz = iz0 + np.arange(cz * 16)
        X, Y, Z = np.meshgrid(s.ox + ix * s.dx, (s.oy + iy * s.dy) if s.dim == 3 else np.zeros(1),
                              s.oz + iz * s.dz, indexing="ij")
        # the tile's centre: the box centre of its first and last samples
        c = (0.5 * (X.min() + X.max()), 0.5 * (Y.min() + Y.max()), 0.5 * (Z.min() + Z.max()))
        for _ in range(16):
            ax = rng.uniform(s.ox - 3000.0, s.ox + s.nx * s.dx + 3000.0)
            ay = rng.uniform(s.oy - 3000.0, s.oy + ny * s.dy + 3000.0) if s.dim == 3 else 0.0
            t = _leg_time(X, Y, Z, ax, ay, s.v0, s.k)
            tc = _leg_time(*c, ax, ay, s.v0, s.k)
            assert abs(s.k) * np.max(np.abs(t - tc)) <= b


def _horner_f32(coef, n, x):
    """sum_{j>=1} coef[j] x^(j-1) by FP32 steps p = fma(p, x, coef[j]) (products of two FP32
    numbers are exact in FP64, so one rounding to FP32 per step)."""
    c = np.asarray(coef, dtype=np.float32)
    p = np.full_like(x, c[n - 1])
    for j in range(n - 2, 0, -1):
        p = (p.astype(np.float64) * x.astype(np.float64) + np.float64(c[j])).astype(np.float32)
    return p


@pytest.mark.parametrize("name,make,tile,two,leg", CASES, ids=[c[0] for c in CASES])
def test_leg_fit_within_its_share_of_the_budget(name, make, tile, two, leg):
    s = make()
    r = _report(s, tile)
    b, n = r["leg_bound"], r["leg_terms"]
    rho = np.linspace(math.expm1(-b), math.expm1(b), 20001).astype(np.float32)
    x = rho if n <= 8 else (rho.astype(np.float64) * r["scale"] + r["offset"]).astype(np.float32)
    p = _horner_f32(r["coef"], n, x)
    rho64 = rho.astype(np.float64)
    approx = rho64 * (np.float64(r["coef"][0]) + rho64 * p.astype(np.float64))
    # the linear term's scale is the FP32 C1 (coef[0]): its rounding, C1lo rho, is FP32
    # evaluation error kept out of the fit budget, as the polynomial's own rounding is
    exact = np.float64(r["coef"][0]) * np.log1p(rho64)
    err = np.max(np.abs(approx - exact))   # in samples (C1 = 1 / (|k| dt))
    print(f"{name}: {n} terms, b = {b:.4f}, max error {err:.2e} samples")
    assert err <= 2.5e-6 * 1.05


def test_refusals():
    s = survey_3d_gradient()
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.kirchhoff_fit_report(kh.desc_from(s.replace(k=0.0)), (16, 16, 1))
    assert ei.value.status == kh.KH_ERR_INVALID_ARG
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.kirchhoff_fit_report(kh.desc_from(s), (16, 16, 2))      # 512 threads
    assert ei.value.status == kh.KH_ERR_INVALID_ARG
    coarse = s.replace(nx=64, ny=64, nz=64, dx=400.0, dy=400.0, dz=400.0)
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.kirchhoff_fit_report(kh.desc_from(coarse), (16, 16, 1))  # rho beyond every fit
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED


def test_random_descriptors_meet_the_budget_or_are_refused():
    """Random grids, spacings, gradients and tiles: every accepted tile's per-leg fit meets its
    share of the budget over its bound, and the bound covers the tile's leg times."""
    rng = np.random.default_rng(1204)
    tiles3 = [(16, 16, 1), (32, 8, 1), (16, 8, 2), (8, 8, 4), (8, 4, 8), (64, 4, 1)]
    tiles2 = [(64, 1, 4), (32, 1, 8), (128, 1, 2), (16, 1, 16), (256, 1, 1)]
    accepted = refused = 0
    for trial in range(40):
        dim = 3 if trial % 2 == 0 else 2
        h = float(rng.choice([2.5, 5.0, 10.0, 12.5, 25.0, 50.0]))
        v0 = float(rng.uniform(1200.0, 3000.0))
        k = float(rng.choice([-1.0, 1.0]) * rng.uniform(0.05, 1.5))
        dt = float(rng.choice([0.001, 0.002, 0.004]))
        nz = 64
        if k < 0:   # keep v > 0 over the grid
            nz = int(min(64, 0.8 * v0 / (-k * h)))
            if nz < 16:
                continue
        s = survey_3d_gradient(1, 64).replace(dim=dim, nx=64, ny=64 if dim == 3 else 1, nz=nz, dx=h,
                                              dy=h, dz=h, ox=0.0, oy=0.0, oz=0.0, v0=v0, k=k, dt=dt)
        tile = (tiles3 if dim == 3 else tiles2)[int(rng.integers(0, 5))]
        try:
            r = _report(s, tile)
        except kh.KirchhoffError as e:
            assert e.status == kh.KH_ERR_UNSUPPORTED
            refused += 1
            continue
        accepted += 1
        b, n = r["leg_bound"], r["leg_terms"]
        rho = np.linspace(math.expm1(-b), math.expm1(b), 4001).astype(np.float32)
        x = rho if n <= 8 else (rho.astype(np.float64) * r["scale"] + r["offset"]).astype(np.float32)
        p = _horner_f32(r["coef"], n, x)
        rho64 = rho.astype(np.float64)
        c1f = np.float64(r["coef"][0])
        err = np.max(np.abs(rho64 * (c1f + rho64 * p.astype(np.float64)) - c1f * np.log1p(rho64)))
        assert err <= 2.5e-6 * 1.05, (trial, n, b, err)
        # bound: the first tile's corners and centre against surface positions around the grid
        cx, cy, cz = tile
        xs = np.array([0.0, (min(cx, s.nx) - 1) * h])
        ys = np.array([0.0, (min(cy, s.ny) - 1) * h]) if dim == 3 else np.array([0.0])
        zs = np.array([0.0, (min(cz * 16, s.nz) - 1) * h])
        X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
        c = (xs.mean(), ys.mean(), zs.mean())
        for _ in range(8):
            ax, ay = rng.uniform(-2000.0, 2000.0 + 64 * h, 2)
            if dim == 2:
                ay = 0.0
            t = _leg_time(X, Y, Z, ax, ay, v0, k)
            tc = _leg_time(*c, ax, ay, v0, k)
            assert abs(k) * np.max(np.abs(t - tc)) <= b
    assert accepted >= 20
    print(f"accepted {accepted}, refused {refused}")
