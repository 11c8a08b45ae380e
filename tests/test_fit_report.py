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
    exact = r["c1"] * np.log1p(rho64)
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
