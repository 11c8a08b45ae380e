"""Pins of the oracle's true-amplitude weight (weight "ta", constant velocity): the weight of the
asymptotic Kirchhoff inversion for the reflection coefficient, |h| / (a_s a_r |grad tau|^2), with h
the Beylkin determinant of the common-offset traveltime over the midpoint.

Pinned by: its closed form at zero offset (2 cos theta in 3D, cos theta in 2D); the determinant
from central differences of grad tau over the midpoint (no derivative formula); its reduction to
z (R_s + R_r)(1/R_s^2 + 1/R_r^2)/2 (3D) derived by hand (the kernels evaluate that form); reciprocity and
invariance under horizontal translation and rotation; and what the weight is for: a horizontal
reflector modelled with the exact specular amplitude R / (4 pi L) of a point source, migrated with
the weight from time-differentiated data, images with the same peak in every offset bin and at
every depth (the obliquity weight and W = 1 do not).  Planted mistakes make a pin fail."""
import math

import numpy as np
import pytest

import oracle
from paper_1204_1225_gb300 import survey as sv


def base(dim=3):
    s = sv.survey_random(np.random.default_rng(1), dim, 4, 8, 8, 8, 16).replace(weight="ta")
    return s


def rand_points(rng, n, dim=3):
    x, y = rng.uniform(-500, 500, n), rng.uniform(-500, 500, n) if dim == 3 else np.zeros(n)
    z = rng.uniform(50, 1500, n)
    sx, sy = rng.uniform(-800, 800, n), rng.uniform(-800, 800, n) if dim == 3 else np.zeros(n)
    rx, ry = rng.uniform(-800, 800, n), rng.uniform(-800, 800, n) if dim == 3 else np.zeros(n)
    return np.stack([x, y, z, sx, sy, rx, ry], 1)


def fd_weight(p, dim):
    """The weight from its definition with the midpoint derivatives of grad tau taken by central
    differences (v = 1; the determinant's v factors are global)."""
    x, y, z, sx, sy, rx, ry = p

    def grad_tau(mx, my):
        out = np.zeros(3)
        for ax, ay in ((sx + mx, sy + my), (rx + mx, ry + my)):
            e = np.array([x - ax, y - ay, z])
            out += e / np.linalg.norm(e)
        return out

    d = 1e-3
    g = grad_tau(0.0, 0.0)
    c1 = (grad_tau(d, 0.0) - grad_tau(-d, 0.0)) / (2 * d)
    Rs = math.sqrt((x - sx) ** 2 + (y - sy) ** 2 + z * z)
    Rr = math.sqrt((x - rx) ** 2 + (y - ry) ** 2 + z * z)
    if dim == 2:
        h = g[0] * c1[2] - g[2] * c1[0]
        return math.sqrt(Rs * Rr) * abs(h) / g.dot(g)
    c2 = (grad_tau(0.0, d) - grad_tau(0.0, -d)) / (2 * d)
    return Rs * Rr * abs(np.linalg.det(np.stack([g, c1, c2]))) / g.dot(g)


def check_zero_offset():
    rng = np.random.default_rng(2)
    for dim, c in ((3, 2.0), (2, 1.0)):
        p = rand_points(rng, 200, dim)
        p[:, 5], p[:, 6] = p[:, 3], p[:, 4]
        W = oracle.ta_weight(base(dim), p)
        R = np.sqrt((p[:, 0] - p[:, 3]) ** 2 + (p[:, 1] - p[:, 4]) ** 2 + p[:, 2] ** 2)
        assert np.max(np.abs(W - c * p[:, 2] / R)) < 1e-12


def check_finite_differences():
    rng = np.random.default_rng(3)
    for dim in (3, 2):
        p = rand_points(rng, 100, dim)
        W = oracle.ta_weight(base(dim), p)
        ref = np.array([fd_weight(q, dim) for q in p])
        assert np.max(np.abs(W - ref) / ref) < 1e-6


def check_reduced_form():
    # with c = e_s . e_r the determinant reduces to (1/R_s + 1/R_r)(1 + c)(z/R_s^2 + z/R_r^2) (3D;
    # 2D: (1 + c)(z/R_s^2 + z/R_r^2)) and |g|^2 = 2 (1 + c): W = z (R_s + R_r)(1/R_s^2 + 1/R_r^2)/2 (3D),
    # z sqrt(R_s R_r)(1/R_s^2 + 1/R_r^2)/2 (2D)
    rng = np.random.default_rng(9)
    for dim in (3, 2):
        p = rand_points(rng, 300, dim)
        W = oracle.ta_weight(base(dim), p)
        Rs = np.sqrt((p[:, 0] - p[:, 3]) ** 2 + (p[:, 1] - p[:, 4]) ** 2 + p[:, 2] ** 2)
        Rr = np.sqrt((p[:, 0] - p[:, 5]) ** 2 + (p[:, 1] - p[:, 6]) ** 2 + p[:, 2] ** 2)
        lat = (Rs + Rr) if dim == 3 else np.sqrt(Rs * Rr)
        assert np.max(np.abs(W - 0.5 * p[:, 2] * lat * (1 / Rs ** 2 + 1 / Rr ** 2)) / W) < 1e-12


def check_symmetries():
    rng = np.random.default_rng(4)
    s = base(3)
    p = rand_points(rng, 100)
    W = oracle.ta_weight(s, p)
    swapped = p[:, [0, 1, 2, 5, 6, 3, 4]]
    assert np.max(np.abs(oracle.ta_weight(s, swapped) - W) / W) < 1e-13          # reciprocity
    t = p.copy()
    for c in (0, 3, 5):
        t[:, c] += 137.0
    for c in (1, 4, 6):
        t[:, c] -= 61.0
    assert np.max(np.abs(oracle.ta_weight(s, t) - W) / W) < 1e-11               # translation
    a = 0.7
    r = p.copy()
    for cx, cy in ((0, 1), (3, 4), (5, 6)):
        r[:, cx] = math.cos(a) * p[:, cx] - math.sin(a) * p[:, cy]
        r[:, cy] = math.sin(a) * p[:, cx] + math.cos(a) * p[:, cy]
    assert np.max(np.abs(oracle.ta_weight(s, r) - W) / W) < 1e-11               # rotation about z


def reflector_peaks(weight, offsets, zr, v=2000.0, spacing=10.0, half=500.0):
    """Peak of the image of a horizontal reflector at depth zr below the centre of a common-offset
    grid of midpoints, per offset bin: data = R / (4 pi L) times the time derivative of a 25 Hz
    Ricker at the specular time L / v (L the specular path length), R = 1."""
    g = np.arange(-half, half + 1e-9, spacing)
    MX, MY = np.meshgrid(g, g, indexing="ij")
    mx, my = MX.ravel(), MY.ravel()
    sx = np.concatenate([mx - o / 2 for o in offsets]).astype(np.float32)
    rx = np.concatenate([mx + o / 2 for o in offsets]).astype(np.float32)
    sy = np.concatenate([my for _ in offsets]).astype(np.float32)
    dt, nt = 0.0005, int(2.6 * math.hypot(max(offsets), 2 * zr) / v / 0.0005)
    L = np.hypot(sx.astype(np.float64) - rx, 2 * zr)
    t = np.arange(nt) * dt
    u = t[None, :] - (L / v)[:, None]
    ricker = (1 - 2 * (math.pi * 25 * u) ** 2) * np.exp(-(math.pi * 25 * u) ** 2)
    D = (1.0 / (4 * math.pi * L))[:, None] * np.gradient(ricker, dt, axis=1)
    nb = int(max(offsets) // 200.0) + 1   # offsets at bin centres of 200 m bins
    s = sv.Survey(dim=3, nx=1, ny=1, nz=61, ox=0.0, oy=0.0, oz=zr - 30.0, dx=1.0, dy=1.0, dz=1.0,
                  n_bins=nb, bin_width=200.0, vel="const", v0=v, k=0.0, weight=weight, r0=1000.0,
                  aperture=half, nt=nt, t0=0.0, dt=dt, sx=sx, sy=sy, rx=rx, ry=sy.copy(), taper=0.5)
    img = oracle.migrate(s, D)
    return np.abs(img).max(axis=(1, 2, 3))[[int(o // 200.0) for o in offsets]]


OFFSETS = [100.0, 300.0, 500.0, 700.0]


def check_flat_reflector_offsets():
    p = reflector_peaks("ta", OFFSETS, 500.0)
    assert np.max(np.abs(p / p[0] - 1.0)) < 0.005
    # the obliquity weight and W = 1 do not keep the amplitude (here +21 % and +47 % at 700 m)
    for w in ("one", "obliq"):
        q = reflector_peaks(w, OFFSETS, 500.0)
        assert q[-1] / q[0] > 1.15


def check_flat_reflector_depths():
    peaks = [reflector_peaks("ta", [300.0], zr)[0] for zr in (350.0, 500.0, 700.0)]
    assert np.max(np.abs(np.array(peaks) / peaks[0] - 1.0)) < 0.005


def test_zero_offset_closed_form():
    check_zero_offset()


def test_finite_difference_determinant():
    check_finite_differences()


def test_reduced_form():
    check_reduced_form()


def test_reciprocity_translation_rotation():
    check_symmetries()


def test_flat_reflector_same_peak_at_every_offset():
    check_flat_reflector_offsets()


def test_flat_reflector_same_peak_at_every_depth():
    check_flat_reflector_depths()


MUTATIONS = [
    (20, check_finite_differences),       # a sign error in one entry of the determinant
    (21, check_zero_offset),              # a spreading factor off
    (21, check_reduced_form),
    (22, check_flat_reflector_offsets),   # the |grad tau|^2 of the reflectivity inversion dropped
]


@pytest.mark.parametrize("mutation,check", MUTATIONS, ids=[f"m{m}-{c.__name__}" for m, c in MUTATIONS])
def test_ta_pins_catch_planted_mistakes(mutation, check):
    oracle.set_mutation(mutation)
    try:
        with pytest.raises(AssertionError):
            check()
    finally:
        oracle.set_mutation(0)
