"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each ``check_*`` helper asserts one fact fixed by the paper or by mathematics:
closed forms of the traveltime, a Fermat-principle minimisation, hand-derived single
contributions, the MapReduce reduce identity of the forward flow (Sec. 4, Forward PKTM,
items 6-7: per-trace partial images summed per image point), operator invariants, the
adjoint identity, finite differences and the focusing of a point diffractor.  The last
test plants each plausible mistake in the oracle (on the CPU) and shows a pin fails.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.optimize

import oracle
from paper_1204_1225_gb300 import survey as sv


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def tiny_survey(**kw):
    base = dict(dim=2, nx=1, ny=1, nz=1, ox=0.0, oy=0.0, oz=0.0, dx=10.0, dy=10.0, dz=10.0,
                n_bins=1, bin_width=10000.0, vel="const", v0=2500.0, k=0.0, weight="one",
                r0=1000.0, aperture=0.0, nt=400, t0=0.0, dt=0.004,
                sx=np.zeros(1, np.float32), sy=np.zeros(1, np.float32),
                rx=np.zeros(1, np.float32), ry=np.zeros(1, np.float32))
    base.update(kw)
    for key in ("sx", "sy", "rx", "ry"):
        base[key] = np.asarray(base[key], dtype=np.float32)
    return sv.Survey(**base)


# ---------------------------------------------------------------- traveltime (T of Eq. 1)

GRAD = tiny_survey(vel="linear", v0=1500.0, k=0.5)


def check_vertical_closed_form():
    # straight vertical ray in v = v0 + k z: T = integral dz / (v0 + k z) = ln(1 + k z / v0) / k
    z = np.array([1.0, 10.0, 250.0, 1000.0, 3200.0])
    T = oracle.traveltime(GRAD, z, z)
    expect = np.log1p(GRAD.k * z / GRAD.v0) / GRAD.k
    assert rel(T, expect) < 1e-14


def check_textbook_arccosh():
    # textbook linear-gradient traveltime T = arccosh(1 + k^2 R^2 / (2 v_a v_b)) / k
    rng = np.random.default_rng(3)
    R = rng.uniform(200.0, 4000.0, 64)
    z = R * rng.uniform(0.05, 1.0, 64)
    vb = GRAD.v0 + GRAD.k * z
    expect = np.arccosh(1.0 + GRAD.k ** 2 * R ** 2 / (2.0 * GRAD.v0 * vb)) / GRAD.k
    assert rel(oracle.traveltime(GRAD, R, z), expect) < 1e-12


def test_traveltime_closed_forms():
    check_vertical_closed_form()
    check_textbook_arccosh()


def test_traveltime_k_to_zero():
    R = np.array([10.0, 500.0, 3000.0])
    z = np.array([5.0, 300.0, 2000.0])
    for k in (0.0, 1e-12, 1e-9):
        s = tiny_survey(vel="linear", v0=1800.0, k=k)
        assert rel(oracle.traveltime(s, R, z), R / 1800.0) < 1e-9
    assert rel(oracle.traveltime(tiny_survey(v0=1800.0), R, z), R / 1800.0) < 1e-15


def _arc_time(v0, k, h, z):
    # the ray in a linear gradient is a circle centred at depth -v0/k; along it
    # ds = rho dtheta and v = k rho sin(theta), so dt = dtheta / (k sin(theta))
    zc = -v0 / k
    xc = (h * h + z * z - 2.0 * z * zc) / (2.0 * h)
    ta = math.atan2(0.0 - zc, 0.0 - xc)
    tb = math.atan2(z - zc, h - xc)
    val, _ = scipy.integrate.quad(lambda t: 1.0 / (k * math.sin(t)), min(ta, tb), max(ta, tb),
                                  epsabs=0.0, epsrel=1e-13, limit=200)
    return val


def _fermat_polyline(v0, k, h, z, n=48):
    # Fermat's principle: minimise the time of a polyline from (0, 0) to (h, z); the
    # exact time of a straight segment in v = v0 + k z is L ln(v_b / v_a) / (k dz).
    def seg(x1, z1, x2, z2):
        L = np.hypot(x2 - x1, z2 - z1)
        dz = z2 - z1
        va, vb = v0 + k * z1, v0 + k * z2
        small = np.abs(k * dz) < 1e-9 * va
        safe = np.where(small, 1.0, dz)
        return np.where(small, L / va, L * np.log(vb / va) / (k * safe))

    s = np.linspace(0.0, 1.0, n + 1)[1:-1]

    def total(p):
        xs = np.concatenate([[0.0], p[: n - 1], [h]])
        zs = np.concatenate([[0.0], p[n - 1:], [z]])
        return float(np.sum(seg(xs[:-1], zs[:-1], xs[1:], zs[1:])))

    p0 = np.concatenate([s * h, s * z])
    res = scipy.optimize.minimize(total, p0, method="L-BFGS-B",
                                  options=dict(maxiter=20000, ftol=1e-15, gtol=1e-12))
    return res.fun


def test_traveltime_circular_ray_and_fermat():
    for h, z in [(300.0, 800.0), (1500.0, 600.0), (2500.0, 2500.0), (40.0, 3000.0)]:
        R = math.hypot(h, z)
        T = float(oracle.traveltime(GRAD, np.array([R]), np.array([z]))[0])
        assert abs(_arc_time(GRAD.v0, GRAD.k, h, z) - T) < 1e-11 * T
        tf = _fermat_polyline(GRAD.v0, GRAD.k, h, z)
        assert T <= tf * (1 + 1e-12)          # Fermat: the true path is the fastest
        assert tf <= T * (1 + 2e-5)           # and the polyline converges to it


def check_traveltime_derivatives():
    rng = np.random.default_rng(5)
    R = rng.uniform(50.0, 4000.0, 32)
    z = R * rng.uniform(0.02, 1.0, 32)
    for k in (0.5, 0.02, 1e-4, 0.0):
        s = tiny_survey(vel="linear", v0=1500.0, k=k)
        T, gv, gk = oracle.traveltime(s, R, z, grad=True)
        hv, hk = 1e-3, 1e-5
        fd_v = (oracle.traveltime(s.replace(v0=1500.0 + hv), R, z)
                - oracle.traveltime(s.replace(v0=1500.0 - hv), R, z)) / (2 * hv)
        fd_k = (oracle.traveltime(s.replace(k=k + hk), R, z)
                - oracle.traveltime(s.replace(k=k - hk), R, z)) / (2 * hk)
        assert rel(gv, fd_v) < 1e-7
        assert rel(gk, fd_k) < 1e-6


def test_traveltime_derivatives_fd():
    check_traveltime_derivatives()


# ----------------------------------------------------- single contributions derived by hand

def check_hand_contributions():
    # v = 2500 m/s, dt = 4 ms: one sample is 10 m of two-way path.  Ramp data D[i] = 3 + 0.5 i
    # is reproduced exactly by linear interpolation, so each contribution is W (3 + 0.5 tau).
    d = (3.0 + 0.5 * np.arange(400.0))[None, :]
    # (a) point (0, 400), source -300, receiver +300: R_s = R_r = 500, tau = 100
    s = tiny_survey(ox=0.0, oz=400.0, sx=[-300.0], rx=[300.0])
    assert abs(oracle.migrate(s, d)[0, 0, 0, 0] - (3.0 + 50.0)) < 1e-12
    # (b) source -300 (R_s = 500), receiver 0 (R_r = 400): tau = 90
    s = tiny_survey(ox=0.0, oz=400.0, sx=[-300.0], rx=[0.0])
    assert abs(oracle.migrate(s, d)[0, 0, 0, 0] - (3.0 + 45.0)) < 1e-12
    # (c) fractional tau: source -300, receiver 0, point depth 400, t0 = 1.3 ms -> tau = 89.675
    s = tiny_survey(ox=0.0, oz=400.0, sx=[-300.0], rx=[0.0], t0=0.0013)
    assert abs(oracle.migrate(s, d)[0, 0, 0, 0] - (3.0 + 0.5 * 89.675)) < 1e-11
    # (d) obliquity x spreading: W = 1/2 (0.8 + 0.8) * 500 * 500 / 1000^2 = 0.2 at tau = 100
    s = tiny_survey(ox=0.0, oz=400.0, dz=400.0, sx=[-300.0], rx=[300.0], weight="obliq")
    assert abs(oracle.migrate(s, d)[0, 0, 0, 0] - 0.2 * 53.0) < 1e-12
    # (e) asymmetric legs with W: cos_s = 0.8, cos_r = 1, W = 1/2 (1.8) 500*400/1e6 = 0.18
    s = tiny_survey(ox=0.0, oz=400.0, dz=400.0, sx=[-300.0], rx=[0.0], weight="obliq")
    assert abs(oracle.migrate(s, d)[0, 0, 0, 0] - 0.18 * 48.0) < 1e-12


def test_hand_contributions():
    check_hand_contributions()


def check_time_window_edges():
    # zero-offset trace at x = 0; v = 2000, dt = 4 ms: tau = z / 4 - t0 / dt.
    d = (1.0 + np.arange(101.0))[None, :]             # D[i] = i + 1, nt = 101
    z = np.array([396.0, 400.0, 402.0, 404.0])
    s = tiny_survey(v0=2000.0, nt=101, nz=410, oz=0.0, dz=1.0, sx=[0.0], rx=[0.0])
    img = oracle.migrate_points(s, d, (z).astype(np.int64))
    # tau = 99, 100 (= nt - 1, kept, D[100] = 101), 100.5 and 101 (beyond the trace: 0)
    assert np.allclose(img, [100.0, 101.0, 0.0, 0.0], rtol=0, atol=1e-12)
    # with t0 = 0.2 s, tau = z/4 - 50: z = 196 -> -1 (dropped), z = 200 -> 0 (kept, D[0] = 1)
    s2 = s.replace(t0=0.2)
    img = oracle.migrate_points(s2, d, np.array([196, 198, 200, 204], dtype=np.int64))
    assert np.allclose(img, [0.0, 0.0, 1.0, 2.0], rtol=0, atol=1e-12)


def test_time_window_edges():
    check_time_window_edges()


def check_offset_bins():
    # 8 uniform bins of 40 m over [0, 320]: interior edges go up, 320 is in the last bin,
    # beyond 320 there is no bin (Eq. 1's delta selects no offset image).
    off = np.array([0.0, 39.5, 40.0, 80.0, 319.5, 320.0, 320.5, 1000.0], dtype=np.float32)
    s = tiny_survey(n_bins=8, bin_width=40.0, sx=np.zeros(8), rx=off)
    assert list(oracle.bins(s)) == [0, 0, 1, 2, 7, 7, -1, -1]
    # 3D offsets are horizontal Euclidean distances: (24, 32) -> 40 m -> bin 1
    s3 = tiny_survey(dim=3, n_bins=8, bin_width=40.0, sx=[0.0], sy=[0.0], rx=[24.0], ry=[32.0])
    assert list(oracle.bins(s3)) == [1]


def test_offset_bins():
    check_offset_bins()


# ----------------------------------------------------------------- operator-level pins

def small3d(vel="linear", weight="obliq", aperture=180.0, seed=11, ntr=40):
    rng = np.random.default_rng(seed)
    s = sv.survey_random(rng, 3, ntr, 6, 5, 9, 160, vel=vel, weight=weight,
                         aperture=aperture, n_bins=3, h=25.0, v0=1600.0,
                         k=0.7 if vel == "linear" else 0.0)
    return s


def test_linearity_and_reduce_identity():
    s = small3d()
    d1 = sv.random_traces(s, 1, smooth=3).astype(np.float64)
    d2 = sv.random_traces(s, 2, smooth=3).astype(np.float64)
    a = oracle.migrate(s, 2.5 * d1 - 0.75 * d2)
    b = 2.5 * oracle.migrate(s, d1) - 0.75 * oracle.migrate(s, d2)
    assert rel(a, b) < 1e-13
    # Forward PKTM (Sec. 4): each map task migrates its own traces; the reduce sums the
    # partial images per image point.  Any split of the traces gives the same image.
    idx = np.random.default_rng(4).permutation(s.ntr)
    A, B = idx[:17], idx[17:]
    full = oracle.migrate(s, d1)
    parts = oracle.migrate(s.subset(A), d1[A]) + oracle.migrate(s.subset(B), d1[B])
    assert rel(parts, full) < 1e-13


def test_reciprocity():
    s = small3d()
    d = sv.random_traces(s, 3, smooth=3)
    swapped = s.replace(sx=s.rx, sy=s.ry, rx=s.sx, ry=s.sy)
    assert rel(oracle.migrate(swapped, d), oracle.migrate(s, d)) < 1e-13


def test_sum_over_bins_is_single_bin():
    s = small3d(aperture=0.0)
    d = sv.random_traces(s, 5, smooth=3)
    one = s.replace(n_bins=1, bin_width=s.bin_width * s.n_bins)
    assert rel(oracle.migrate(s, d).sum(axis=0), oracle.migrate(one, d)[0]) < 1e-13


def test_translation_invariance():
    s = small3d(aperture=0.0)
    d = sv.random_traces(s, 6, smooth=3)
    sh = 250.0
    moved = s.replace(ox=s.ox + sh, oy=s.oy - sh, sx=s.sx + np.float32(sh), rx=s.rx + np.float32(sh),
                      sy=s.sy - np.float32(sh), ry=s.ry - np.float32(sh))
    # the shift is exact in FP32 only where the headers keep their bits; compare in FP64
    assert rel(oracle.migrate(moved, d), oracle.migrate(s, d)) < 1e-6


def check_adjoint():
    for vel, weight in (("const", "one"), ("linear", "obliq")):
        s = small3d(vel=vel, weight=weight)
        d = sv.random_traces(s, 7).astype(np.float64)
        m = sv.random_image(s, 8).astype(np.float64)
        lhs = float(np.vdot(oracle.migrate(s, d), m))
        rhs = float(np.vdot(d, oracle.demigrate(s, m)))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_adjoint_dot_product():
    check_adjoint()


def check_vgrad_fd():
    rng = np.random.default_rng(9)
    s = sv.survey_random(rng, 2, 24, 12, 1, 16, 300, vel="linear", weight="one", n_bins=2,
                         h=20.0, v0=1800.0, k=0.6)
    d = sv.random_traces(s, 10, smooth=15).astype(np.float64)
    m = sv.random_image(s, 11).astype(np.float64)
    g = oracle.vgrad(s, m, d)

    def B(v0, k):
        return float(np.vdot(m, oracle.migrate(s.replace(v0=v0, k=k), d)))

    hv, hk = 1e-3, 1e-6
    fd_v = (B(s.v0 + hv, s.k) - B(s.v0 - hv, s.k)) / (2 * hv)
    fd_k = (B(s.v0, s.k + hk) - B(s.v0, s.k - hk)) / (2 * hk)
    assert abs(g[0] - fd_v) < 2e-4 * abs(fd_v)
    assert abs(g[1] - fd_k) < 2e-4 * abs(fd_k)


def test_velocity_gradient_fd():
    check_vgrad_fd()


def check_focusing():
    # A noise-free point diffractor on an image node focuses at that node in every offset
    # image (Sec. 3: reflectors are built by constructive interference), with a peak of
    # N_b r(0) reduced at worst by linear interpolation midway between samples:
    # r(2 ms) at 25 Hz = 0.9275.
    s = sv.survey_2d_const()
    sc = sv.point_scatterers_2d(np.random.default_rng(sv.BASE_SEED))
    d = sv.synthesize(s, sc, oracle.arrival_times, 25.0, noise_sigma=0.0).numpy()
    img = oracle.migrate(s, d)[:, 0]                       # [bin, x, z]
    off = np.abs(s.sx.astype(np.float64) - s.rx)
    nb = np.bincount(np.minimum((off // 40.0).astype(int), 7), minlength=8)
    for b in range(8):
        for x, _, z, _ in sc:
            ix, iz = int(round(x / 10.0)), int(round(z / 10.0))
            win = img[b, ix - 1:ix + 2, iz - 1:iz + 2]
            assert img[b, ix, iz] == win.max()
            assert 0.92 * nb[b] <= img[b, ix, iz] <= 1.02 * nb[b]


def test_point_diffractor_focusing():
    check_focusing()


def test_count_full_aperture():
    s = small3d(aperture=0.0)
    nvalid = int(np.sum(oracle.bins(s) >= 0))
    assert oracle.count(s) == nvalid * s.nx * s.ny * s.nz


def test_cgls_reaches_least_squares_solution():
    rng = np.random.default_rng(12)
    s = sv.survey_random(rng, 2, 6, 3, 1, 4, 32, vel="const", n_bins=1, h=30.0, v0=1500.0,
                         dt=0.01)
    n = int(np.prod(s.image_shape))
    A = np.stack([oracle.demigrate(s, np.eye(n)[p].reshape(s.image_shape)).ravel()
                  for p in range(n)], axis=1)
    d = sv.random_traces(s, 13).astype(np.float64)
    m_ls = np.linalg.lstsq(A, d.ravel(), rcond=None)[0]
    m, rn, gn = oracle.cgls(s, d, n_iter=n)
    assert np.all(np.diff(rn) <= 1e-12 * rn[0])           # residual norm never grows
    assert rel(m.ravel(), m_ls) < 1e-6


# ------------------------------------------- aperture ("traces close enough", after Eq. 2)

# One image column at the origin and A = 300 m.  Each trace carries one constant value,
# 2^j for trace j, so with W = 1 and every tau inside the trace the image at any depth is
# the sum of the codes of the traces kept there.  The geometry is chosen by hand:
APERTURE_TRACES = [
    # (sx, sy, rx, ry), kept?  -- reason
    ((300.0, 0.0, 300.0, 0.0), True),     # midpoint exactly A from the column: <= is inside
    ((302.0, 0.0, 300.0, 0.0), False),    # midpoint at A + 1 m
    ((0.0, 0.0, 700.0, 0.0), False),      # source on the column, midpoint 350 m away
    ((-500.0, 0.0, 500.0, 0.0), True),    # source 500 m away, midpoint on the column
    ((180.0, 0.0, 180.0, 480.0), True),   # midpoint (180, 240): exactly 300 m in 2D
    ((180.0, 0.0, 180.0, 482.0), False),  # midpoint (180, 241): 301 m
    ((100.0, 0.0, 300.0, 0.0), True),     # midpoint 200 m away
]
APERTURE_DEPTHS = 5                        # z = 0, 250, 500, 750, 1000 m


def aperture_survey():
    g = np.array([t for t, _ in APERTURE_TRACES], dtype=np.float64)
    return tiny_survey(dim=3, nz=APERTURE_DEPTHS, dz=250.0, aperture=300.0, nt=400,
                       sx=g[:, 0], sy=g[:, 1], rx=g[:, 2], ry=g[:, 3])


def check_aperture_hand_geometry():
    s = aperture_survey()
    codes = 2.0 ** np.arange(len(APERTURE_TRACES))
    d = np.repeat(codes[:, None], s.nt, axis=1)
    want = sum(c for c, (_, kept) in zip(codes, APERTURE_TRACES) if kept)
    img = oracle.migrate(s, d)[0, 0, 0]
    # the decision is horizontal only: the same traces are kept at every depth
    assert np.allclose(img, want, rtol=0, atol=1e-9), (img, want)
    assert oracle.count(s) == sum(kept for _, kept in APERTURE_TRACES) * s.nz


def check_aperture_count_row():
    # nine columns x = -400 ... 400 (100 m apart), one trace with its midpoint at x = 50
    # and A = 250 m: the columns -200 ... 300 are within 250 m (the two ends exactly),
    # so the Eq. 2 count is 6 columns x nz
    s = tiny_survey(nx=9, ox=-400.0, dx=100.0, nz=3, aperture=250.0, sx=[0.0], rx=[100.0])
    assert oracle.count(s) == 6 * s.nz


def check_taper_hand_values():
    # one column at x = 0, A = 300 m, taper 0.5 (core 150 m); a trace whose midpoint is d from the
    # column carries the constant 1, so the image is the taper factor: 1 in the core, then
    # (1 + cos(pi (d - 150) / 150)) / 2
    for dist, want in ((100.0, 1.0), (150.0, 1.0), (187.5, 0.5 * (1 + math.cos(math.pi / 4))),
                       (225.0, 0.5), (299.0, 0.5 * (1 + math.cos(math.pi * 149.0 / 150.0)))):
        s = tiny_survey(aperture=300.0, taper=0.5, sx=[dist - 50.0], rx=[dist + 50.0])
        img = oracle.migrate(s, np.ones((1, s.nt)))[0, 0, 0, 0]
        assert abs(img - want) < 1e-12, (dist, img, want)


def check_taper_keeps_operators_paired():
    s = small3d(aperture=180.0).replace(taper=0.4)
    d = sv.random_traces(s, 7).astype(np.float64)
    m = sv.random_image(s, 8).astype(np.float64)
    lhs = float(np.vdot(oracle.migrate(s, d), m))
    rhs = float(np.vdot(d, oracle.demigrate(s, m)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    # the taper changes the image only where some midpoint lies in the taper band
    assert rel(oracle.migrate(s, d), oracle.migrate(s.replace(taper=0.0), d)) > 1e-3


def test_aperture_taper_hand_values():
    check_taper_hand_values()


def test_aperture_taper_keeps_operators_paired():
    check_taper_keeps_operators_paired()


def test_aperture_hand_geometry():
    check_aperture_hand_geometry()


def test_aperture_count_hand_row():
    check_aperture_count_row()


# -------------------------------------------------------------- the pins catch mistakes

MUTATIONS = [
    (1, check_hand_contributions),     # weight dropped
    (2, check_time_window_edges),      # sign of t0
    (3, check_hand_contributions),     # receiver leg replaced by the source leg
    (4, check_offset_bins),            # offset bin rounded instead of floored
    (5, check_traveltime_derivatives), # sign of a derivative term
    (5, check_vgrad_fd),
    (6, check_hand_contributions),     # interpolation weights swapped
    (7, check_aperture_hand_geometry), # aperture centred on the source, not the midpoint
    (7, check_aperture_count_row),
    (8, check_aperture_hand_geometry), # strict < at the aperture edge
    (8, check_aperture_count_row),
    (9, check_aperture_hand_geometry), # midpoint without its 1/2
    (9, check_aperture_count_row),
    (10, check_aperture_hand_geometry),  # depth term in the aperture distance
    (13, check_taper_hand_values),     # taper reversed across its band
]


@pytest.mark.parametrize("mutation,check", MUTATIONS,
                         ids=[f"m{m}-{c.__name__}" for m, c in MUTATIONS])
def test_pins_catch_planted_mistakes(mutation, check):
    oracle.set_mutation(mutation)
    try:
        with pytest.raises(AssertionError):
            check()
    finally:
        oracle.set_mutation(0)


# ------------------------------------------------------------------ table traveltimes

def test_table_traveltime_nodes_and_cells():
    # nodes reproduce the closed form; a cell centre is the mean of its four corners
    # (bilinear interpolation); the error against the closed form shrinks ~D^2.  With
    # dz = D/4 the depth nodes fall every D (m = 4) and, at spacing D/4, every dz (m = 1).
    base = tiny_survey(vel="table", v0=1500.0, k=0.5, oz=0.0, dz=6.25, nz=400)
    D = base.table_spacing
    assert D == 4 * base.dz
    lin = base.replace(vel="linear")
    h = np.array([0.0, D, 7 * D, 40 * D])
    z = np.array([0.0, 3 * D, 11 * D, 60 * D])
    T = oracle.table_traveltime(base, h, z)
    assert rel(T, oracle.traveltime(lin, np.hypot(h, z), z)) < 1e-15
    hc, zc = 7.5 * D, 11.5 * D
    corners = oracle.traveltime(lin, np.hypot([7 * D, 7 * D, 8 * D, 8 * D], [11 * D, 12 * D, 11 * D, 12 * D]),
                                np.array([11 * D, 12 * D, 11 * D, 12 * D]))
    assert abs(oracle.table_traveltime(base, [hc], [zc])[0] - corners.mean()) < 1e-14
    rng = np.random.default_rng(1)
    hh, zz = rng.uniform(200, 2000, 200), rng.uniform(200, 2000, 200)
    exact = oracle.traveltime(lin, np.hypot(hh, zz), zz)
    e1 = np.max(np.abs(oracle.table_traveltime(base, hh, zz) - exact))
    e2 = np.max(np.abs(oracle.table_traveltime(base.replace(table_spacing=D / 4), hh, zz) - exact))
    assert 8.0 < e1 / e2 < 24.0                       # second-order convergence


def test_table_depth_nodes_sit_on_image_depths():
    # depth nodes at z_min + j m dz, m the largest power of two <= min(4, D/dz): with
    # dz = 10 m and D = 25 m the nodes are every 20 m from the first image depth, so the
    # table is exact there and bilinear (here: linear in z) between them
    s = tiny_survey(vel="table", v0=1500.0, k=0.5, oz=30.0, dz=10.0, nz=100)
    assert s.table_spacing == 25.0
    lin = s.replace(vel="linear")
    h = np.array([0.0, 50.0, 125.0, 250.0])
    for zn in (30.0, 50.0, 230.0, 630.0):                # nodes: 30 + 20 j
        z = np.full(4, zn)
        assert rel(oracle.table_traveltime(s, h, z), oracle.traveltime(lin, np.hypot(h, z), z)) < 1e-15
    z = np.full(4, 40.0)                                 # halfway between the nodes at 30 and 50
    mid = 0.5 * (oracle.table_traveltime(s, h, np.full(4, 30.0)) + oracle.table_traveltime(s, h, np.full(4, 50.0)))
    assert rel(oracle.table_traveltime(s, h, z), mid) < 1e-14
    # the old node at 25 m (a multiple of D) is not a node any more: interpolated, not exact
    z25 = np.full(1, 25.0 + 30.0)
    assert abs(oracle.table_traveltime(s, [125.0], z25)[0] -
               oracle.traveltime(lin, np.hypot([125.0], z25), z25)[0]) > 1e-9
