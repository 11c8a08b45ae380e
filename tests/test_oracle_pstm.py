"""Pins of the oracle's prestack time migration (the PKTM the paper names in Sec. 4): the image's
vertical axis is the two-way vertical time t0, and each leg takes the double-square-root time
T = sqrt((t0/2)^2 + h^2 / v_rms(t0)^2) with the RMS velocity of v(z) = v0 + k z.  Pinned by the
identity with constant-velocity depth migration at k = 0 (z = v0 t0 / 2), the RMS velocity
against a numerical Dix integral of the model, the vertical two-way time, the exact hyperbola
in h^2, and the focusing of a diffractor in time; planted mistakes make a pin fail."""
import math

import numpy as np
import pytest
import scipy.integrate

import oracle
from paper_1204_1225_gb300 import survey as sv


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def pstm_survey(k=0.5, weight="one", aperture=0.0, seed=3):
    rng = np.random.default_rng(seed)
    s = sv.survey_random(rng, 3, 40, 7, 6, 30, 400, vel="pstm", weight=weight, aperture=aperture,
                         n_bins=3, h=25.0, v0=1600.0, k=k)
    return s.replace(oz=0.0, dz=0.02)       # t0 = 0 .. 0.58 s


def check_constant_velocity_identity():
    # k = 0: sqrt((t0/2)^2 + h^2/v0^2) = sqrt(h^2 + z^2)/v0 with z = v0 t0 / 2, and the weight's
    # straight rays are the same: the time image is the depth image on the mapped axis
    for weight in ("one", "obliq"):
        s = pstm_survey(k=0.0, weight=weight, aperture=90.0)
        d = sv.random_traces(s, 4, smooth=5).astype(np.float64)
        depth = s.replace(vel="const", oz=s.v0 * s.oz / 2, dz=s.v0 * s.dz / 2)
        a, b = oracle.migrate(s, d), oracle.migrate(depth, d)
        assert np.count_nonzero(b) > 0
        assert rel(a, b) < 1e-12


def check_rms_velocity_dix():
    # v_rms(t0)^2 = (2/t0) integral_0^{t0/2} v(tau)^2 dtau, with z(tau) from dz/dtau = v0 + k z
    # integrated numerically; read back from the hyperbola T^2 - (t0/2)^2 = h^2 / v_rms^2
    s = pstm_survey(k=0.6)
    for t0 in (0.1, 0.8, 2.0, 3.5):
        sol = scipy.integrate.solve_ivp(lambda t, z: s.v0 + s.k * z, (0.0, t0 / 2), [0.0], rtol=1e-12,
                                        atol=1e-9, dense_output=True)
        v2, _ = scipy.integrate.quad(lambda t: (s.v0 + s.k * sol.sol(t)[0]) ** 2, 0.0, t0 / 2,
                                     epsabs=0.0, epsrel=1e-12)
        vrms2 = v2 / (t0 / 2)
        h = 900.0
        T = float(oracle.traveltime(s, np.array([h]), np.array([t0]))[0])
        assert abs(h * h / (T * T - t0 * t0 / 4) - vrms2) < 1e-8 * vrms2


def check_vertical_and_hyperbola():
    s = pstm_survey(k=0.6)
    t0 = np.array([0.05, 0.4, 1.3, 2.7])
    # zero offset, vertical: each leg is half the two-way vertical time
    assert np.allclose(oracle.traveltime(s, np.zeros(4), t0), t0 / 2, rtol=0, atol=1e-15)
    # T^2 is exactly linear in h^2 at fixed t0
    h = np.array([0.0, 300.0, 700.0, 1500.0, 3000.0])
    for t in t0:
        T2 = oracle.traveltime(s, h, np.full(h.size, t)) ** 2
        slope = (T2[1:] - T2[0]) / h[1:] ** 2
        assert np.max(np.abs(slope - slope[0])) < 1e-12 * slope[0]


def check_diffractor_focuses_in_time():
    s = sv.survey_2d_const().replace(vel="pstm", v0=1800.0, k=0.4, oz=0.0, dz=0.008, nz=160)
    sc = np.array([[640.0, 0.0, 0.6, 1.0], [320.0, 0.0, 0.96, 1.0]])   # (x, -, t0, amplitude)
    d = sv.synthesize(s, sc, oracle.arrival_times, 25.0).numpy()
    img = oracle.migrate(s, d)[:, 0]
    for x, _, t0, _ in sc:
        ix, it = int(round(x / s.dx)), int(round(t0 / s.dz))
        for b in range(s.n_bins):
            win = img[b, ix - 2:ix + 3, it - 2:it + 3]
            if np.max(np.abs(win)) > 0:
                assert img[b, ix, it] == win.max()


def test_constant_velocity_identity():
    check_constant_velocity_identity()


def test_rms_velocity_dix():
    check_rms_velocity_dix()


def test_vertical_time_and_hyperbola():
    check_vertical_and_hyperbola()


def test_diffractor_focuses_in_time():
    check_diffractor_focuses_in_time()


MUTATIONS = [
    (11, check_rms_velocity_dix),           # interval velocity instead of the RMS velocity
    (12, check_vertical_and_hyperbola),     # t0 instead of t0/2 in the vertical leg
    (12, check_constant_velocity_identity),
]


@pytest.mark.parametrize("mutation,check", MUTATIONS, ids=[f"m{m}-{c.__name__}" for m, c in MUTATIONS])
def test_pstm_pins_catch_planted_mistakes(mutation, check):
    oracle.set_mutation(mutation)
    try:
        with pytest.raises(AssertionError):
            check()
    finally:
        oracle.set_mutation(0)
