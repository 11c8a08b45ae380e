"""Pins of the oracle's velocity-analysis objective (Sec. 2: redundant offset images whose
differences measure the velocity error; the model is corrected until they agree and are
stacked).  The objective is the normalised variance of the weighted offset images across the
bins, V = sum_b ||w_b I_b - m||^2 / sum_b ||w_b I_b||^2.  Pinned by closed forms (identical
images, disjoint supports), invariances, finite differences of both gradients, and the
position of its minimum on noise-free diffractor data; planted mistakes make a pin fail."""
import numpy as np
import pytest

import oracle
from paper_1204_1225_gb300 import survey as sv


def check_closed_forms():
    rng = np.random.default_rng(1)
    w = np.array([0.5, 0.25, 0.0, 0.125])            # bin 2 holds no trace
    base = rng.standard_normal((3, 5, 7))
    # identical weighted images: nothing to correct, V = 0 and no gradient
    img = np.stack([base / wb if wb > 0 else rng.standard_normal((3, 5, 7)) for wb in w])
    V, G = oracle.semblance(img, w)
    assert abs(V) < 1e-15 and np.max(np.abs(G)) < 1e-15
    # weighted images of equal energy on disjoint supports: V = 1 - 1/N (N = 3 bins with traces)
    img = np.zeros((4, 3, 5, 7))
    for i, b in enumerate((0, 1, 3)):
        img[b, i, :, :] = 2.0 / w[b]
    V, _ = oracle.semblance(img, w)
    assert abs(V - (1.0 - 1.0 / 3.0)) < 1e-15
    # two bins, unit weights, images e_1 and e_2: m = (1/2, 1/2), D = 1, B = 2, V = 1/2
    V, G = oracle.semblance(np.array([[1.0, 0.0], [0.0, 1.0]]), np.ones(2))
    assert V == 0.5
    # by the quotient rule, dV/dI = (dD/dI B - D dB/dI) / B^2 with dD/dI_b = 2 (I_b - m) and
    # dB/dI_b = 2 I_b: for bin 0, ((2 (1/2) 2 - 1 (2)) / 4, (2 (-1/2) 2 - 0) / 4) = (0, -1/2)
    assert np.allclose(G, [[0.0, -0.5], [-0.5, 0.0]], rtol=0, atol=1e-15)


def check_invariances():
    rng = np.random.default_rng(2)
    img = rng.standard_normal((4, 6, 5))
    w = np.array([1.0, 0.5, 2.0, 0.25])
    V, _ = oracle.semblance(img, w)
    assert abs(oracle.semblance(3.7 * img, w)[0] - V) < 1e-14        # scale of the data
    perm = [2, 0, 3, 1]
    assert abs(oracle.semblance(img[perm], w[perm])[0] - V) < 1e-14  # order of the bins
    assert 0.0 <= V <= 1.0


def check_image_gradient_fd():
    rng = np.random.default_rng(3)
    img = rng.standard_normal((3, 4, 6))
    w = np.array([0.3, 0.7, 0.2])
    V, G = oracle.semblance(img, w)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 3), (2, 3, 5), (1, 0, 4)]:
        e = np.zeros_like(img)
        e[idx] = h
        fd = (oracle.semblance(img + e, w)[0] - oracle.semblance(img - e, w)[0]) / (2 * h)
        assert abs(fd - G[idx]) < 1e-7 * max(1.0, abs(G[idx])) + 1e-9


def pin_line():
    s = sv.survey_25d_velan(nx=64, nz=60, h=25.0)
    sc = sv.diffractors_2d(np.random.default_rng(3), s)
    d = sv.synthesize(s, sc, oracle.arrival_times, 12.0).numpy()
    return s, d


def check_velocity_gradient_fd():
    s, d = pin_line()
    v0, k = 1740.0, 0.52
    V, g0, g1 = oracle.velocity_objective(s, d, v0, k)
    hv, hk = 1e-2, 1e-5
    fv = (oracle.velocity_objective(s, d, v0 + hv, k)[0] - oracle.velocity_objective(s, d, v0 - hv, k)[0]) / (2 * hv)
    fk = (oracle.velocity_objective(s, d, v0, k + hk)[0] - oracle.velocity_objective(s, d, v0, k - hk)[0]) / (2 * hk)
    # the linear interpolant's slope jumps at samples: agreement to ~1e-3
    assert abs(g0 - fv) < 2e-3 * abs(fv)
    assert abs(g1 - fk) < 2e-3 * abs(fk)


def check_minimum_at_true_velocity():
    # noise-free diffractors: with k at its true value the offset images agree best at the true
    # v0 (20 m/s grid), and with v0 true the best k lies within 0.05 of the true 0.6
    s, d = pin_line()
    v0s = np.arange(1700.0, 1901.0, 20.0)
    Vv = [oracle.velocity_objective(s, d, v, s.k)[0] for v in v0s]
    assert v0s[int(np.argmin(Vv))] == s.v0
    ks = np.arange(0.45, 0.751, 0.05)
    Vk = [oracle.velocity_objective(s, d, s.v0, kk)[0] for kk in ks]
    assert abs(ks[int(np.argmin(Vk))] - s.k) <= 0.05 + 1e-9


def test_semblance_closed_forms():
    check_closed_forms()


def test_semblance_invariances():
    check_invariances()


def test_semblance_image_gradient_fd():
    check_image_gradient_fd()


def test_velocity_gradient_fd():
    check_velocity_gradient_fd()


def test_minimum_at_true_velocity():
    check_minimum_at_true_velocity()


MUTATIONS = [
    (1, check_closed_forms),          # bin weights dropped
    (2, check_closed_forms),          # wrong bin count in the mean image
    (3, check_image_gradient_fd),     # sign of the quotient term of the gradient
    (3, check_velocity_gradient_fd),
]


@pytest.mark.parametrize("mutation,check", MUTATIONS, ids=[f"m{m}-{c.__name__}" for m, c in MUTATIONS])
def test_velan_pins_catch_planted_mistakes(mutation, check):
    oracle._va_mutation = mutation
    try:
        with pytest.raises(AssertionError):
            check()
    finally:
        oracle._va_mutation = 0
