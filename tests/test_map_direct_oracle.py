"""Pins of the direct aperture-mass oracle (Sect. 5.2, Eq. MapDirectEstimator) against
brute force, closed forms and invariances; no GPU."""
import itertools
import math

import numpy as np
import pytest

import oracle


def test_elementary_symmetric_is_the_distinct_product_sum():
    """e_k is the sum over index sets of k distinct galaxies; the ordered sum over distinct
    quadruplets i != j != k != l of Eq. MapDirectEstimator is 4! e_4."""
    x = np.random.default_rng(5).normal(size=8)
    e = oracle.elementary_symmetric(x, 4)
    assert e[0] == 1.0
    for k in range(1, 5):
        bf = sum(np.prod(c) for c in itertools.combinations(x, k))
        assert e[k] == pytest.approx(bf, rel=1e-13, abs=1e-13)
    ordered = sum(x[i] * x[j] * x[k] * x[l]
                  for i, j, k, l in itertools.permutations(range(x.size), 4))
    assert 24 * e[4] == pytest.approx(ordered, rel=1e-12)
    # fewer values than the order: the distinct sum is empty
    assert oracle.elementary_symmetric(x[:3], 4)[4] == 0.0
    assert oracle.elementary_symmetric([], 4)[1] == 0.0
    # all equal: binomial coefficients
    e = oracle.elementary_symmetric(np.full(11, 0.5), 4)
    assert e[4] == pytest.approx(math.comb(11, 4) * 0.5 ** 4, rel=1e-14)


def _brute_aperture(pos, shear, w, c, theta):
    """Eq. MapDirectEstimator for one aperture written as the nested distinct sums."""
    d = pos - c
    r = np.hypot(d[:, 0], d[:, 1])
    idx = np.flatnonzero(r < 4 * theta)
    zeta = np.arctan2(d[idx, 1], d[idx, 0])
    gt = -(shear[idx, 0] * np.cos(2 * zeta) + shear[idx, 1] * np.sin(2 * zeta))
    q = r[idx] ** 2 / (4 * np.pi * theta ** 4) * np.exp(-r[idx] ** 2 / (2 * theta ** 2))
    a = w[idx] * q * gt
    num = den = 0.0
    for i, j, k, l in itertools.permutations(range(idx.size), 4):
        num += a[i] * a[j] * a[k] * a[l]
        den += w[idx[i]] * w[idx[j]] * w[idx[k]] * w[idx[l]]
    num2 = sum(a[i] * a[j] for i, j in itertools.permutations(range(idx.size), 2))
    den2 = sum(w[idx[i]] * w[idx[j]] for i, j in itertools.permutations(range(idx.size), 2))
    return num, den, num2, den2, idx.size


def test_aperture_record_matches_nested_sums():
    rng = np.random.default_rng(11)
    pos = rng.uniform(-5, 5, size=(40, 2))
    shear = rng.normal(0, 0.3, size=(40, 2))
    w = rng.uniform(0.5, 1.5, 40)
    theta = 0.55
    c = np.array([0.3, -0.2])
    rec = oracle.aperture_record(pos, shear, w, c, theta)
    num, den, num2, den2, n = _brute_aperture(pos, shear, w, c, theta)
    assert 6 <= n <= 14 and rec[6] == n
    assert rec[2] * 24 == pytest.approx(num, rel=1e-10, abs=1e-16)
    assert rec[5] * 24 == pytest.approx(den, rel=1e-12)
    assert rec[1] * 2 == pytest.approx(num2, rel=1e-10, abs=1e-16)
    assert rec[4] * 2 == pytest.approx(den2, rel=1e-12)


def _tangential_lattice(theta, h, g, cross=False):
    """Galaxies on a square lattice (spacing h) around the origin with a constant tangential
    (or cross) shear g about the origin: gamma_c = -g e^{2i phi} (or -i g e^{2i phi})."""
    m = int(round(4 * theta / h))
    u = (np.arange(-m, m) + 0.5) * h
    x, y = np.meshgrid(u, u)
    pos = np.stack([x.ravel(), y.ravel()], 1)
    phi = np.arctan2(pos[:, 1], pos[:, 0])
    gc = -g * np.exp(2j * phi) * (1j if cross else 1.0)
    return pos, np.stack([gc.real, gc.imag], 1)


def test_tangential_pattern_closed_form():
    """Constant tangential shear g: the aperture measure is g times the integral of Q over
    the disc of radius 4 theta, g (1 - 9 e^{-8}) (Eq. CrittendenQ integrated in closed
    form); the cross pattern gives zero (E/B separation, Eq. MapGamma)."""
    theta, h, g = 1.3, 1.3 / 16, 0.05
    pos, sh = _tangential_lattice(theta, h, g)
    w = np.full(len(pos), 1.0)
    rec = oracle.aperture_record(pos, sh, w, np.zeros(2), theta)
    m_int = g * (1.0 - 9.0 * math.exp(-8.0))
    # Riemann sum of Q gamma_t over the disc (midpoint rule): h^2 sum a_i / w
    assert h * h * rec[0] == pytest.approx(m_int, rel=2e-4)
    # the estimator: area times the weighted mean over the disc, then fourth power
    area = math.pi * (4 * theta) ** 2
    mean_ap = area * rec[0] / rec[3]
    m4 = area ** 4 * rec[2] / rec[5]
    m2 = area ** 2 * rec[1] / rec[4]
    assert m4 == pytest.approx(mean_ap ** 4, rel=2e-3)
    assert m2 == pytest.approx(mean_ap ** 2, rel=1e-3)
    # sign: tangential shear counts positive
    assert mean_ap > 0
    mom = oracle.moments_from_records(rec[None], theta)
    assert mom[5] == pytest.approx(m4, rel=1e-12) and mom[6] == pytest.approx(m2, rel=1e-12)
    assert mom[7] == pytest.approx(m4 - 3 * m2 ** 2, rel=1e-12)
    # a deterministic field is far from Gaussian: connected part -2 M^4
    assert mom[7] == pytest.approx(-2 * mean_ap ** 4, rel=5e-3)
    pos, sh = _tangential_lattice(theta, h, g, cross=True)
    rec = oracle.aperture_record(pos, sh, w, np.zeros(2), theta)
    assert abs(rec[0]) < 1e-13 * len(pos) * g and abs(rec[2]) < 1e-20


def test_rotation_invariance():
    """Rotating positions, aperture centre and shear frame together (gamma_c -> gamma_c
    e^{2 i alpha}) leaves every record unchanged (gamma_t is a spin-0 projection)."""
    rng = np.random.default_rng(3)
    pos = rng.uniform(-6, 6, size=(3000, 2))
    shear = rng.normal(0, 0.3, size=(3000, 2))
    w = rng.uniform(0.5, 1.5, 3000)
    c = np.array([0.4, 0.7])
    rec = oracle.aperture_record(pos, shear, w, c, 1.1)
    al = 0.7
    rot = np.array([[math.cos(al), -math.sin(al)], [math.sin(al), math.cos(al)]])
    gc = (shear[:, 0] + 1j * shear[:, 1]) * np.exp(2j * al)
    rec2 = oracle.aperture_record(pos @ rot.T, np.stack([gc.real, gc.imag], 1), w, rot @ c, 1.1)
    assert rec2[6] == rec[6]
    np.testing.assert_allclose(rec2, rec, rtol=1e-9, atol=1e-12 * np.abs(rec).max())


def test_cut_and_degenerate_apertures():
    theta = 1.0
    # galaxies at exactly 4 theta are outside the hard cut; those inside are counted
    pos = np.array([[4.0, 0.0], [0.0, -4.0], [1.0, 1.0], [2.0, -1.0], [0.5, 3.0], [-2.0, 0.1],
                    [10.0, 10.0]])
    rng = np.random.default_rng(0)
    shear = rng.normal(0, 0.3, (len(pos), 2))
    w = np.ones(len(pos))
    rec = oracle.aperture_record(pos, shear, w, np.zeros(2), theta)
    assert rec[6] == 4 and rec[5] == pytest.approx(1.0)
    # fewer than four galaxies: no quadruplet, zero numerator and denominator
    rec3 = oracle.aperture_record(pos[:4], shear[:4], w[:4], np.zeros(2), theta)
    assert rec3[6] == 2 and rec3[2] == 0 and rec3[5] == 0 and rec3[4] == pytest.approx(1.0)
    mom = oracle.moments_from_records(rec3[None], theta)
    assert mom[5] == 0 and mom[1] == 0
    # an empty aperture
    rec0 = oracle.aperture_record(pos, shear, w, np.array([100.0, 0.0]), theta)
    assert not rec0.any()


def test_inverse_shot_noise_average():
    """The radius record adds numerators and denominators over apertures, i.e. averages the
    per-aperture ratios with weights equal to their denominators."""
    rng = np.random.default_rng(8)
    recs = np.zeros((5, 8))
    recs[:, [1, 2]] = rng.normal(size=(5, 2))
    recs[:, [4, 5]] = rng.uniform(1, 3, size=(5, 2))
    theta = 0.8
    mom = oracle.moments_from_records(recs, theta)
    area = math.pi * 3.2 ** 2
    ratio4 = recs[:, 2] / recs[:, 5]
    assert mom[5] == pytest.approx(area ** 4 * np.average(ratio4, weights=recs[:, 5]), rel=1e-12)
    assert mom[4] == 5
