"""Pins of the N-th order oracle (App. F): the enumeration of natural components and the
brute-force multipoles, against the paper's 4PCF definitions, the pinned 4PCF brute force,
the two-point accumulators and rotation invariance; no GPU."""
import math

import numpy as np
import pytest

import oracle


def test_beta_matrix_reproduces_the_4pcf_components():
    """Eqs. Gamma0_def .. Gamma7_def: which of the four shears is conjugated in Gamma_0..7."""
    conj = [(), (0,), (1,), (2,), (3,), (0, 1), (0, 2), (0, 3)]
    want = np.ones((8, 4), dtype=int)
    for mu, c in enumerate(conj):
        want[mu, list(c)] = -1
    np.testing.assert_array_equal(oracle.beta_matrix(4), want)


@pytest.mark.parametrize("order", range(2, 11))
def test_beta_matrix_counts_and_completeness(order):
    """2^{N-1} rows (App. F.1), all distinct, and together with their global conjugates
    (every sign flipped) they cover all 2^N patterns exactly once."""
    b = oracle.beta_matrix(order)
    assert b.shape == (2 ** (order - 1), order)
    rows = {tuple(r) for r in b}
    conj = {tuple(-r) for r in b}
    assert len(rows) == b.shape[0] and not rows & conj
    assert len(rows | conj) == 2 ** order
    # ordered by the number of conjugated shears
    p = (b < 0).sum(axis=1)
    assert np.all(np.diff(p) >= 0) and p.max() == order // 2


def _catalogue(n, side, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, side, (n, 2))
    sh = rng.normal(0, 0.3, (n, 2))
    w = rng.uniform(0.5, 1.5, n)
    return pos, sh, w


def test_fourth_order_matches_the_pinned_quadruplet_brute_force():
    pos, sh, w = _catalogue(40, 6.0, 3)
    edges = np.array([0.8, 1.6, 3.0])
    g = oracle.bruteforce_multipoles(4, pos, sh, w, edges, 2)
    ref = oracle.bruteforce(pos, sh, w, edges, 2, distinct=False)
    assert g.shape == ref.shape
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_distinct_tuples_match_the_pinned_quadruplet_brute_force():
    """Excluding coinciding neighbours gives the distinct-quadruplet estimator."""
    pos, sh, w = _catalogue(40, 6.0, 7)
    edges = np.array([0.8, 1.6, 3.0])
    g = oracle.bruteforce_multipoles(4, pos, sh, w, edges, 2, distinct=True)
    ref = oracle.bruteforce(pos, sh, w, edges, 2, distinct=True)
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    full = oracle.bruteforce_multipoles(4, pos, sh, w, edges, 2)
    assert np.abs(full - g).max() > 1e-3 * np.abs(ref).max()  # coinciding neighbours matter


def test_second_order_is_the_xi_accumulators():
    """N = 2: Upsilon_0 = sum_i x_i G_-4, Upsilon_1 = sum_i x_i^* G_0 and the normalisation
    sum_i w_i W_0, the accumulators of xi_- and xi_+."""
    pos, sh, w = _catalogue(120, 10.0, 4)
    edges = np.array([0.5, 1.5, 3.0, 5.0])
    g = oracle.bruteforce_multipoles(2, pos, sh, w, edges, 0)
    _, xi = oracle.measure(pos, sh, w, edges, 1, with_xi=True)
    xi = np.asarray(xi).reshape(len(edges) - 1, 3)
    np.testing.assert_allclose(g[0], xi[:, 1], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(g[1], xi[:, 0], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(g[2], xi[:, 2], rtol=1e-12, atol=1e-13)


def test_third_order_rotation_invariance():
    """Natural components in the x-projection are invariant when positions and the shear
    frame rotate together (gamma_c -> gamma_c e^{2 i alpha})."""
    pos, sh, w = _catalogue(50, 6.0, 5)
    edges = np.array([0.7, 1.5, 2.8])
    g = oracle.bruteforce_multipoles(3, pos, sh, w, edges, 3)
    al = 0.9
    rot = np.array([[math.cos(al), -math.sin(al)], [math.sin(al), math.cos(al)]])
    gc = (sh[:, 0] + 1j * sh[:, 1]) * np.exp(2j * al)
    g2 = oracle.bruteforce_multipoles(3, pos @ rot.T, np.stack([gc.real, gc.imag], 1), w, edges, 3)
    assert np.abs(g).max() > 0
    np.testing.assert_allclose(g2, g, rtol=0, atol=1e-11 * np.abs(g).max())
    # reflection y -> -y: every polar angle changes sign and gamma_c -> gamma_c^*, so each
    # projected shear and the Fourier kernel become their conjugates: Upsilon -> Upsilon^*
    g3 = oracle.bruteforce_multipoles(3, pos * [1, -1], sh * [1, -1], w, edges, 3)
    np.testing.assert_allclose(g3, np.conj(g), rtol=0, atol=1e-11 * np.abs(g).max())
