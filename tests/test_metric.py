"""The bin triples that empty_slabs flags are exactly those where the oracle's distinct-index
brute force (the definition, no corrections involved) has no term; no GPU."""
import numpy as np

from metric import empty_slabs, rel_err


def test_empty_slabs_are_those_without_distinct_quadruplets(oracle):
    rng = np.random.default_rng(11)
    pos = rng.uniform(0, 10, (60, 2))
    pos[5] = pos[4]  # a duplicated position: two distinct galaxies at zero separation
    sh = rng.normal(0, 0.3, pos.shape)
    w = rng.uniform(0.5, 1.5, 60)
    edges = np.geomspace(0.4, 6.0, 9)
    bf = oracle.bruteforce(pos, sh, w, edges, 1)
    flagged = empty_slabs(pos, edges)
    zero = np.all(bf == 0, axis=(0, 1, 2))
    assert flagged.any() and (~flagged).any()
    np.testing.assert_array_equal(flagged, zero)


def test_rel_err_measures_empty_slabs_against_the_component_scale():
    b = np.zeros((9, 3, 3, 2, 2, 2), complex)
    b[:, :, :, 1, 1, 1] = 1.0
    a = b.copy()
    a[:, :, :, 0, 0, 0] = 1e-15  # residue where the reference is exactly zero
    empty = np.zeros((2, 2, 2), bool)
    empty[0, 0, 0] = True
    assert rel_err(a, b, empty=empty).max() == 1e-15
    assert rel_err(a, b).max() == 1e-15 / 1e-12
