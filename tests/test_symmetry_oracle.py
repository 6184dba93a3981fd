"""Symmetry-reduced storage of the multipoles (Table tab:4PCFSymm), oracle side; no GPU."""
import numpy as np
import pytest

import oracle
from oracle import symmetry


@pytest.mark.parametrize("nmax,edges", [(2, [0.8, 1.6, 3.0, 5.0]), (3, [0.7, 1.3, 2.5, 4.0, 6.0])])
def test_sorted_triples_rebuild_every_ordered_triple(nmax, edges):
    """Multipoles of the sorted triples, kept up to |n| <= 2N + 1, give all ordered triples at
    |n| <= N through the table (corrected estimator, all nine components)."""
    rng = np.random.default_rng(13 + nmax)
    pos = rng.uniform(0, 9, (45, 2))
    sh = rng.normal(0, 0.3, (45, 2))
    w = rng.uniform(0.5, 1.5, 45)
    edges = np.array(edges)
    nb = len(edges) - 1
    M = symmetry.enlarged_nmax(nmax)
    big = oracle.measure(pos, sh, w, edges, M)
    full = oracle.measure(pos, sh, w, edges, nmax)
    stored = symmetry.restrict(big, M)
    assert stored.shape[-1] == nb * (nb + 1) * (nb + 2) // 6
    rebuilt = symmetry.expand(stored, nb, nmax, M)
    np.testing.assert_allclose(rebuilt, full, rtol=0, atol=1e-12 * np.abs(full).max())


def test_reached_region_fits_the_enlarged_range():
    for nmax in (1, 3, 10, 20):
        M = symmetry.enlarged_nmax(nmax)
        reg = symmetry.reached_region(nmax)
        for mu, pairs in reg.items():
            a = np.array(sorted(pairs))
            assert np.abs(a).max() <= M
            assert len(pairs) >= (2 * nmax + 1) ** 2
            assert {(n2, n3) for n2 in range(-nmax, nmax + 1) for n3 in range(-nmax, nmax + 1)} <= pairs
