"""Pins of the tree-approximation oracle (Sect. 3.2, App. F.3); no GPU."""
import numpy as np
import pytest

import oracle


def _catalogue(n, side, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, side, (n, 2)), rng.normal(0, 0.3, (n, 2)), rng.uniform(0.5, 1.5, n)


def test_exact_path_is_the_uncorrected_quadruplet_estimator():
    """Without approximation the per-centre multipoles contract into the C oracle's Upsilon_0
    and N_n without multiple-counting corrections."""
    pos, sh, w = _catalogue(250, 20.0, 5)
    edges = np.array([1.0, 2.0, 4.0, 8.0])
    nmax = 2
    n_lo = -2 * nmax - 3
    G, W = oracle.neighbour_multipoles(pos, sh, w, edges, n_lo, 2 * nmax)
    x = w * (sh[:, 0] + 1j * sh[:, 1])
    ups, nrm = oracle.upsilon0_from_multipoles(x, w, G, W, n_lo, nmax)
    ref = oracle.measure(pos, sh, w, edges, nmax, corrections=False)
    np.testing.assert_allclose(ups, ref[0], rtol=0, atol=1e-13 * np.abs(ref[0]).max())
    np.testing.assert_allclose(nrm, ref[8], rtol=0, atol=1e-13 * np.abs(ref[8]).max())


def test_reduced_catalogue_conserves_weight_and_shear():
    pos, sh, w = _catalogue(3000, 30.0, 6)
    x = w * (sh[:, 0] + 1j * sh[:, 1])
    origin = pos.min(axis=0)
    for delta in (0.5, 1.0, 4.0):
        com, X, W = oracle.reduced_catalogue(pos, sh, w, delta, origin)
        assert W.sum() == pytest.approx(w.sum(), rel=1e-12)
        assert abs(X.sum() - x.sum()) < 1e-10 * np.abs(x).sum()
        assert len(W) <= len(w) and np.all(W > 0)
        # every centre of mass lies in a cell that holds galaxies (to rounding: a galaxy on
        # the grid origin may give a centre of mass one ulp below it)
        cells = {tuple(v) for v in np.floor((pos - origin) / delta).astype(int)}
        for eps in (-1e-9, 1e-9):
            c = np.floor((com - origin) / delta + eps).astype(int)
            inside = np.array([tuple(v) in cells for v in c])
            if eps < 0:
                first = inside
        assert np.all(first | inside)


def test_one_galaxy_per_cell_is_exact():
    """On a lattice with one galaxy at the centre of every finest cell the level-1 reduced
    catalogue is the catalogue itself."""
    d = 0.25
    u = (np.arange(60) + 0.5) * d
    gx, gy = np.meshgrid(u, u)
    pos = np.stack([gx.ravel(), gy.ravel()], 1)
    rng = np.random.default_rng(2)
    sh = rng.normal(0, 0.3, (len(pos), 2))
    w = rng.uniform(0.5, 1.5, len(pos))
    # edges that no lattice separation (0.25 sqrt(k^2 + l^2)) comes near, so that the centre
    # of mass (the galaxy's position up to rounding) never crosses one
    edges = np.array([1.01, 2.03, 4.07])
    G, W = oracle.neighbour_multipoles(pos, sh, w, edges, -3, 3)
    Gt, Wt = oracle.neighbour_multipoles(pos, sh, w, edges, -3, 3, delta1=d, n_levels=1, r_min=2.0,
                                         origin=np.zeros(2))
    assert (oracle.bin_levels(edges, d, 1, 2.0) == 1).all()
    np.testing.assert_allclose(Gt, G, rtol=0, atol=1e-12 * np.abs(G).max())
    np.testing.assert_allclose(Wt, W, rtol=0, atol=1e-12 * np.abs(W).max())


def test_level_choice_of_the_paper_setting():
    """Resolutions {0.5', 1', 2'} and r_min = 40 (Sect. 6.2): a bin uses the coarsest grid
    with Theta_low / Delta >= 40, else the galaxies themselves."""
    lows = np.array([10.0, 19.9, 20.0, 39.9, 45.0, 79.9, 80.0, 166.0])
    edges = np.append(lows, 170.0)
    np.testing.assert_array_equal(oracle.bin_levels(edges, 0.5, 3, 40.0), [0, 0, 1, 1, 2, 2, 3, 3])


def test_error_shrinks_as_r_min_grows():
    """Every approximated bin uses a finer grid at r_min = 40 than at r_min = 10 (Delta_1 =
    0.05, four levels); the RMS error of Upsilon_0 against the exact path falls."""
    pos, sh, w = _catalogue(600, 30.0, 9)
    edges = np.array([2.0, 4.0, 8.0, 12.0])
    nmax = 2
    n_lo = -2 * nmax - 3
    x = w * (sh[:, 0] + 1j * sh[:, 1])
    G, W = oracle.neighbour_multipoles(pos, sh, w, edges, n_lo, 2 * nmax)
    ups, _ = oracle.upsilon0_from_multipoles(x, w, G, W, n_lo, nmax)
    np.testing.assert_array_equal(oracle.bin_levels(edges, 0.05, 4, 10.0), [3, 4, 4])
    np.testing.assert_array_equal(oracle.bin_levels(edges, 0.05, 4, 40.0), [1, 2, 3])
    errs = []
    for r_min in (10.0, 40.0):
        Gt, Wt = oracle.neighbour_multipoles(pos, sh, w, edges, n_lo, 2 * nmax, delta1=0.05, n_levels=4,
                                             r_min=r_min)
        ut, _ = oracle.upsilon0_from_multipoles(x, w, Gt, Wt, n_lo, nmax)
        errs.append(np.sqrt(np.mean(np.abs(ut - ups) ** 2) / np.mean(np.abs(ups) ** 2)))
    assert 0 < errs[1] < 0.5 * errs[0]


def test_approximation_error_at_the_papers_setting():
    """Error of the tree approximation against the exact multipoles (Sect. 3.2): a seeded
    4000-galaxy GRF on 60' x 60', 8 log bins 1'-30', n_max = 5, grids of 0.125', 0.25', 0.5'.
    Bins kept exact stay exact; at the paper's r_min = 40 every approximated bin holds the
    largest error of G_n to 7%, of Upsilon_0 on diagonal triples to 5% and of N_n to 3e-4
    (each relative to the largest value of its bin; measured 4-6%, 2-4%, <= 1.2e-4), and
    the errors shrink from r_min = 10 to r_min = 40."""
    import synth
    pos, sh, w = synth.grf_catalog(4000, 60.0, 9, grid=512)
    edges = synth.log_edges(1.0, 30.0, 8)
    nmax = 5
    n_lo, n_hi = -2 * nmax - 3, 2 * nmax
    x = w * (sh[:, 0] + 1j * sh[:, 1])
    G, W = oracle.neighbour_multipoles(pos, sh, w, edges, n_lo, n_hi)
    u, nr = oracle.upsilon0_from_multipoles(x, w, G, W, n_lo, nmax)
    nb = len(edges) - 1
    worst = {}
    for r_min in (10, 40):
        Gt, Wt = oracle.neighbour_multipoles(pos, sh, w, edges, n_lo, n_hi, delta1=0.125, n_levels=3, r_min=r_min)
        ut, nt = oracle.upsilon0_from_multipoles(x, w, Gt, Wt, n_lo, nmax)
        lev = oracle.bin_levels(edges, 0.125, 3, r_min)
        eg = np.abs(Gt - G).max(axis=(0, 1)) / np.abs(G).max(axis=(0, 1))
        eu = np.array([np.abs(ut[..., b, b, b] - u[..., b, b, b]).max() / np.abs(u[..., b, b, b]).max()
                       for b in range(nb)])
        en = np.array([np.abs(nt[..., b, b, b] - nr[..., b, b, b]).max() / np.abs(nr[..., b, b, b]).max()
                       for b in range(nb)])
        exact = np.asarray(lev) == 0
        assert exact.any() and (~exact).any()
        assert eg[exact].max() < 1e-12 and en[exact].max() < 1e-12
        worst[r_min] = (eg[~exact].max(), eu[~exact].max(), en[~exact].max())
    g, ups, nrm = worst[40]
    assert g < 0.07 and ups < 0.05 and nrm < 3e-4
    assert all(worst[40][k] < worst[10][k] for k in range(3))
