"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from the
definition (brute force over quadruplets), a closed form, a count printed in the paper,
an exact invariance, the symmetry table printed separately from the estimator equations,
DFT orthogonality, or direct numerical quadrature of the aperture-mass definition.
"""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_err(a, b):
    """|a-b| per element over max(|b|, rms floor) -- the floor is the rms over (n2, n3)
    of the reference for each (mu, Theta1, Theta2, Theta3)."""
    floor = np.sqrt(np.mean(np.abs(b) ** 2, axis=(1, 2), keepdims=True))
    # slabs that vanish in exact arithmetic hold only rounding residue: floor them at
    # 1e-12 of the component's largest value
    scale = np.abs(b).reshape(b.shape[0], -1).max(axis=1).reshape((-1,) + (1,) * (b.ndim - 1))
    den = np.maximum(np.maximum(np.abs(b), floor), 1e-12 * scale)
    den = np.where(den > 0, den, 1.0)
    return np.abs(a - b) / den


def tiny_catalogue(n=22, seed=3, side=8.0, dup=0):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, side, (n, 2))
    sh = rng.normal(0, 0.3, (n, 2))
    w = rng.uniform(0.5, 1.5, n)
    if dup:
        pos = np.concatenate([pos, pos[:dup]])
        sh = np.concatenate([sh, sh[:dup]])
        w = np.concatenate([w, w[:dup]])
    return pos, sh, w


EDGES = np.array([0.6, 1.5, 3.0, 7.0])


# --------------------------------------------------------------------------------------
# Definition: the factorised estimator equals the O(N^4) quadruplet sum
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("seed,nmax", [(3, 2), (4, 3)])
def test_factorised_equals_bruteforce_distinct(oracle, seed, nmax):
    pos, sh, w = tiny_catalogue(seed=seed)
    f = oracle.measure(pos, sh, w, EDGES, nmax)
    b = oracle.bruteforce(pos, sh, w, EDGES, nmax, distinct=True)
    assert np.abs(b).max() > 0
    assert rel_err(f, b).max() < 1e-11


def test_uncorrected_equals_bruteforce_all_indices(oracle):
    pos, sh, w = tiny_catalogue(seed=5)
    f = oracle.measure(pos, sh, w, EDGES, 2, corrections=False)
    b = oracle.bruteforce(pos, sh, w, EDGES, 2, distinct=False)
    assert rel_err(f, b).max() < 1e-11


def test_duplicated_galaxies_are_distinct_points(oracle):
    """Distinct indices at the same position are different galaxies: only equal-index
    terms are removed by the correction."""
    pos, sh, w = tiny_catalogue(n=16, seed=6, dup=4)
    f = oracle.measure(pos, sh, w, EDGES, 2)
    b = oracle.bruteforce(pos, sh, w, EDGES, 2, distinct=True)
    assert rel_err(f, b).max() < 1e-11


def test_centre_mask_is_a_sum_over_centres(oracle):
    pos, sh, w = tiny_catalogue(seed=7)
    mask = np.zeros(len(w), np.uint8)
    mask[::3] = 1
    a = oracle.measure(pos, sh, w, EDGES, 2, centre_mask=mask)
    b = oracle.measure(pos, sh, w, EDGES, 2, centre_mask=1 - mask)
    full = oracle.measure(pos, sh, w, EDGES, 2)
    assert rel_err(a + b, full).max() < 1e-12
    bf = oracle.bruteforce(pos, sh, w, EDGES, 2, centre_mask=mask)
    assert rel_err(a, bf).max() < 1e-11


# --------------------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------------------
def test_single_centre_three_neighbours_closed_form(oracle):
    """One centre, one neighbour in each of three bins: each ordered assignment (j,k,l)
    of the neighbours gives exactly one term.  mu = 0 and N are printed explicitly in
    Eq. QuadrupletUpsilon and Eq. TripletNorm:  x_i x_j x_k x_l e^{-i(3phi_ij + 2phi_ik +
    3phi_il)} and w_i w_j w_k w_l, each times e^{-i n2 phi_ijk} e^{-i n3 phi_ijl}."""
    N = 3
    phis = np.array([0.3, 2.2, -1.9])
    radii = np.array([1.0, 2.0, 5.0])  # bins 0, 1, 2 of EDGES
    pos = np.vstack([[0.0, 0.0], np.c_[radii * np.cos(phis), radii * np.sin(phis)]])
    rng = np.random.default_rng(11)
    sh = rng.normal(0, 0.3, (4, 2))
    w = np.array([1.3, 0.7, 1.1, 0.9])
    mask = np.array([1, 0, 0, 0], np.uint8)
    U = oracle.measure(pos, sh, w, EDGES, N, centre_mask=mask)
    x = w * (sh[:, 0] + 1j * sh[:, 1])
    n = np.arange(-N, N + 1)
    import itertools
    for perm in itertools.permutations(range(3)):
        j, k, l = perm
        pj, pk, pl = phis[j], phis[k], phis[l]
        proj = np.exp(-1j * n[:, None] * (pk - pj)) * np.exp(-1j * n[None, :] * (pl - pj))
        exp0 = x[0] * x[1 + j] * x[1 + k] * x[1 + l] * np.exp(-1j * (3 * pj + 2 * pk + 3 * pl)) * proj
        expN = w[0] * w[1 + j] * w[1 + k] * w[1 + l] * proj
        assert np.allclose(U[0, :, :, j, k, l], exp0, rtol=1e-13, atol=1e-15)
        assert np.allclose(U[8, :, :, j, k, l], expN, rtol=1e-13, atol=1e-15)
    # every bin triple with a repeated bin holds only multiple-counting terms -> zero
    for b1 in range(3):
        for b2 in range(3):
            for b3 in range(3):
                if len({b1, b2, b3}) < 3:
                    assert np.abs(U[:, :, :, b1, b2, b3]).max() < 1e-14


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "worked_count.json")))["cases"])
def test_worked_count_app_a1(oracle, case):
    """App. A.1: unit weights, m galaxies in one annulus, all radial bins equal:
    N_0 = m^3 uncorrected and m(m-1)(m-2) for distinct quadruplets."""
    m = case["m"]
    ang = 2 * np.pi * np.arange(m) / m + 0.1
    pos = np.vstack([[0.0, 0.0], np.c_[2.0 * np.cos(ang), 2.0 * np.sin(ang)]])
    sh = np.zeros((m + 1, 2))
    w = np.ones(m + 1)
    mask = np.zeros(m + 1, np.uint8)
    mask[0] = 1
    edges = np.array([1.5, 2.5, 4.5])
    U0 = oracle.measure(pos, sh, w, edges, 1, centre_mask=mask, corrections=False)
    U1 = oracle.measure(pos, sh, w, edges, 1, centre_mask=mask)
    assert abs(U0[8, 1, 1, 0, 0, 0] - case["uncorrected"]) < 1e-9
    assert abs(U1[8, 1, 1, 0, 0, 0] - case["corrected"]) < 1e-9


def test_memory_footprint_matches_paper(oracle):
    g = json.load(open(os.path.join(GOLDEN, "memory_footprint.json")))
    nb, N, nphi = g["n_bins"], g["n_max"], g["n_phi"]
    multipole = np.prod(oracle.ups_shape(nb, N)) * 16 / 1e9
    real_space = 9 * nb ** 3 * nphi ** 2 * 16 / 1e9
    assert round(multipole) == g["multipole_GB"]
    assert round(real_space) == g["real_space_GB"]


# --------------------------------------------------------------------------------------
# Exact invariances
# --------------------------------------------------------------------------------------
def test_rotation_invariance(oracle):
    """Rotating positions by alpha rotates the Cartesian shear by e^{2 i alpha}; the
    natural components in the x-projection do not change."""
    pos, sh, w = tiny_catalogue(seed=8)
    a = 0.7
    R = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    g = (sh[:, 0] + 1j * sh[:, 1]) * np.exp(2j * a)
    U = oracle.measure(pos, sh, w, EDGES, 3)
    Ur = oracle.measure(pos @ R.T, np.c_[g.real, g.imag], w, EDGES, 3)
    assert rel_err(Ur, U).max() < 1e-10


def test_reflection_conjugates(oracle):
    pos, sh, w = tiny_catalogue(seed=9)
    U = oracle.measure(pos, sh, w, EDGES, 3)
    Uf = oracle.measure(pos * [1, -1], sh * [1, -1], w, EDGES, 3)
    assert rel_err(Uf, np.conj(U)).max() < 1e-10


def test_translation_and_weight_scaling(oracle):
    pos, sh, w = tiny_catalogue(seed=10)
    U = oracle.measure(pos, sh, w, EDGES, 2)
    Ut = oracle.measure(pos + [37.0, -11.5], sh, w, EDGES, 2)
    assert rel_err(Ut, U).max() < 1e-10
    Us = oracle.measure(pos, sh, 1.7 * w, EDGES, 2)
    assert rel_err(Us, 1.7 ** 4 * U).max() < 1e-12


def test_global_shear_phase(oracle):
    """gamma -> gamma e^{i beta}: components with p unconjugated and q conjugated shears
    pick up e^{i (p - q) beta}; N is unchanged."""
    pos, sh, w = tiny_catalogue(seed=12)
    beta = 0.9
    g = (sh[:, 0] + 1j * sh[:, 1]) * np.exp(1j * beta)
    U = oracle.measure(pos, sh, w, EDGES, 2)
    Ub = oracle.measure(pos, np.c_[g.real, g.imag], w, EDGES, 2)
    k = np.array([4, 2, 2, 2, 2, 0, 0, 0, 0])
    expect = U * np.exp(1j * k * beta)[:, None, None, None, None, None]
    assert rel_err(Ub, expect).max() < 1e-12


# --------------------------------------------------------------------------------------
# Table tab:4PCFSymm: permutations of the radial bins
# --------------------------------------------------------------------------------------
# the table as typed into the oracle (bin permutation per column, mu' per (mu, column) and the
# multipole map); pinned here against the estimator itself
from oracle.symmetry import BIN_PERM as _BIN_PERM, MU_MAP as _MU_MAP, n_map as _n_map  # noqa: E402


def test_symmetry_table(oracle):
    pos, sh, w = tiny_catalogue(n=40, seed=13, side=9.0)
    N = 3
    U = oracle.measure(pos, sh, w, EDGES, N)
    scale = np.abs(U).max()
    nb = len(EDGES) - 1
    checked = 0
    for mu in range(9):
        for col in range(5):
            mup = _MU_MAP[mu][col]
            perm = _BIN_PERM[col]
            for n2 in range(-N, N + 1):
                for n3 in range(-N, N + 1):
                    m2, m3 = _n_map(mu, col, n2, n3)
                    if abs(m2) > N or abs(m3) > N:
                        continue
                    for b1 in range(nb):
                        for b2 in range(nb):
                            for b3 in range(nb):
                                bb = (b1, b2, b3)
                                lhs = U[mu, n2 + N, n3 + N, b1, b2, b3]
                                rhs = U[mup, m2 + N, m3 + N, bb[perm[0]], bb[perm[1]], bb[perm[2]]]
                                assert abs(lhs - rhs) < 1e-11 * scale
                                checked += 1
    assert checked > 1000


# --------------------------------------------------------------------------------------
# Real space: bin-integrated reconstruction and DFT orthogonality
# --------------------------------------------------------------------------------------
def test_real_space_orthogonality(oracle):
    """For nphi > 4N+1 uniform bins, the bin sums of the reconstructed density project
    back onto the multipoles: Upsilon_m = sum_{p,q} C(p,q) e^{-i m.phi_c} / sinc(m dphi/2)^2."""
    pos, sh, w = tiny_catalogue(seed=14)
    N = 3
    U = oracle.measure(pos, sh, w, EDGES, N)
    nphi = 4 * N + 6
    gam, nrm = oracle.to_real_space(U, nphi)
    dphi = 2 * np.pi / nphi
    pc = (np.arange(nphi) + 0.5) * dphi
    n = np.arange(-N, N + 1)
    E = np.exp(-1j * n[:, None] * pc[None, :])  # [n, p]
    sinc = np.sinc(n * dphi / 2 / np.pi)
    counts = gam * nrm[None]
    rec = np.einsum("ap,bq,mxyzpq->mabxyz", E, E, counts) / (sinc[:, None] * sinc[None, :])[None, :, :, None, None, None]
    assert rel_err(rec, U[:8]).max() < 1e-10
    recN = np.einsum("ap,bq,xyzpq->abxyz", E, E, nrm) / (sinc[:, None] * sinc[None, :])[:, :, None, None, None]
    assert np.abs(recN - U[8]).max() < 1e-10 * np.abs(U[8]).max()


def test_real_space_total_count(oracle):
    """Summing the bin counts over all angular bins gives the n = 0 multipole."""
    pos, sh, w = tiny_catalogue(seed=15)
    U = oracle.measure(pos, sh, w, EDGES, 2)
    gam, nrm = oracle.to_real_space(U, 7)
    assert np.allclose(nrm.sum(axis=(-1, -2)), U[8, 2, 2].real, rtol=1e-12, atol=1e-12)
    tot = (gam * nrm[None]).sum(axis=(-1, -2))
    assert np.allclose(tot, U[:8, 2, 2], rtol=1e-10, atol=1e-12 * np.abs(U).max())


# --------------------------------------------------------------------------------------
# Aperture measures: the closed-form filter against quadrature of Eq. MapGamma
# --------------------------------------------------------------------------------------
_BETA = [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (1, 1, 0, 0),
         (1, 0, 1, 0), (1, 0, 0, 1)]


def _q_times_phase(v, theta, conj):
    """Q_theta(|v|) e^{-+2i arg v} with Q of Eq. CrittendenQ."""
    r = np.abs(v)
    Q = r ** 2 / (4 * np.pi * theta ** 4) * np.exp(-r ** 2 / (2 * theta ** 2))
    return Q * np.exp((2j if conj else -2j) * np.angle(v))


@pytest.mark.parametrize("mu", range(8))
def test_map4_filter_against_quadrature(oracle, mu):
    """F_mu / (2 pi t1 t2 t3) = e^{2 i sum_a s_a zeta_a} int d^2y prod_a Q(|y+vt_a|)
    e^{-+2i arg(y+vt_a)}: the aperture centre integrated numerically on a grid."""
    theta = 1.3
    t1, t2, t3, p12, p13 = 0.9, 1.6, 2.1, 1.1, 3.7
    vt = np.array([0.0, t1, t2 * np.exp(1j * p12), t3 * np.exp(1j * p13)])
    L, M = 9.0 * theta, 1201
    g = np.linspace(-L, L, M)
    yy = g[None, :] + 1j * g[:, None]
    prod = np.ones_like(yy)
    for a in range(4):
        prod = prod * _q_times_phase(yy + vt[a], theta, _BETA[mu][a])
    quad = prod.sum() * (g[1] - g[0]) ** 2
    zeta = [0.5 * p13, 0.0, p12, p13]
    phase = np.exp(2j * sum((-1 if _BETA[mu][a] else 1) * zeta[a] for a in range(4)))
    expect = 2 * np.pi * t1 * t2 * t3 * phase * quad
    got = oracle.map4_filter(mu, theta, t1, t2, t3, p12, p13)
    assert abs(got - expect) < 1e-7 * abs(expect)


def test_eb_decomposition_of_one_sample(oracle):
    """With M_a = P_a + i X_a, the 8 correlators of Eq. M4Ordering evaluated on one sample
    decompose into the 16 products of P and X in the order of Eq. 4PCF_rawcomponents."""
    rng = np.random.default_rng(21)
    P = rng.normal(size=4)
    X = rng.normal(size=4)
    M = P + 1j * X
    m4 = [np.prod([np.conj(M[a]) if b[a] else M[a] for a in range(4)]) for b in _BETA]
    order = ["tttt", "xttt", "txtt", "ttxt", "tttx", "ttxx", "txtx", "txxt", "xttx", "xtxt",
             "xxtt", "txxx", "xtxx", "xxtx", "xxxt", "xxxx"]
    expect = [np.prod([P[a] if c[a] == "t" else X[a] for a in range(4)]) for c in order]
    assert np.allclose(oracle.eb_from_m4(np.array(m4)), expect, rtol=1e-12, atol=1e-14)


def _pair_kernel(theta, sep, conj2):
    """int d^2X Q(|Y0-X|) e^{-2i arg} Q(|Y1-X|) e^{-+2i arg} for Y1 - Y0 = sep (real)."""
    L, M = 9.0 * theta, 1201
    g = np.linspace(-L, L, M)
    yy = g[None, :] + 1j * g[:, None]
    k = _q_times_phase(yy, theta, False) * _q_times_phase(yy + sep, theta, conj2)
    return k.sum() * (g[1] - g[0]) ** 2


def test_disconnected_part_two_point_filters(oracle):
    """The Gaussian part uses <M M^*> and <M M> of one aperture built from xi_+/-; check
    them against quadrature of Eq. MapGamma for a pair, via <M_ap^4>_disc = 3 <M_ap^2>^2."""
    theta = 2.0
    edges = np.array([1.0, 3.0])
    tb = 2.0 / 3.0 * (27 - 1) / (9 - 1)
    A = 0.5 * (9 - 1)
    ups = np.zeros(oracle.ups_shape(1, 0), np.complex128)
    # xi_+ only: <M M^*> = xi_+ * 2 pi A_b K_+(tb)  (the cross shear phase cancels)
    xi = np.array([[0.8, 0.0, 0.0, 0.0]])
    _, _, disc = oracle.map4(ups, edges, 4, [theta], xi)
    B = 0.8 * 2 * np.pi * A * _pair_kernel(theta, tb, True).real
    assert abs(disc[0, 0] - 3 * (B / 2) ** 2) < 1e-6 * abs(3 * (B / 2) ** 2)
    # xi_- only: <M M> = xi_- * 2 pi A_b K_-(tb) e^{4 i phi} with phi = 0 here
    xi = np.array([[0.0, 0.0, 0.6, 0.0]])
    _, _, disc = oracle.map4(ups, edges, 4, [theta], xi)
    Am = 0.6 * 2 * np.pi * A * _pair_kernel(theta, tb, False)
    assert abs(disc[0, 0] - 3 * (Am.real / 2) ** 2) < 1e-6 * abs(3 * (Am.real / 2) ** 2)


def test_xi_plus_of_constant_shear(oracle):
    """A noiseless constant shear g with unit weights has xi_+ = |g|^2 in every bin."""
    rng = np.random.default_rng(22)
    pos = rng.uniform(0, 8, (60, 2))
    g = 0.03 - 0.02j
    sh = np.tile([g.real, g.imag], (60, 1))
    _, acc = oracle.measure(pos, sh, np.ones(60), EDGES, 1, with_xi=True)
    xi = oracle.xi_from_acc(acc)
    assert np.allclose(xi[:, 0], abs(g) ** 2, rtol=1e-12)
    assert np.allclose(xi[:, 1], 0, atol=1e-16)


def test_xi_pm_against_tangential_and_cross_pair_sums(oracle):
    """xi_+/- from the estimator's accumulators equal their definition as weighted pair means:
    xi_+ = <gamma_t gamma_t + gamma_x gamma_x>, xi_- = <gamma_t gamma_t - gamma_x gamma_x>
    (plus the imaginary parts <gamma_x gamma_t - gamma_t gamma_x> and
    <gamma_x gamma_t + gamma_t gamma_x> up to sign), each galaxy's shear projected on the
    direction of the pair (Eq. gammatx_def), over ordered pairs i != j in the bin.  A sign of
    the phase, a conjugation or a bin index off by one fails it."""
    rng = np.random.default_rng(31)
    n = 120
    pos = rng.uniform(0, 8, (n, 2))
    sh = rng.normal(0, 0.3, (n, 2))
    w = rng.uniform(0.5, 1.5, n)
    _, acc = oracle.measure(pos, sh, w, EDGES, 4, with_xi=True)
    xi = oracle.xi_from_acc(acc)
    g = sh[:, 0] + 1j * sh[:, 1]
    nb = len(EDGES) - 1
    num_p = np.zeros(nb); num_m = np.zeros(nb); den = np.zeros(nb)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            d = pos[j] - pos[i]
            r2 = d @ d
            b = np.searchsorted(EDGES ** 2, r2, side="right") - 1
            if b < 0 or b >= nb:
                continue
            phi = np.arctan2(d[1], d[0])
            ti, xi_i = (-(g[i] * np.exp(-2j * phi))).real, (-(g[i] * np.exp(-2j * phi))).imag
            tj, xj = (-(g[j] * np.exp(-2j * phi))).real, (-(g[j] * np.exp(-2j * phi))).imag
            num_p[b] += w[i] * w[j] * (ti * tj + xi_i * xj)
            num_m[b] += w[i] * w[j] * (ti * tj - xi_i * xj)
            den[b] += w[i] * w[j]
    ok = den > 0
    assert ok.sum() >= nb - 1
    assert np.allclose(xi[ok, 0], num_p[ok] / den[ok], rtol=1e-10, atol=1e-14)
    assert np.allclose(xi[ok, 2], num_m[ok] / den[ok], rtol=1e-10, atol=1e-14)
    # the imaginary part of xi_+ vanishes over ordered pairs (i, j) and (j, i)
    assert np.allclose(xi[ok, 1], 0.0, atol=1e-14)
