"""The N-th order table generator of the library (App. F; host functions, no GPU):
its enumeration against the oracle's, its order-4 tables against the tables compiled into
the contraction kernels and against the paper's printed example, and the multipoles its
tables define against the oracle's brute force at orders 2, 3, 4 and 5."""
import itertools

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def lib():
    from paper_2509_07974_gb300 import build, ext4pcf
    build.build()
    return ext4pcf


@pytest.mark.parametrize("order", range(2, 13))
def test_components_match_the_oracle_enumeration(lib, order):
    np.testing.assert_array_equal(lib.ext4pcf_nth_order_components(order), oracle.beta_matrix(order))


def test_generated_order_four_tables_are_the_kernels_tables(lib):
    """Code-generation cross-check of the hand-written 4PCF index tables: the factors of
    Upsilon_0..7 and N_n generated from beta equal, entry for entry, those compiled into the
    CUDA-core and the tensor-core contraction."""
    gen = np.array([lib.ext4pcf_nth_order_factors(4, mu) for mu in list(range(8)) + [-1]])
    np.testing.assert_array_equal(lib.ext4pcf_contraction_tables(0), gen)
    np.testing.assert_array_equal(lib.ext4pcf_contraction_tables(1), gen)


@pytest.mark.parametrize("order", [4, 5, 6, 7])
def test_printed_example_of_the_first_p_shears_conjugated(lib, order):
    """App. F.2 prints Upsilon for the component whose first p shears are conjugated:
    x^* conj(G_{-(sum n + 3)})(Th_1) prod_{m=2}^{p-1} conj(G_{n_m - 2})(Th_m)
    prod_{m=p}^{N-2} G_{-(n_m + 2)}(Th_m) G_{-(n_{N-1} + 1)}(Th_{N-1})."""
    beta = lib.ext4pcf_nth_order_components(order)
    for p in range(2, order // 2 + 1):
        row = np.ones(order, dtype=int)
        row[:p] = -1
        mu = int(np.flatnonzero((beta == row).all(axis=1))[0])
        t = lib.ext4pcf_nth_order_factors(order, mu)
        rw = order + 1
        assert t[1] == 1
        want = []
        for m in range(1, order):
            a = np.zeros(order - 2, dtype=int)
            if m == 1:
                a[:] = -1
                want.append([0, 1, *a, -3])
            elif m <= p - 1:
                a[m - 2] = 1
                want.append([0, 1, *a, -2])
            elif m <= order - 2:
                a[m - 2] = -1
                want.append([0, 0, *a, -2])
            else:
                a[m - 2] = -1
                want.append([0, 0, *a, -1])
        np.testing.assert_array_equal(t[2:].reshape(order - 1, rw), np.array(want))


def test_invalid_arguments(lib):
    from paper_2509_07974_gb300.ext4pcf import Ext4pcfError
    for order, mu in ((1, 0), (17, 0), (4, 8), (4, -2)):
        with pytest.raises(Ext4pcfError):
            lib.ext4pcf_nth_order_factors(order, mu)
    with pytest.raises(Ext4pcfError):
        lib.ext4pcf_contraction_tables(3)


def evaluate(order, tables, pos, shear, w, edges, nmax):
    """The multipoles the generated tables define: sign * sum_i t_i prod_l F_l, with G_m and
    W_m of every centre summed directly.  Layout of oracle.bruteforce_multipoles."""
    pos = np.asarray(pos, dtype=np.float64)
    gc = shear[:, 0] + 1j * shear[:, 1]
    nb = len(edges) - 1
    k = order - 1
    mmax = (order - 2) * nmax + 4
    ms = np.arange(-mmax, mmax + 1)
    nvec = list(itertools.product(range(-nmax, nmax + 1), repeat=order - 2))
    out = np.zeros((len(tables), len(nvec)) + (nb,) * k, dtype=np.complex128)
    e2 = np.asarray(edges) ** 2
    for i in range(len(pos)):
        d = pos - pos[i]
        r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
        phi = np.arctan2(d[:, 1], d[:, 0])
        memb = np.stack([(r2 >= e2[b]) & (r2 < e2[b + 1]) for b in range(nb)], 0)       # [nb][n]
        ph = np.exp(1j * np.outer(ms, phi))                                               # [m][n]
        G = (ph * (w * gc)) @ memb.T.astype(float)                                        # [m][nb]
        W = (ph * w) @ memb.T.astype(float)
        for mu, t in enumerate(tables):
            sign, centre = t[0], t[1]
            ti = w[i] * (gc[i] if centre == 0 else np.conj(gc[i]) if centre == 1 else 1.0)
            rows = t[2:].reshape(k, order + 1)
            for q, n in enumerate(nvec):
                acc = np.array(sign * ti, dtype=np.complex128)
                for l in range(k):
                    arr, cj, a, b = rows[l, 0], rows[l, 1], rows[l, 2:order], rows[l, order]
                    m = int(np.dot(a, n)) + int(b)
                    f = (W if arr else G)[m + mmax]
                    acc = np.multiply.outer(acc, np.conj(f) if cj else f)
                out[mu, q] += acc
    return out.reshape((len(tables),) + (2 * nmax + 1,) * (order - 2) + (nb,) * k)


@pytest.mark.parametrize("order,n,side,edges,nmax", [
    (2, 80, 8.0, [0.5, 1.5, 3.0], 0),
    (3, 50, 6.0, [0.7, 1.5, 2.8], 3),
    (4, 35, 6.0, [0.8, 1.6, 3.0], 2),
    (5, 22, 5.0, [0.9, 1.8, 3.0], 1),
])
def test_generated_tables_give_the_brute_force_multipoles(lib, order, n, side, edges, nmax):
    rng = np.random.default_rng(100 + order)
    pos = rng.uniform(0, side, (n, 2))
    sh = rng.normal(0, 0.3, (n, 2))
    w = rng.uniform(0.5, 1.5, n)
    n_mu = 2 ** (order - 1)
    tables = [lib.ext4pcf_nth_order_factors(order, mu) for mu in list(range(n_mu)) + [-1]]
    got = evaluate(order, tables, pos, sh, w, np.array(edges), nmax)
    ref = oracle.bruteforce_multipoles(order, pos, sh, w, np.array(edges), nmax)
    assert got.shape == ref.shape and np.abs(ref).max() > 0
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_tensor_core_swap_map_is_the_papers_symmetry_table():
    """The Theta2 <-> Theta3 map that the reduced tensor-core contraction derives from its own
    factor table equals the column (Theta1, Theta3, Theta2) of Table tab:4PCFSymm in the oracle:
    Upsilon_mu[n2, n3](b1, b2, b3) = Upsilon_mu'[n3 + o, n2 - o](b1, b3, b2)."""
    from oracle import symmetry
    from paper_2509_07974_gb300 import ext4pcf
    m = ext4pcf.ext4pcf_contraction_tables(2)
    col = symmetry.BIN_PERM.index((0, 2, 1))
    for mu in range(9):
        assert m[mu, 0] == symmetry.MU_MAP[mu][col]
        for n2, n3 in ((0, 0), (3, -2), (-4, 1)):
            assert symmetry.n_map(mu, col, n2, n3) == (n3 + m[mu, 1], n2 - m[mu, 1])
