"""Parity of the direct <M_ap^2>, <M_ap^4> estimator (Sect. 5.2, Eq. MapDirectEstimator) of
the CUDA library with the FP64 oracle, through the C ABI.

Per aperture the galaxy counts inside the 4 theta cut must agree exactly (the kernel decides
near-cut galaxies in FP64 like the oracle).  The e_k come from FP32 per-galaxy terms and FP64
power sums; their error is bounded relative to |e_k| + p_2^{k/2} (p_2 = sum a_i^2, the
scale of the Newton-identity terms): measured below 1e-6 in an FP32 emulation, held to 1e-5.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_07974_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def est(torch_cuda):
    from paper_2509_07974_gb300 import ext4pcf
    e = ext4pcf.Estimator(0, "3xtf32")
    yield e
    e.close()


def scaled_err(g, o):
    """|g - o| / (|o| + p2^(k/2)) for the six e_k entries of aperture records [n][8]."""
    g, o = np.atleast_2d(g), np.atleast_2d(o)
    p2a = np.maximum(o[:, 0] ** 2 - 2 * o[:, 1], 0)
    p2w = np.maximum(o[:, 3] ** 2 - 2 * o[:, 4], 0)
    sc = np.stack([np.sqrt(p2a), p2a, p2a ** 2, np.sqrt(p2w), p2w, p2w ** 2], 1)
    den = np.abs(o[:, :6]) + sc
    return np.abs(g[:, :6] - o[:, :6]) / np.where(den > 0, den, 1.0)


def run(torch, est, pos, sh, w, thetas, centres, host=False):
    dev = torch.device("cuda:0")
    if host:
        from paper_2509_07974_gb300 import ext4pcf
        th = np.ascontiguousarray(thetas, dtype=np.float64)
        offs = np.zeros(len(th) + 1, dtype=np.int64)
        offs[1:] = np.cumsum([len(c) for c in centres])
        cen = np.ascontiguousarray(np.vstack(centres), dtype=np.float64)
        rec = np.zeros((int(offs[-1]), 8))
        mom = np.zeros((len(th), 8))
        ext4pcf.ext4pcf_map_direct(est.ctx, np.ascontiguousarray(pos), np.ascontiguousarray(sh),
                                   np.ascontiguousarray(w), len(w), th, len(th), cen, offs, rec, mom)
        return mom, rec
    tp, ts, tw = (torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev) for a in (pos, sh, w))
    mom, rec = est.map_direct(tp, ts, tw, thetas, centres, want_records=True)
    torch.cuda.synchronize()
    return mom.cpu().numpy(), rec.cpu().numpy()


def check(oracle, pos, sh, w, thetas, centres, mom, rec):
    ref_rec, ref_mom = oracle.map_direct(pos, sh, w, thetas, centres)
    np.testing.assert_array_equal(rec[:, 6], ref_rec[:, 6])
    assert scaled_err(rec, ref_rec).max() < TOL
    assert np.all(rec[:, 7] == 0)
    # per-radius sums: errors of the apertures add up
    off = 0
    for t, c in enumerate(centres):
        r = ref_rec[off:off + len(c)]
        p2a = np.maximum(r[:, 0] ** 2 - 2 * r[:, 1], 0)
        p2w = np.maximum(r[:, 3] ** 2 - 2 * r[:, 4], 0)
        assert mom[t, 4] == ref_mom[t, 4] == len(c)
        for i, (col, sc) in enumerate([(2, p2a ** 2), (5, p2w ** 2), (1, p2a), (4, p2w)]):
            bound = TOL * (np.abs(r[:, col]).sum() + sc.sum()) + 1e-300
            assert abs(mom[t, i] - ref_mom[t, i]) <= bound, (t, i, mom[t, i], ref_mom[t, i])
        area = math.pi * (4 * thetas[t]) ** 2
        if mom[t, 1] > 0:
            assert mom[t, 5] == pytest.approx(area ** 4 * mom[t, 0] / mom[t, 1], rel=1e-12)
            assert mom[t, 6] == pytest.approx(area ** 2 * mom[t, 2] / mom[t, 3], rel=1e-12)
            assert mom[t, 7] == pytest.approx(mom[t, 5] - 3 * mom[t, 6] ** 2, rel=1e-9, abs=1e-12 * abs(mom[t, 5]))
        off += len(c)
    return ref_rec, ref_mom


def test_small_catalogue_several_radii(torch_cuda, est, oracle):
    """Random weights and shears, apertures on a lattice inside the field, near its edges,
    partly and wholly outside it; radii that span many cells and a ragged split of rows."""
    import synth
    from paper_2509_07974_gb300 import ext4pcf
    pos, sh, w = synth.grf_catalog(40000, 60.0, 21, grid=512)
    thetas = [0.6, 1.7, 3.9]
    rng = np.random.default_rng(4)
    centres = []
    for th in thetas:
        lat = ext4pcf.aperture_lattice((0, 0, 60, 60), th, 1.3 * th)
        extra = np.vstack([rng.uniform(-3 * th, 60 + 3 * th, (25, 2)), [[0.0, 0.0], [60.0, 60.0], [-100, 30]]])
        centres.append(np.vstack([lat, extra]))
    mom, rec = run(torch_cuda, est, pos, sh, w, thetas, centres)
    check(oracle, pos, sh, w, thetas, centres, mom, rec)


def test_host_buffers_match_device_buffers(torch_cuda, est, oracle):
    import synth
    pos, sh, w = synth.uniform_catalog(3000, 20.0, 9)
    w = np.random.default_rng(1).uniform(0.5, 1.5, len(w))
    thetas = [0.8, 2.0]
    centres = [np.random.default_rng(2).uniform(0, 20, (30, 2)), np.array([[10.0, 10.0], [3.0, 17.0]])]
    m_d, r_d = run(torch_cuda, est, pos, sh, w, thetas, centres)
    m_h, r_h = run(torch_cuda, est, pos, sh, w, thetas, centres, host=True)
    np.testing.assert_array_equal(r_h, r_d)
    np.testing.assert_array_equal(m_h, m_d)
    check(oracle, pos, sh, w, thetas, centres, m_d, r_d)


def test_tangential_pattern_closed_form(torch_cuda, est):
    """Constant tangential shear g about the aperture centre: A e1(a)/e1(w) is the integral of
    Q over the 4 theta disc times g, g (1 - 9 e^{-8}) up to the lattice's quadrature error;
    the cross pattern gives zero."""
    theta, h, g = 1.3, 1.3 / 16, 0.05
    m = int(round(4 * theta / h))
    u = (np.arange(-m, m) + 0.5) * h
    x, y = np.meshgrid(u, u)
    pos = np.stack([x.ravel(), y.ravel()], 1) + 7.0
    phi = np.arctan2(pos[:, 1] - 7.0, pos[:, 0] - 7.0)
    w = np.ones(len(pos))
    for cross in (False, True):
        gc = -g * np.exp(2j * phi) * (1j if cross else 1.0)
        sh = np.stack([gc.real, gc.imag], 1)
        mom, rec = run(torch_cuda, est, pos, sh, w, [theta], [np.array([[7.0, 7.0]])])
        area = math.pi * (4 * theta) ** 2
        m_ap = area * rec[0, 0] / rec[0, 3]
        if cross:
            assert abs(m_ap) < 1e-6 * g
        else:
            # h^2 sum a_i = g (1 - 9 e^-8) within the midpoint rule's error
            assert h * h * rec[0, 0] == pytest.approx(g * (1 - 9 * math.exp(-8)), rel=3e-4)
            assert mom[0, 5] == pytest.approx(m_ap ** 4, rel=3e-3)


def test_degenerate_cases(torch_cuda, est):
    """Empty catalogue, empty radius, apertures with fewer than four (two) galaxies, and the
    accumulation of the per-radius sums over calls."""
    torch = torch_cuda
    dev = torch.device("cuda:0")
    pos = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.2], [5.0, 5.0], [5.3, 5.1]])
    sh = np.random.default_rng(0).normal(0, 0.3, (5, 2))
    w = np.array([1.0, 2.0, 0.5, 1.5, 1.0])
    cen = [np.array([[0.2, 0.2], [5.1, 5.0], [50.0, 50.0]]), np.zeros((0, 2))]
    mom, rec = run(torch, est, pos, sh, w, [0.5, 1.0], cen)
    assert rec[0, 6] == 3 and rec[1, 6] == 2 and rec[2, 6] == 0
    assert rec[0, 2] == 0 and rec[0, 5] == 0 and rec[1, 2] == 0 and rec[1, 5] == 0
    assert rec[1, 4] == pytest.approx(1.5, rel=1e-6)  # e2(w) of the pair (1.5, 1.0)
    assert not rec[2].any()
    assert mom[0, 4] == 3 and mom[1, 4] == 0 and mom[0, 5] == 0 and not mom[1].any()
    # empty catalogue
    from paper_2509_07974_gb300 import ext4pcf
    z = torch.zeros((0, 2), dtype=torch.float64, device=dev)
    m0, r0 = est.map_direct(z, z, torch.zeros(0, dtype=torch.float64, device=dev), [1.0], [np.array([[0.0, 0.0]])],
                            want_records=True)
    assert not r0.cpu().numpy().any() and m0.cpu().numpy()[0, 4] == 1
    # accumulation: a second call on the same moments doubles the sums, keeps the ratios
    pos, sh, w = (np.random.default_rng(5).uniform(0, 10, (2000, 2)), np.random.default_rng(6).normal(0, .3, (2000, 2)),
                  np.ones(2000))
    tp, ts, tw = (torch.tensor(a, device=dev) for a in (pos, sh, w))
    m1, _ = est.map_direct(tp, ts, tw, [1.0], [np.array([[5.0, 5.0], [4.0, 6.0]])])
    first = m1.cpu().numpy().copy()
    est.map_direct(tp, ts, tw, [1.0], [np.array([[5.0, 5.0], [4.0, 6.0]])], moments=m1)
    second = m1.cpu().numpy()
    np.testing.assert_allclose(second[0, :5], 2 * first[0, :5], rtol=1e-15)
    np.testing.assert_allclose(second[0, 5:], first[0, 5:], rtol=1e-12)


def test_invalid_arguments(torch_cuda, est):
    from paper_2509_07974_gb300 import ext4pcf
    pos = np.zeros((1, 2))
    mom = np.zeros((1, 8))
    cen = np.zeros((1, 2))
    for th, offs in (([0.0], [0, 1]), ([float("nan")], [0, 1]), ([1.0], [1, 1]), ([1.0, 2.0], [0, 1, 0])):
        t = np.ascontiguousarray(th, dtype=np.float64)
        m = np.zeros((len(th), 8))
        with pytest.raises(ext4pcf.Ext4pcfError) as ei:
            ext4pcf.ext4pcf_map_direct(est.ctx, pos, pos, np.ones(1), 1, t, len(t), cen,
                                       np.ascontiguousarray(offs, dtype=np.int64), None, m)
        assert ei.value.code == ext4pcf.EXT4PCF_E_INVALID_ARG
    assert not mom.any()


def test_full_size_sampled_apertures(torch_cuda, est, oracle):
    """The 2e6-galaxy GRF workload with all 24 radii and their full aperture lattices, in one
    call (the configuration the benchmark times); sampled apertures of every fourth radius
    against the oracle, and the per-radius aperture counts."""
    import synth
    from paper_2509_07974_gb300 import ext4pcf
    c = synth.GRF2E6
    pos, sh, w = synth.grf_catalog(c["n"], c["side"], c["seed"], grid=c["grid"])
    thetas = synth.direct_radii()
    centres = [ext4pcf.aperture_lattice((0, 0, c["side"], c["side"]), t, synth.DIRECT["spacing"] * t) for t in thetas]
    mom, rec = run(torch_cuda, est, pos, sh, w, thetas, centres)
    off = np.concatenate([[0], np.cumsum([len(x) for x in centres])])
    rng = np.random.default_rng(12)
    for t in range(0, len(thetas), 4):
        n_t = len(centres[t])
        assert n_t > 0 and mom[t, 4] == n_t
        pick = rng.choice(n_t, size=min(4, n_t), replace=False)
        ref = np.array([oracle.aperture_record(pos, sh, w, centres[t][i], thetas[t]) for i in pick])
        got = rec[off[t] + pick]
        np.testing.assert_array_equal(got[:, 6], ref[:, 6])
        assert scaled_err(got, ref).max() < TOL
    # every aperture lies 4 theta inside the field: the counts follow the mean density
    dens = c["n"] / c["side"] ** 2
    for t in (0, len(thetas) - 1):
        r = rec[off[t]:off[t + 1], 6]
        assert abs(r.mean() / (dens * math.pi * (4 * thetas[t]) ** 2) - 1) < 0.02
