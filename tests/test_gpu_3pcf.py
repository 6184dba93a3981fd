"""The shear 3PCF multipoles of ext4pcf_measure3 (order 3 of App. F, contracted with the
generated tables) against the oracle's brute force over triplets of distinct galaxies."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_07974_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("nmax,wave,edges", [(4, 0, (0.6, 1.2, 2.2, 3.5)), (2, 37, (0.6, 1.2, 2.2, 3.5)),
                                             (8, 0, (0.5, 0.9, 1.5, 2.2, 3.0, 4.0))])
def test_third_order_matches_distinct_brute_force(torch_cuda, oracle, nmax, wave, edges):
    torch = torch_cuda
    from paper_2509_07974_gb300 import ext4pcf
    rng = np.random.default_rng(31 + nmax)
    n = 150
    pos = rng.uniform(0, 8.0, (n, 2))
    pos[1] = pos[0]  # two galaxies at one position: distinct galaxies, separation in no bin
    sh = rng.normal(0, 0.3, (n, 2))
    w = rng.uniform(0.5, 1.5, n)
    edges = np.array(edges)
    nb = len(edges) - 1
    dev = torch.device("cuda:0")
    tp, ts, tw = (torch.tensor(a, dtype=torch.float64, device=dev) for a in (pos, sh, w))
    est = ext4pcf.Estimator(0, "fp64", wave_centres=wave)
    ups = torch.zeros((5, 2 * nmax + 1, nb, nb, 2), dtype=torch.float64, device=dev)
    ext4pcf.ext4pcf_measure3(est.ctx, tp, ts, tw, n, edges, nb, nmax, ups)
    # accumulation: a second call adds the same values
    ext4pcf.ext4pcf_measure3(est.ctx, tp, ts, tw, n, edges, nb, nmax, ups)
    torch.cuda.synchronize()
    got = torch.view_as_complex(ups).cpu().numpy() / 2
    est.close()
    ref = oracle.bruteforce_multipoles(3, pos, sh, w, edges, nmax, distinct=True)
    assert got.shape == ref.shape and np.abs(ref).max() > 0
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_third_order_fp32_gather_matches_distinct_brute_force(torch_cuda, oracle):
    """Every precision but FP64 gathers in FP32 (products and sums of the contraction in FP64):
    the same brute force within the FP32 records' rounding, on 600 galaxies in several waves."""
    torch = torch_cuda
    from paper_2509_07974_gb300 import ext4pcf
    rng = np.random.default_rng(77)
    n, nmax = 600, 6
    pos = rng.uniform(0, 14.0, (n, 2))
    sh = rng.normal(0, 0.3, (n, 2))
    w = rng.uniform(0.5, 1.5, n)
    edges = np.array((0.5, 1.0, 1.8, 2.6, 3.5))
    nb = len(edges) - 1
    dev = torch.device("cuda:0")
    tp, ts, tw = (torch.tensor(a, dtype=torch.float64, device=dev) for a in (pos, sh, w))
    est = ext4pcf.Estimator(0, "f16x3", wave_centres=256)
    ups = torch.zeros((5, 2 * nmax + 1, nb, nb, 2), dtype=torch.float64, device=dev)
    ext4pcf.ext4pcf_measure3(est.ctx, tp, ts, tw, n, edges, nb, nmax, ups)
    torch.cuda.synchronize()
    got = torch.view_as_complex(ups).cpu().numpy()
    est.close()
    ref = oracle.bruteforce_multipoles(3, pos, sh, w, edges, nmax, distinct=True)
    scale = np.abs(ref).reshape(5, -1).max(axis=1).reshape(5, 1, 1, 1)
    assert (np.abs(got - ref) <= 2e-5 * scale).all(), (np.abs(got - ref) / scale).max()


def test_every_accepted_nmax_has_order3_tables(torch_cuda):
    """The generated order-3 tables stay inside the gathered multipole range for every n_max
    the entry point accepts (0..40): an empty catalogue returns EXT4PCF_OK, not
    EXT4PCF_E_UNSUPPORTED, and n_max = 41 is refused as an invalid argument."""
    torch = torch_cuda
    from paper_2509_07974_gb300 import ext4pcf
    dev = torch.device("cuda:0")
    edges = np.array([0.5, 1.0, 2.0])
    est = ext4pcf.Estimator(0, "fp64")
    for nmax in range(0, 41):
        ups = torch.zeros((5, 2 * nmax + 1, 2, 2, 2), dtype=torch.float64, device=dev)
        assert ext4pcf.ext4pcf_measure3(est.ctx, None, None, None, 0, edges, 2, nmax, ups) == ext4pcf.EXT4PCF_OK
    ups = torch.zeros((5, 83, 2, 2, 2), dtype=torch.float64, device=dev)
    with pytest.raises(ext4pcf.Ext4pcfError) as e:
        ext4pcf.ext4pcf_measure3(est.ctx, None, None, None, 0, edges, 2, 41, ups)
    assert e.value.code == ext4pcf.EXT4PCF_E_INVALID_ARG
    est.close()
