"""The C ABI's synchronisation contract (device-only ext4pcf_measure returns after enqueueing;
failures recorded on the device are reported by the next synchronising call) and a measure
call captured into a CUDA graph."""
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


@pytest.fixture(scope="module")
def catalogue():
    """A 2e5-galaxy GRF patch at the density of the 2e6 workload (seconds of GPU work)."""
    import synth
    side = 600.0 * np.sqrt(0.1)
    pos, sh, w = synth.grf_catalog(200_000, side, 17, grid=1024)
    return pos, sh, w, synth.log_edges(0.5, 40.0, 10), 20


def _measure(torch, est, tp, ts, tw, edges, nmax, ups, mask=None):
    from paper_2509_07974_gb300 import ext4pcf
    nb = len(edges) - 1
    ext4pcf.ext4pcf_measure(est.ctx, tp, ts, tw, tp.shape[0], np.ascontiguousarray(edges), nb, nmax, None, 1,
                            mask, ups, None)


def test_device_only_measure_returns_before_the_gpu_finishes(torch_cuda, catalogue):
    torch = torch_cuda
    from paper_2509_07974_gb300 import ext4pcf
    pos, sh, w, edges, nmax = catalogue
    dev = torch.device("cuda:0")
    tp, ts, tw = (torch.tensor(a, device=dev) for a in (pos, sh, w))
    stream = torch.cuda.Stream()
    est = ext4pcf.Estimator(0, "3xtf32", stream=stream)
    nb = len(edges) - 1
    ups = torch.zeros(ext4pcf.Estimator.ups_shape(nb, nmax), dtype=torch.float64, device=dev)
    _measure(torch, est, tp, ts, tw, edges, nmax, ups)  # sizes the scratch buffers
    ext4pcf.ext4pcf_synchronize(est.ctx)
    first = ups.clone()
    ups.zero_()
    torch.cuda.synchronize()
    _measure(torch, est, tp, ts, tw, edges, nmax, ups)
    done = torch.cuda.Event()
    done.record(stream)
    pending = not done.query()  # checked right after the call returned
    ext4pcf.ext4pcf_synchronize(est.ctx)
    assert done.query()
    assert pending, "ext4pcf_measure waited for the GPU"
    assert torch.equal(ups, first)
    est.close()


def test_measure_captured_in_a_cuda_graph(torch_cuda, oracle):
    """A whole measure call (grid, gather, contraction, corrections, expansion) captured once
    and replayed: the replay gives the result of a direct call, bit for bit."""
    torch = torch_cuda
    import synth
    from paper_2509_07974_gb300 import ext4pcf
    pos, sh, w, edges, nmax = synth.small_workload()
    dev = torch.device("cuda:0")
    tp, ts, tw = (torch.tensor(a, device=dev) for a in (pos, sh, w))
    stream = torch.cuda.Stream()
    est = ext4pcf.Estimator(0, "3xtf32", stream=stream)
    nb = len(edges) - 1
    ups = torch.zeros(ext4pcf.Estimator.ups_shape(nb, nmax), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        _measure(torch, est, tp, ts, tw, edges, nmax, ups)  # sizes buffers, uploads tables
    ext4pcf.ext4pcf_synchronize(est.ctx)
    direct = ups.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
        ups.zero_()
        _measure(torch, est, tp, ts, tw, edges, nmax, ups)
    ups.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ups, direct)
    ref = oracle.measure(pos, sh, w, edges, nmax)
    got = torch.view_as_complex(ups[0]).cpu().numpy()
    assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()
    est.close()


def test_nonfinite_positions_are_reported_by_synchronize(torch_cuda):
    torch = torch_cuda
    from paper_2509_07974_gb300 import ext4pcf
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, 10, (100, 2))
    pos[17, 1] = np.nan
    dev = torch.device("cuda:0")
    tp = torch.tensor(pos, device=dev)
    ts = torch.tensor(rng.normal(0, 0.3, (100, 2)), device=dev)
    tw = torch.ones(100, dtype=torch.float64, device=dev)
    edges = np.array([0.5, 1.0, 2.0])
    est = ext4pcf.Estimator(0, "fp64")
    ups = torch.zeros(ext4pcf.Estimator.ups_shape(2, 2), dtype=torch.float64, device=dev)
    _measure(torch, est, tp, ts, tw, edges, 2, ups)  # enqueued; nothing read back
    with pytest.raises(ext4pcf.Ext4pcfError) as e:
        ext4pcf.ext4pcf_synchronize(est.ctx)
    assert e.value.code == ext4pcf.EXT4PCF_E_INVALID_ARG
    assert "non-finite" in ext4pcf.ext4pcf_last_error(est.ctx)
    # the status word was read and cleared; a finite catalogue measures cleanly
    pos[17, 1] = 3.0
    tp.copy_(torch.tensor(pos))
    _measure(torch, est, tp, ts, tw, edges, 2, ups)
    assert ext4pcf.ext4pcf_synchronize(est.ctx) == ext4pcf.EXT4PCF_OK
    est.close()


def _run(torch, est, tp, ts, tw, edges, nmax):
    from paper_2509_07974_gb300 import ext4pcf
    nb = len(edges) - 1
    ups = torch.zeros(ext4pcf.Estimator.ups_shape(nb, nmax), dtype=torch.float64, device=tp.device)
    st = ext4pcf.Stats()
    ext4pcf.ext4pcf_measure(est.ctx, tp, ts, tw, tp.shape[0], np.ascontiguousarray(edges), nb, nmax, None, 1, None,
                            ups, None, st)
    torch.cuda.synchronize()
    return torch.view_as_complex(ups[0]).cpu().numpy(), st.as_dict()


def test_autotuner_picks_a_wave_size_and_keeps_it(torch_cuda, catalogue):
    """autotune = 1: the first call times its first waves at the candidate sizes and keeps the
    fastest; the result is that of a fixed wave size to the form's rounding, and later calls
    reuse the choice (and repeat bit for bit)."""
    torch = torch_cuda
    from metric import rel_err
    from paper_2509_07974_gb300 import ext4pcf
    pos, sh, w, edges, nmax = catalogue
    nmax = 6  # the wave size, not the multipole count, is what is tuned
    dev = torch.device("cuda:0")
    tp, ts, tw = (torch.tensor(a, device=dev) for a in (pos, sh, w))
    fixed = ext4pcf.Estimator(0, "3xtf32")
    ref, _ = _run(torch, fixed, tp, ts, tw, edges, nmax)
    fixed.close()
    est = ext4pcf.Estimator(0, "3xtf32", autotune=True)
    a, sa = _run(torch, est, tp, ts, tw, edges, nmax)
    b, sb = _run(torch, est, tp, ts, tw, edges, nmax)
    c, _ = _run(torch, est, tp, ts, tw, edges, nmax)
    est.close()
    assert sa["wave_centres"] in (2048, 4096, 8192, 16384) and sb["wave_centres"] == sa["wave_centres"]
    assert rel_err(a, ref).max() < 1e-4 and rel_err(b, ref).max() < 1e-4
    assert np.array_equal(b, c)


def test_workspace_cap_shrinks_the_wave(torch_cuda):
    import synth
    torch = torch_cuda
    from metric import rel_err
    from paper_2509_07974_gb300 import ext4pcf
    pos, sh, w, edges, nmax = synth.small_workload()
    dev = torch.device("cuda:0")
    tp, ts, tw = (torch.tensor(a, device=dev) for a in (pos, sh, w))
    ref, s0 = _run(torch, ext4pcf.Estimator(0, "3xtf32"), tp, ts, tw, edges, nmax)
    est = ext4pcf.Estimator(0, "3xtf32", workspace_bytes=16 << 20)
    got, s1 = _run(torch, est, tp, ts, tw, edges, nmax)
    est.close()
    assert s0["wave_centres"] == 2000 and s1["wave_centres"] < 2000 and s1["waves"] > 1
    assert rel_err(got, ref).max() < 1e-4
    tiny = ext4pcf.Estimator(0, "3xtf32", workspace_bytes=4096)
    with pytest.raises(ext4pcf.Ext4pcfError) as e:
        _run(torch, tiny, tp, ts, tw, edges, nmax)
    assert e.value.code == ext4pcf.EXT4PCF_E_OOM
    tiny.close()
