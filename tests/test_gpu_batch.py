"""Batched measurement (ext4pcf_measure_batch): many catalogues in one call, waves packing the
centres of several catalogues, catalogues accumulating into shared output slots (the patches
of one survey), and a batched call captured in a CUDA graph."""
import numpy as np
import pytest

import oracle
import synth
from metric import empty_slabs, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_07974_gb300 import build
    build.build()
    return torch


def _suite():
    """Five uneven uniform catalogues (one of them tiny) with their own extents."""
    cats, offs = [], [0]
    for k, (n, side) in enumerate(((300, 20.0), (1200, 35.0), (60, 10.0), (800, 30.0), (2500, 45.0))):
        p, s, w = synth.uniform_catalog(n, side, seed=70 + k, weights="uniform")
        cats.append((p + 1000.0 * k, s, w))  # far apart: no catalogue sees another
        offs.append(offs[-1] + n)
    pos = np.concatenate([c[0] for c in cats])
    sh = np.concatenate([c[1] for c in cats])
    w = np.concatenate([c[2] for c in cats])
    return pos, sh, w, np.array(offs, dtype=np.int64), synth.log_edges(0.8, 8.0, 6), 4


def _ctx(torch, prec, wave=0):
    from paper_2509_07974_gb300 import ext4pcf
    cfg = ext4pcf.Config(device=0, stream=torch.cuda.current_stream().cuda_stream, precision=ext4pcf.PRECISION[prec],
                         autotune=0, workspace_bytes=0, timeout_cycles=0, deterministic=1, wave_centres=wave)
    return ext4pcf.ext4pcf_create(cfg)


def _run(torch, prec, pos, sh, w, offs, edges, nmax, slots=None, n_out=None, mask=None, wave=0):
    from paper_2509_07974_gb300 import ext4pcf
    dev = torch.device("cuda:0")
    n_cat = len(offs) - 1
    n_out = n_out or n_cat
    nb = len(edges) - 1
    ups = torch.zeros((n_out,) + tuple(ext4pcf.Estimator.ups_shape(nb, nmax)[1:]), dtype=torch.float64, device=dev)
    tp, ts, tw = (torch.tensor(a, device=dev) for a in (pos, sh, w))
    ctx = _ctx(torch, prec, wave)
    sl = None if slots is None else np.ascontiguousarray(slots, dtype=np.int32)
    ext4pcf.ext4pcf_measure_batch(ctx, tp, ts, tw, len(w), np.ascontiguousarray(edges), nb, nmax,
                                  np.ascontiguousarray(offs), n_cat, sl, n_out if slots is not None else 0,
                                  mask, ups, None)
    torch.cuda.synchronize()
    ext4pcf.ext4pcf_destroy(ctx)
    u = ups.cpu().numpy()
    return u[..., 0] + 1j * u[..., 1]


def test_fp64_batch_equals_one_catalogue_calls_bitwise(torch_cuda):
    pos, sh, w, offs, edges, nmax = _suite()
    both = _run(torch_cuda, "fp64", pos, sh, w, offs, edges, nmax)
    for k in range(len(offs) - 1):
        a, b = offs[k], offs[k + 1]
        one = _run(torch_cuda, "fp64", pos[a:b], sh[a:b], w[a:b], np.array([0, b - a]), edges, nmax)
        assert np.array_equal(both[k], one[0]), k


def test_f16x3_packed_waves_match_the_oracle_per_catalogue(torch_cuda):
    """Waves of 512 records pack the runs of several catalogues (and split the larger ones);
    a host mask makes the centre counts known on the host.  Every catalogue's slot matches the
    FP64 oracle on its own centres."""
    pos, sh, w, offs, edges, nmax = _suite()
    rng = np.random.default_rng(8)
    mask = (rng.uniform(size=len(w)) < 0.6).astype(np.uint8)
    got = _run(torch_cuda, "f16x3", pos, sh, w, offs, edges, nmax, mask=mask, wave=512)
    for k in range(len(offs) - 1):
        a, b = offs[k], offs[k + 1]
        ref = oracle.measure(pos[a:b], sh[a:b], w[a:b], edges, nmax, centre_mask=mask[a:b])
        err = rel_err(got[k], ref, empty=empty_slabs(pos[a:b], edges))
        assert err.max() < 1e-4, (k, err.max())


def test_patched_survey_equals_the_unpatched_catalogue(torch_cuda):
    """3 x 3 patches with margins wider than the largest separation, cores as centres, all in
    slot 0: the same sums as the whole catalogue (FP64 to rounding; split-FP16 to its bound)."""
    side = 60.0
    pos, sh, w = synth.lognormal_catalog(6000, side, seed=12, grid=256)
    edges, nmax = synth.log_edges(0.6, 6.0, 5), 3
    idx, offs, mask = synth.flat_patches(pos, side, 3, 6.5)
    whole64 = _run(torch_cuda, "fp64", pos, sh, w, np.array([0, len(w)]), edges, nmax)[0]
    patch64 = _run(torch_cuda, "fp64", pos[idx], sh[idx], w[idx], offs, edges, nmax,
                   slots=np.zeros(9, np.int32), n_out=1, mask=mask)[0]
    scale = np.abs(whole64).reshape(9, -1).max(axis=1).reshape(9, 1, 1, 1, 1, 1)
    assert (np.abs(patch64 - whole64) <= 1e-10 * scale).all()
    patch16 = _run(torch_cuda, "f16x3", pos[idx], sh[idx], w[idx], offs, edges, nmax,
                   slots=np.zeros(9, np.int32), n_out=1, mask=mask, wave=1024)[0]
    assert rel_err(patch16, whole64, empty=empty_slabs(pos, edges)).max() < 1e-4


def test_batched_call_captured_in_a_cuda_graph(torch_cuda):
    """The whole batched call (grids, packed waves, expansion, corrections) captured once and
    replayed gives the direct call's result bit for bit; the mask is a pinned host buffer, so
    its counts are known on the host and its copy is part of the graph."""
    torch = torch_cuda
    from paper_2509_07974_gb300 import ext4pcf
    pos, sh, w, offs, edges, nmax = _suite()
    dev = torch.device("cuda:0")
    nb, n_cat = len(edges) - 1, len(offs) - 1
    mask = torch.tensor((np.random.default_rng(3).uniform(size=len(w)) < 0.5).astype(np.uint8)).pin_memory()
    tp, ts, tw = (torch.tensor(a, device=dev) for a in (pos, sh, w))
    ups = torch.zeros((n_cat,) + tuple(ext4pcf.Estimator.ups_shape(nb, nmax)[1:]), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream()
    cfg = ext4pcf.Config(device=0, stream=stream.cuda_stream, precision=ext4pcf.PRECISION["f16x3"], autotune=0,
                         workspace_bytes=0, timeout_cycles=0, deterministic=1, wave_centres=1024)
    ctx = ext4pcf.ext4pcf_create(cfg)
    args = (ctx, tp, ts, tw, len(w), np.ascontiguousarray(edges), nb, nmax, np.ascontiguousarray(offs), n_cat,
            None, 0, mask, ups, None)
    with torch.cuda.stream(stream):
        ext4pcf.ext4pcf_measure_batch(*args)  # sizes the scratch buffers
    ext4pcf.ext4pcf_synchronize(ctx)
    direct = ups.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
        ups.zero_()
        ext4pcf.ext4pcf_measure_batch(*args)
    ups.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ups, direct)
    assert ext4pcf.ext4pcf_synchronize(ctx) == ext4pcf.EXT4PCF_OK
    ext4pcf.ext4pcf_destroy(ctx)


def test_out_slot_out_of_range_is_an_argument_error(torch_cuda):
    from paper_2509_07974_gb300 import ext4pcf
    pos, sh, w, offs, edges, nmax = _suite()
    with pytest.raises(ext4pcf.Ext4pcfError) as e:
        _run(torch_cuda, "fp64", pos, sh, w, offs, edges, nmax, slots=np.array([0, 1, 2, 3, 7]), n_out=4)
    assert e.value.code == ext4pcf.EXT4PCF_E_INVALID_ARG


def test_batched_grid_build_equals_per_catalogue_build(torch_cuda):
    """Up to 128 catalogues a call sorts them all at once; beyond that each is sorted on its
    own.  130 small catalogues in one call (built one by one) and the same catalogues in two
    calls of 65 (built at once) give the same FP64 sums bit for bit."""
    rng = np.random.default_rng(21)
    sizes = rng.integers(0, 60, 130)
    sizes[7] = 0  # an empty catalogue
    cats = [synth.uniform_catalog(int(m), 12.0, seed=300 + k, weights="uniform") if m > 0
            else (np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(0)) for k, m in enumerate(sizes)]
    pos = np.concatenate([c[0] + 100.0 * k for k, c in enumerate(cats)])
    sh = np.concatenate([c[1] for c in cats])
    w = np.concatenate([c[2] for c in cats])
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    edges, nmax = synth.log_edges(0.8, 6.0, 4), 3
    one = _run(torch_cuda, "fp64", pos, sh, w, offs, edges, nmax)
    a, b = offs[65], offs[130]
    first = _run(torch_cuda, "fp64", pos[:a], sh[:a], w[:a], offs[:66], edges, nmax)
    second = _run(torch_cuda, "fp64", pos[a:b], sh[a:b], w[a:b], offs[65:] - a, edges, nmax)
    assert np.array_equal(one[:65], first)
    assert np.array_equal(one[65:], second)
    assert np.abs(one).max() > 0
