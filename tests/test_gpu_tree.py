"""Neighbour multipole records (ext4pcf_multipoles) against the tree oracle: exact records, and
the tree approximation of Sect. 3.2 / App. F.3 (reduced catalogues on cells of side
Delta_d = Delta_1 2^(d-1), each bin from the coarsest level with Theta_lo / Delta_d >= r_min)
against oracle/tree.py:neighbour_multipoles with the same setting."""
import numpy as np
import pytest

import synth
from oracle import tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_07974_gb300 import build
    build.build()
    return torch


def _records(torch, prec, pos, sh, w, edges, nmax, centres, delta1=0.0, levels=0, rmin=0.0):
    from paper_2509_07974_gb300 import ext4pcf
    cfg = ext4pcf.Config(device=0, stream=torch.cuda.current_stream().cuda_stream, precision=ext4pcf.PRECISION[prec],
                         autotune=0, workspace_bytes=0, timeout_cycles=0, deterministic=1, wave_centres=0,
                         tree_delta1=delta1, tree_levels=levels, tree_rmin=rmin)
    ctx = ext4pcf.ext4pcf_create(cfg)
    nb = len(edges) - 1
    lay = ext4pcf.record_layout(nb, nmax)
    out = np.zeros((len(centres), lay["rec"], 2))
    dev = torch.device("cuda:0")
    tp, ts, tw = (torch.tensor(a, device=dev) for a in (pos, sh, w))
    ext4pcf.ext4pcf_multipoles(ctx, tp, ts, tw, len(w), np.ascontiguousarray(edges), nb, nmax,
                               np.ascontiguousarray(centres, dtype=np.int64), len(centres), out)
    ext4pcf.ext4pcf_destroy(ctx)
    rec = out[..., 0] + 1j * out[..., 1]
    g0, gfirst, gcnt = lay["G"]
    w0, _, wcnt = lay["W"]
    G = rec[:, g0:g0 + gcnt * nb].reshape(len(centres), gcnt, nb)
    W = rec[:, w0:w0 + wcnt * nb].reshape(len(centres), wcnt, nb)
    return G, W, gfirst


def _check(G, W, gfirst, refG, refW, nmax, tol):
    """G over its index range, W for m >= 0, against the oracle's [centre][n][bin] arrays that
    run over n = gfirst .. 2N (W: the same range, m >= 0 taken)."""
    gcnt = G.shape[1]
    rg = refG[:, :gcnt]
    rw = refW[:, -gfirst:-gfirst + W.shape[1]]
    scale_g = np.abs(rg).max()
    scale_w = np.abs(rw).max()
    assert scale_g > 0 and scale_w > 0
    assert np.abs(G - rg).max() <= tol * scale_g, np.abs(G - rg).max() / scale_g
    assert np.abs(W - rw).max() <= tol * scale_w, np.abs(W - rw).max() / scale_w


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("f16x3", 2e-6)])
def test_exact_records_match_the_oracle(torch_cuda, prec, tol):
    pos, sh, w = synth.uniform_catalog(4000, 60.0, seed=21, weights="uniform")
    edges, nmax = synth.log_edges(0.5, 12.0, 6), 4
    centres = np.random.default_rng(2).choice(len(w), 40, replace=False)
    G, W, gfirst = _records(torch_cuda, prec, pos, sh, w, edges, nmax, centres)
    refG, refW = tree.neighbour_multipoles(pos[:], sh, w, edges, gfirst, 2 * nmax)
    _check(G, W, gfirst, refG[centres], refW[centres], nmax, tol)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("f16x3", 2e-6)])
def test_tree_records_match_the_tree_oracle(torch_cuda, prec, tol):
    """The paper's setting scaled to a small catalogue: three resolutions 0.5, 1, 2 (powers of
    two, so that both sides find the same cells) and r_min = 4, so that the outer bins take
    levels 1, 2 and 3 and the inner bins the galaxies."""
    pos, sh, w = synth.lognormal_catalog(20000, 80.0, seed=23, grid=256)
    edges, nmax = synth.log_edges(0.5, 16.0, 8), 3
    lv = tree.bin_levels(edges, 0.5, 3, 4.0)
    assert set(lv.tolist()) >= {0, 1, 2, 3}
    centres = np.random.default_rng(4).choice(len(w), 30, replace=False)
    G, W, gfirst = _records(torch_cuda, prec, pos, sh, w, edges, nmax, centres, 0.5, 3, 4.0)
    refG, refW = tree.neighbour_multipoles(pos, sh, w, edges, gfirst, 2 * nmax, delta1=0.5, n_levels=3, r_min=4.0)
    _check(G, W, gfirst, refG[centres], refW[centres], nmax, tol)
    # the approximation changed the outer bins (it is not the exact answer)
    eG, _, _ = _records(torch_cuda, prec, pos, sh, w, edges, nmax, centres)
    outer = lv > 0
    assert np.abs(G[..., outer] - eG[..., outer]).max() > 1e-6 * np.abs(eG[..., outer]).max()
    # the inner bins come from the galaxies in both runs (summed in other chunks: to rounding)
    assert np.abs(G[..., ~outer] - eG[..., ~outer]).max() <= tol * np.abs(eG[..., ~outer]).max()
