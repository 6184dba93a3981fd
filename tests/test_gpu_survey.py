"""The survey form at the survey's density and binning (lognormal shear, 12 log bins 0.5'-120',
n_max = 30), split into patches with 120' margins: sampled centres of the patched, batched,
split-FP16 measurement against the FP64 oracle on the whole catalogue."""
import numpy as np
import pytest

import oracle
import synth
from metric import rel_err

pytestmark = pytest.mark.gpu


def test_patched_survey_matches_the_oracle_on_sampled_centres():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_07974_gb300 import build, ext4pcf
    build.build()
    c = synth.SURVEY
    n = 1_500_000
    side = c["side"] * (n / c["n"]) ** 0.5  # the survey's density, ~7 per arcmin^2
    pos, sh, w = synth.lognormal_catalog(n, side, seed=51, grid=1024)
    edges, nmax = synth.log_edges(c["lo"], c["hi"], c["nb"]), c["nmax"]
    idx, offs, core = synth.flat_patches(pos, side, 2, c["margin"])
    # three sampled centres per patch core, as original indices and in the patched layout
    rng = np.random.default_rng(52)
    chosen = []
    for k in range(len(offs) - 1):
        cidx = offs[k] + np.flatnonzero(core[offs[k]:offs[k + 1]])
        chosen.extend(rng.choice(cidx, 3, replace=False).tolist())
    pmask = np.zeros(len(idx), np.uint8)
    pmask[chosen] = 1
    omask = np.zeros(n, np.uint8)
    omask[idx[chosen]] = 1
    assert omask.sum() == len(chosen)  # each sampled galaxy is a centre once
    dev = torch.device("cuda:0")
    tp, ts, tw = (torch.tensor(a, device=dev) for a in (pos[idx], sh[idx], w[idx]))
    nb = len(edges) - 1
    ups = torch.zeros(ext4pcf.Estimator.ups_shape(nb, nmax), dtype=torch.float64, device=dev)
    est = ext4pcf.Estimator(0, "f16x3")
    ext4pcf.ext4pcf_measure_batch(est.ctx, tp, ts, tw, len(idx), np.ascontiguousarray(edges), nb, nmax,
                                  np.ascontiguousarray(offs, dtype=np.int64), len(offs) - 1,
                                  np.zeros(len(offs) - 1, np.int32), 1, pmask, ups, None)
    torch.cuda.synchronize()
    est.close()
    got = torch.view_as_complex(ups[0]).cpu().numpy()
    ref = oracle.measure(pos, sh, w, edges, nmax, centre_mask=omask)
    # with ~3e5 neighbours per centre no bin triple is empty
    err = rel_err(got, ref)
    assert err.max() < 1e-4, err.max()
