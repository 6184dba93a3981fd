"""Error metric of the parity tests (floor-relative error per component) and the bin triples
that hold no quadruplet of distinct galaxies.  Test infrastructure: numpy and scipy only."""
import numpy as np


def rel_err(a, b, unc=None, empty=None):
    """Floor-relative error |a - b| / max(|b|, floor), floor = rms over (n2, n3) of the
    reference for each (mu, Theta1, Theta2, Theta3), and at least 1e-12 of the component's
    largest value.
    `empty` ([nb, nb, nb] bool, from empty_slabs): bin triples that hold no quadruplet of
    distinct galaxies, where the corrected multipoles vanish in exact arithmetic and both
    sides hold only rounding residue of the uncorrected terms; there the error is measured
    against the component's largest value instead.
    `unc` (the reference without multiple-counting corrections), when given, also sets the
    floor (a corrected value is a difference of uncorrected terms, and its rounding scales
    with them); only the FP32, BF16x3 and TF32 forms use it, on 60-galaxy catalogues."""
    floor = np.sqrt(np.mean(np.abs(b) ** 2, axis=(1, 2), keepdims=True))
    if unc is not None:
        floor = np.maximum(floor, np.sqrt(np.mean(np.abs(unc) ** 2, axis=(1, 2), keepdims=True)))
    scale = np.abs(b).reshape(b.shape[0], -1).max(axis=1).reshape((-1,) + (1,) * (b.ndim - 1))
    den = np.maximum(np.maximum(np.abs(b), floor), 1e-12 * scale)
    if empty is not None:
        den = np.where(np.broadcast_to(empty, b.shape), np.broadcast_to(scale, b.shape), den)
    den = np.where(den > 0, den, 1.0)
    return np.abs(a - b) / den


def empty_slabs(pos, edges):
    """[nb, nb, nb] bool: bin triples (Theta1, Theta2, Theta3) for which no centre has
    neighbours j, k, l, pairwise different, in those bins (a bin that appears m times in the
    triple needs m neighbours of the centre in it).  Counted with the bin rule of the
    estimator, lo^2 <= dx^2 + dy^2 < hi^2 in FP64; every galaxy a centre."""
    from scipy.spatial import cKDTree
    pos = np.asarray(pos, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.float64)
    e2 = edges * edges
    nb = len(edges) - 1
    tri = np.array(np.meshgrid(*[np.arange(nb)] * 3, indexing="ij")).reshape(3, -1).T
    need = np.stack([(tri == b).sum(axis=1) for b in range(nb)], axis=1)  # [nb^3][nb]
    occupied = np.zeros(len(tri), bool)
    tree = cKDTree(pos)
    for i, nbrs in enumerate(tree.query_ball_point(pos, edges[-1] * (1 + 1e-9))):
        d = pos[nbrs] - pos[i]
        r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
        c = np.array([np.count_nonzero((r2 >= e2[b]) & (r2 < e2[b + 1])) for b in range(nb)])
        occupied |= np.all(c[None, :] >= need, axis=1)
    return (~occupied).reshape(nb, nb, nb)
