"""FP64 CPU oracle of the tree approximation of the neighbour multipoles (arXiv:2509.07974,
Sect. 3.2 and App. F.3), and its error against the exact multipoles.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; the product library never uses it.

The catalogue is binned on a hierarchy of square grids of side Delta_d = 2^{d-1} Delta_1
(d = 1..D), all anchored at the same origin.  The galaxies of each non-empty cell are
replaced by one "reduced" galaxy at their weighted centre of mass, carrying the summed weight
sum w and the summed weighted shear sum w gamma_c.  A radial bin Theta uses the coarsest
level d with Theta_low / Delta_d >= r_min; when no level qualifies it uses the galaxies
themselves.  The centres stay the discrete galaxies; the neighbour multipoles of a bin are
    G_n(theta_i, Theta) = sum_c X_c e^{i n phi_ic},  W_n = sum_c W_c e^{i n phi_ic}
over the reduced galaxies c of that bin's level whose separation from theta_i lies in the bin
(lo^2 <= r^2 < hi^2).  ``upsilon0_from_multipoles`` contracts them into Upsilon_0 and N_n of
Eq. 4PCFUpsilon0 and Eq. Nnmultipoles (all index triples, no multiple-counting corrections).
"""
from __future__ import annotations

import numpy as np

__all__ = ["reduced_catalogue", "bin_levels", "neighbour_multipoles", "upsilon0_from_multipoles"]


def reduced_catalogue(pos, shear, w, delta, origin):
    """Cells of side ``delta`` anchored at ``origin``: (centre-of-mass positions [m][2],
    summed w gamma_c [m] complex, summed w [m]) over the non-empty cells."""
    pos = np.asarray(pos, dtype=np.float64)
    x = np.asarray(w) * (np.asarray(shear)[:, 0] + 1j * np.asarray(shear)[:, 1])
    cx = np.floor((pos[:, 0] - origin[0]) / delta).astype(np.int64)
    cy = np.floor((pos[:, 1] - origin[1]) / delta).astype(np.int64)
    key = (cy - cy.min()) * (cx.max() - cx.min() + 1) + (cx - cx.min())
    uniq, inv = np.unique(key, return_inverse=True)
    m = uniq.size
    W = np.bincount(inv, weights=w, minlength=m)
    X = np.bincount(inv, weights=x.real, minlength=m) + 1j * np.bincount(inv, weights=x.imag, minlength=m)
    com = np.stack([np.bincount(inv, weights=w * pos[:, 0], minlength=m),
                    np.bincount(inv, weights=w * pos[:, 1], minlength=m)], 1) / W[:, None]
    return com, X, W


def bin_levels(edges, delta1, n_levels, r_min):
    """Level per radial bin: the coarsest d in 1..n_levels with lo / (2^{d-1} delta1) >= r_min,
    else 0 (the galaxies themselves)."""
    lv = []
    for lo in np.asarray(edges, dtype=np.float64)[:-1]:
        d_ok = [d for d in range(1, n_levels + 1) if lo / (2.0 ** (d - 1) * delta1) >= r_min]
        lv.append(max(d_ok) if d_ok else 0)
    return np.array(lv, dtype=int)


def neighbour_multipoles(pos, shear, w, edges, n_lo, n_hi, delta1=None, n_levels=0, r_min=np.inf,
                         origin=None):
    """G_n and W_n (n = n_lo..n_hi) of every galaxy as centre, per radial bin, each bin from
    its level of the hierarchy (exact when r_min is infinite).  Returns G, W of shape
    [n_gal][n_hi - n_lo + 1][nb], complex128."""
    pos = np.asarray(pos, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.float64)
    nb = edges.size - 1
    if origin is None:
        origin = pos.min(axis=0)
    levels = bin_levels(edges, delta1, n_levels, r_min) if delta1 else np.zeros(nb, dtype=int)
    cats = {0: (pos, w * (shear[:, 0] + 1j * shear[:, 1]), w)}
    for d in set(levels.tolist()) - {0}:
        cats[d] = reduced_catalogue(pos, shear, w, 2.0 ** (d - 1) * delta1, origin)
    ns = np.arange(n_lo, n_hi + 1)
    G = np.zeros((pos.shape[0], ns.size, nb), dtype=np.complex128)
    Wn = np.zeros_like(G)
    e2 = edges * edges
    for i in range(pos.shape[0]):
        for b in range(nb):
            cpos, cx, cw = cats[levels[b]]
            dx = cpos[:, 0] - pos[i, 0]
            dy = cpos[:, 1] - pos[i, 1]
            r2 = dx * dx + dy * dy
            sel = (r2 >= e2[b]) & (r2 < e2[b + 1])
            if not sel.any():
                continue
            ph = np.exp(1j * np.outer(ns, np.arctan2(dy[sel], dx[sel])))
            G[i, :, b] = ph @ cx[sel]
            Wn[i, :, b] = ph @ cw[sel]
    return G, Wn


def upsilon0_from_multipoles(x, w, G, Wn, n_lo, nmax):
    """Upsilon_0 (Eq. 4PCFUpsilon0) and N_n (Eq. Nnmultipoles) from per-centre multipoles:
    sum_i x_i G_{n2+n3-3}(Th1) G_{-n2-2}(Th2) G_{-n3-3}(Th3) and
    sum_i w_i W_{n2+n3}(Th1) W_{-n2}(Th2) W_{-n3}(Th3).  Shapes [2N+1][2N+1][nb]^3."""
    nn = 2 * nmax + 1
    nb = G.shape[2]
    ups = np.zeros((nn, nn, nb, nb, nb), dtype=np.complex128)
    nrm = np.zeros_like(ups)
    for a, n2 in enumerate(range(-nmax, nmax + 1)):
        for c, n3 in enumerate(range(-nmax, nmax + 1)):
            g1, g2, g3 = G[:, n2 + n3 - 3 - n_lo], G[:, -n2 - 2 - n_lo], G[:, -n3 - 3 - n_lo]
            ups[a, c] = np.einsum("i,ia,ib,ic->abc", x, g1, g2, g3)
            w1, w2, w3 = Wn[:, n2 + n3 - n_lo], Wn[:, -n2 - n_lo], Wn[:, -n3 - n_lo]
            nrm[a, c] = np.einsum("i,ia,ib,ic->abc", w, w1, w2, w3)
    return ups, nrm
