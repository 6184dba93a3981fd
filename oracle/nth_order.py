"""FP64 CPU oracle of the N-th order shear correlation multipoles (arXiv:2509.07974, App. F).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; the product library never uses it, and it
uses nothing of the product (its enumeration and its estimator are written here from the
paper's definitions).

``beta_matrix(N)`` enumerates the natural components as App. F.1 describes: first no
conjugated shear, then one, two, ... up to floor(N/2); for p conjugated shears, the
conjugated positions start packed at the left, the rightmost one walks to the end, then the
next one steps right with the previous ones packed behind it; for even N only the first
half of the p = N/2 rows is kept (the rest are their complex conjugates).  Row mu holds
beta^mu_l = -1 where the l-th shear is conjugated, else +1.

``bruteforce_multipoles`` evaluates the multipole components of App. F.2 directly from
their definition: for every centre galaxy and every tuple of neighbours (one per radial bin,
any indices), the product of the weights, the x-projected shears (Eq. gammatx_def with
zeta_0 = (phi_1 + phi_{N-1}) / 2 and zeta_l = phi_l) and the Fourier kernel
exp(-i sum_{l>=2} n_l (phi_l - phi_1)), summed without factorising.  Bin membership is
lo^2 <= r^2 < hi^2 with r^2 = dx*dx + dy*dy.
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = ["beta_matrix", "bruteforce_multipoles"]


def beta_matrix(order):
    """[2^{N-1}][N] int array of +-1 in the enumeration order of App. F.1."""
    rows = []
    for p in range(order // 2 + 1):
        combos = list(itertools.combinations(range(order), p))
        if 2 * p == order:
            combos = combos[: len(combos) // 2]
        for c in combos:
            r = np.ones(order, dtype=int)
            r[list(c)] = -1
            rows.append(r)
    return np.array(rows, dtype=int)


def _projected(gc, zeta2, beta):
    """x-projected shear (Eq. gammatx_def) or its conjugate; zeta2 = 2 zeta."""
    g = -gc * np.exp(-1j * zeta2)
    return g if beta > 0 else np.conj(g)


def bruteforce_multipoles(order, pos, shear, w, edges, nmax, distinct=False):
    """Upsilon_{mu, n}(Theta_1..Theta_{N-1}) for every natural component (rows 0 .. 2^{N-1}-1)
    and the normalisation (last row), over all neighbour tuples, or (distinct=True) only over
    tuples of pairwise different galaxies (the centre always differs from its neighbours).
    Shape [2^{N-1} + 1] + [2 nmax + 1] * (N - 2) + [nb] * (N - 1), axes n_l + nmax for
    l = 2..N-1, complex128."""
    pos = np.asarray(pos, dtype=np.float64)
    gc_all = np.asarray(shear, dtype=np.float64) @ np.array([1.0, 1j])
    w = np.asarray(w, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.float64)
    nb = edges.size - 1
    beta = beta_matrix(order)
    nmu = beta.shape[0]
    k = order - 1                     # neighbours per tuple
    nvec = list(itertools.product(range(-nmax, nmax + 1), repeat=order - 2))
    nvec_arr = np.array(nvec, dtype=np.float64).reshape(len(nvec), order - 2)
    out = np.zeros((nmu + 1, len(nvec)) + (nb,) * k, dtype=np.complex128)
    e2 = edges * edges
    for i in range(pos.shape[0]):
        dx = pos[:, 0] - pos[i, 0]
        dy = pos[:, 1] - pos[i, 1]
        r2 = dx * dx + dy * dy
        phi = np.arctan2(dy, dx)
        members = [np.flatnonzero((r2 >= e2[b]) & (r2 < e2[b + 1])) for b in range(nb)]
        for bins in itertools.product(range(nb), repeat=k):
            sets = [members[b] for b in bins]
            if any(s.size == 0 for s in sets):
                continue
            grids = np.meshgrid(*sets, indexing="ij")   # neighbour index per tuple slot
            ph = [phi[g] for g in grids]                  # phi_1 .. phi_{N-1}
            wt = w[i] * np.prod([w[g] for g in grids], axis=0)
            if distinct:
                for a in range(k):
                    for b in range(a + 1, k):
                        wt = np.where(grids[a] == grids[b], 0.0, wt)
            # Fourier kernel exp(-i sum_{l=2}^{N-1} n_l (phi_l - phi_1)) for every n
            if order > 2:
                rel = np.stack([ph[l] - ph[0] for l in range(1, k)], axis=0)   # [N-2][...]
                arg = np.tensordot(nvec_arr, rel, axes=([1], [0]))             # [n][...]
                kern = np.exp(-1j * arg)
            else:
                kern = np.ones((1,) + wt.shape)
            zeta0_2 = ph[0] + ph[-1]                      # 2 zeta_0
            for mu in range(nmu):
                val = wt * _projected(gc_all[i], zeta0_2, beta[mu, 0])
                for l in range(k):
                    val = val * _projected(gc_all[grids[l]], 2.0 * ph[l], beta[mu, l + 1])
                out[(mu, slice(None)) + bins] += np.tensordot(kern, val, axes=(list(range(1, k + 1)),
                                                                              list(range(k))))
            out[(nmu, slice(None)) + bins] += np.tensordot(kern, wt, axes=(list(range(1, k + 1)),
                                                                           list(range(k))))
    return out.reshape((nmu + 1,) + (2 * nmax + 1,) * (order - 2) + (nb,) * k)
