"""Symmetry-reduced storage of the 4PCF multipoles (arXiv:2509.07974, Sect. 3.1, Table
tab:4PCFSymm) in FP64 numpy.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; the product library never uses it.

Table tab:4PCFSymm relates a permutation of the radial bins (Theta1, Theta2, Theta3) to another
natural component mu' at shifted multipoles (n2', n3'):
    Upsilon_mu[n2, n3](b1, b2, b3) = Upsilon_mu'[n2', n3'](b_{p0}, b_{p1}, b_{p2}).
So the multipoles of the sorted triples b1 <= b2 <= b3 determine all others, provided they are
kept over the larger multipole range the maps reach (|n'| <= 2N + 1 for |n| <= N).
``restrict`` keeps the sorted triples of a computation at that larger range; ``expand``
rebuilds every ordered triple at |n| <= N from them.
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = ["BIN_PERM", "MU_MAP", "n_map", "sorted_triples", "enlarged_nmax", "restrict", "expand",
           "reached_region"]

# columns of Table tab:4PCFSymm: (Theta2,Theta3,Theta1), (Theta3,Theta1,Theta2),
# (Theta1,Theta3,Theta2), (Theta2,Theta1,Theta3), (Theta3,Theta2,Theta1)
BIN_PERM = [(1, 2, 0), (2, 0, 1), (0, 2, 1), (1, 0, 2), (2, 1, 0)]
# component mu' per component mu (rows; mu = 8 the normalisation) and column
MU_MAP = {0: [0, 0, 0, 0, 0], 1: [1, 1, 1, 1, 1], 2: [4, 3, 2, 3, 4], 3: [2, 4, 4, 2, 3],
          4: [3, 2, 3, 4, 2], 5: [7, 6, 5, 6, 7], 6: [5, 7, 7, 5, 6], 7: [6, 5, 6, 7, 5],
          8: [8, 8, 8, 8, 8]}
_OFFSET = {0: 1, 2: 1, 3: 1, 4: 1, 1: -1, 5: -1, 6: -1, 7: -1, 8: 0}


def n_map(mu, col, n2, n3):
    """(n2', n3') of Table tab:4PCFSymm for component mu and column col."""
    s = n2 + n3
    o = _OFFSET[mu]
    return [(n3 + o, -s), (-s + o, n2 - o), (n3 + o, n2 - o), (-s + o, n3), (n2, -s)][col]


def sorted_triples(nb):
    return [t for t in itertools.product(range(nb), repeat=3) if t[0] <= t[1] <= t[2]]


def enlarged_nmax(nmax):
    """Multipole range the maps reach from |n2|, |n3| <= nmax."""
    return 2 * nmax + 1


def restrict(ups_big, nmax_big):
    """Sorted-triple storage [9][2M+1][2M+1][n_sorted] from full multipoles computed at
    nmax_big = M (layout [9][2M+1][2M+1][nb][nb][nb])."""
    nb = ups_big.shape[3]
    tri = sorted_triples(nb)
    return np.stack([ups_big[:, :, :, a, b, c] for a, b, c in tri], axis=-1)


def expand(stored, nb, nmax, nmax_big):
    """All ordered triples at |n| <= nmax, [9][2N+1][2N+1][nb][nb][nb], from the sorted-triple
    storage of ``restrict``."""
    index = {t: k for k, t in enumerate(sorted_triples(nb))}
    N, M = nmax, nmax_big
    out = np.zeros((9, 2 * N + 1, 2 * N + 1, nb, nb, nb), dtype=stored.dtype)
    for b in itertools.product(range(nb), repeat=3):
        if b in index:
            out[:, :, :, b[0], b[1], b[2]] = stored[:, M - N:M + N + 1, M - N:M + N + 1, index[b]]
            continue
        col = next(c for c, p in enumerate(BIN_PERM) if b[p[0]] <= b[p[1]] <= b[p[2]])
        p = BIN_PERM[col]
        k = index[(b[p[0]], b[p[1]], b[p[2]])]
        for mu in range(9):
            mup = MU_MAP[mu][col]
            for n2 in range(-N, N + 1):
                for n3 in range(-N, N + 1):
                    m2, m3 = n_map(mu, col, n2, n3)
                    out[mu, n2 + N, n3 + N, b[0], b[1], b[2]] = stored[mup, m2 + M, m3 + M, k]
    return out


def reached_region(nmax):
    """For each component mu', the set of (n2', n3') that some ordered triple at |n| <= nmax
    reads from a sorted triple (identity included): the multipoles a symmetry-reduced
    contraction has to produce."""
    need = {m: set() for m in range(9)}
    for mu in range(9):
        for n2 in range(-nmax, nmax + 1):
            for n3 in range(-nmax, nmax + 1):
                need[mu].add((n2, n3))
                for col in range(5):
                    need[MU_MAP[mu][col]].add(n_map(mu, col, n2, n3))
    return need
