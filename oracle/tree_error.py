"""Error of the tree approximation against the exact neighbour multipoles (oracle only; a
measurement, not a test):  python -m oracle.tree_error

A GRF catalogue of 4000 galaxies on 60' x 60' (the seeded generator of ``synth``), 8 log bins
1'-30', n_max = 5, grids of 0.125', 0.25', 0.5' and r_min in {10, 20, 40}.  Prints, per radial
bin, the level used and the largest error of G_n, W_n (over centres and n) and of Upsilon_0,
N_n on the diagonal bin triples, each relative to the largest value of that bin.
"""
import numpy as np

from . import tree


def main():
    import synth
    pos, sh, w = synth.grf_catalog(4000, 60.0, 9, grid=512)
    edges = synth.log_edges(1.0, 30.0, 8)
    nmax = 5
    n_lo, n_hi = -2 * nmax - 3, 2 * nmax
    x = w * (sh[:, 0] + 1j * sh[:, 1])
    G, W = tree.neighbour_multipoles(pos, sh, w, edges, n_lo, n_hi)
    u, nr = tree.upsilon0_from_multipoles(x, w, G, W, n_lo, nmax)
    nb = len(edges) - 1
    print("bins (arcmin):", np.array2string(edges, precision=2))
    for r_min in (10, 20, 40):
        Gt, Wt = tree.neighbour_multipoles(pos, sh, w, edges, n_lo, n_hi, delta1=0.125, n_levels=3, r_min=r_min)
        ut, nt = tree.upsilon0_from_multipoles(x, w, Gt, Wt, n_lo, nmax)
        eg = np.abs(Gt - G).max(axis=(0, 1)) / np.abs(G).max(axis=(0, 1))
        ew = np.abs(Wt - W).max(axis=(0, 1)) / np.abs(W).max(axis=(0, 1))
        eu = [np.abs(ut[..., b, b, b] - u[..., b, b, b]).max() / np.abs(u[..., b, b, b]).max() for b in range(nb)]
        en = [np.abs(nt[..., b, b, b] - nr[..., b, b, b]).max() / np.abs(nr[..., b, b, b]).max() for b in range(nb)]
        print("r_min", r_min, "levels", tree.bin_levels(edges, 0.125, 3, r_min))
        for name, e in (("G_n", eg), ("W_n", ew), ("Upsilon_0 (b,b,b)", eu), ("N_n (b,b,b)", en)):
            print("  %-18s" % name, " ".join("%.1e" % v for v in e))


if __name__ == "__main__":
    main()
