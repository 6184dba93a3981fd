"""Multipole structure of the 4PCF of a Gaussian field (App. B), oracle side; no GPU.

For a Gaussian shear field Wick's theorem writes the 4PCF as products of two-point functions.
At equal radii (thin bins, Theta1 = Theta2 = Theta3), for the sixth natural component
(conjugated shears at the centre and at the second neighbour, Upsilon_6 here), App. B derives
that the three Wick terms are each non-zero only on one line of the (n2, n3) plane --
n2 = -2, n3 = -1 and n2 + n3 = 1 -- and that the largest value sits at (n2, n3) = (2, -1),
where two of those lines cross.

The pin averages the oracle's (corrected, distinct-quadruplet) Upsilon_6 over an ensemble of
seeded noise-free Gaussian random fields (as the paper does with its GRF ensemble), at one thin
radial bin, and checks that structure.  A sign error in the multipole phases, a transposed
(n2, n3), or a wrong conjugation pattern moves the peak or the lines.
"""
import numpy as np

import synth

N = 4


def on_lines(n2, n3):
    """The lines n3 = -1 and n2 + n3 = 1, and the largest value of the line n2 = -2, which the
    derivation puts at n3 = 1."""
    return n3 == -1 or n2 + n3 == 1 or (n2, n3) == (-2, 1)


def test_equal_radii_multipoles_of_a_gaussian_field(oracle):
    edges = np.array([1.0, 1.15])  # one thin bin: Theta1 = Theta2 = Theta3
    acc = np.zeros((2 * N + 1, 2 * N + 1), complex)
    for r in range(16):
        pos, sh, _ = synth.grf_catalog(20000, 60.0, 100 + r, grid=512, sigma_e=0.0)
        ups = oracle.measure(pos, sh, np.ones(len(pos)), edges, N)
        acc += ups[6, :, :, 0, 0, 0]
    a = np.abs(acc) / np.abs(acc).max()
    n2, n3 = np.unravel_index(np.argmax(a), a.shape)
    assert (n2 - N, n3 - N) == (2, -1)
    cells = [(i - N, j - N) for i in range(2 * N + 1) for j in range(2 * N + 1)]
    on = [a[n2 + N, n3 + N] for n2, n3 in cells if on_lines(n2, n3)]
    # the rest of the line n2 = -2 belongs to neither set
    off = [a[n2 + N, n3 + N] for n2, n3 in cells if not on_lines(n2, n3) and n2 != -2]
    # measured: every entry of the set >= 0.10 of the peak, every entry off it <= 0.04
    assert min(on) > 1.5 * max(off)
    # along n2 = -2 the largest value is at n3 = 1 or where the other two lines cross it
    row = a[-2 + N]
    assert row[1 + N] >= 0.9 * row.max() and row[1 + N] > 2.0 * np.median(row)
