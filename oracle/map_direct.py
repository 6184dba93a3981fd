"""FP64 CPU oracle of the direct aperture-mass estimator (arXiv:2509.07974, Sect. 5.2,
Eq. MapDirectEstimator).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py``; the product library never uses it.

For one aperture of radius theta centred at vartheta, Eq. MapDirectEstimator takes the sum
over ordered quadruplets of distinct galaxies of w Q_theta gamma_t (numerator) and of w
(denominator).  Both are 4! times the elementary symmetric polynomial e_4 of the per-galaxy
values; this module evaluates e_k literally as the coefficient of t^k in prod_i (1 + x_i t)
(the product taken pairwise, degree truncated at k_max), so the ratio is the paper's.

Readings of the passage (the paper is terse here):
  * Q_theta is the filter of Eq. CrittendenQ; galaxies enter an aperture when
    |vartheta_i - vartheta| < 4 theta (the hard cut at 4 theta).
  * gamma_t is the real part of Eq. gammatx_def with zeta the polar angle of
    vartheta_i - vartheta.
  * The printed ratio leaves out the area of the sampled disc: Eq. MapGamma integrates
    Q gamma_t over the plane, which the weighted galaxy mean over the disc of radius 4 theta
    estimates only after multiplication by its area A = pi (4 theta)^2.  The estimate of
    <M_ap^4> per aperture is therefore A^4 e_4(w Q gamma_t) / e_4(w) (and A^2 e_2 / e_2 for
    <M_ap^2>).
  * Apertures are averaged with inverse shot-noise weights: the shot-noise variance of an
    aperture's ratio falls as its denominator grows, so each aperture is weighted by its
    denominator and <M_ap^4> = A^4 sum_a e_4(a) / sum_a e_4(w) over the apertures.
  * The Gaussian (disconnected) part of <M_ap^4> is 3 <M_ap^2>^2 with <M_ap^2> from the
    same apertures (order-two form of the same estimator); connected = full - 3 <M_ap^2>^2.

Per-aperture record (float64 [8]): e1(a), e2(a), e4(a), e1(w), e2(w), e4(w), n, 0 with
a_i = w_i Q_theta,i gamma_t,i and n the number of galaxies inside the cut.
Per-radius record (float64 [8]): sum e4(a), sum e4(w), sum e2(a), sum e2(w), apertures,
<M_ap^4>, <M_ap^2>, <M_ap^4> - 3 <M_ap^2>^2.
"""
from __future__ import annotations

import numpy as np

__all__ = ["crittenden_q", "tangential_shear", "elementary_symmetric", "aperture_record",
           "map_direct", "moments_from_records"]


def crittenden_q(r, theta):
    """Eq. CrittendenQ: Q_theta(r) = r^2 / (4 pi theta^4) exp(-r^2 / (2 theta^2))."""
    r = np.asarray(r, dtype=np.float64)
    return r * r / (4.0 * np.pi * theta ** 4) * np.exp(-r * r / (2.0 * theta * theta))


def tangential_shear(g1, g2, dx, dy):
    """Real part of Eq. gammatx_def, gamma(theta; zeta) = -gamma_c exp(-2 i zeta), with zeta
    the polar angle of (dx, dy)."""
    zeta = np.arctan2(dy, dx)
    return (-(np.asarray(g1) + 1j * np.asarray(g2)) * np.exp(-2j * zeta)).real


def elementary_symmetric(x, kmax=4):
    """e_0 .. e_kmax of the values x: the coefficients of prod_i (1 + x_i t) up to t^kmax,
    i.e. e_k = sum over index sets i_1 < ... < i_k of x_{i_1} ... x_{i_k}."""
    x = np.asarray(x, dtype=np.float64).ravel()
    polys = np.zeros((max(x.size, 1), kmax + 1))
    polys[:, 0] = 1.0
    polys[:x.size, 1] = x
    while polys.shape[0] > 1:
        if polys.shape[0] % 2:
            polys = np.vstack([polys, np.eye(1, kmax + 1)])
        a, b = polys[0::2], polys[1::2]
        prod = np.zeros_like(a)
        for k in range(kmax + 1):
            for m in range(k + 1):
                prod[:, k] += a[:, m] * b[:, k - m]
        polys = prod
    return polys[0]


def aperture_record(pos, shear, w, centre, theta):
    """Per-aperture record (see the module docstring) of one aperture."""
    R = 4.0 * theta
    dx = pos[:, 0] - centre[0]
    dy = pos[:, 1] - centre[1]
    r2 = dx * dx + dy * dy
    inside = r2 < R * R
    dx, dy, r2 = dx[inside], dy[inside], r2[inside]
    wi = w[inside]
    a = wi * crittenden_q(np.sqrt(r2), theta) * tangential_shear(shear[inside, 0], shear[inside, 1], dx, dy)
    ea = elementary_symmetric(a, 4)
    ew = elementary_symmetric(wi, 4)
    return np.array([ea[1], ea[2], ea[4], ew[1], ew[2], ew[4], float(inside.sum()), 0.0])


def moments_from_records(records, theta):
    """Per-radius record from the per-aperture records of one radius."""
    rec = np.asarray(records, dtype=np.float64).reshape(-1, 8)
    out = np.zeros(8)
    out[0] = rec[:, 2].sum()
    out[1] = rec[:, 5].sum()
    out[2] = rec[:, 1].sum()
    out[3] = rec[:, 4].sum()
    out[4] = rec.shape[0]
    area = np.pi * (4.0 * theta) ** 2
    out[5] = area ** 4 * out[0] / out[1] if out[1] > 0 else 0.0
    out[6] = area ** 2 * out[2] / out[3] if out[3] > 0 else 0.0
    out[7] = out[5] - 3.0 * out[6] ** 2
    return out


def map_direct(pos, shear, w, thetas, centres):
    """Direct estimator over apertures.  ``centres`` is a list (one entry per radius) of
    [n_a][2] arrays of aperture centres.  Returns (per-aperture records [sum n_a][8],
    per-radius records [n_theta][8])."""
    pos = np.asarray(pos, dtype=np.float64)
    shear = np.asarray(shear, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    recs, moms = [], []
    for theta, cen in zip(thetas, centres):
        cen = np.asarray(cen, dtype=np.float64).reshape(-1, 2)
        r = np.array([aperture_record(pos, shear, w, c, theta) for c in cen]).reshape(-1, 8)
        recs.append(r)
        moms.append(moments_from_records(r, theta))
    return np.vstack(recs) if recs else np.zeros((0, 8)), np.array(moms).reshape(-1, 8)
