"""Pin of the oracle's fourth-order aperture integration (Eq. 4PCF2M4), assembly included.

The oracle evaluates <M_mu> as a sum over radial and angular bins of the real-space 4PCF times
its closed-form kernel F_mu (aperture centre integrated analytically), with the radial area
element (hi^2 - lo^2)/2 at the r-weighted mean radius and the angular bins at their centres.
The kernel alone is pinned elsewhere by quadrature of the aperture-centre integral; this file
pins the whole assembly -- radial area elements, angular rule, every Jacobian factor, the
projection phases and the component routing -- against an independent numerical integration
of the defining integral, for a 4PCF whose natural components are constant, Gamma_mu = C_mu,
on the radial range [r_lo, r_hi) of the bins.

Defining integral (Eq. MapGamma inserted for four apertures sharing one centre at the origin,
the Cartesian correlator written in the x-projection of Eq. xprojection with Eq. gammatx_def):
    <M_mu> = int d^2y d^2v1 d^2v2 d^2v3  prod_{a=0..3} q_{beta_a}(Y_a)  C_mu  e^{2i sum_a s_a zeta_a},
    Y_0 = y, Y_a = y + v_a,  q_0(Y) = conj(Y)^2 g(Y), q_1(Y) = Y^2 g(Y),
    g(Y) = exp(-|Y|^2 / 2 theta^2) / (4 pi theta^4)  (Q_theta of Eq. CrittendenQ times the spin
    phase of Eq. MapGamma),  s_a = +1 (-1) for an unconjugated (conjugated) aperture,
    zeta_0 = (phi_1 + phi_3)/2, zeta_a = phi_a (the polar angle of v_a).
The quadrature here shares nothing with the oracle's closed form: Gauss-Hermite nodes for the
y integral (its integrand is a polynomial of degree 8 times a Gaussian, so 6 nodes per axis are
exact), Gauss-Legendre nodes in each radius with the Jacobian r, uniform periodic grids in
phi_12 and phi_13, and phi_1 fixed by the rotation invariance of the integrand (checked).
The oracle's binned rule converges to it at second order in the bin width.
"""
import numpy as np
import pytest

# conjugation pattern beta of the correlators of Eq. M4Ordering (1 = conjugated aperture)
BETA = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
                 [1, 1, 0, 0], [1, 0, 1, 0], [1, 0, 0, 1]])


def defining_integral(theta, r_lo, r_hi, phi1=0.0, n_r=8, n_phi=32, n_h=6):
    """[8] complex: the integral above with C_mu = 1, vartheta_a in [r_lo, r_hi)."""
    xr, wr = np.polynomial.legendre.leggauss(n_r)
    r = 0.5 * (r_hi - r_lo) * xr + 0.5 * (r_hi + r_lo)
    wr = 0.5 * (r_hi - r_lo) * wr * r
    phi = 2.0 * np.pi * np.arange(n_phi) / n_phi
    wphi = 2.0 * np.pi / n_phi
    # y = -c + u with c the mean of (0, v1, v2, v3): sum_a |Y_a|^2 = 4|u|^2 + sum_a |v_a - c|^2,
    # so the y integral carries the weight exp(-|u|^2 / 2 s^2), s = theta / 2
    xh, wh = np.polynomial.hermite_e.hermegauss(n_h)
    s = theta / 2.0
    ux, uy = np.meshgrid(xh * s, xh * s, indexing="ij")
    u = (ux + 1j * uy).ravel()
    wu = np.outer(wh, wh).ravel() * s * s * np.exp(np.abs(u) ** 2 / (2 * s * s))
    P2, P3 = np.meshgrid(phi, phi, indexing="ij")
    out = np.zeros(8, complex)
    for a in range(n_r):
        R2, R3 = np.meshgrid(r, r, indexing="ij")
        v1 = np.full(R2.shape + P2.shape, r[a] * np.exp(1j * phi1))
        v2 = R2[:, :, None, None] * np.exp(1j * (phi1 + P2))[None, None]
        v3 = R3[:, :, None, None] * np.exp(1j * (phi1 + P3))[None, None]
        cen = (v1 + v2 + v3) / 4.0
        Y = np.stack([np.zeros_like(v1), v1, v2, v3], 0)[..., None] - cen[None, ..., None] + u
        g = np.exp(-np.sum(np.abs(Y) ** 2, axis=0) / (2 * theta * theta)) / (4 * np.pi * theta ** 4) ** 4
        zeta = [0.5 * (2 * phi1 + P3), np.full(P2.shape, phi1), phi1 + P2, phi1 + P3]
        wt = (wr[a] * np.outer(wr, wr))[:, :, None, None] * wphi * wphi * 2.0 * np.pi
        for mu in range(8):
            f = g.copy()
            ph = np.zeros(P2.shape)
            for q in range(4):
                f = f * (np.conj(Y[q]) ** 2 if BETA[mu, q] == 0 else Y[q] ** 2)
                ph = ph + (1.0 if BETA[mu, q] == 0 else -1.0) * zeta[q]
            out[mu] += np.sum((f @ wu) * np.exp(2j * ph)[None, None] * wt)
    return out


def constant_4pcf(C, nb):
    """Multipoles (n_max = 0) whose real-space natural components are C_mu on every bin:
    only n2 = n3 = 0 is non-zero, and N_0 = 1 (every angular bin has the same weight)."""
    ups = np.zeros((9, 1, 1, nb, nb, nb), complex)
    for mu in range(8):
        ups[mu, 0, 0] = C[mu]
    ups[8, 0, 0] = 1.0
    return ups


def test_defining_integral_is_rotation_invariant():
    a = defining_integral(2.0, 1.0, 4.0, phi1=0.0, n_r=3, n_phi=12)
    b = defining_integral(2.0, 1.0, 4.0, phi1=0.9, n_r=3, n_phi=12)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_binned_integration_converges_to_the_defining_integral(oracle):
    theta, lo, hi = 2.0, 1.0, 4.0
    C = (1.0 + 0.1 * np.arange(8)) * np.exp(0.3j * np.arange(8))
    ref = C * defining_integral(theta, lo, hi)
    assert np.abs(ref).min() > 1e-3 * np.abs(ref).max()
    err = {}
    for nb in (10, 20):
        m4, _, _ = oracle.map4(constant_4pcf(C, nb), np.geomspace(lo, hi, nb + 1), 48, [theta])
        err[nb] = np.abs(m4[0] - ref) / np.abs(ref)
    # measured: 0.6-1.2% at 10 bins of 0.06 dex, a quarter of that at 20 bins
    assert err[10].max() < 0.02
    assert err[20].max() < 0.005
    ratio = err[10] / err[20]
    assert np.all((ratio > 3.0) & (ratio < 5.0))
