"""Seeded synthetic shear catalogues shaped like the paper's workloads.

This module holds no estimator arithmetic: it only draws inputs (positions, shears,
weights, radial bin edges).  Both the CUDA path and the CPU oracle consume its output.

Recipes (the paper's data are not available; these stand in with its shapes):
  * ``uniform_catalog``  -- positions U([0, side)^2), unit (or uniform) weights, shear
    components i.i.d. N(0, sigma_e^2): the small parity workload.
  * ``grf_catalog``      -- Gaussian random field convergence with a power-law spectrum
    P(l) ~ l^slope on an FFT grid, Kaiser-Squires to shear, sampled at uniform positions
    (the shear of the pixel containing the position, i.e. a random pixel plus a random
    in-pixel displacement as in the paper's Sect. 4.1 mocks), plus shape noise sigma_e per
    component and weights U[0.5, 1.5].  The amplitude is set by the pixel rms of kappa.
"""
from __future__ import annotations

import numpy as np


def log_edges(lo: float, hi: float, nb: int) -> np.ndarray:
    """nb logarithmic radial bins between lo and hi (nb+1 edges)."""
    return np.geomspace(float(lo), float(hi), int(nb) + 1)


def uniform_catalog(n: int, side: float, seed: int, sigma_e: float = 0.26,
                    weights: str = "unit"):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, side, size=(n, 2))
    shear = rng.normal(0.0, sigma_e, size=(n, 2))
    if weights == "unit":
        w = np.ones(n)
    else:
        w = rng.uniform(0.5, 1.5, size=n)
    return pos, shear, w


def grf_shear_field(grid: int, side: float, seed: int, slope: float = -1.2,
                    sigma_kappa: float = 0.02):
    """Convergence GRF with P(l) ~ l^slope (P(0) = 0) and its Kaiser-Squires shear on a
    grid x grid periodic map of the given side.  Returns (gamma1, gamma2) float32 maps."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((grid, grid))
    k = np.fft.fftfreq(grid, d=side / grid)
    k1, k2 = np.meshgrid(k, k, indexing="xy")
    ksq = k1 * k1 + k2 * k2
    amp = np.zeros_like(ksq)
    nz = ksq > 0
    amp[nz] = ksq[nz] ** (0.25 * slope)          # sqrt(P(l)), P ~ l^slope
    kap_hat = np.fft.fft2(white) * amp
    kappa = np.fft.ifft2(kap_hat).real
    scale = sigma_kappa / kappa.std()
    kap_hat *= scale
    D = np.zeros(ksq.shape, dtype=np.complex128)
    D[nz] = ((k1[nz] ** 2 - k2[nz] ** 2) + 2j * k1[nz] * k2[nz]) / ksq[nz]
    gam = np.fft.ifft2(kap_hat * D)
    return gam.real.astype(np.float32), gam.imag.astype(np.float32)


def grf_catalog(n: int, side: float, seed: int, grid: int = 4096, slope: float = -1.2,
                sigma_kappa: float = 0.02, sigma_e: float = 0.26):
    """n galaxies on a side x side flat patch (units of side, e.g. arcmin)."""
    g1, g2 = grf_shear_field(grid, side, seed, slope, sigma_kappa)
    rng = np.random.default_rng(seed + 7919)
    pos = rng.uniform(0.0, side, size=(n, 2))
    ix = np.minimum((pos[:, 0] * (grid / side)).astype(np.int64), grid - 1)
    iy = np.minimum((pos[:, 1] * (grid / side)).astype(np.int64), grid - 1)
    shear = np.empty((n, 2))
    shear[:, 0] = g1[iy, ix]
    shear[:, 1] = g2[iy, ix]
    shear += rng.normal(0.0, sigma_e, size=(n, 2))
    w = rng.uniform(0.5, 1.5, size=n)
    return pos, shear, w


# Workloads with the paper's shapes (arcmin units).
SMALL = dict(name="uniform 2000 gal, 60'x60', 8 log bins 1'-30', n_max=10",
             n=2000, side=60.0, seed=1, lo=1.0, hi=30.0, nb=8, nmax=10)
GRF2E6 = dict(name="GRF 2e6 gal, 600'x600', 10 log bins 0.5'-40', n_max=20",
              n=2_000_000, side=600.0, seed=2, lo=0.5, hi=40.0, nb=10, nmax=20, grid=4096)


def small_workload():
    c = SMALL
    pos, shear, w = uniform_catalog(c["n"], c["side"], c["seed"])
    return pos, shear, w, log_edges(c["lo"], c["hi"], c["nb"]), c["nmax"]


def grf2e6_workload(n: int | None = None, grid: int | None = None):
    c = GRF2E6
    pos, shear, w = grf_catalog(n or c["n"], c["side"], c["seed"], grid=grid or c["grid"])
    return pos, shear, w, log_edges(c["lo"], c["hi"], c["nb"]), c["nmax"]


# Direct aperture-mass estimator: the GRF catalogue above, 24 logarithmically spaced aperture
# radii 1'-32' (the radii of the paper's comparison of the two estimators, Sect. 5.3),
# centres on a square lattice of spacing theta at least 4 theta inside the field.
DIRECT = dict(name="direct M_ap^4: GRF 2e6 gal, 600'x600', 24 log radii 1'-32', lattice spacing theta",
              lo=1.0, hi=32.0, n_radii=24, spacing=1.0)


def direct_radii():
    c = DIRECT
    return np.geomspace(c["lo"], c["hi"], c["n_radii"])
