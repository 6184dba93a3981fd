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
  * ``lognormal_catalog`` -- the same with a lognormal convergence: a Gaussian field G of
    pixel variance sigma_g^2 mapped to kappa = kappa0 (exp(G - sigma_g^2 / 2) - 1), scaled to
    the requested pixel rms (a skewed field bounded below, as weak-lensing convergence is).
  * ``mock_suite``        -- many GRF mocks of uneven size and density, concatenated with
    catalogue offsets (the batched workload).
  * ``flat_patches``      -- a footprint split into n x n square core patches, each patch
    holding its core plus every galaxy within a margin of it; a centre mask marks the core,
    so that every galaxy is a centre in exactly one patch (the survey workload, split the
    way the paper splits its survey data into overlapping flat-sky patches).
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


def lognormal_convergence(grid: int, side: float, seed: int, slope: float = -1.2, sigma_kappa: float = 0.02,
                          sigma_g: float = 1.0):
    """Lognormal convergence on a grid x grid periodic map: G, a Gaussian field with
    P(l) ~ l^slope and pixel standard deviation sigma_g, mapped to exp(G - sigma_g^2 / 2) - 1,
    then made zero-mean and scaled to pixel rms sigma_kappa (float64 map)."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((grid, grid))
    k = np.fft.fftfreq(grid, d=side / grid)
    k1, k2 = np.meshgrid(k, k, indexing="xy")
    ksq = k1 * k1 + k2 * k2
    amp = np.zeros_like(ksq)
    nz = ksq > 0
    amp[nz] = ksq[nz] ** (0.25 * slope)
    g = np.fft.ifft2(np.fft.fft2(white) * amp).real
    del white
    g *= sigma_g / g.std()
    kap = np.expm1(g - 0.5 * sigma_g * sigma_g)
    del g
    kap -= kap.mean()
    kap *= sigma_kappa / kap.std()
    return kap


def kaiser_squires_shear(kappa, side: float):
    """Shear of a periodic convergence map (flat-sky Kaiser-Squires): (gamma1, gamma2) float32."""
    grid = kappa.shape[0]
    k = np.fft.fftfreq(grid, d=side / grid)
    k1, k2 = np.meshgrid(k, k, indexing="xy")
    ksq = k1 * k1 + k2 * k2
    nz = ksq > 0
    D = np.zeros(ksq.shape, dtype=np.complex128)
    D[nz] = ((k1[nz] ** 2 - k2[nz] ** 2) + 2j * k1[nz] * k2[nz]) / ksq[nz]
    gam = np.fft.ifft2(np.fft.fft2(kappa) * D)
    return gam.real.astype(np.float32), gam.imag.astype(np.float32)


def lognormal_shear_field(grid: int, side: float, seed: int, slope: float = -1.2,
                          sigma_kappa: float = 0.02, sigma_g: float = 1.0):
    """Shear maps (gamma1, gamma2) of lognormal_convergence."""
    return kaiser_squires_shear(lognormal_convergence(grid, side, seed, slope, sigma_kappa, sigma_g), side)


def _sample_field(g1, g2, n, side, rng, sigma_e):
    grid = g1.shape[0]
    pos = rng.uniform(0.0, side, size=(n, 2))
    ix = np.minimum((pos[:, 0] * (grid / side)).astype(np.int64), grid - 1)
    iy = np.minimum((pos[:, 1] * (grid / side)).astype(np.int64), grid - 1)
    shear = np.empty((n, 2))
    shear[:, 0] = g1[iy, ix]
    shear[:, 1] = g2[iy, ix]
    del ix, iy
    shear += rng.normal(0.0, sigma_e, size=(n, 2))
    w = rng.uniform(0.5, 1.5, size=n)
    return pos, shear, w


def lognormal_catalog(n: int, side: float, seed: int, grid: int = 4096, slope: float = -1.2,
                      sigma_kappa: float = 0.02, sigma_e: float = 0.26):
    """n galaxies uniform on a side x side flat footprint with lognormal shear plus shape noise."""
    g1, g2 = lognormal_shear_field(grid, side, seed, slope, sigma_kappa)
    return _sample_field(g1, g2, n, side, np.random.default_rng(seed + 7919), sigma_e)


def mock_suite(n_mocks: int, seed: int, side_range=(300.0, 900.0), density_range=(5.0, 8.0),
               n_range=(500_000, 5_000_000), grid: int = 1024, scale: float = 1.0):
    """n_mocks GRF mocks of uneven size: side U(side_range) arcmin, density U(density_range)
    per arcmin^2, galaxy count clipped to n_range (the density follows), each its own field
    and seed.  scale < 1 shrinks every mock's area (same densities) for small test suites.
    Returns concatenated (pos, shear, w), int64 catalogue offsets [n_mocks + 1] and sides."""
    rng = np.random.default_rng(seed)
    parts, offs, sides = [], [0], []
    for k in range(n_mocks):
        side = rng.uniform(*side_range)
        dens = rng.uniform(*density_range)
        n = int(np.clip(round(dens * side * side), *n_range))
        side_k = side * np.sqrt(scale)
        n_k = max(1, int(round(n * scale)))
        parts.append(grf_catalog(n_k, side_k, seed * 1000 + k, grid=grid))
        offs.append(offs[-1] + n_k)
        sides.append(side_k)
    pos = np.concatenate([p[0] for p in parts])
    shear = np.concatenate([p[1] for p in parts])
    w = np.concatenate([p[2] for p in parts])
    return pos, shear, w, np.array(offs, dtype=np.int64), np.array(sides)


def flat_patches(pos, extent: float, n_side: int = 10, margin: float = 120.0, origin=(0.0, 0.0)):
    """Split the square footprint [origin, origin + extent)^2 into n_side x n_side core patches
    of side extent / n_side (margin < core side).  Patch p holds every galaxy of its core and
    every galaxy within `margin` of the core (along each axis, i.e. the core grown by the
    margin on each side); the cores partition the catalogue.  Returns (index, offsets, mask):
    patch p is pos[index[offsets[p]:offsets[p+1]]], and mask (uint8, aligned with index) is 1
    for the galaxies of p's core, so that every galaxy is a centre in exactly one patch."""
    pos = np.asarray(pos, dtype=np.float64)
    core = extent / n_side
    if not margin < core:
        raise ValueError("the margin must be smaller than a patch")
    x = pos[:, 0] - origin[0]
    y = pos[:, 1] - origin[1]
    px = np.clip(np.floor(x / core), 0, n_side - 1).astype(np.int16)
    py = np.clip(np.floor(y / core), 0, n_side - 1).astype(np.int16)
    pids, idxs, cores = [], [], []
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            qx = px + np.int16(dx)
            qy = py + np.int16(dy)
            sel = (qx >= 0) & (qx < n_side) & (qy >= 0) & (qy < n_side)
            if dx:
                sel &= (x >= qx * core - margin) & (x < (qx + 1) * core + margin)
            if dy:
                sel &= (y >= qy * core - margin) & (y < (qy + 1) * core + margin)
            i = np.flatnonzero(sel)
            idxs.append(i)
            pids.append((qy[i].astype(np.int16) * np.int16(n_side) + qx[i]).astype(np.int16))
            cores.append(np.full(i.size, 1 if (dx == 0 and dy == 0) else 0, dtype=np.uint8))
            del sel, qx, qy
    pid = np.concatenate(pids)
    idx = np.concatenate(idxs)
    core_flag = np.concatenate(cores)
    del pids, idxs, cores
    order = np.argsort(pid, kind="stable")
    counts = np.bincount(pid, minlength=n_side * n_side)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return idx[order], offsets, core_flag[order]


# Workloads with the paper's shapes (arcmin units).
SMALL = dict(name="uniform 2000 gal, 60'x60', 8 log bins 1'-30', n_max=10",
             n=2000, side=60.0, seed=1, lo=1.0, hi=30.0, nb=8, nmax=10)
GRF2E6 = dict(name="GRF 2e6 gal, 600'x600', 10 log bins 0.5'-40', n_max=20",
              n=2_000_000, side=600.0, seed=2, lo=0.5, hi=40.0, nb=10, nmax=20, grid=4096)


# Batched form: 64 GRF mocks of uneven size (sides 5-15 deg, 0.5e6-5e6 galaxies at 5-8 per
# arcmin^2), 12 log bins 0.5'-60', n_max = 20.  The shear maps use 1024^2 grids (one FFT pair per
# mock keeps generation short; the estimator's work does not depend on the map resolution).
BATCH64 = dict(name="64 GRF mocks, sides 300'-900', 0.5e6-5e6 gal at 5-8/arcmin^2, 12 log bins 0.5'-60', n_max=20",
               n_mocks=64, seed=40, lo=0.5, hi=60.0, nb=12, nmax=20, grid=1024)
# Survey scale: 1e8 galaxies over 3795' x 3795' (~4000 deg^2, ~7 per arcmin^2) of lognormal
# shear, split into 10 x 10 patches with 120' margins, 12 log bins 0.5'-120', n_max = 30.
SURVEY = dict(name="lognormal survey 1e8 gal, 3795'x3795' (~4000 deg^2), 10x10 patches + 120' margins, "
                   "12 log bins 0.5'-120', n_max=30",
              n=100_000_000, side=3795.0, seed=50, lo=0.5, hi=120.0, nb=12, nmax=30, grid=4096,
              n_side=10, margin=120.0)


def batch64_workload(scale: float = 1.0, n_mocks: int | None = None):
    c = BATCH64
    pos, sh, w, offs, sides = mock_suite(n_mocks or c["n_mocks"], c["seed"], grid=c["grid"], scale=scale)
    return pos, sh, w, offs, log_edges(c["lo"], c["hi"], c["nb"]), c["nmax"]


def survey_workload(n: int | None = None, side: float | None = None, grid: int | None = None,
                    n_side: int | None = None):
    """The survey catalogue and its patches: (pos, shear, w) of the patched catalogue (galaxies
    in patch order, margins repeated), catalogue offsets, the core mask, edges, n_max.  A
    smaller n keeps the density (side scaled) and, unless n_side is given, patches of about
    the survey's size (at least 2 x 2, each wider than the margin)."""
    c = SURVEY
    n = n or c["n"]
    side = side or c["side"] * (n / c["n"]) ** 0.5
    if n_side is None:
        n_side = max(2, min(c["n_side"], int(side / (c["side"] / c["n_side"]) + 0.5)))
        while side / n_side <= c["margin"] and n_side > 1:
            n_side -= 1
    pos, sh, w = lognormal_catalog(n, side, c["seed"], grid=grid or c["grid"])
    idx, offs, mask = flat_patches(pos, side, n_side, c["margin"])
    return pos[idx], sh[idx], w[idx], offs, mask, log_edges(c["lo"], c["hi"], c["nb"]), c["nmax"]


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
