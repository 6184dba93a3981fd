"""Input generators of the batched and survey workloads (host code, no GPU): the patcher's
cores partition the catalogue and every patch holds exactly its core grown by the margin;
the mock suite's sizes and densities stay in their ranges; the lognormal field is skewed."""
import numpy as np

import synth


def test_patch_cores_partition_the_catalogue_and_margins_are_complete():
    side, n_side, margin = 90.0, 3, 12.0
    pos, _, _ = synth.uniform_catalog(6000, side, seed=3)
    pos[:3] = [[0.0, 0.0], [side - 1e-9, side - 1e-9], [30.0, 60.0]]  # corners and a core edge
    idx, offs, mask = synth.flat_patches(pos, side, n_side, margin)
    n = len(pos)
    assert offs[0] == 0 and offs[-1] == len(idx) == len(mask)
    assert np.array_equal(np.sort(idx[mask == 1]), np.arange(n))  # a centre exactly once
    core = side / n_side
    x, y = pos[:, 0], pos[:, 1]
    cx = np.clip(np.floor(x / core), 0, n_side - 1)
    cy = np.clip(np.floor(y / core), 0, n_side - 1)
    for p in range(n_side * n_side):
        qy, qx = divmod(p, n_side)
        members = idx[offs[p]:offs[p + 1]]
        grown = (x >= qx * core - margin) & (x < (qx + 1) * core + margin) & \
                (y >= qy * core - margin) & (y < (qy + 1) * core + margin)
        in_core = (cx == qx) & (cy == qy)
        assert np.array_equal(np.sort(members), np.flatnonzero(grown | in_core))
        assert np.array_equal(np.sort(members[mask[offs[p]:offs[p + 1]] == 1]), np.flatnonzero(in_core))
        # every galaxy closer than the margin to a core galaxy of p is in p
        cpos = pos[in_core]
        if len(cpos):
            d2 = ((pos[None, :, :] - cpos[:200, None, :]) ** 2).sum(-1)
            near = np.flatnonzero((d2 < margin * margin).any(0))
            assert np.isin(near, members).all()


def test_mock_suite_sizes_and_densities():
    pos, sh, w, offs, sides = synth.mock_suite(6, seed=9, grid=128, scale=0.01)
    n = np.diff(offs)
    assert len(n) == 6 and offs[-1] == len(pos) == len(sh) == len(w)
    full = n / 0.01
    assert np.all((full >= 5e5 * 0.999) & (full <= 5e6 * 1.001))
    assert np.all((sides >= 300 * 0.1) & (sides <= 900 * 0.1))
    for k in range(6):
        p = pos[offs[k]:offs[k + 1]]
        assert p.min() >= 0 and p.max() < sides[k]
    assert len(set(np.round(sides, 6))) == 6


def test_lognormal_convergence_is_skewed_zero_mean_and_scaled():
    kap = synth.lognormal_convergence(256, 200.0, seed=4, sigma_kappa=0.02, sigma_g=1.0)
    assert abs(kap.mean()) < 1e-12 and abs(kap.std() - 0.02) < 1e-12
    z = (kap - kap.mean()) / kap.std()
    assert (z ** 3).mean() > 1.0  # a Gaussian field has zero skewness
    assert kap.min() > -3 * kap.std()  # bounded below (long tail upwards)
    g1, g2 = synth.kaiser_squires_shear(kap, 200.0)
    assert np.isfinite(g1).all() and np.isfinite(g2).all()


def test_kaiser_squires_single_modes():
    """Flat-sky Kaiser-Squires on single Fourier modes of the convergence: a mode along x
    gives gamma_1 = kappa, gamma_2 = 0; along y gamma_1 = -kappa; along the diagonal
    gamma_1 = 0, gamma_2 = kappa (gamma = (k1^2 - k2^2 + 2 i k1 k2) / k^2 kappa in Fourier
    space); the mean of kappa carries no shear."""
    grid, side = 64, 30.0
    x = (np.arange(grid) * side / grid)[None, :]
    y = (np.arange(grid) * side / grid)[:, None]
    m = 3
    for kap, want1, want2 in (
            (np.cos(2 * np.pi * m * x / side) + 0 * y, 1.0, 0.0),
            (np.cos(2 * np.pi * m * y / side) + 0 * x, -1.0, 0.0),
            (np.cos(2 * np.pi * m * (x + y) / side), 0.0, 1.0)):
        g1, g2 = synth.kaiser_squires_shear(kap + 0.25, side)
        assert np.allclose(g1, want1 * kap, atol=2e-6)
        assert np.allclose(g2, want2 * kap, atol=2e-6)


def test_grf_shear_field_power_law_pure_e_mode_and_scale():
    """The GRF shear maps: pure E mode (inverse Kaiser-Squires gives no B-mode convergence),
    pixel rms of the convergence sigma_kappa (|gamma_hat| = |kappa_hat| away from l = 0, so
    <|gamma|^2> = sigma_kappa^2 by Parseval), and an azimuthally averaged power spectrum with
    the requested slope."""
    grid, side, slope, sk = 256, 100.0, -1.2, 0.02
    g1, g2 = synth.grf_shear_field(grid, side, 4, slope=slope, sigma_kappa=sk)
    gam = g1.astype(np.float64) + 1j * g2.astype(np.float64)
    assert abs(np.mean(np.abs(gam) ** 2) - sk * sk) < 1e-6 * sk * sk + 1e-12
    k = np.fft.fftfreq(grid, d=side / grid)
    k1, k2 = np.meshgrid(k, k, indexing="xy")
    ksq = k1 * k1 + k2 * k2
    nz = ksq > 0
    D = np.zeros(ksq.shape, dtype=np.complex128)
    D[nz] = ((k1[nz] ** 2 - k2[nz] ** 2) + 2j * k1[nz] * k2[nz]) / ksq[nz]
    kap = np.fft.ifft2(np.fft.fft2(gam) * np.conj(D))
    assert np.abs(kap.imag).max() < 1e-5 * np.abs(kap.real).max()
    p = np.abs(np.fft.fft2(kap.real)) ** 2
    kk = np.sqrt(ksq)
    bands = np.geomspace(4 / side, 0.3 * grid / side, 9)
    lk, lp = [], []
    for lo, hi in zip(bands[:-1], bands[1:]):
        sel = (kk >= lo) & (kk < hi)
        lk.append(np.log(np.sqrt(lo * hi)))
        lp.append(np.log(p[sel].mean()))
    fit = np.polyfit(lk, lp, 1)[0]
    assert abs(fit - slope) < 0.15, fit
