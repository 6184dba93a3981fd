"""Models, on the CPU, of two arguments the direct-estimator kernel (aperture.cu) rests on; the
kernel itself is compared with the oracle in tests/test_gpu_map_direct.py.

1. Coverage: the FP32 row and chord limits (cell units, relative to the aperture's cell,
   widened by a 1e-3-cell slack and the squared half-chord by 1e-6 (R/cell + 2)^2) scan every
   galaxy inside the 4 theta cut exactly once, for power-of-two cells chosen as the library
   chooses them, up to a cut radius of ~4096 cells.
2. Precision: per-galaxy terms formed in FP32 as the kernel forms them, summed in FP32 over
   32-galaxy partials and combined in FP64 with Newton's identities, stay within 1e-6 of
   |e_k| + p_2^{k/2} of the oracle's e_k (the GPU tests hold the kernel to 1e-5).
"""
import math

import numpy as np
import pytest

import oracle

f32 = np.float32


def _grid(pos, thetas):
    x0, y0 = pos[:, 0].min(), pos[:, 1].min()
    ext = max(pos[:, 0].max() - x0, pos[:, 1].max() - y0)
    target = max(0.5 * min(thetas), ext / 2048, 4 * max(thetas) / 2048)
    cell = math.ldexp(1.0, math.frexp(target)[1] - 1)
    ncx = int(math.floor((pos[:, 0].max() - x0) / cell)) + 1
    ncy = int(math.floor((pos[:, 1].max() - y0) / cell)) + 1
    cx = np.clip(np.floor((pos[:, 0] - x0) / cell).astype(int), 0, ncx - 1)
    cy = np.clip(np.floor((pos[:, 1] - y0) / cell).astype(int), 0, ncy - 1)
    order = np.argsort(cy * ncx + cx, kind="stable")
    start = np.searchsorted((cy * ncx + cx)[order], np.arange(ncx * ncy + 1))
    return x0, y0, cell, ncx, ncy, order, start


def _scanned(ax, ay, theta, x0, y0, cell, ncx, ncy, start):
    """Sorted indices the kernel's row/chord logic visits for one aperture (all splits)."""
    rc = f32(4.0 * theta / cell)
    rs = f32(rc + f32(1e-3))
    h2err = f32(f32(1e-6) * f32(rc + f32(2)) * f32(rc + f32(2)))
    mx = 4.0 * theta + 2.0 * cell
    if not (x0 - mx <= ax <= x0 + ncx * cell + mx and y0 - mx <= ay <= y0 + ncy * cell + mx):
        return np.zeros(0, dtype=int)
    acx, acy = math.floor((ax - x0) / cell), math.floor((ay - y0) / cell)
    ox, oy = f32(((ax - x0) - acx * cell) / cell), f32(((ay - y0) - acy * cell) / cell)
    ylo = max(acy + int(math.floor(f32(oy - rs))), 0)
    yhi = min(acy + int(math.floor(f32(oy + rs))), ncy - 1)
    seen = []
    for cyy in range(ylo, yhi + 1):
        k = f32(cyy - acy)
        dymin = max(f32(0), max(f32(k - oy), f32(oy - f32(k + f32(1)))))
        if dymin < rs:
            h2 = f32(float(rs) * float(rs) - float(f32(dymin * dymin)))  # fmaf: one rounding
            h = f32(f32(np.sqrt(f32(h2 + h2err))) + f32(1e-3))
            xl = max(acx + int(math.floor(f32(ox - h))), 0)
            xh = min(acx + int(math.floor(f32(ox + h))), ncx - 1)
            if xl <= xh:
                seen.extend(range(start[cyy * ncx + xl], start[cyy * ncx + xh + 1]))
    return np.array(seen, dtype=int)


@pytest.mark.parametrize("n,side,thetas,clustered", [
    (20000, 60.0, [0.7, 1.5, 3.0], False),
    (5000, 10.0, [0.05, 2.0], True),
    (40000, 100.0, [0.3, 255.0], False),   # cut radius ~4080 cells
])
def test_rows_and_chords_cover_the_cut_exactly_once(n, side, thetas, clustered):
    rng = np.random.default_rng(1)
    pos = rng.uniform(0, side, (n, 2))
    if clustered:
        pos[: n // 2] = rng.normal(side / 2, side / 50, (n // 2, 2))
    x0, y0, cell, ncx, ncy, order, start = _grid(pos, thetas)
    ps = pos[order]
    for theta in thetas:
        cen = np.vstack([rng.uniform(-4 * theta, side + 4 * theta, (12, 2)), [[x0, y0], [x0 + 3 * cell, y0]]])
        for ax, ay in cen:
            seen = _scanned(ax, ay, theta, x0, y0, cell, ncx, ncy, start)
            assert len(np.unique(seen)) == len(seen)
            d = ps - (ax, ay)
            inside = np.flatnonzero(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] < (4.0 * theta) ** 2)
            assert np.setdiff1d(inside, seen).size == 0


def _kernel_model(pos, sh, w, c, theta):
    R = 4.0 * theta
    d = pos - c
    ins = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] < R * R
    u = (d[ins, 0] / theta).astype(f32)
    v = (d[ins, 1] / theta).astype(f32)
    xr, xi = (w[ins] * sh[ins, 0]).astype(f32), (w[ins] * sh[ins, 1]).astype(f32)
    wf = w[ins].astype(f32)
    e = np.exp(f32(-0.5) * (u * u + v * v)).astype(f32)
    b = (-e * (xr * (u * u - v * v) + f32(2) * xi * u * v)).astype(f32)
    P = np.zeros(8)
    for s in range(0, b.size, 32):
        for k in range(4):
            P[k] += float(np.sum(b[s:s + 32] ** (k + 1), dtype=f32))
            P[4 + k] += float(np.sum(wf[s:s + 32] ** (k + 1), dtype=f32))
    cc = 1.0 / (4 * math.pi * theta * theta)

    def newton(p):
        e1 = p[1]
        e2 = (e1 * p[1] - p[2]) / 2
        e3 = (e2 * p[1] - e1 * p[2] + p[3]) / 3
        return e1, e2, (e3 * p[1] - e2 * p[2] + e1 * p[3] - p[4]) / 4

    a = newton([0, P[0] * cc, P[1] * cc ** 2, P[2] * cc ** 3, P[3] * cc ** 4])
    return np.array([*a, *newton([0, *P[4:]]), ins.sum()])


def test_fp32_terms_stay_well_inside_the_tolerance():
    import synth
    pos, sh, w = synth.grf_catalog(60000, 120.0, 5, grid=512)
    rng = np.random.default_rng(0)
    worst = 0.0
    for theta in (1.0, 4.0, 9.0):
        for c in rng.uniform(40, 80, (3, 2)):
            o = oracle.aperture_record(pos, sh, w, c, theta)
            g = _kernel_model(pos, sh, w, c, theta)
            assert g[6] == o[6]
            p2a, p2w = o[0] ** 2 - 2 * o[1], o[3] ** 2 - 2 * o[4]
            sc = np.array([math.sqrt(p2a), p2a, p2a ** 2, math.sqrt(p2w), p2w, p2w ** 2])
            worst = max(worst, float((np.abs(g[:6] - o[:6]) / (np.abs(o[:6]) + sc)).max()))
    assert worst < 1e-6


def test_model_constants_are_the_kernel_sources_constants():
    """The coverage model above restates the kernel's slack, half-chord widening, row and chord
    limits and the library's cell rule; a change to any of them in the CUDA sources fails here
    until the model follows."""
    import os
    import re
    csrc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2509_07974_gb300", "csrc")
    ap = open(os.path.join(csrc, "aperture.cu")).read()
    api = open(os.path.join(csrc, "api.cu")).read()
    assert re.search(r"constexpr float kSlack = 1e-3f;", ap)
    assert "const float Rs = A.rc + kSlack;" in ap
    assert "const float h2err = 1e-6f * (A.rc + 2.f) * (A.rc + 2.f);" in ap
    assert "const int ylo = max(acy + (int)floorf(oy - Rs), 0);" in ap
    assert "const int yhi = min(acy + (int)floorf(oy + Rs), A.ncy - 1);" in ap
    assert "const float dymin = fmaxf(0.f, fmaxf(k - oy, oy - (k + 1.f)));" in ap
    assert "const float h = sqrtf(fmaf(Rs, Rs, -dymin * dymin) + h2err) + kSlack;" in ap
    assert "const int xl = max(acx + (int)floorf(ox - h), 0);" in ap
    assert "const int xh = min(acx + (int)floorf(ox + h), A.ncx - 1);" in ap
    assert "std::fmax(0.5 * tmin, std::fmax(extent / 2048.0, 4.0 * tmax / 2048.0))" in api
    assert "cell = std::ldexp(1.0, ex - 1);" in api
    assert "A.rc = (float)(4.0 * theta / cat.cell);" in ap
