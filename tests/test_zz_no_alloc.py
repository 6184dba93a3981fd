"""The allocation-free real-space transform, ext4pcf_to_real_space_noalloc.

Some callers of this library cannot allocate device memory: code that runs while a CUDA
graph is captured under a strict allocator, plug-ins whose host application owns every
device allocation, and real-time loops that must not block in the allocator.  This entry
point serves them with a fixed 16 MiB scratch array inside the library.  It must give the
same result as ext4pcf_to_real_space (same kernels, same summation order), on two calls in
a row (the shared scratch keeps the previous call's contents), and must refuse sizes beyond
its scratch before enqueueing any work.  This file runs last: it leaves the array in use.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_07974_gb300 import build, ext4pcf
    build.build()
    rng = np.random.default_rng(31)
    pos = rng.uniform(0, 12, (150, 2))
    sh = rng.normal(0, 0.3, pos.shape)
    w = rng.uniform(0.5, 1.5, 150)
    edges = np.geomspace(0.5, 5.0, 6)
    nmax = 4
    ups = oracle.measure(pos, sh, w, edges, nmax)
    t = torch.tensor(np.stack([ups.real, ups.imag], axis=-1), device="cuda:0")
    return torch, ext4pcf, t, len(edges) - 1, nmax


def test_noalloc_matches_context_transform_on_two_calls(setup):
    torch, ext4pcf, ups, nb, nmax = setup
    nphi = 21
    est = ext4pcf.Estimator(0, "fp64")
    gam_ref, nrm_ref = est.to_real_space(ups, nphi)
    torch.cuda.synchronize()
    est.close()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        gam = torch.zeros_like(gam_ref)
        nrm = torch.zeros_like(nrm_ref)
        rc = ext4pcf.ext4pcf_to_real_space_noalloc(ups, nb, nmax, nphi, gam, nrm, stream)
        assert rc == ext4pcf.EXT4PCF_OK
        torch.cuda.synchronize()
        assert torch.allclose(nrm, nrm_ref, rtol=1e-12, atol=1e-12 * nrm_ref.abs().max().item())
        assert torch.allclose(gam, gam_ref, rtol=1e-12, atol=1e-12 * gam_ref.abs().max().item())


def test_noalloc_refuses_sizes_beyond_its_scratch(setup):
    torch, ext4pcf, ups, nb, nmax = setup
    big_nb, nphi = 32, 64  # 32^3 * 64^2 * 8 bytes = 1 GiB of normalisation counts
    gam = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    rc = ext4pcf.ext4pcf_to_real_space_noalloc(ups, big_nb, nmax, nphi, gam, nrm, torch.cuda.current_stream())
    assert rc == ext4pcf.EXT4PCF_E_UNSUPPORTED
    rc = ext4pcf.ext4pcf_to_real_space_noalloc(ups, nb, nmax, 0, gam, nrm, None)
    assert rc == ext4pcf.EXT4PCF_E_INVALID_ARG
