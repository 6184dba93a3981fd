"""Host-side failure paths of the C ABI.  Faults are injected on the host only
(EXT4PCF_FAULT=alloc|arg); no kernel is made to fault, trap or hang."""
import numpy as np
import pytest


def test_alloc_fault_on_create_is_an_oom_code(monkeypatch):
    """EXT4PCF_FAULT=alloc makes ext4pcf_create report a failed device allocation before it
    touches any device, so this runs without a GPU."""
    from paper_2509_07974_gb300 import build, ext4pcf
    build.build()
    monkeypatch.setenv("EXT4PCF_FAULT", "alloc")
    with pytest.raises(ext4pcf.Ext4pcfError) as e:
        ext4pcf.ext4pcf_create(ext4pcf.Config(device=0, precision=0))
    assert e.value.code == ext4pcf.EXT4PCF_E_OOM


def test_invalid_precision_is_refused_without_a_device():
    from paper_2509_07974_gb300 import build, ext4pcf
    build.build()
    with pytest.raises(ext4pcf.Ext4pcfError) as e:
        ext4pcf.ext4pcf_create(ext4pcf.Config(device=0, precision=99))
    assert e.value.code in (ext4pcf.EXT4PCF_E_INVALID_ARG, ext4pcf.EXT4PCF_E_UNSUPPORTED)


@pytest.mark.gpu
def test_arg_fault_on_measure_leaves_the_context_usable(monkeypatch):
    """EXT4PCF_FAULT=arg makes ext4pcf_measure fail its argument check with a message; the
    same context then measures normally once the variable is gone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_07974_gb300 import build, ext4pcf
    build.build()
    rng = np.random.default_rng(4)
    dev = torch.device("cuda:0")
    pos = torch.tensor(rng.uniform(0, 5, (50, 2)), device=dev)
    sh = torch.tensor(rng.normal(0, 0.3, (50, 2)), device=dev)
    w = torch.ones(50, dtype=torch.float64, device=dev)
    edges = np.array([0.5, 1.0, 2.0])
    est = ext4pcf.Estimator(0, "fp64")
    ups = torch.zeros(ext4pcf.Estimator.ups_shape(2, 2), dtype=torch.float64, device=dev)
    monkeypatch.setenv("EXT4PCF_FAULT", "arg")
    with pytest.raises(ext4pcf.Ext4pcfError) as e:
        ext4pcf.ext4pcf_measure(est.ctx, pos, sh, w, 50, edges, 2, 2, None, 1, None, ups, None)
    assert e.value.code == ext4pcf.EXT4PCF_E_INVALID_ARG
    assert "fault injection" in ext4pcf.ext4pcf_last_error(est.ctx)
    assert float(ups.abs().max()) == 0.0
    monkeypatch.delenv("EXT4PCF_FAULT")
    ext4pcf.ext4pcf_measure(est.ctx, pos, sh, w, 50, edges, 2, 2, None, 1, None, ups, None)
    torch.cuda.synchronize()
    assert float(ups.abs().max()) > 0.0
    est.close()
