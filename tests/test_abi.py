"""The C-ABI library builds, loads and exports every entry point that include/*.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names.update(re.findall(r"EXT4PCF_API\s+[\w\s\*]*?\b(ext4pcf_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2509_07974_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("ext4pcf_create", "ext4pcf_destroy", "ext4pcf_measure", "ext4pcf_to_real_space",
              "ext4pcf_to_map4", "ext4pcf_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_binding_names_match_the_abi():
    from paper_2509_07974_gb300 import ext4pcf
    for n in declared_symbols():
        assert callable(getattr(ext4pcf, n)), n


def test_struct_layouts_match_header():
    from paper_2509_07974_gb300 import ext4pcf
    # int, void*, int, int, int64, int64, int, int  (x86-64 / aarch64 LP64 alignment)
    assert ctypes.sizeof(ext4pcf.Config) == 48
    assert ctypes.sizeof(ext4pcf.Stats) == 9 * 8


def test_create_without_gpu_is_an_error_code(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_07974_gb300 import ext4pcf
    cfg = ext4pcf.Config(device=0, precision=0)
    with pytest.raises(ext4pcf.Ext4pcfError):
        ext4pcf.ext4pcf_create(cfg)
