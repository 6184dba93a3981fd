"""GB300 (sm_103a) implementation of the multipole estimator of the shear four-point
correlation function (arXiv:2509.07974).

The compute path is the CUDA library ``libext4pcf.so`` (sources in ``csrc/``, C ABI in
``include/ext4pcf.h``); ``ext4pcf`` is its ctypes binding (the library is loaded on first
use) and ``build`` compiles it.
"""
from . import build, ext4pcf  # noqa: F401

__all__ = ["build", "ext4pcf"]
