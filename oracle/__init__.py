"""FP64 CPU oracle for the shear 4PCF multipole estimator (arXiv:2509.07974).

TEST INFRASTRUCTURE ONLY.  The product library never imports, links or calls this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
use it.  The C source (``oracle4pcf.c``) follows the paper's equations step by step; this
module builds it with gcc and wraps it with ctypes, returning numpy arrays.

Layouts (numpy, complex128 unless stated):
    upsilon  [9, 2N+1, 2N+1, nb, nb, nb]   mu = 0..7 natural components, mu = 8 the
                                            normalisation; axes 1, 2 are n2+N, n3+N.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle4pcf.c")
_LIB_PATH = os.path.join(_HERE, "liboracle4pcf.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction) into liboracle4pcf.so."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC[:-1] + "h")):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int
            lib.o4_measure.argtypes = [i64, P, P, P, P, i32, i32, P, i32, i32, P, P]
            lib.o4_bruteforce.argtypes = [i64, P, P, P, P, i32, i32, P, i32, P]
            lib.o4_to_real_space.argtypes = [P, i32, i32, i32, P, P]
            lib.o4_map4_filter.argtypes = [i32, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, P]
            lib.o4_map4_filter.restype = None
            lib.o4_map4.argtypes = [P, P, i32, i32, i32, P, i32, P, P, P, P]
            lib.o4_eb_from_m4.argtypes = [P, P]
            lib.o4_eb_from_m4.restype = None
            for f in ("o4_measure", "o4_bruteforce", "o4_to_real_space", "o4_map4"):
                getattr(lib, f).restype = i32
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def ups_shape(nb: int, nmax: int):
    return (9, 2 * nmax + 1, 2 * nmax + 1, nb, nb, nb)


def measure(pos, shear, w, edges, nmax, centre_mask=None, corrections=True, n_threads=0,
            with_xi=False):
    """Factorised estimator (paper Sect. 3.1 + App. A.1).  Returns upsilon (and the
    xi accumulators [nb, 3] complex when with_xi)."""
    lib = _load()
    pos = _f64(pos)
    n = pos.shape[0] if pos.size else 0
    pos = pos.reshape(n, 2)
    shear = _f64(shear).reshape(n, 2)
    w = _f64(w).reshape(n)
    edges = _f64(edges)
    nb = edges.size - 1
    out = np.zeros(ups_shape(nb, nmax), dtype=np.complex128)
    xi = np.zeros((nb, 3), dtype=np.complex128) if with_xi else None
    mask = None
    if centre_mask is not None:
        mask = np.ascontiguousarray(centre_mask, dtype=np.uint8).reshape(n)
    rc = lib.o4_measure(n, _ptr(pos), _ptr(shear), _ptr(w), _ptr(edges), nb, nmax, _ptr(mask),
                        1 if corrections else 0, int(n_threads), _ptr(out), _ptr(xi))
    if rc != 0:
        raise ValueError("o4_measure failed (%d)" % rc)
    return (out, xi) if with_xi else out


def bruteforce(pos, shear, w, edges, nmax, centre_mask=None, distinct=True):
    """O(N^4) sum over quadruplets of the definition (Eq. QuadrupletUpsilon / TripletNorm
    on the multipole basis)."""
    lib = _load()
    pos = _f64(pos)
    n = pos.shape[0]
    pos = pos.reshape(n, 2)
    shear = _f64(shear).reshape(n, 2)
    w = _f64(w).reshape(n)
    edges = _f64(edges)
    nb = edges.size - 1
    out = np.zeros(ups_shape(nb, nmax), dtype=np.complex128)
    mask = None
    if centre_mask is not None:
        mask = np.ascontiguousarray(centre_mask, dtype=np.uint8).reshape(n)
    rc = lib.o4_bruteforce(n, _ptr(pos), _ptr(shear), _ptr(w), _ptr(edges), nb, nmax,
                           _ptr(mask), 1 if distinct else 0, _ptr(out))
    if rc != 0:
        raise ValueError("o4_bruteforce failed (%d)" % rc)
    return out


def to_real_space(ups, nphi):
    """Multipoles -> bin-integrated real space.  Returns (gamma [8,nb,nb,nb,nphi,nphi]
    complex, norm [nb,nb,nb,nphi,nphi] real)."""
    lib = _load()
    ups = np.ascontiguousarray(ups, dtype=np.complex128)
    nb = ups.shape[3]
    nmax = (ups.shape[1] - 1) // 2
    gam = np.zeros((8, nb, nb, nb, nphi, nphi), dtype=np.complex128)
    nrm = np.zeros((nb, nb, nb, nphi, nphi), dtype=np.float64)
    rc = lib.o4_to_real_space(_ptr(ups), nb, nmax, nphi, _ptr(gam), _ptr(nrm))
    if rc != 0:
        raise ValueError("o4_to_real_space failed (%d)" % rc)
    return gam, nrm


def map4_filter(mu, theta, t1, t2, t3, phi12, phi13):
    """F_mu of Eq. 4PCF2M4 (Crittenden filter), Jacobian included."""
    lib = _load()
    out = np.zeros(2)
    lib.o4_map4_filter(int(mu), float(theta), float(t1), float(t2), float(t3), float(phi12),
                       float(phi13), _ptr(out))
    return complex(out[0], out[1])


def eb_from_m4(m4):
    lib = _load()
    m4 = np.ascontiguousarray(m4, dtype=np.complex128).reshape(8)
    out = np.zeros(16)
    lib.o4_eb_from_m4(_ptr(m4), _ptr(out))
    return out


def map4(ups, edges, nphi, ap_radii, xi_pm=None):
    """Fourth-order aperture statistics.  Returns (m4 [n_ap,8] complex, map4 [n_ap,16],
    disc [n_ap,16])."""
    lib = _load()
    ups = np.ascontiguousarray(ups, dtype=np.complex128)
    nb = ups.shape[3]
    nmax = (ups.shape[1] - 1) // 2
    edges = _f64(edges)
    ap = _f64(ap_radii)
    n_ap = ap.size
    m4 = np.zeros((n_ap, 8), dtype=np.complex128)
    eb = np.zeros((n_ap, 16))
    disc = np.zeros((n_ap, 16))
    xi = None if xi_pm is None else _f64(xi_pm).reshape(nb, 4)
    rc = lib.o4_map4(_ptr(ups), _ptr(edges), nb, nmax, nphi, _ptr(ap), n_ap, _ptr(xi),
                     _ptr(m4), _ptr(eb), _ptr(disc))
    if rc != 0:
        raise ValueError("o4_map4 failed (%d)" % rc)
    return m4, eb, disc


def xi_from_acc(xi_acc):
    """xi_+ and xi_- per radial bin from the accumulators of measure(with_xi=True):
    xi_+ = sum x_i^* G_0 / sum w_i W_0, xi_- = sum x_i G_-4 / sum w_i W_0.
    Returns [nb, 4] = (xi+ re, im, xi- re, im)."""
    acc = np.asarray(xi_acc).reshape(-1, 3)
    den = acc[:, 2].real
    safe = np.where(den != 0, den, 1.0)
    xp = np.where(den != 0, acc[:, 0] / safe, 0)
    xm = np.where(den != 0, acc[:, 1] / safe, 0)
    return np.stack([xp.real, xp.imag, xm.real, xm.imag], axis=1)


# direct estimator of <M_ap^2> and <M_ap^4> (Sect. 5.2, Eq. MapDirectEstimator); numpy only
from .map_direct import (aperture_record, crittenden_q, elementary_symmetric,  # noqa: E402
                         map_direct, moments_from_records, tangential_shear)

# N-th order natural components and multipoles by brute force (App. F); numpy only
from .nth_order import beta_matrix, bruteforce_multipoles  # noqa: E402

# tree approximation of the neighbour multipoles (Sect. 3.2, App. F.3); numpy only
from .tree import bin_levels, neighbour_multipoles, reduced_catalogue, upsilon0_from_multipoles  # noqa: E402

# symmetry-reduced storage of the multipoles (Table tab:4PCFSymm); numpy only
from . import symmetry  # noqa: E402
