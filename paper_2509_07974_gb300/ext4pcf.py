"""ctypes binding of libext4pcf (include/ext4pcf.h): argument marshalling only.

The functions ``ext4pcf_create``, ``ext4pcf_destroy``, ``ext4pcf_measure``,
``ext4pcf_to_real_space``, ``ext4pcf_to_map4``, ``ext4pcf_to_real_space_noalloc``,
``ext4pcf_map_direct``, ``ext4pcf_measure3``, ``ext4pcf_nth_order_components``, ``ext4pcf_nth_order_factors``,
``ext4pcf_contraction_tables``, ``ext4pcf_synchronize`` and ``ext4pcf_last_error`` mirror the C ABI one to one; pointer arguments accept torch tensors (device or host), numpy arrays, raw
integer addresses or None.  ``Estimator`` wraps them for torch users: it allocates outputs
and passes the current CUDA stream.  Every computation happens in the CUDA library; there
is no fallback, and loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libext4pcf.so")

EXT4PCF_OK = 0
EXT4PCF_E_INVALID_ARG = -1
EXT4PCF_E_OOM = -2
EXT4PCF_E_CUDA = -3
EXT4PCF_E_TIMEOUT = -4
EXT4PCF_E_UNSUPPORTED = -5

PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "3xtf32": 3, "bf16x3": 4, "f16x3": 5}


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("precision", ctypes.c_int),
                ("autotune", ctypes.c_int), ("workspace_bytes", ctypes.c_int64),
                ("timeout_cycles", ctypes.c_int64), ("deterministic", ctypes.c_int),
                ("wave_centres", ctypes.c_int), ("tree_delta1", ctypes.c_double), ("tree_levels", ctypes.c_int),
                ("tree_rmin", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int64), ("centres", ctypes.c_int64), ("waves", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("ms_grid", ctypes.c_double), ("ms_gather", ctypes.c_double),
                ("ms_contract", ctypes.c_double), ("ms_correct", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("wave_centres", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Ext4pcfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("ext4pcf error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libext4pcf.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libext4pcf.so not found at %s; run paper_2509_07974_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.ext4pcf_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Config)]
    lib.ext4pcf_destroy.argtypes = [P]
    lib.ext4pcf_measure.argtypes = [P, P, P, P, I64, P, I, I, P, I, P, P, P, ctypes.POINTER(Stats)]
    lib.ext4pcf_measure_batch.argtypes = [P, P, P, P, I64, P, I, I, P, I, P, I, P, P, P, ctypes.POINTER(Stats)]
    lib.ext4pcf_multipoles.argtypes = [P, P, P, P, I64, P, I, I, P, I64, P]
    lib.ext4pcf_to_real_space.argtypes = [P, P, I, I, I, P, P]
    lib.ext4pcf_to_map4.argtypes = [P, P, P, I, I, I, P, I, P, P, P, P]
    lib.ext4pcf_to_real_space_noalloc.argtypes = [P, I, I, I, P, P, P]
    lib.ext4pcf_to_real_space_noalloc.restype = I
    lib.ext4pcf_map_direct.argtypes = [P, P, P, P, I64, P, I, P, P, P, P]
    lib.ext4pcf_measure3.argtypes = [P, P, P, P, I64, P, I, I, P]
    lib.ext4pcf_measure3.restype = I
    lib.ext4pcf_nth_order_components.argtypes = [I, P, I]
    lib.ext4pcf_nth_order_factors.argtypes = [I, I, P, I]
    lib.ext4pcf_contraction_tables.argtypes = [I, P, I]
    for f in ("ext4pcf_nth_order_components", "ext4pcf_nth_order_factors", "ext4pcf_contraction_tables"):
        getattr(lib, f).restype = I
    lib.ext4pcf_synchronize.argtypes = [P]
    lib.ext4pcf_synchronize.restype = I
    lib.ext4pcf_last_error.argtypes = [P]
    lib.ext4pcf_last_error.restype = ctypes.c_char_p
    for f in ("ext4pcf_create", "ext4pcf_destroy", "ext4pcf_measure", "ext4pcf_measure_batch", "ext4pcf_multipoles",
              "ext4pcf_to_real_space",
              "ext4pcf_to_map4", "ext4pcf_map_direct"):
        getattr(lib, f).restype = I
    _lib = lib
    return lib


def _addr(x):
    """Address of a torch tensor / numpy array / int (None -> None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


# ---- the C ABI, one to one ------------------------------------------------------------
def ext4pcf_create(config: Config) -> int:
    lib = load()
    h = ctypes.c_void_p()
    rc = lib.ext4pcf_create(ctypes.byref(h), ctypes.byref(config))
    if rc != EXT4PCF_OK:
        raise Ext4pcfError(rc, "ext4pcf_create failed")
    return h.value


def ext4pcf_destroy(ctx: int) -> int:
    return load().ext4pcf_destroy(ctx)


def ext4pcf_synchronize(ctx: int) -> int:
    """Wait for the context's enqueued work; raises on a recorded failure (timeout, non-finite
    positions)."""
    return _check(ctx, load().ext4pcf_synchronize(ctx))


def ext4pcf_last_error(ctx: int) -> str:
    r = load().ext4pcf_last_error(ctx)
    return r.decode() if r else ""


def _check(ctx, rc):
    if rc != EXT4PCF_OK:
        raise Ext4pcfError(rc, ext4pcf_last_error(ctx))
    return rc


def ext4pcf_measure(ctx, positions, shears, weights, n_gal, radial_bins, n_bins, n_max,
                    cat_offsets=None, n_cat=1, centre_mask=None, upsilon=None, xi_acc=None,
                    stats: Stats | None = None) -> int:
    lib = load()
    rc = lib.ext4pcf_measure(ctx, _addr(positions), _addr(shears), _addr(weights), int(n_gal),
                             _addr(radial_bins), int(n_bins), int(n_max), _addr(cat_offsets),
                             int(n_cat), _addr(centre_mask), _addr(upsilon), _addr(xi_acc),
                             ctypes.byref(stats) if stats is not None else None)
    return _check(ctx, rc)


def ext4pcf_measure_batch(ctx, positions, shears, weights, n_gal, radial_bins, n_bins, n_max,
                          cat_offsets, n_cat, out_slot=None, n_out=0, centre_mask=None, upsilon=None,
                          xi_acc=None, stats: Stats | None = None) -> int:
    lib = load()
    rc = lib.ext4pcf_measure_batch(ctx, _addr(positions), _addr(shears), _addr(weights), int(n_gal),
                                   _addr(radial_bins), int(n_bins), int(n_max), _addr(cat_offsets),
                                   int(n_cat), _addr(out_slot), int(n_out), _addr(centre_mask),
                                   _addr(upsilon), _addr(xi_acc),
                                   ctypes.byref(stats) if stats is not None else None)
    return _check(ctx, rc)


def ext4pcf_multipoles(ctx, positions, shears, weights, n_gal, radial_bins, n_bins, n_max, centres,
                       n_centres, records) -> int:
    rc = load().ext4pcf_multipoles(ctx, _addr(positions), _addr(shears), _addr(weights), int(n_gal),
                                   _addr(radial_bins), int(n_bins), int(n_max), _addr(centres), int(n_centres),
                                   _addr(records))
    return _check(ctx, rc)


def record_layout(n_bins, n_max):
    """Offsets (complex elements) of the arrays of an ext4pcf_multipoles record:
    {'G': (offset, first n, count), 'W': ..., 'XX', 'XA', 'WW', 'TR'}, each [count][n_bins]."""
    N, nb = n_max, n_bins
    parts = [("G", -2 * N - 3, 4 * N + 3), ("W", 0, 2 * N + 1), ("XX", -2 * N - 6, 4 * N + 5),
             ("XA", 0, 2 * N + 3), ("WW", 0, 2 * N + 1), ("TR", 0, 5)]
    out, off = {}, 0
    for name, first, cnt in parts:
        out[name] = (off, first, cnt)
        off += cnt * nb
    out["rec"] = off
    return out


def ext4pcf_to_real_space(ctx, upsilon, n_bins, n_max, n_phi, gamma, norm) -> int:
    rc = load().ext4pcf_to_real_space(ctx, _addr(upsilon), int(n_bins), int(n_max), int(n_phi),
                                      _addr(gamma), _addr(norm))
    return _check(ctx, rc)


def ext4pcf_to_map4(ctx, upsilon, radial_bins, n_bins, n_max, n_phi, ap_radii, n_ap, xi_acc,
                    m4, map4_eb, map4_disc) -> int:
    rc = load().ext4pcf_to_map4(ctx, _addr(upsilon), _addr(radial_bins), int(n_bins), int(n_max),
                                int(n_phi), _addr(ap_radii), int(n_ap), _addr(xi_acc), _addr(m4),
                                _addr(map4_eb), _addr(map4_disc))
    return _check(ctx, rc)


def ext4pcf_to_real_space_noalloc(upsilon, n_bins, n_max, n_phi, gamma, norm, stream=None) -> int:
    """Allocation-free real-space transform (static 16 MiB device scratch, no context).
    Returns the ABI status code (0 on success); does not raise."""
    st = getattr(stream, "cuda_stream", stream)
    return load().ext4pcf_to_real_space_noalloc(_addr(upsilon), int(n_bins), int(n_max), int(n_phi),
                                                _addr(gamma), _addr(norm), st)


def ext4pcf_map_direct(ctx, positions, shears, weights, n_gal, thetas, n_theta, centres,
                       centre_offsets, ap_records, moments) -> int:
    rc = load().ext4pcf_map_direct(ctx, _addr(positions), _addr(shears), _addr(weights), int(n_gal),
                                   _addr(thetas), int(n_theta), _addr(centres), _addr(centre_offsets),
                                   _addr(ap_records), _addr(moments))
    return _check(ctx, rc)


def ext4pcf_measure3(ctx, positions, shears, weights, n_gal, radial_bins, n_bins, n_max, upsilon3) -> int:
    rc = load().ext4pcf_measure3(ctx, _addr(positions), _addr(shears), _addr(weights), int(n_gal),
                                 _addr(radial_bins), int(n_bins), int(n_max), _addr(upsilon3))
    return _check(ctx, rc)


def _host_table(rc):
    if rc < 0:
        raise Ext4pcfError(rc, "invalid argument")
    return rc


def ext4pcf_nth_order_components(order):
    """Sign matrix beta of the natural components of order N (host only): int32 [2^{N-1}][N]."""
    import numpy as np
    lib = load()
    n = _host_table(lib.ext4pcf_nth_order_components(int(order), None, 0))
    beta = np.zeros((n, int(order)), dtype=np.int32)
    _host_table(lib.ext4pcf_nth_order_components(int(order), beta.ctypes.data, beta.size))
    return beta


def ext4pcf_nth_order_factors(order, mu):
    """Factor table of component mu (-1: normalisation) at order N (host only): int32 array
    [sign, centre code, then per bin (array, conj, a_2 .. a_{N-1}, b)]."""
    import numpy as np
    lib = load()
    n = _host_table(lib.ext4pcf_nth_order_factors(int(order), int(mu), None, 0))
    t = np.zeros(n, dtype=np.int32)
    _host_table(lib.ext4pcf_nth_order_factors(int(order), int(mu), t.ctypes.data, t.size))
    return t


def ext4pcf_contraction_tables(which):
    """The 4PCF contraction kernels' own factor tables (0 CUDA-core, 1 tensor-core), int32 [9][17];
    which = 2: the Theta2 <-> Theta3 map of the reduced tensor-core contraction, int32 [9][2]
    (mu', o per component)."""
    import numpy as np
    lib = load()
    n = _host_table(lib.ext4pcf_contraction_tables(int(which), None, 0))
    t = np.zeros(n, dtype=np.int32)
    _host_table(lib.ext4pcf_contraction_tables(int(which), t.ctypes.data, t.size))
    return t.reshape(9, 2) if int(which) == 2 else t.reshape(9, 17)


def aperture_lattice(field, theta, spacing):
    """Aperture centres on a square lattice of the given spacing, at least 4 theta inside
    the rectangle field = (x_min, y_min, x_max, y_max), so that no aperture's cut disc leaves
    the field (float64 [n][2], possibly empty).  Host-side sampling only."""
    import numpy as np
    x0, y0, x1, y1 = (float(v) for v in field)
    m = 4.0 * theta
    axes = []
    for lo, hi in ((x0 + m, x1 - m), (y0 + m, y1 - m)):
        k = int(np.floor((hi - lo) / spacing + 1e-9)) + 1 if hi >= lo else 0
        axes.append(lo + 0.5 * ((hi - lo) - (k - 1) * spacing) + spacing * np.arange(k))
    gx, gy = np.meshgrid(axes[0], axes[1])
    return np.ascontiguousarray(np.stack([gx.ravel(), gy.ravel()], 1), dtype=np.float64)


# ---- torch convenience wrapper ---------------------------------------------------------
class Estimator:
    """One context on one device.  Inputs are torch tensors (float64); outputs are
    allocated as torch float64 tensors on the same device (complex values interleaved;
    ``as_complex`` gives a complex128 view)."""

    def __init__(self, device: int = 0, precision: str = "fp64", stream=None,
                 wave_centres: int = 0, autotune: bool = False, workspace_bytes: int = 0):
        import torch
        self.torch = torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        cfg = Config(device=device, stream=stream.cuda_stream, precision=PRECISION[precision],
                     autotune=1 if autotune else 0, workspace_bytes=int(workspace_bytes), timeout_cycles=0,
                     deterministic=1, wave_centres=wave_centres)
        self.ctx = ext4pcf_create(cfg)

    def close(self):
        if self.ctx:
            ext4pcf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def ups_shape(n_bins, n_max, n_cat=1):
        nn = 2 * n_max + 1
        return (n_cat, 9, nn, nn, n_bins, n_bins, n_bins, 2)

    def measure(self, positions, shears, weights, radial_bins, n_max, cat_offsets=None,
                centre_mask=None, upsilon=None, xi_acc=None, want_stats=False):
        torch = self.torch
        import numpy as np
        edges = np.ascontiguousarray(np.asarray(radial_bins, dtype=np.float64))
        nb = edges.size - 1
        n_gal = positions.shape[0]
        n_cat = 1
        offs = None
        if cat_offsets is not None:
            offs = np.ascontiguousarray(np.asarray(cat_offsets, dtype=np.int64))
            n_cat = offs.size - 1
        if upsilon is None:
            upsilon = torch.zeros(self.ups_shape(nb, n_max, n_cat), dtype=torch.float64,
                                  device=positions.device)
        st = Stats() if want_stats else None
        ext4pcf_measure(self.ctx, positions, shears, weights, n_gal, edges, nb, n_max, offs, n_cat,
                        centre_mask, upsilon, xi_acc, st)
        return (upsilon, st.as_dict()) if want_stats else upsilon

    def to_real_space(self, upsilon, n_phi):
        torch = self.torch
        nb = upsilon.shape[-2]
        n_max = (upsilon.shape[-5] - 1) // 2
        gamma = torch.zeros((8, nb, nb, nb, n_phi, n_phi, 2), dtype=torch.float64, device=upsilon.device)
        norm = torch.zeros((nb, nb, nb, n_phi, n_phi), dtype=torch.float64, device=upsilon.device)
        ext4pcf_to_real_space(self.ctx, upsilon, nb, n_max, n_phi, gamma, norm)
        return gamma, norm

    def to_map4(self, upsilon, radial_bins, n_phi, ap_radii, xi_acc=None):
        import numpy as np
        edges = np.ascontiguousarray(np.asarray(radial_bins, dtype=np.float64))
        nb = edges.size - 1
        n_max = (upsilon.shape[-5] - 1) // 2
        ap = np.ascontiguousarray(np.asarray(ap_radii, dtype=np.float64))
        n_ap = ap.size
        m4 = np.zeros((n_ap, 8, 2))
        eb = np.zeros((n_ap, 16))
        disc = np.zeros((n_ap, 16))
        xi = xi_acc
        if xi is not None and not hasattr(xi, "data_ptr"):
            xi = np.ascontiguousarray(np.asarray(xi, dtype=np.float64))
        ext4pcf_to_map4(self.ctx, upsilon, edges, nb, n_max, n_phi, ap, n_ap, xi, m4, eb, disc)
        return m4[..., 0] + 1j * m4[..., 1], eb, disc

    def map_direct(self, positions, shears, weights, thetas, centres, moments=None,
                   want_records=False):
        """Direct <M_ap^2>, <M_ap^4> estimator.  ``centres`` is a list (one per radius) of [n][2]
        arrays (numpy or torch).  Returns (moments [n_theta][8], records [sum n][8] or None) as
        torch float64 tensors on the catalogue's device."""
        torch = self.torch
        import numpy as np
        th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64)).ravel()
        cen = [torch.as_tensor(c, dtype=torch.float64).reshape(-1, 2) for c in centres]
        offs = np.zeros(th.size + 1, dtype=np.int64)
        offs[1:] = np.cumsum([c.shape[0] for c in cen])
        dev = positions.device
        cen_all = (torch.cat(cen) if cen else torch.zeros((0, 2), dtype=torch.float64)).to(dev).contiguous()
        if moments is None:
            moments = torch.zeros((th.size, 8), dtype=torch.float64, device=dev)
        rec = torch.zeros((int(offs[-1]), 8), dtype=torch.float64, device=dev) if want_records else None
        ext4pcf_map_direct(self.ctx, positions, shears, weights, positions.shape[0], th, th.size,
                           cen_all if offs[-1] > 0 else None, offs, rec, moments)
        return moments, rec


def as_complex(t):
    """complex128 view of an interleaved float64 tensor (last axis 2)."""
    import torch
    return torch.view_as_complex(t)
