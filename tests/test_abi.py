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
    # int, void*, int, int, int64, int64, int, int, double, int, double  (LP64 alignment)
    assert ctypes.sizeof(ext4pcf.Config) == 72
    assert ctypes.sizeof(ext4pcf.Stats) == 10 * 8


def test_create_without_gpu_is_an_error_code(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_07974_gb300 import ext4pcf
    cfg = ext4pcf.Config(device=0, precision=0)
    with pytest.raises(ext4pcf.Ext4pcfError):
        ext4pcf.ext4pcf_create(cfg)


def test_aperture_lattice_stays_four_radii_inside():
    """Host-side aperture sampling of the direct estimator: a square lattice of the given
    spacing whose centres all lie at least 4 theta inside the field, centred in it."""
    import numpy as np
    from paper_2509_07974_gb300 import ext4pcf
    for field, theta, sp in (((0, 0, 60, 40), 1.3, 1.3), ((-5, 2, 30, 9), 0.5, 0.7), ((0, 0, 10, 10), 3.0, 1.0)):
        c = ext4pcf.aperture_lattice(field, theta, sp)
        if len(c) == 0:
            assert field[2] - field[0] < 8 * theta or field[3] - field[1] < 8 * theta
            continue
        assert c[:, 0].min() >= field[0] + 4 * theta - 1e-12 and c[:, 0].max() <= field[2] - 4 * theta + 1e-12
        assert c[:, 1].min() >= field[1] + 4 * theta - 1e-12 and c[:, 1].max() <= field[3] - 4 * theta + 1e-12
        xs, ys = np.unique(c[:, 0]), np.unique(c[:, 1])
        assert len(c) == len(xs) * len(ys)
        for a in (xs, ys):
            if len(a) > 1:
                np.testing.assert_allclose(np.diff(a), sp, rtol=1e-12)
        # no room for another lattice column or row
        assert (xs.max() - xs.min()) + sp > (field[2] - field[0]) - 8 * theta


def test_struct_offsets_match_the_c_compiler(tmp_path):
    """Every field of the binding's ctypes structs sits at the offset the C compiler gives the
    header's struct (and the sizes agree): a field added, dropped or reordered on one side
    fails here."""
    import shutil
    import subprocess
    from paper_2509_07974_gb300 import ext4pcf
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ext4pcf.h"', "int main(void) {"]
    for cname, cls in (("ext4pcf_config", ext4pcf.Config), ("ext4pcf_stats", ext4pcf.Stats)):
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        *key, val = line.split()
        got[tuple(key)] = int(val)
    for cname, cls in (("ext4pcf_config", ext4pcf.Config), ("ext4pcf_stats", ext4pcf.Stats)):
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_status_codes_and_precisions_match_the_header(tmp_path):
    """The binding's status codes and precision names carry the header's enum values."""
    import shutil
    import subprocess
    from paper_2509_07974_gb300 import ext4pcf
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    codes = [n for n in dir(ext4pcf) if re.fullmatch(r"EXT4PCF_(OK|E_\w+)", n)]
    prec = {"fp64": "EXT4PCF_FP64", "fp32": "EXT4PCF_FP32", "tf32": "EXT4PCF_TF32", "3xtf32": "EXT4PCF_3XTF32",
            "bf16x3": "EXT4PCF_SPLIT_BF16", "f16x3": "EXT4PCF_SPLIT_F16"}
    assert sorted(prec) == sorted(ext4pcf.PRECISION)
    body = ['  printf("%s %%d\\n", (int)%s);' % (n, n) for n in codes + sorted(prec.values())]
    src = tmp_path / "codes.c"
    src.write_text('#include <stdio.h>\n#include "ext4pcf.h"\nint main(void) {\n' + "\n".join(body)
                   + "\n  return 0;\n}\n")
    exe = tmp_path / "codes"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict((k, int(v)) for k, v in (line.split() for line in subprocess.run(
        [str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()))
    assert {"EXT4PCF_OK", "EXT4PCF_E_INVALID_ARG", "EXT4PCF_E_TIMEOUT"} <= set(codes)
    for n in codes:
        assert got[n] == getattr(ext4pcf, n), n
    for name, cname in prec.items():
        assert got[cname] == ext4pcf.PRECISION[name], name


def _prototypes():
    """{name: (return type, [argument declarations])} of every EXT4PCF_API function."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", " ", open(h).read(), flags=re.S)
        for m in re.finditer(r"EXT4PCF_API\s+([\w\s\*]*?)\b(ext4pcf_\w+)\s*\(([^;]*?)\)\s*;", src):
            args = [a.strip() for a in m.group(3).split(",") if a.strip() and a.strip() != "void"]
            out[m.group(2)] = (" ".join(m.group(1).split()), args)
    return out


def test_binding_argtypes_follow_the_prototypes(lib):
    """Every argument the binding declares has the width the C prototype gives it (int,
    int64_t, double, or a pointer), in the same number and order, and the return types agree:
    a scalar of the wrong width would pass garbage in the upper bits."""
    from paper_2509_07974_gb300 import ext4pcf
    bound = ext4pcf.load()
    protos = _prototypes()
    assert set(protos) == set(declared_symbols())
    scalar = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "double": ctypes.c_double}
    for name, (ret, args) in protos.items():
        fn = getattr(bound, name)
        assert fn.argtypes is not None and len(fn.argtypes) == len(args), name
        for decl, t in zip(args, fn.argtypes):
            if "*" in decl:
                assert t is ctypes.c_void_p or issubclass(t, ctypes._Pointer), (name, decl, t)
            else:
                base = decl.replace("const", "").split()[0]
                assert t is scalar[base], (name, decl, t)
        if ret == "int":
            assert fn.restype is ctypes.c_int, name
        else:
            assert "char" in ret and "*" in ret and fn.restype is ctypes.c_char_p, name
