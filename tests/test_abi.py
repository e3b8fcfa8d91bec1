"""CPU-side checks of the C ABI: the library builds, loads, and exports every
function include/hdmd.h declares (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hdmd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_][a-z_0-9]*\s*\**\s*([a-z_][a-z_0-9]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2112_12271_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("create_system", "set_state", "get_state", "build_neighbors", "get_neighbors",
              "compute_forces", "md_steps", "fire_minimize", "swap_sweep", "destroy_system",
              "hdmd_last_error"):
        assert n in names, n


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_errors_without_gpu_are_reported_not_raised(libpath):
    # argument validation happens before any device work
    from paper_2112_12271_gb300 import hdmd
    lib = hdmd.lib()
    h = ctypes.c_void_p()
    pot = hdmd.potential(1.0, 0.3)
    import numpy as np
    diam = np.ones(10)
    st = lib.create_system(11, 10, 5.0, diam.ctypes.data, ctypes.byref(pot), 0, None, ctypes.byref(h))
    assert st == 8   # HDMD_E_UNSUPPORTED_D
    assert b"d must be" in lib.hdmd_last_error(None)
    st = lib.create_system(3, 10, 2.0, diam.ctypes.data, ctypes.byref(pot), 0, None, ctypes.byref(h))
    assert st == 1   # box not longer than twice the largest diameter
    assert b"box too small" in lib.hdmd_last_error(None)
    bad = diam.copy(); bad[3] = -1.0
    st = lib.create_system(3, 10, 9.0, bad.ctypes.data, ctypes.byref(pot), 0, None, ctypes.byref(h))
    assert st == 1
    bad_law = hdmd.potential(1.0, 0.3, law="morse", a=-1.0)
    st = lib.create_system(3, 10, 9.0, diam.ctypes.data, ctypes.byref(bad_law), 0, None, ctypes.byref(h))
    assert st == 1 and b"Morse stiffness" in lib.hdmd_last_error(None)
    assert lib.destroy_system(None) == 0


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2112_12271_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "hdmd_oracle" not in txt, f


def test_footprint_needs_no_gpu(libpath):
    from paper_2112_12271_gb300 import hdmd
    import numpy as np
    small = hdmd.system_footprint(6, 4096, 5.0, np.ones(4096))
    big = hdmd.system_footprint(6, 32768, 10.0, np.ones(32768))
    assert 0 < small < big
    with pytest.raises(hdmd.HDMDError):
        hdmd.system_footprint(3, 10, 2.0, np.ones(10))      # box too small


@pytest.mark.parametrize("case", [
    dict(d=1), dict(d=11), dict(N=1), dict(L=0.0), dict(L=float("inf")),
    dict(L=float("nan")), dict(diam_nan=True), dict(diam_zero=True), dict(eps=0.0),
    dict(skin=-0.1), dict(skin=float("nan")), dict(law="morse", a=0.0),
    dict(law="mie", n=0), dict(law="mie", n=25), dict(precision=7), dict(L=2.0),
])
def test_every_argument_rule_is_checked_without_a_gpu(libpath, case):
    """Each argument rule of create_system (same checks as system_footprint)
    answers HDMD_E_INVALID or HDMD_E_UNSUPPORTED_D with a message, before any
    device work."""
    from paper_2112_12271_gb300 import hdmd
    import numpy as np
    c = dict(d=3, N=10, L=9.0, eps=1.0, skin=0.3, precision=hdmd.HDMD_MIXED,
             law="harmonic", a=30.0, n=6)
    c.update(case)
    diam = np.ones(max(c["N"], 1))[: c["N"]]
    if c.pop("diam_nan", False):
        diam[2] = float("nan")
    if c.pop("diam_zero", False):
        diam[5] = 0.0
    with pytest.raises(hdmd.HDMDError) as e:
        hdmd.system_footprint(c["d"], c["N"], c["L"], diam, eps=c["eps"], skin=c["skin"],
                              precision=c["precision"], law=c["law"], a=c["a"], n=c["n"])
    assert e.value.status in (1, 8)
    assert len(str(e.value)) > 10


def test_footprint_grows_with_the_system(libpath):
    """Footprint: linear growth with N at a fixed density, FP64 systems no
    smaller than mixed ones, and the laws change no array sizes."""
    from paper_2112_12271_gb300 import hdmd
    import numpy as np
    base = [hdmd.system_footprint(4, N, 6.0 * (N / 4096) ** 0.25, np.ones(N)) for N in (4096, 8192, 16384)]
    assert base[0] < base[1] < base[2]
    assert 1.6 < base[2] / base[1] < 2.4
    s = np.ones(4096)
    mixed = hdmd.system_footprint(4, 4096, 6.0, s, precision=hdmd.HDMD_MIXED)
    fp64 = hdmd.system_footprint(4, 4096, 6.0, s, precision=hdmd.HDMD_FP64)
    assert fp64 >= mixed
    assert hdmd.system_footprint(4, 4096, 6.0, s, law="morse") == mixed


@pytest.mark.parametrize("args,status,text", [
    ((1, 100, 5.0, 1.0), 8, b"d must be"),
    ((11, 100, 5.0, 1.0), 8, b"d must be"),
    ((3, 1, 5.0, 1.0), 1, b"N must be"),
    ((3, 524289, 5.0, 1.0), 1, b"scratch limit"),
    ((3, 100, 0.0, 1.0), 1, b"positive and finite"),
    ((3, 100, 5.0, -1.0), 1, b"positive and finite"),
    ((3, 100, 5.0, 1.0), 1, b"NULL buffer"),
])
def test_noalloc_arguments_checked_before_device_work(libpath, args, status, text):
    """The allocation-free force call rejects bad sizes, its scratch limit
    (524,288 atoms) and missing buffers before it touches the device (NULL
    buffers here, so nothing could be launched)."""
    lib = ctypes.CDLL(libpath)
    f = lib.compute_forces_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    lib.hdmd_noalloc_last_error.restype = ctypes.c_char_p
    d, N, L, eps = args
    assert f(d, N, L, None, None, eps, None, None, None) == status
    assert text in lib.hdmd_noalloc_last_error()
