"""The allocation-free force entry point (compute_forces_noalloc), for
callers that cannot allocate GPU memory (graph capture, host-framework memory
pools, allocation-free loops).  It is called through the C ABI with device
buffers the caller owns and compared with the regular compute_forces of a
system on the same positions, within the FP64 force tolerance of the other
parity tests (1e-12, relative to the largest force), on two calls in a row
that reuse the shared scratch array."""
import ctypes

import numpy as np
import pytest

from paper_2112_12271_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_12271_gb300 import build, hdmd
    path = build.build()
    lib = ctypes.CDLL(path)
    f = lib.compute_forces_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    lib.hdmd_noalloc_last_error.restype = ctypes.c_char_p
    return torch, hdmd, lib


def reference(hdmd, s):
    with hdmd.System(s.d, s.L, s.sigma, s.x, precision=hdmd.HDMD_FP64) as g:
        return g.forces()


def call_noalloc(torch, lib, s):
    x = torch.tensor(s.x, dtype=torch.float64, device="cuda").contiguous()
    sg = torch.tensor(s.sigma, dtype=torch.float64, device="cuda").contiguous()
    F = torch.empty_like(x)
    ew = torch.empty(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = lib.compute_forces_noalloc(s.d, s.N, s.L, x.data_ptr(), sg.data_ptr(), 1.0,
                                    F.data_ptr(), ew.data_ptr(), stream.cuda_stream)
    assert st == 0, lib.hdmd_noalloc_last_error()
    stream.synchronize()
    return F.cpu().numpy(), float(ew[0]), float(ew[1])


def test_noalloc_matches_compute_forces_twice(env):
    torch, hdmd, lib = env
    systems = [W.make_system(4, 3000, phi=0.4, dist="poly", T=0.0, seed=5),
               W.make_system(6, 2500, L=4.6, dist="poly", T=0.0, seed=6)]
    for s in systems:        # two calls in a row through the shared scratch
        F0, E0, W0 = reference(hdmd, s)
        F1, E1, W1 = call_noalloc(torch, lib, s)
        assert E0 > 0
        assert np.abs(F1 - F0).max() <= TOL * np.abs(F0).max()
        assert E1 == pytest.approx(E0, rel=TOL)
        assert W1 == pytest.approx(W0, rel=TOL)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, hdmd, lib = env
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    st = lib.compute_forces_noalloc(3, 524289, 10.0, p, p, 1.0, p, p, None)
    assert st == 1
    assert b"scratch limit" in lib.hdmd_noalloc_last_error()
