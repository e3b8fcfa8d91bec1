"""The allocation-free force entry point (compute_forces_noalloc).

Some callers cannot allocate GPU memory at the moment they need forces: a
plug-in inside a host framework whose memory pool owns the device, or a loop
that must not allocate after start-up.  They call compute_forces_noalloc with
device buffers they own; its only scratch is a static device array.  Called
here through the C ABI, twice in a row on each system (the second call reuses
the scratch the first one left behind), and compared element by element with
the FP64 oracle's all-pairs forces, energy and virial (1e-12 relative to the
largest force, as in the other FP64 parity tests) and with the library's own
compute_forces of a system on the same positions."""
import ctypes

import numpy as np
import pytest

import oracle
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
    oracle.build()
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


def call_noalloc(torch, lib, d, x, sigma, L):
    x = torch.tensor(x, dtype=torch.float64, device="cuda").contiguous()
    sg = torch.tensor(sigma, dtype=torch.float64, device="cuda").contiguous()
    F = torch.full_like(x, np.nan)
    ew = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = lib.compute_forces_noalloc(d, x.shape[0], L, x.data_ptr(), sg.data_ptr(), 1.0,
                                    F.data_ptr(), ew.data_ptr(), stream.cuda_stream)
    assert st == 0, lib.hdmd_noalloc_last_error()
    stream.synchronize()
    return F.cpu().numpy(), float(ew[0]), float(ew[1])


def check(got, ref):
    F1, E1, W1 = got
    F0, E0, W0 = ref
    assert E0 > 0
    assert np.abs(F1 - F0).max() <= TOL * np.abs(F0).max()
    assert E1 == pytest.approx(E0, rel=TOL)
    assert W1 == pytest.approx(W0, rel=TOL)


# ragged N (not multiples of the 128-atom block), d from 2 to 10
SYSTEMS = [(2, 1001, dict(phi=0.7)), (3, 777, dict(phi=0.6)), (6, 1531, dict(L=4.2)),
           (10, 389, dict(L=2.6))]


@pytest.mark.parametrize("d,N,kw", SYSTEMS)
def test_noalloc_matches_oracle_twice(env, d, N, kw):
    torch, hdmd, lib = env
    s = W.make_system(d, N, dist="poly", T=0.0, seed=5 + d, **kw)
    assert s.L >= 2 * s.sigma.max()
    ref = oracle.forces(s.x, s.sigma, s.L)
    for _ in range(2):       # two calls in a row through the shared scratch
        check(call_noalloc(torch, lib, d, s.x, s.sigma, s.L), ref)


def test_noalloc_matches_compute_forces_twice(env):
    torch, hdmd, lib = env
    systems = [W.make_system(4, 3000, phi=0.4, dist="poly", T=0.0, seed=5),
               W.make_system(6, 2500, L=4.6, dist="poly", T=0.0, seed=6)]
    for s in systems:
        ref = reference(hdmd, s)
        for _ in range(2):
            check(call_noalloc(torch, lib, s.d, s.x, s.sigma, s.L), ref)


def test_noalloc_at_the_smallest_box(env):
    """At L = 2 sigma_max (the smallest box the call accepts) a pair still
    overlaps through one periodic image at most, the nearest, which is what
    the kernel evaluates: the count of overlapping images over all 3^d
    shifts is checked here, and the result against the oracle."""
    torch, hdmd, lib = env
    d, N = 3, 61
    rng = np.random.default_rng(11)
    sigma = rng.uniform(0.8, 1.2, N)
    L = 2.0 * sigma.max() * (1.0 + 1e-12)
    x = rng.uniform(-L / 2, L / 2, (N, d))
    shifts = np.array(np.meshgrid(*[[-1, 0, 1]] * d, indexing="ij")).reshape(d, -1).T * L
    dx = x[:, None, :] - x[None, :, :]
    dx -= L * np.round(dx / L)
    r = np.linalg.norm(dx[:, :, None, :] + shifts[None, None], axis=-1)
    sij = 0.5 * (sigma[:, None] + sigma[None, :])
    over = (r < sij[:, :, None]).sum(-1)
    np.fill_diagonal(over, 0)
    assert over.max() == 1 and over.sum() > N
    ref = oracle.forces(x, sigma, L)
    for _ in range(2):
        check(call_noalloc(torch, lib, d, x, sigma, L), ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, hdmd, lib = env
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    st = lib.compute_forces_noalloc(3, 524289, 10.0, p, p, 1.0, p, p, None)
    assert st == 1
    assert b"scratch limit" in lib.hdmd_noalloc_last_error()
