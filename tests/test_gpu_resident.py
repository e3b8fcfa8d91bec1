"""GPU tests of the resident MD kernel (one cooperative launch runs the steps
between list builds, Sec. II.B-II.C): its NVE trajectories equal those of one
kernel launch per step bit for bit (same pair loop, same kick and drift
arithmetic, same rebuild steps), through CUDA graphs and eagerly; with masses
and the Morse law too; its NVT and NVE trajectories follow the FP64 oracle
within the mixed-precision tolerance of the other parity tests."""
import numpy as np
import pytest

import oracle
from paper_2112_12271_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_12271_gb300 import build, hdmd
    build.build()
    oracle.build()
    return hdmd


def run(H, s, nsteps, resident, graphs=1, mass=None, law=None, pieces=None, **kw):
    args = dict(law) if law else {}
    with H.System(s.d, s.L, s.sigma, s.x, s.v, mass, precision=H.HDMD_MIXED, **args, **kw) as g:
        g.tune(use_graphs=graphs)
        g.resident(resident)
        info = g.info()
        rebuilds = 0
        for n in (pieces or (nsteps,)):
            t = g.md_steps(n, 0.005)
            rebuilds += t["rebuilds"]
        return g.state(), t, rebuilds, info


@pytest.mark.parametrize("d,N,kw", [(6, 32768, dict(L=6.0)), (3, 1000, dict(phi=0.6)),
                                    (4, 5000, dict(phi=0.3)), (2, 777, dict(phi=0.7))])
def test_resident_equals_one_launch_per_step_bitwise(H, d, N, kw):
    s = W.make_system(d, N, dist="poly", T=0.02, seed=60 + d, **kw)
    a = run(H, s, 300, resident=False)
    b = run(H, s, 300, resident=True)
    c = run(H, s, 300, resident=True, graphs=0)
    assert a[3]["resident"] == 0 and b[3]["resident"] > 0
    assert a[2] >= 3, a[2]                               # several list builds in the run
    for other in (b, c):
        assert other[2] == a[2]
        assert np.array_equal(other[0]["x"], a[0]["x"])
        assert np.array_equal(other[0]["v"], a[0]["v"])
        assert other[1]["E_pair"] == a[1]["E_pair"]


def test_resident_with_masses_and_morse_bitwise(H):
    """The paper's model (Morse law, prefactors and masses sigma^d) at d = 4,
    from a relaxed start: resident and per-step launches agree bit for bit."""
    import dataclasses
    s = W.paper_model(4, 4000, seed=5)
    with H.System(4, s.L, s.sigma, s.x, precision=H.HDMD_MIXED) as g:
        g.fire(max_iter=20000)
        x0 = g.state(v=False, img=False)["x"]
    s0 = dataclasses.replace(s, x=x0)
    law = dict(skin=0.25, law="morse", a=W.MORSE_A, eps_scale=True)
    a = run(H, s0, 400, resident=False, mass=s.mass, law=law)
    b = run(H, s0, 400, resident=True, mass=s.mass, law=law)
    assert b[3]["resident"] > 0
    assert b[2] == a[2] >= 1
    assert np.array_equal(b[0]["x"], a[0]["x"]) and np.array_equal(b[0]["v"], a[0]["v"])


@pytest.mark.parametrize("d,N,kw", [(3, 2000, dict(phi=0.6)), (6, 4000, dict(L=5.0))])
def test_resident_nve_and_nvt_follow_oracle(H, d, N, kw):
    """100 steps against the FP64 oracle (1e-5 of positions, E and K
    relative), NVE and Berendsen NVT; in pieces of 37 + 63 steps, so that
    the resident launches start from a state left by an earlier call."""
    s = W.make_system(d, N, dist="poly", T=1e-3, seed=70 + d, **kw)
    for tau in (0.0, 0.05):
        ref = oracle.md_steps(s.x, s.v, s.sigma, s.L, 100, 0.005, T_target=2e-3 if tau else 0.0,
                              tau=tau)
        with H.System(d, s.L, s.sigma, s.x, s.v, precision=H.HDMD_MIXED) as g:
            assert g.info()["resident"] > 0
            if tau:
                g.thermostat(2e-3, tau)
            g.md_steps(37, 0.005)
            t = g.md_steps(63, 0.005)
            st = g.state()
        dx = st["x"] - ref["x"]
        dx -= s.L * np.round(dx / s.L)
        assert np.abs(dx).max() < 1e-5, (tau, np.abs(dx).max())
        assert t["E_pair"] == pytest.approx(ref["E"], rel=1e-5)
        assert t["K"] == pytest.approx(ref["K"], rel=1e-5)


def test_resident_not_used_where_it_does_not_apply(H):
    s = W.make_system(3, 1000, phi=0.6, dist="poly", T=1e-3, seed=3)
    with H.System(3, s.L, s.sigma, s.x, s.v, precision=H.HDMD_FP64) as g:
        assert g.info()["resident"] == 0          # FP64 pair forces
    with H.System(3, s.L, s.sigma, s.x, s.v, precision=H.HDMD_MIXED) as g:
        assert g.info()["resident"] > 0
        g.rebuild_rule("paper", 5)
        assert g.info()["resident"] == 0          # the paper's rebuild rule
