"""GPU parity for the Mie law of Sec. II.A, truncated at sigma_ij and
shifted (n = 6 is WCA), with one eps and with volume-scaled prefactors:
forces, energy and virial (1e-12 FP64, 1e-5 mixed), 100 steps of MD
(1e-9 / 1e-5) and SWAP decisions, against the oracle under the same law."""
import numpy as np
import pytest

import oracle
from paper_2112_12271_gb300 import workloads as W
from test_gpu_morse import _start

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


@pytest.mark.parametrize("d,N,n,scale", [(3, 700, 6, False), (4, 900, 12, True), (6, 1200, 6, True)])
def test_forces_energy_virial(H, d, N, n, scale):
    s, x = _start(d, N, 50 + d, 0.02)
    with oracle.law("mie", n, eps_scale=scale):
        Fo, Eo, Wo = oracle.forces(x, s.sigma, s.L)
    assert Eo > 0
    for prec, tol in ((H.HDMD_FP64, 1e-12), (H.HDMD_MIXED, 1e-5)):
        with H.System(d, s.L, s.sigma, x, precision=prec, law="mie", n=n, eps_scale=scale) as g:
            F, E, Wv = g.forces()
        assert np.abs(F - Fo).max() <= tol * np.abs(Fo).max(), prec
        assert E == pytest.approx(Eo, rel=tol)
        assert Wv == pytest.approx(Wo, rel=tol)


def test_100_steps_and_swap_match_oracle(H):
    s, x0 = _start(3, 800, 61, 0.005)
    with oracle.law("mie", 6, eps_scale=True):
        ref = oracle.md_steps(x0, s.v, s.sigma, s.L, 100, 0.002, skin=0.25, mass=s.mass)
        pairs, u = W.swap_pairs(np.random.default_rng(5), s.N, s.N // 3)
        sref = oracle.swap(ref["x"], s.sigma, s.L, 0.25, pairs, u, mass=s.mass, v=ref["v"])
    assert 0 < sref["naccepted"] < len(pairs)
    for prec, tol in ((H.HDMD_FP64, 1e-9), (H.HDMD_MIXED, 1e-5)):
        with H.System(3, s.L, s.sigma, x0, s.v, s.mass, skin=0.25, precision=prec,
                      law="mie", n=6, eps_scale=True) as g:
            t = g.md_steps(100, 0.002)
            st = g.state()
            dx = st["x"] - ref["x"]
            dx -= s.L * np.round(dx / s.L)
            assert np.abs(dx).max() < tol, (prec, np.abs(dx).max())
            assert t["E_pair"] == pytest.approx(ref["E"], rel=max(tol, 1e-11))
            if prec == H.HDMD_FP64:
                g.set_state(ref["x"], ref["v"], s.mass)
                nacc, flags = g.swap(0.25, pairs=pairs, uniforms=u)
                assert nacc == sref["naccepted"]
                assert (flags == sref["accepted"]).all()
