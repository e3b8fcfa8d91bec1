"""GPU parity of the Berendsen thermostat (NVT) fused into the second kick:
against the oracle's NVT trajectory (same tolerances as the NVE one: 1e-9
FP64, 1e-5 mixed over 100 steps), against the closed-form relaxation of an
ideal gas, and, for the paper's model, the temperature it holds."""
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


def test_nvt_trajectory_matches_oracle(H):
    s = W.c0_bidisperse_d3()
    Tt, tau = 5e-3, 0.05
    ref = oracle.md_steps(s.x, s.v, s.sigma, s.L, 100, 0.005, T_target=Tt, tau=tau)
    for prec, tol in ((H.HDMD_FP64, 1e-9), (H.HDMD_MIXED, 1e-5)):
        with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=prec) as g:
            g.thermostat(Tt, tau)
            t = g.md_steps(100, 0.005)
            st = g.state()
        dx = st["x"] - ref["x"]
        dx -= s.L * np.round(dx / s.L)
        assert np.abs(dx).max() < tol, (prec, np.abs(dx).max())
        assert np.abs(st["v"] - ref["v"]).max() < 10 * tol
        assert t["K"] == pytest.approx(ref["K"], rel=max(tol, 1e-11))
        assert t["E_pair"] == pytest.approx(ref["E"], rel=max(tol, 1e-11))


def test_nvt_in_pieces_equals_one_call(H):
    s = W.make_system(4, 1200, phi=0.4, dist="poly", T=1e-2, seed=3)
    outs = []
    for pieces in ((90,), (17, 73)):
        with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=H.HDMD_FP64) as g:
            g.thermostat(0.05, 0.02)
            for n in pieces:
                g.md_steps(n, 0.005)
            outs.append(g.state())
    assert np.abs(outs[0]["x"] - outs[1]["x"]).max() < 1e-12


def test_ideal_gas_relaxes_in_closed_form(H):
    rng = np.random.default_rng(3)
    d, N, L = 3, 400, 6.0
    x = W.uniform_positions(rng, N, d, L)
    v = W.thermal_velocities(rng, N, d, 0.7)
    sigma = np.full(N, 1e-3)
    dt, tau, Tt = 0.005, 0.1, 0.25
    for n in (1, 7, 40):
        with H.System(d, L, sigma, x, v, skin=2.0, precision=H.HDMD_MIXED) as g:
            g.thermostat(Tt, tau)
            t = g.md_steps(n, dt)
        assert t["T"] - Tt == pytest.approx((0.7 - Tt) * (1 - dt / tau) ** n, rel=1e-9)


def test_paper_model_holds_its_temperature(H):
    """The paper's runs are NVT at T = 0.25 (Sec. III): started at T = 0.5,
    the Morse liquid at phi*_3 settles to a mean kinetic temperature within
    3 % of the target over time units 5-10."""
    s = W.paper_model(3, 8000, T=0.5, seed=9)
    with H.System(3, s.L, s.sigma, s.x, precision=H.HDMD_MIXED) as g:
        g.fire(max_iter=20000)
        x0 = g.state(v=False, img=False)["x"]
    per_tau = int(round(1.0 / W.PAPER_DT))
    with H.System(3, s.L, s.sigma, x0, s.v, s.mass, skin=0.25, precision=H.HDMD_MIXED,
                  law="morse", a=W.MORSE_A, eps_scale=True) as g:
        g.thermostat(W.PAPER_T, 0.1)
        g.md_steps(5 * per_tau, W.PAPER_DT)
        Ts = [g.md_steps(per_tau // 5, W.PAPER_DT)["T"] for _ in range(25)]
    assert np.mean(Ts) == pytest.approx(W.PAPER_T, rel=0.03)
