"""Edge cases of the GPU path against the oracle: the extreme dimensions
d = 2 and d = 10 through MD and FIRE, ragged N around the 64-atom padding,
positions on the box faces and far outside the box (wrapped with image
counts), coincident atoms (the force at r = 0 is 0), zero-step calls."""
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


@pytest.mark.parametrize("d,N,L", [(2, 400, 22.0), (10, 300, 3.0)])
def test_extreme_dimensions_md_and_fire(H, d, N, L):
    s = W.make_system(d, N, L=L, dist="poly", T=1e-2, seed=d)
    assert s.L > 2 * s.sigma.max()
    ref = oracle.md_steps(s.x, s.v, s.sigma, s.L, 50, 0.005)
    fref = oracle.fire(s.x, s.sigma, s.L, max_iter=30)
    assert oracle.forces(s.x, s.sigma, s.L)[1] > 0
    for prec, tol in ((H.HDMD_FP64, 1e-9), (H.HDMD_MIXED, 1e-5)):
        with H.System(d, s.L, s.sigma, s.x, s.v, precision=prec) as g:
            t = g.md_steps(50, 0.005)
            st = g.state()
        dx = st["x"] - ref["x"]
        dx -= s.L * np.round(dx / s.L)
        assert np.abs(dx).max() < tol, (d, prec)
        assert t["E_pair"] == pytest.approx(ref["E"], rel=max(tol, 1e-11), abs=1e-300)
    with H.System(d, s.L, s.sigma, s.x, precision=H.HDMD_FP64) as g:
        r = g.fire(max_iter=30)
        xs = g.state()["x"]
    assert r["iterations"] == fref["iters"] == 30
    dx = xs - fref["x"]
    dx -= s.L * np.round(dx / s.L)
    assert np.abs(dx).max() < 1e-10


@pytest.mark.parametrize("N", [2, 63, 64, 65, 127, 129])
def test_ragged_sizes(H, N):
    s = W.make_system(3, N, L=max(2.9, (N / 0.8) ** (1 / 3)), dist="poly", T=1e-2, seed=N)
    Fo, Eo, _ = oracle.forces(s.x, s.sigma, s.L)
    for lanes in (1, 4, 32):
        with H.System(3, s.L, s.sigma, s.x, s.v, precision=H.HDMD_FP64) as g:
            g.tune(lanes_per_atom=lanes)
            F, E, _ = g.forces()
        assert np.abs(F - Fo).max() <= 1e-12 * max(np.abs(Fo).max(), 1e-300)
        assert E == pytest.approx(Eo, rel=1e-12, abs=1e-300)


def test_box_faces_outside_positions_and_coincident_atoms(H):
    L, d = 6.0, 3
    x = np.array([[3.0, -3.0, 0.0],          # on the upper face: wraps to -L/2
                  [-3.0, 3.0, 0.1],
                  [15.2, -20.9, 7.7],         # several boxes away
                  [15.2, -20.9, 7.7],         # coincident with the previous atom
                  [0.0, 0.0, 0.0],
                  [0.3, 0.0, 0.0]])
    sigma = np.ones(len(x))
    xw = x - L * np.floor((x + 0.5 * L) / L)  # the same points inside the box
    Fo, Eo, _ = oracle.forces(xw, sigma, L)
    for prec in (H.HDMD_FP64, H.HDMD_MIXED):
        with H.System(d, L, sigma, x, precision=prec) as g:
            F, E, _ = g.forces()
            st = g.state()
        assert np.isfinite(F).all()
        assert np.abs(F - Fo).max() <= 1e-5 * np.abs(Fo).max()
        assert E == pytest.approx(Eo, rel=1e-5)
        assert np.all(st["x"] >= -0.5 * L) and np.all(st["x"] < 0.5 * L)
        assert np.abs(st["x"] + L * st["img"] - x).max() < 1e-12


def test_zero_step_calls(H):
    s = W.c0_bidisperse_d3()
    with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=H.HDMD_FP64) as g:
        t = g.md_steps(0, 0.005)
        r = g.fire(max_iter=0)
        st = g.state()
    Fo, Eo, _ = oracle.forces(s.x, s.sigma, s.L)
    assert t["E_pair"] == pytest.approx(Eo, rel=1e-12) and t["steps"] == 0
    assert r["iterations"] == 0 and r["E_pair"] == pytest.approx(Eo, rel=1e-12)
    assert np.abs(st["x"] - s.x).max() < 1e-12
