"""GPU parity at the benchmark sizes, in the configuration the benchmark times
(library-default lanes per atom, CUDA graphs):

* d = 6, N = 32768, L = 6 (the MD benchmark system): whole neighbour lists,
  forces, energy and virial against the oracle, FP64 and mixed; 100 steps of
  velocity Verlet against the oracle's trajectory; over one timed bench step
  (1000 steps) the energy error scales as dt^2 (FP64) and the mixed form
  conserves energy as well as the FP64 form up to its FP32 rounding floor;
* d = 6, N = 2^21 (the HBM-bound size): sampled atoms' lists and forces
  against the oracle's single-atom definitions, list symmetry and Newton's
  third law over the whole system;
* the paper's systems at d = 3..6 (N = 10^5): sampled lists and symmetry;
* the dimension-sweep systems (N = 65536, d = 4): a FIRE minimum checked by
  the oracle's forces, and one seeded SWAP sweep against the serial oracle.

Tolerances are those of test_gpu_parity: lists identical except pairs within
1e-6 of sigma_ij + skin; forces max|dF| <= tol max|F| with tol = 1e-12 (FP64)
and 1e-5 (mixed); 100-step positions within 1e-9 (FP64) and 1e-5 (mixed).
"""
import numpy as np
import pytest

import oracle
from paper_2112_12271_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TIE = 1e-6
SKIN = 0.3


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_12271_gb300 import build, hdmd
    build.build()
    oracle.build()
    return hdmd


@pytest.fixture(scope="module")
def c1():
    return W.c1_poly_d6(0)


@pytest.fixture(scope="module")
def c1_ref(c1):
    s = c1
    return dict(lists=oracle.neighbors_cells(s.x, s.sigma, s.L, SKIN),
                forces=oracle.forces(s.x, s.sigma, s.L,
                                     lists=oracle.neighbors_cells(s.x, s.sigma, s.L, 0.0)),
                md100=oracle.md_steps(s.x, s.v, s.sigma, s.L, 100, 0.005, skin=SKIN))


def _is_tie(x, sigma, L, i, j, skin=SKIN):
    dx = x[j] - x[i]
    dx -= L * np.round(dx / L)
    r = float(np.sqrt(dx @ dx))
    return abs(r - (0.5 * (sigma[i] + sigma[j]) + skin)) <= TIE


def _check_row(x, sigma, L, i, gpu_row, ref_row, skin=SKIN):
    for j in set(int(a) for a in gpu_row) ^ set(int(b) for b in ref_row):
        assert _is_tie(x, sigma, L, i, j, skin), (i, j)


def _rows(counts, idx):
    off = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
    return lambda i: idx[off[i]:off[i + 1]]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_c1_lists_forces_energy_virial(H, c1, c1_ref, prec):
    p, tol = (H.HDMD_FP64, 1e-12) if prec == "fp64" else (H.HDMD_MIXED, 1e-5)
    s = c1
    with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=p) as g:
        counts, idx = g.neighbors()
        F, E, Wv = g.forces()
    rc, ri = c1_ref["lists"]
    gr, rr = _rows(counts, idx), _rows(rc, ri)
    for i in np.nonzero((counts != rc))[0]:
        _check_row(s.x, s.sigma, s.L, i, gr(i), rr(i))
    same = np.nonzero(counts == rc)[0]
    for i in same[:: max(1, len(same) // 2000)]:
        _check_row(s.x, s.sigma, s.L, i, gr(i), rr(i))
    Fo, Eo, Wo = c1_ref["forces"]
    assert Eo > 0
    assert np.abs(F - Fo).max() <= tol * np.abs(Fo).max()
    assert E == pytest.approx(Eo, rel=tol)
    assert Wv == pytest.approx(Wo, rel=tol)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_c1_100_steps_match_oracle(H, c1, c1_ref, prec):
    p, tol = (H.HDMD_FP64, 1e-9) if prec == "fp64" else (H.HDMD_MIXED, 1e-5)
    s = c1
    ref = c1_ref["md100"]
    with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=p) as g:
        t = g.md_steps(100, 0.005)
        st = g.state()
    dx = st["x"] - ref["x"]
    dx -= s.L * np.round(dx / s.L)
    assert np.abs(dx).max() < tol, np.abs(dx).max()
    assert np.abs(st["v"] - ref["v"]).max() < 10 * tol
    assert t["E_pair"] == pytest.approx(ref["E"], rel=max(tol, 1e-11))
    assert t["K"] == pytest.approx(ref["K"], rel=max(tol, 1e-11))


def test_c1_bench_step_energy_error(H, c1, c1_ref):
    """One timed bench step is 1000 MD steps (t = 5).  The energy error of
    velocity Verlet at fixed t scales as dt^2: halving dt (2000 steps) divides
    the FP64 error by about 4.  The mixed form's error stays within twice the
    FP64 form's plus its FP32 rounding floor (1e-6 of E + K)."""
    s = c1
    H0 = c1_ref["forces"][1] + oracle.kinetic(s.v)
    err = {}
    for p, dt, n in ((H.HDMD_FP64, 0.005, 1000), (H.HDMD_FP64, 0.0025, 2000),
                     (H.HDMD_MIXED, 0.005, 1000)):
        with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=p) as g:
            t = g.md_steps(n, dt)
        err[(p, dt)] = abs(t["E_pair"] + t["K"] - H0)
    ratio = err[(H.HDMD_FP64, 0.005)] / err[(H.HDMD_FP64, 0.0025)]
    assert 2.5 < ratio < 6.5, (ratio, err)
    assert err[(H.HDMD_MIXED, 0.005)] <= 2.0 * err[(H.HDMD_FP64, 0.005)] + 1e-6 * abs(H0), err


def test_c1_large_sampled_lists_forces_and_symmetry(H):
    s = W.c1_poly_d6(0, N=2 ** 21)
    N = s.N
    with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=H.HDMD_MIXED) as g:
        counts, idx = g.neighbors()
        F, E, Wv = g.forces()
    rows = _rows(counts, idx)
    # j in list(i) <=> i in list(j), over the whole system
    ii = np.repeat(np.arange(N, dtype=np.int64), counts)
    jj = idx.astype(np.int64)
    assert np.array_equal(np.sort(ii * N + jj), np.sort(jj * N + ii))
    # Newton's third law: the pair forces cancel to FP32 rounding
    assert np.abs(F.sum(axis=0)).max() <= 1e-6 * np.abs(F).sum(axis=0).max()
    rng = np.random.default_rng(21)
    fmax = np.abs(F).max()
    for i in rng.choice(N, size=48, replace=False):
        _check_row(s.x, s.sigma, s.L, i, rows(i), oracle.neighbors_of(s.x, s.sigma, s.L, SKIN, i))
        Fi, _, _ = oracle.force_on(s.x, s.sigma, s.L, i)
        assert np.abs(F[i] - Fi).max() <= 1e-5 * fmax, i


@pytest.mark.parametrize("d", [3, 4, 5, 6])
def test_paper_model_sampled_lists_and_symmetry(H, d):
    """The paper's own systems (N = 10^5 at phi*_d, skin 0.25, Sec. III):
    13 (d = 5) and 24 (d = 6) atoms per subcell, so a stencil row spans
    several 32-wide chunks and the reach test drops whole subcells along the
    last axis; at d = 3, 4 (4 and 7 atoms per subcell) the build tests every
    home atom of a batch at once.  Sampled atoms' lists against the oracle's
    single-atom search, and list symmetry over the whole system."""
    skin = 0.25
    s = W.paper_model(d, 100000, seed=0)
    N = s.N
    with H.System(d, s.L, s.sigma, s.x, s.v, skin=skin, precision=H.HDMD_MIXED) as g:
        counts, idx = g.neighbors()
    rows = _rows(counts, idx)
    ii = np.repeat(np.arange(N, dtype=np.int64), counts)
    jj = idx.astype(np.int64)
    assert np.array_equal(np.sort(ii * N + jj), np.sort(jj * N + ii))
    rng = np.random.default_rng(100 + d)
    for i in rng.choice(N, size=128, replace=False):
        _check_row(s.x, s.sigma, s.L, i, rows(i),
                   oracle.neighbors_of(s.x, s.sigma, s.L, skin, i), skin)


def test_sweep_d4_fire_minimum_checked_by_oracle(H):
    s = W.c2_sweep(4, seed=0, N=65536)
    with H.System(s.d, s.L, s.sigma, s.x, precision=H.HDMD_MIXED) as g:
        r = g.fire(max_iter=200000)
        xs = g.state(v=False, img=False)["x"]
    assert r["converged"], r
    Fo, Eo, _ = oracle.forces(xs, s.sigma, s.L, lists=oracle.neighbors_cells(xs, s.sigma, s.L, 0.0))
    assert np.linalg.norm(Fo, axis=1).max() < 1e-10
    assert r["E_pair"] == pytest.approx(Eo, rel=1e-6, abs=1e-20)


def test_sweep_d4_seeded_swap_sweep_matches_serial_oracle(H):
    s = W.c2_sweep(4, seed=0, N=65536)
    T, seed = 1e-3, 7
    pairs, u = oracle.swap_draw(seed, 0, round(0.1 * s.N), s.N)
    ref = oracle.swap(s.x, s.sigma, s.L, T, pairs, u)
    assert 0 < ref["naccepted"] < len(pairs)
    with H.System(s.d, s.L, s.sigma, s.x, precision=H.HDMD_MIXED) as g:
        nacc, _ = g.swap(T, p=0.1, nsweeps=1, seed=seed)
        sig = g.state(sigma=True)["sigma"]
    assert nacc == ref["naccepted"]
    assert (sig == ref["sigma"]).all()
