"""The list build's FP32 pair test against the bound that widens its guard
band (CPU).

For n_cell >= 3 the kernel decides r^2 < (rho_j + rho_h)^2 from
  diff = (|r_j|^2 - rho_j^2) + (|x_h|^2 - rho_h^2) - 2 (r_j . x_h + rho_j rho_h)
in FP32 and hands pairs with |diff| inside the guard band to FP64.  The band
is widened by (d + 3)(4d + 1) 2u L_sc^2, twice the rounding bound of that
expression for cell-relative coordinates |x_hk| <= L_sc/2, |r_jk| <= 3 L_sc/2
and rho_j + rho_h <= L_sc.  Here the kernel's operation order is replayed in
FP32 (each fused multiply-add rounded once: the product of two FP32 values
is exact in FP64) on random and extreme inputs, and the error against the
exact value of the same FP32 inputs stays below that widening."""
import numpy as np
import pytest

f32 = np.float32


def fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def expanded_diff(xh, rj, rhoj, rh):
    D = xh.shape[1]
    Aj = (-(rhoj * rhoj)).astype(f32)
    for k in range(D):
        Aj = fma(rj[:, k], rj[:, k], Aj)
    Bh = (-(rh * rh)).astype(f32)
    for k in range(D):
        Bh = fma(xh[:, k], xh[:, k], Bh)
    dot = (rhoj * rh).astype(f32)
    for k in range(D):
        dot = fma(rj[:, k], xh[:, k], dot)
    return fma(np.full(len(xh), -2, f32), dot, (Aj + Bh).astype(f32))


@pytest.mark.parametrize("D", range(2, 11))
def test_expanded_pair_test_error_within_the_band(D):
    rng = np.random.default_rng(D)
    Lsc, skin, M = f32(1.5), f32(0.3), 100000
    xh = (rng.uniform(-0.5, 0.5, (M, D)) * Lsc).astype(f32)
    rj = (rng.uniform(-0.5, 0.5, (M, D)) * Lsc).astype(f32)
    # extreme magnitudes: corners of the home subcell and of the far neighbours
    xh[: M // 4] = (np.sign(rng.uniform(-1, 1, (M // 4, D))) * 0.5 * Lsc).astype(f32)
    rj[: M // 4] = (np.sign(rng.uniform(-1, 1, (M // 4, D))) * 0.5 * Lsc).astype(f32)
    off = rng.integers(-1, 2, (M, D)).astype(f32)
    rj = (rj + off * Lsc).astype(f32)                       # the row's offsets, in FP32
    rhoj = rng.uniform(0.4, 0.6, M).astype(f32)
    rh = (rng.uniform(0.4, 0.6, M).astype(f32) + skin).astype(f32)
    diff = expanded_diff(xh, rj, rhoj, rh)
    X, R = xh.astype(np.float64), rj.astype(np.float64)
    exact = ((R - X) ** 2).sum(1) - (rhoj.astype(np.float64) + rh.astype(np.float64)) ** 2
    widening = (D + 3) * (4 * D + 1) * 1.2e-7 * float(Lsc) ** 2
    err = np.abs(diff.astype(np.float64) - exact).max()
    assert err < 0.5 * widening, (err, widening)
