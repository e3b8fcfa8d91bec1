"""Seeded synthetic inputs for the d-dimensional soft-sphere workloads.

This module only draws inputs: diameters, positions in the periodic box,
velocities and SWAP candidate pairs.  It holds none of the method's
arithmetic (no binning, lists, forces or integration), imports nothing from
the CUDA binding or from the oracle, and is the one module both sides use.
All draws use numpy's PCG64 generator with an explicit seed.

The box side follows the paper's recipe (Sec. II.A): the particle volume is
the sum of d-sphere volumes (Eq. (2)) and L = (V_part / phi)^(1/d), with the
box centred at the origin.  The workloads below restate the benchmark
configurations; the paper measures on none of these (it has no public
dataset), so all of them are synthetic stand-ins.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def sphere_volume(d: int, sigma) -> np.ndarray:
    """Eq. (2): pi^(d/2) sigma^d / (2^d Gamma(1 + d/2))."""
    return math.pi ** (0.5 * d) * np.asarray(sigma, dtype=np.float64) ** d / (
        2.0 ** d * math.gamma(1.0 + 0.5 * d))


def box_side(d: int, sigma, phi: float) -> float:
    """L = (sum_i v(d, sigma_i) / phi)^(1/d) (Sec. II.A)."""
    return float((sphere_volume(d, sigma).sum() / phi) ** (1.0 / d))


def jamming_estimate(d: int) -> float:
    """The packing-fraction scale 1.5 d 2^-d, clamped to 0.7."""
    return min(1.5 * d * 2.0 ** (-d), 0.7)


@dataclass
class System:
    """Host-side description of one synthetic system (row-major x[N, d])."""
    d: int
    L: float
    sigma: np.ndarray
    x: np.ndarray
    v: np.ndarray
    mass: np.ndarray | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.sigma.shape[0])


def uniform_positions(rng, N: int, d: int, L: float) -> np.ndarray:
    """Uniform in the periodic box [-L/2, L/2)^d."""
    x = rng.uniform(-0.5 * L, 0.5 * L, size=(N, d))
    return np.where(x >= 0.5 * L, x - L, x)


def thermal_velocities(rng, N: int, d: int, T: float, mass=None) -> np.ndarray:
    """Gaussian N(0, T/m) per component, centre-of-mass motion removed, then
    rescaled so that the kinetic energy is d (N - 1) T / 2."""
    m = np.ones(N) if mass is None else np.asarray(mass, dtype=np.float64)
    v = rng.normal(size=(N, d)) * np.sqrt(T / m)[:, None]
    if T <= 0.0:
        return np.zeros((N, d))
    p = (m[:, None] * v).sum(axis=0) / m.sum()
    v -= p
    K = 0.5 * (m[:, None] * v * v).sum()
    return v * math.sqrt(0.5 * d * (N - 1) * T / K)


def bidisperse(rng, N: int, a: float = 1.0, b: float = 1.4) -> np.ndarray:
    """50:50 mixture of diameters a and b in random order."""
    s = np.where(np.arange(N) < N // 2, a, b).astype(np.float64)
    rng.shuffle(s)
    return s


def polydisperse(rng, N: int, lo: float = 0.8, hi: float = 1.2) -> np.ndarray:
    """Diameters uniform in [lo, hi]."""
    return rng.uniform(lo, hi, size=N)


def power_law_diameters(rng, N: int, d: int, R: float) -> np.ndarray:
    """Diameters from Eq. (3): P(sigma) proportional to sigma^-d on
    [R^(-1/2d), R^(1/2d)] (R = ratio of largest to smallest particle volume),
    by inverting its cumulative distribution."""
    lo, hi = R ** (-0.5 / d), R ** (0.5 / d)
    a, b = lo ** (1 - d), hi ** (1 - d)
    u = rng.random(N)
    return (a - u * (a - b)) ** (1.0 / (1 - d))


# Table III: packing fractions phi*_d of the paper's d = 3..6 benchmark runs
# (the hard-sphere dynamical glass transition mapped to the Morse law with
# a = 30 at T = 0.25).
PHI_STAR = {3: 0.5980, 4: 0.4232, 5: 0.2847, 6: 0.1850}
MORSE_A = 30.0      # Morse stiffness of the benchmark runs (Sec. II.A)
PAPER_DT = 0.0016   # time step 6/(125 a) (Sec. II.A)
PAPER_T = 0.25      # temperature of the benchmark runs (Sec. III)


def paper_model(d, N, phi=None, T=PAPER_T, seed=0, R=None):
    """The paper's own model (Sec. II.A): diameters from Eq. (3) with R = d,
    masses m_i = sigma_i^d (prefactors eps_i = sigma_i^d are the pair law's
    business), phi = phi*_d of Table III unless given, uniform positions,
    Gaussian velocities at T for those masses.  The random positions overlap
    badly: the paper removes that with a partial FIRE pushoff before MD."""
    rng = np.random.default_rng(seed)
    sigma = power_law_diameters(rng, N, d, float(d if R is None else R))
    phi = PHI_STAR[d] if phi is None else phi
    L = box_side(d, sigma, phi)
    x = uniform_positions(rng, N, d, L)
    mass = sigma ** d
    v = thermal_velocities(rng, N, d, T, mass)
    return System(d=d, L=float(L), sigma=sigma, x=x, v=v, mass=mass,
                  name="paper_model_d%d_N%d" % (d, N), meta=dict(phi=phi, T=T, seed=seed))


def make_system(d, N, *, phi=None, L=None, dist="poly", T=1e-3, seed=0, name=""):
    """One system: diameters, box, uniform positions, thermal velocities."""
    rng = np.random.default_rng(seed)
    sigma = bidisperse(rng, N) if dist == "bi" else polydisperse(rng, N)
    if L is None:
        L = box_side(d, sigma, phi)
    x = uniform_positions(rng, N, d, L)
    v = thermal_velocities(rng, N, d, T)
    return System(d=d, L=float(L), sigma=sigma, x=x, v=v, name=name,
                  meta=dict(phi=phi, T=T, seed=seed, dist=dist))


# ---------------------------------------------------------------- workloads
def c0_bidisperse_d3(seed=0):
    """d=3, N=1000, 50:50 diameters 1.0/1.4, phi=0.60, T=1e-3."""
    return make_system(3, 1000, phi=0.60, dist="bi", T=1e-3, seed=seed,
                       name="d3_N1000_bidisperse_phi0.60")


def c1_poly_d6(seed=0, N=32768):
    """d=6 polydisperse [0.8, 1.2]; N=32768 in a box of side 6 (about 6 mean
    diameters).  Larger N keeps the number density (L = 6 (N/32768)^(1/6))."""
    L = 6.0 * (N / 32768.0) ** (1.0 / 6.0)
    return make_system(6, N, L=L, dist="poly", T=1e-3, seed=seed,
                       name="d6_N%d_poly_L%.3g" % (N, L))


def c2_sweep(d, seed=0, N=65536):
    """Dimension sweep: polydisperse, phi = min(1.5 d 2^-d, 0.7), T = 0."""
    return make_system(d, N, phi=jamming_estimate(d), dist="poly", T=0.0, seed=seed,
                       name="d%d_N%d_poly_fire" % (d, N))


def c3_batch_specs(n_jobs=512, seed=0):
    """Batched FIRE jobs: N log-uniform in [256, 8192], d in {3,4,5,6},
    bidisperse, phi = U[0.6, 1.2] x min(1.5 d 2^-d, 0.7)."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(n_jobs):
        N = int(round(math.exp(rng.uniform(math.log(256), math.log(8192)))))
        d = int(rng.integers(3, 7))
        phi = float(rng.uniform(0.6, 1.2) * jamming_estimate(d))
        specs.append(dict(d=d, N=N, phi=phi, seed=seed * 100003 + k))
    return specs


def c3_job(spec):
    return make_system(spec["d"], spec["N"], phi=spec["phi"], dist="bi", T=0.0,
                       seed=spec["seed"], name="batch_job")


def swap_pairs(rng, N: int, npairs: int):
    """Candidate pairs (i != j, each uniform) and Metropolis uniforms in [0, 1)."""
    i = rng.integers(0, N, size=npairs)
    j = rng.integers(0, N - 1, size=npairs)
    j = j + (j >= i)
    u = rng.random(npairs)
    return np.stack([i, j], axis=1).astype(np.int32), u


def lattice(d: int, n: int, spacing: float = 1.0):
    """Hypercubic lattice Z^d with n sites per axis, in a box of side n*spacing,
    shifted so that every coordinate lies in [-L/2, L/2)."""
    g = np.stack(np.meshgrid(*([np.arange(n)] * d), indexing="ij"), axis=-1).reshape(-1, d)
    L = n * spacing
    x = (g + 0.5) * spacing - 0.5 * L
    return x.astype(np.float64), float(L)


def min_valid_N(d, phi, hi=1.2, lo=0.8):
    """Smallest N whose box (polydisperse U[lo, hi] at packing fraction phi)
    is longer than twice the largest diameter."""
    mean_v = float(np.mean(sphere_volume(d, np.linspace(lo, hi, 201))))
    return int(math.ceil(phi * (2.0 * hi * 1.02) ** d / mean_v))


def c4_requests(duration=2.0, rate=200.0, seed=0):
    """Poisson stream of MD and FIRE requests: arrivals at `rate` per second
    over `duration` seconds; 50 % MD (steps uniform in 1000..10000, T = 1e-3,
    dt = 0.005), 50 % FIRE; N lognormal with median 4096 and log-sd 1, clipped
    to [256, 131072] and raised where needed so that the box exceeds twice the
    largest diameter; d uniform in 3..8; polydisperse U[0.8, 1.2] at
    phi = min(1.5 d 2^-d, 0.7)."""
    rng = np.random.default_rng(seed)
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        d = int(rng.integers(3, 9))
        phi = jamming_estimate(d)
        N = int(np.clip(round(math.exp(rng.normal(math.log(4096), 1.0))), 256, 131072))
        N = max(N, min_valid_N(d, phi))
        kind = int(rng.integers(0, 2))
        steps = int(rng.integers(1000, 10001))
        reqs.append(dict(t=t, d=d, N=N, phi=phi, kind=kind, nsteps=steps,
                         seed=int(rng.integers(0, 2 ** 31))))
    return reqs


def c4_system(req):
    T = 1e-3 if req["kind"] == 0 else 0.0
    return make_system(req["d"], req["N"], phi=req["phi"], dist="poly", T=T, seed=req["seed"],
                       name="request")
