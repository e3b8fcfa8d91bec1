"""Plain FP64 CPU oracle for the d-dimensional soft-sphere MD hot path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never imports, links or
executes anything here, and this package imports nothing from the product.

The arithmetic lives in ``hdmd_oracle.c`` (serial C, double precision, every
function citing the passage of arXiv:2112.12271 it follows).  This module
compiles it with gcc on first use and wraps it with ctypes + numpy.  Arrays
are row-major ``x[N, d]``.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  sphere_volume, n_cell, cell_index ... closed forms, hand-built examples
  neighbors_brute / neighbors_cells .. each other, hypercubic-lattice counts
                                       (2d, 2d^2), symmetry, O(N^2) brute force
  neighbors_of / force_on ............ rows of the all-pairs routines,
                                       lattice counts, shares summing to E, W
  forces ............................. two-body closed form, central finite
                                       differences of E, Newton's third law,
                                       virial = -sum x.grad U (both laws)
  mie ................................ the textbook WCA form for n = 6,
                                       closed-form values for other n
  morse / law ........................ closed-form values of Eq. (1), the
                                       volume-scaled prefactors on two bodies
  sigma_eff .......................... Table III of the paper (4 digits)
  observables ........................ uniform translation in closed form,
                                       alpha2 -> 0 for Gaussian displacements,
                                       Z on hypercubic lattices (2d, 2d^2)
  md_steps ........................... time reversibility, energy drift ~ dt^2,
                                       head-on two-body collision; Berendsen:
                                       ideal-gas relaxation in closed form
  md_npt ............................. ideal-gas volume relaxation in closed
                                       form
  fire ............................... |F|max < 1e-10, E -> 0 below jamming,
                                       two spheres relax to contact
  swap ............................... brute dE, equal diameters always
                                       accepted, exact detailed balance (3 atoms)
  philox4x32_10 ...................... published known-answer vectors
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hdmd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FMA contraction) into oracle/_build.
    openmp=True builds the threaded variant used only to time the oracle on
    all host cores (the tests use the serial build)."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO_OMP if openmp else _SO
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + ".tmp.%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared"]
            + (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)
    return so


def _load(openmp: bool = False):
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if openmp else _lib) is None:
            lib = C.CDLL(build(openmp=openmp))
            i64, i32, dbl, vp = C.c_int64, C.c_int, C.c_double, C.c_void_p
            lib.orc_sphere_volume.restype = dbl
            lib.orc_sphere_volume.argtypes = [i32, dbl]
            lib.orc_n_cell.restype = i32
            lib.orc_n_cell.argtypes = [dbl, dbl]
            lib.orc_cell_index.restype = i64
            lib.orc_cell_index.argtypes = [i32, i32, vp]
            lib.orc_min_image.restype = dbl
            lib.orc_min_image.argtypes = [dbl, dbl]
            for fn in (lib.orc_neighbors_brute, lib.orc_neighbors_cells):
                fn.restype = i64
                fn.argtypes = [i32, i64, dbl, vp, vp, dbl, i32, vp, vp, i64]
            lib.orc_neighbors_of.restype = i64
            lib.orc_neighbors_of.argtypes = [i32, i64, dbl, vp, vp, dbl, i32, i64, vp, i64]
            lib.orc_force_on.restype = None
            lib.orc_force_on.argtypes = [i32, i64, dbl, vp, vp, dbl, i64, vp,
                                         C.POINTER(dbl), C.POINTER(dbl)]
            lib.orc_morse.restype = dbl
            lib.orc_morse.argtypes = [dbl, dbl, dbl, dbl, C.POINTER(dbl)]
            lib.orc_mie.restype = dbl
            lib.orc_mie.argtypes = [dbl, dbl, dbl, i32, C.POINTER(dbl)]
            lib.orc_set_law.restype = i32
            lib.orc_set_law.argtypes = [i32, dbl, i32]
            lib.orc_sigma_eff.restype = dbl
            lib.orc_sigma_eff.argtypes = [dbl, dbl, i64]
            lib.orc_observables.restype = None
            lib.orc_observables.argtypes = [i32, i64, dbl, vp, vp, vp, dbl, i32, dbl, vp, vp]
            lib.orc_harmonic.restype = dbl
            lib.orc_harmonic.argtypes = [dbl, dbl, dbl, C.POINTER(dbl)]
            lib.orc_forces.restype = None
            lib.orc_forces.argtypes = [i32, i64, dbl, vp, vp, dbl, vp, vp, vp,
                                       C.POINTER(dbl), C.POINTER(dbl)]
            lib.orc_kinetic.restype = dbl
            lib.orc_kinetic.argtypes = [i32, i64, vp, vp]
            lib.orc_md_steps.restype = i64
            lib.orc_md_steps.argtypes = [i32, i64, dbl, vp, vp, vp, vp, vp, dbl, dbl,
                                         dbl, i64, vp, i32, vp, dbl, dbl, i32, i64, vp]
            lib.orc_md_npt.restype = i64
            lib.orc_md_npt.argtypes = [i32, i64, vp, vp, vp, vp, vp, vp, dbl, dbl, dbl, i64,
                                       dbl, dbl, dbl, dbl, dbl, i64, vp, vp]
            lib.orc_fire.restype = i32
            lib.orc_fire.argtypes = [i32, i64, dbl, vp, vp, vp, vp, vp, dbl, dbl, vp,
                                     vp, vp]
            lib.orc_swap.restype = i64
            lib.orc_swap.argtypes = [i32, i64, dbl, vp, vp, vp, vp, dbl, dbl, i64, vp,
                                     vp, vp]
            lib.orc_philox4x32_10.restype = None
            lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
            lib.orc_swap_draw.restype = None
            lib.orc_swap_draw.argtypes = [C.c_uint64, i64, i64, i64, vp, vp]
            lib.orc_set_threads.restype = i32
            lib.orc_set_threads.argtypes = [i32]
            if openmp:
                _lib_omp = lib
            else:
                _lib = lib
    return _lib_omp if openmp else _lib


def set_threads(n: int) -> int:
    """Threads of the OpenMP build for later calls with threads > 1; returns
    the count it will use."""
    return int(_load(openmp=True).orc_set_threads(int(n)))


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------- geometry
def sphere_volume(d: int, sigma: float) -> float:
    """Eq. (2): volume of a d-sphere of diameter sigma."""
    return _load().orc_sphere_volume(d, sigma)


def n_cell(L: float, rc_max: float) -> int:
    """Eq. (7): subcells per axis."""
    return _load().orc_n_cell(L, rc_max)


def cell_index(d: int, n: int, C_: np.ndarray) -> int:
    """Eq. (9): linear subcell index, axis 1 most significant."""
    c = np.ascontiguousarray(C_, dtype=np.int32)
    return _load().orc_cell_index(d, n, _p(c))


def min_image(dx: float, L: float) -> float:
    return _load().orc_min_image(dx, L)


# --------------------------------------------------------------- lists
def _neighbors(fn, x, sigma, L, skin, global_cut):
    x = _f64(x)
    N, d = x.shape
    sigma = _f64(sigma)
    counts = np.zeros(N, dtype=np.int32)
    tot = fn(d, N, L, _p(x), _p(sigma), skin, int(global_cut), _p(counts), None, 0)
    if tot < 0:
        raise ValueError("oracle neighbor build failed (%d)" % tot)
    idx = np.zeros(max(tot, 1), dtype=np.int32)
    tot2 = fn(d, N, L, _p(x), _p(sigma), skin, int(global_cut), _p(counts), _p(idx), tot)
    assert tot2 == tot
    return counts, idx[:tot]


def neighbors_brute(x, sigma, L, skin, global_cut=False):
    """Full Verlet lists by all-pairs search; (counts[N], idx[sum]) ascending."""
    return _neighbors(_load().orc_neighbors_brute, x, sigma, L, skin, global_cut)


def neighbors_cells(x, sigma, L, skin, global_cut=False):
    """Full Verlet lists with the linked-subcell loop nest of Sec. II.C."""
    return _neighbors(_load().orc_neighbors_cells, x, sigma, L, skin, global_cut)


def neighbors_of(x, sigma, L, skin, i, global_cut=False):
    """The list of atom i alone (ascending), by the all-pairs definition."""
    x = _f64(x)
    N, d = x.shape
    sigma = _f64(sigma)
    lib = _load()
    c = lib.orc_neighbors_of(d, N, L, _p(x), _p(sigma), skin, int(global_cut), int(i), None, 0)
    idx = np.zeros(max(c, 1), dtype=np.int32)
    c2 = lib.orc_neighbors_of(d, N, L, _p(x), _p(sigma), skin, int(global_cut), int(i), _p(idx), c)
    assert c2 == c
    return idx[:c]


def lists_as_sets(counts, idx):
    out, off = [], 0
    for c in counts:
        out.append(set(int(j) for j in idx[off:off + c]))
        off += c
    return out


# --------------------------------------------------------------- forces
def harmonic(r: float, s: float, eps: float = 1.0):
    """(U, |f|/r) of the harmonic soft-sphere law."""
    fr = C.c_double()
    u = _load().orc_harmonic(r, s, eps, C.byref(fr))
    return u, fr.value


def morse(r: float, s: float, eps: float = 1.0, a: float = 30.0):
    """(U, |f|/r) of the truncated and shifted Morse law, Eq. (1)."""
    fr = C.c_double()
    u = _load().orc_morse(r, s, eps, a, C.byref(fr))
    return u, fr.value


def mie(r: float, s: float, eps: float = 1.0, n: int = 6):
    """(U, |f|/r) of the Mie law truncated at r = s and shifted (Sec. II.A)."""
    fr = C.c_double()
    u = _load().orc_mie(r, s, eps, int(n), C.byref(fr))
    return u, fr.value


def sigma_eff(a: float, T: float, npts: int = 200000) -> float:
    """Effective hard-sphere diameter of the Morse law, Eq. (12)."""
    return _load().orc_sigma_eff(a, T, npts)


class law:
    """Context manager selecting the pair law of every oracle routine:
    kind "harmonic", "morse" (stiffness a) or "mie" (exponent n = a),
    eps_scale for the volume-scaled
    prefactors eps_i = eps sigma_i^d mixed as sqrt(eps_i eps_j).  The setting
    is process-wide while the block runs; the harmonic law with one eps is
    restored on exit."""

    def __init__(self, kind="harmonic", a=30.0, eps_scale=False):
        self.args = ({"harmonic": 0, "morse": 1, "mie": 2}[kind], float(a), int(bool(eps_scale)))

    def __enter__(self):
        if _load().orc_set_law(*self.args) != 0:
            raise ValueError("bad pair law")
        return self

    def __exit__(self, *exc):
        _load().orc_set_law(0, 30.0, 0)
        return False


def forces(x, sigma, L, eps=1.0, lists=None):
    """(F[N,d], E_pair, W) by brute force, or over full lists (counts, idx)."""
    x = _f64(x)
    N, d = x.shape
    sigma = _f64(sigma)
    F = np.zeros_like(x)
    E, W = C.c_double(), C.c_double()
    if lists is None:
        cnt = idx = None
    else:
        cnt = np.ascontiguousarray(lists[0], dtype=np.int32)
        idx = np.ascontiguousarray(lists[1], dtype=np.int32)
        if idx.size == 0:
            idx = np.zeros(1, dtype=np.int32)
    _load().orc_forces(d, N, L, _p(x), _p(sigma), eps, _p(cnt), _p(idx), _p(F),
                       C.byref(E), C.byref(W))
    return F, E.value, W.value


def force_on(x, sigma, L, i, eps=1.0):
    """(F_i[d], e_i, w_i): force on atom i over all other atoms and its half
    shares of the pair energy and virial."""
    x = _f64(x)
    N, d = x.shape
    sigma = _f64(sigma)
    Fi = np.zeros(d)
    e, w = C.c_double(), C.c_double()
    _load().orc_force_on(d, N, L, _p(x), _p(sigma), eps, int(i), _p(Fi), C.byref(e), C.byref(w))
    return Fi, e.value, w.value


def observables(x, xref, sigma, L, a, nbins=0, r_max=1.0):
    """dict(msd, mqd, alpha2, f_ov, Z[, G_s]) of unwrapped x against xref
    (sigma None: Z is not computed)."""
    x = _f64(x)
    N, d = x.shape
    out = np.zeros(5)
    gs = np.zeros(max(nbins, 1))
    sg = None if sigma is None else _f64(sigma)
    _load().orc_observables(d, N, L, _p(x), _p(_f64(xref)), _p(sg), float(a),
                            int(nbins), float(r_max), _p(out), _p(gs))
    r = dict(msd=out[0], mqd=out[1], alpha2=out[2], f_ov=out[3], Z=out[4])
    if nbins > 0:
        r["G_s"] = gs[:nbins]
    return r


def kinetic(v, mass=None):
    v = _f64(v)
    N, d = v.shape
    m = None if mass is None else _f64(mass)
    return _load().orc_kinetic(d, N, _p(v), _p(m))


# --------------------------------------------------------------- integrators
def md_steps(x, v, sigma, L, nsteps, dt, skin=0.3, eps=1.0, mass=None, img=None, F=None,
             T_target=0.0, tau=0.0, rule="exact", n_bet=1, step=0, openmp=False):
    """Velocity Verlet on copies (NVE, or NVT with the Berendsen factor
    when tau > 0), lists rebuilt by the exact rule or the paper's (checked
    every n_bet steps, step = steps already counted); returns dict(x, v, img,
    F, E, W, K, builds, step).  openmp=True runs the threaded build (for
    timing; its E and W may differ from the serial build's in rounding)."""
    x = _f64(x).copy()
    v = _f64(v).copy()
    N, d = x.shape
    sigma = _f64(sigma)
    m = None if mass is None else _f64(mass)
    img = np.zeros((N, d), dtype=np.int32) if img is None else np.array(img, dtype=np.int32)
    have_F = F is not None
    F = np.zeros_like(x) if F is None else _f64(F).copy()
    th = np.zeros(3)
    stp = np.array([int(step)], dtype=np.int64)
    b = _load(openmp).orc_md_steps(d, N, L, _p(x), _p(v), _p(img), _p(sigma), _p(m), eps, skin,
                             dt, int(nsteps), _p(F), int(have_F), _p(th), float(T_target),
                             float(tau), {"exact": 0, "paper": 1}[rule], int(n_bet), _p(stp))
    return dict(x=x, v=v, img=img, F=F, E=th[0], W=th[1], K=th[2], builds=int(b),
                step=int(stp[0]))


def md_npt(x, v, sigma, L, nsteps, dt, P_target, tau_P, beta, n_baro, skin=0.3, eps=1.0,
           mass=None, img=None, T_target=0.0, tau=0.0, count=0):
    """NPT with the Berendsen barostat on copies: dict(x, v, img, L, E, W, K,
    rescales, count)."""
    x = _f64(x).copy()
    v = _f64(v).copy()
    N, d = x.shape
    m = None if mass is None else _f64(mass)
    img = np.zeros((N, d), dtype=np.int32) if img is None else np.array(img, dtype=np.int32)
    Lb = np.array([float(L)])
    cnt = np.array([int(count)], dtype=np.int64)
    th = np.zeros(3)
    n = _load().orc_md_npt(d, N, _p(Lb), _p(x), _p(v), _p(img), _p(_f64(sigma)), _p(m), eps,
                           skin, dt, int(nsteps), float(T_target), float(tau), float(P_target),
                           float(tau_P), float(beta), int(n_baro), _p(cnt), _p(th))
    if n < 0:
        raise ValueError("barostat step would make the box vanish")
    return dict(x=x, v=v, img=img, L=float(Lb[0]), E=th[0], W=th[1], K=th[2], rescales=int(n),
                count=int(cnt[0]))


FIRE_DEFAULTS = dict(dt0=0.005, dt_max=0.05, dt_min=1e-4, f_inc=1.1, f_dec=0.5,
                     alpha0=0.25, f_alpha=0.99, f_tol=1e-10, n_delay=20, n_neg_max=2000,
                     max_iter=1000000, initial_delay=1, e_thres=0.0, f_thres=0.0, dx_max=0.0)


class _FireParams(C.Structure):
    _fields_ = [("dt0", C.c_double), ("dt_max", C.c_double), ("dt_min", C.c_double),
                ("f_inc", C.c_double), ("f_dec", C.c_double), ("alpha0", C.c_double),
                ("f_alpha", C.c_double), ("f_tol", C.c_double), ("n_delay", C.c_int64),
                ("n_neg_max", C.c_int64), ("max_iter", C.c_int64),
                ("initial_delay", C.c_int), ("e_thres", C.c_double), ("f_thres", C.c_double),
                ("dx_max", C.c_double)]


def fire(x, sigma, L, skin=0.3, eps=1.0, mass=None, **params):
    """FIRE 2.0 minimisation; returns dict(x, F, E, fmax, iters, status, builds)."""
    p = dict(FIRE_DEFAULTS)
    p.update(params)
    fp = _FireParams(**p)
    x = _f64(x).copy()
    N, d = x.shape
    v = np.zeros_like(x)
    F = np.zeros_like(x)
    img = np.zeros((N, d), dtype=np.int32)
    sigma = _f64(sigma)
    m = None if mass is None else _f64(mass)
    out = np.zeros(4)
    st = _load().orc_fire(d, N, L, _p(x), _p(v), _p(img), _p(sigma), _p(m), eps, skin,
                          C.addressof(fp), _p(F), _p(out))
    return dict(x=x, v=v, img=img, F=F, E=out[1], fmax=out[2], iters=int(out[0]),
                status=int(st), builds=int(out[3]))


# --------------------------------------------------------------- SWAP
def swap(x, sigma, L, T, pairs, uniforms, eps=1.0, mass=None, v=None):
    """Serial SWAP pass; returns dict(sigma, mass, v, accepted[npairs], naccepted)."""
    x = _f64(x)
    N, d = x.shape
    sigma = _f64(sigma).copy()
    m = None if mass is None else _f64(mass).copy()
    vv = None if v is None else _f64(v).copy()
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    u = _f64(uniforms)
    acc = np.zeros(len(pairs), dtype=np.int8)
    n = _load().orc_swap(d, N, L, _p(x), _p(sigma), _p(m), _p(vv), eps, T, len(pairs),
                         _p(pairs), _p(u), _p(acc))
    return dict(sigma=sigma, mass=m, v=vv, accepted=acc.astype(bool), naccepted=int(n))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def swap_draw(seed: int, sweep: int, npairs: int, N: int):
    """The seeded candidate pairs and uniforms of one SWAP pass."""
    pairs = np.zeros((npairs, 2), dtype=np.int32)
    u = np.zeros(npairs)
    _load().orc_swap_draw(seed, sweep, npairs, N, _p(pairs), _p(u))
    return pairs, u
