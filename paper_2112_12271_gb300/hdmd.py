"""Python binding of the hdmd C ABI (include/hdmd.h): argument marshalling only.

Every computation runs in the CUDA kernels of ``libhdmd.so``; this module
converts numpy arrays to the ABI's row-major host buffers and back.  There is
no CPU fallback: if the library is missing or no GPU is present, the calls
raise.  Functions keep the ABI's names; ``System`` bundles them around one
handle.  The CUDA stream defaults to PyTorch's current stream when PyTorch
is importable with a GPU, else the legacy default stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libhdmd.so")

HDMD_FP64, HDMD_MIXED = 0, 1
STATUS = {0: "HDMD_OK", 1: "HDMD_E_INVALID", 2: "HDMD_E_NOMEM", 3: "HDMD_E_NBR_OVERFLOW",
          4: "HDMD_E_LOST_ATOM", 5: "HDMD_E_NOT_CONVERGED", 6: "HDMD_E_CUDA",
          7: "HDMD_E_TIMEOUT", 8: "HDMD_E_UNSUPPORTED_D"}


class HDMDError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class Potential(C.Structure):
    _fields_ = [("kind", C.c_int), ("eps", C.c_double), ("skin", C.c_double),
                ("a", C.c_double), ("eps_scale", C.c_int), ("n_mie", C.c_int)]


LAWS = {"harmonic": 0, "morse": 1, "mie": 2}


def potential(eps=1.0, skin=0.3, law="harmonic", a=30.0, eps_scale=False, n=6):
    """The pair law of include/hdmd.h: harmonic, the Morse law of Eq. (1)
    (stiffness a) or the truncated and shifted Mie law (exponent n); one eps
    or volume-scaled prefactors eps sigma_i^d."""
    return Potential(LAWS[law], float(eps), float(skin), float(a), int(bool(eps_scale)), int(n))


class Thermo(C.Structure):
    _fields_ = [("E_pair", C.c_double), ("virial", C.c_double), ("K", C.c_double),
                ("T", C.c_double), ("P", C.c_double), ("steps", C.c_int64),
                ("rebuilds", C.c_int64)]


class FireParams(C.Structure):
    _fields_ = [("dt0", C.c_double), ("dt_max", C.c_double), ("dt_min", C.c_double),
                ("f_inc", C.c_double), ("f_dec", C.c_double), ("alpha0", C.c_double),
                ("f_alpha", C.c_double), ("f_tol", C.c_double), ("polish_tol", C.c_double),
                ("n_delay", C.c_int64), ("n_neg_max", C.c_int64), ("max_iter", C.c_int64),
                ("initial_delay", C.c_int), ("e_thres", C.c_double), ("f_thres", C.c_double),
                ("dx_max", C.c_double)]


class FireResult(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("polish_iterations", C.c_int64),
                ("rebuilds", C.c_int64), ("E_pair", C.c_double), ("fmax", C.c_double),
                ("converged", C.c_int)]


class Info(C.Structure):
    _fields_ = [("d", C.c_int), ("N", C.c_int64), ("L", C.c_double), ("n_cell", C.c_int),
                ("n_cells", C.c_int64), ("list_capacity", C.c_int), ("lanes_per_atom", C.c_int),
                ("max_list_length", C.c_int), ("total_list_entries", C.c_int64),
                ("precision", C.c_int), ("graphs", C.c_int), ("device_bytes", C.c_int64),
                ("resident", C.c_int)]


class JobSpec(C.Structure):
    _fields_ = [("kind", C.c_int), ("d", C.c_int), ("N", C.c_int64), ("L", C.c_double),
                ("eps", C.c_double), ("skin", C.c_double), ("dt", C.c_double),
                ("nsteps", C.c_int64), ("list_capacity", C.c_int), ("fire", FireParams)]


class JobResult(C.Structure):
    _fields_ = [("status", C.c_int), ("kind", C.c_int), ("iterations", C.c_int64),
                ("rebuilds", C.c_int64), ("E_pair", C.c_double), ("virial", C.c_double),
                ("K", C.c_double), ("fmax", C.c_double), ("converged", C.c_int),
                ("error", C.c_int)]


JOB_MD, JOB_FIRE = 0, 1
JOB_RUNNING, JOB_DONE, JOB_NOT_CONVERGED, JOB_ERROR = 0, 1, 2, 3

FIRE_DEFAULTS = dict(dt0=0.005, dt_max=0.05, dt_min=1e-4, f_inc=1.1, f_dec=0.5, alpha0=0.25,
                     f_alpha=0.99, f_tol=1e-10, polish_tol=1e-6, n_delay=20, n_neg_max=2000,
                     max_iter=1000000, initial_delay=1, e_thres=0.0, f_thres=0.0, dx_max=0.0)

_lib = None


def lib():
    """Load libhdmd.so; raise if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("hdmd CUDA library not built (%s missing); run "
                               "paper_2112_12271_gb300.build.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
        sig = {
            "create_system": [i32, i64, dbl, vp, vp, i32, vp, C.POINTER(vp)],
            "system_footprint": [i32, i64, dbl, vp, vp, i32, C.POINTER(i64)],
            "set_state": [vp, vp, vp, vp],
            "set_diameters": [vp, vp],
            "get_state": [vp, vp, vp, vp, vp, vp],
            "build_neighbors": [vp, i32, C.POINTER(i32)],
            "get_neighbors": [vp, vp, vp, C.POINTER(i64)],
            "compute_forces": [vp, C.POINTER(dbl), C.POINTER(dbl)],
            "md_steps": [vp, i64, dbl, vp],
            "set_thermostat": [vp, dbl, dbl],
            "set_reference": [vp, vp],
            "set_barostat": [vp, dbl, dbl, dbl, i64],
            "set_rebuild_rule": [vp, i32, i32],
            "set_list_radius": [vp, i32],
            "get_box": [vp, C.POINTER(dbl)],
            "observables": [vp, dbl, i32, dbl, vp, vp],
            "fire_minimize": [vp, vp, vp],
            "swap_sweep": [vp, i32, dbl, dbl, C.c_uint64, vp, vp, i64, C.POINTER(i64), vp],
            "get_info": [vp, vp],
            "set_tuning": [vp, i32, i32],
            "set_resident": [vp, i32],
            "destroy_system": [vp],
            "profile_kernels": [vp, i32, dbl, vp],
            "batch_create": [i64, i32, i32, vp, C.POINTER(vp)],
            "batch_add": [vp, vp, vp, vp, vp, C.POINTER(i32)],
            "batch_run": [vp, i64, C.POINTER(i32)],
            "batch_result": [vp, i32, vp, vp],
            "batch_remove": [vp, i32],
            "batch_info": [vp, C.POINTER(i64), C.POINTER(i32), vp],
            "batch_autotune": [vp, i32],
            "batch_set_lanes": [vp, i32, i32],
            "batch_destroy": [vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.hdmd_last_error.argtypes = [vp]
        L.hdmd_last_error.restype = C.c_char_p
        L.hdmd_batch_last_error.argtypes = [vp]
        L.hdmd_batch_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(st, h=None):
    if st != 0:
        msg = lib().hdmd_last_error(h).decode(errors="replace")
        raise HDMDError(st, msg)


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


# ------------------------------------------------------------------ ABI calls
def create_system(d, N, L, diameters, eps=1.0, skin=0.3, precision=HDMD_MIXED, stream=None,
                  law="harmonic", a=30.0, eps_scale=False, n=6):
    diam = _f64(diameters)
    if diam.shape != (N,):
        raise ValueError("diameters must have shape (N,)")
    pot = potential(eps, skin, law, a, eps_scale, n)
    h = C.c_void_p()
    st = lib().create_system(d, N, L, _p(diam), C.byref(pot), int(precision),
                             stream if stream is not None else default_stream(), C.byref(h))
    _check(st)
    return h


def system_footprint(d, N, L, diameters, eps=1.0, skin=0.3, precision=HDMD_MIXED,
                     law="harmonic", a=30.0, eps_scale=False, n=6):
    """Device bytes create_system would allocate (no device work)."""
    diam = _f64(diameters)
    if diam.shape != (N,):
        raise ValueError("diameters must have shape (N,)")
    pot = potential(eps, skin, law, a, eps_scale, n)
    b = C.c_int64(0)
    _check(lib().system_footprint(d, N, L, _p(diam), C.byref(pot), int(precision), C.byref(b)))
    return b.value


def set_state(h, x, v=None, masses=None):
    x = _f64(x)
    v = None if v is None else _f64(v)
    m = None if masses is None else _f64(masses)
    _check(lib().set_state(h, _p(x), _p(v), _p(m)), h)


def set_diameters(h, diameters):
    _check(lib().set_diameters(h, _p(_f64(diameters))), h)


def get_state(h, N, d, x=True, v=True, img=True, f=False, sigma=False):
    out = {}
    xa = np.empty((N, d)) if x else None
    va = np.empty((N, d)) if v else None
    ia = np.empty((N, d), dtype=np.int32) if img else None
    fa = np.empty((N, d)) if f else None
    sa = np.empty(N) if sigma else None
    _check(lib().get_state(h, _p(xa), _p(va), _p(ia), _p(fa), _p(sa)), h)
    for k, a in (("x", xa), ("v", va), ("img", ia), ("f", fa), ("sigma", sa)):
        if a is not None:
            out[k] = a
    return out


def get_state_into(h, x_out, v_out=None):
    """Positions (and velocities) copied into caller arrays of shape (N, d),
    float64, C-contiguous (pinned host memory makes the copy direct)."""
    for a in (x_out, v_out):
        if a is not None and (a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]):
            raise ValueError("output arrays must be C-contiguous float64")
    _check(lib().get_state(h, _p(x_out), _p(v_out), None, None, None), h)


def build_neighbors(h, force=True):
    r = C.c_int(0)
    _check(lib().build_neighbors(h, 1 if force else 0, C.byref(r)), h)
    return bool(r.value)


def get_neighbors(h, N):
    counts = np.empty(N, dtype=np.int32)
    tot = C.c_int64(0)
    _check(lib().get_neighbors(h, _p(counts), None, C.byref(tot)), h)
    idx = np.empty(max(tot.value, 1), dtype=np.int32)
    _check(lib().get_neighbors(h, _p(counts), _p(idx), C.byref(tot)), h)
    return counts, idx[:tot.value]


def compute_forces(h):
    e, w = C.c_double(), C.c_double()
    _check(lib().compute_forces(h, C.byref(e), C.byref(w)), h)
    return e.value, w.value


def md_steps(h, nsteps, dt):
    t = Thermo()
    _check(lib().md_steps(h, int(nsteps), float(dt), C.byref(t)), h)
    return {k: getattr(t, k) for k, _ in Thermo._fields_}


class Observables(C.Structure):
    _fields_ = [("msd", C.c_double), ("mqd", C.c_double), ("alpha2", C.c_double),
                ("f_ov", C.c_double), ("Z", C.c_double)]


def set_reference(h, x_ref=None):
    """Reference configuration for the observables (None: current positions)."""
    _check(lib().set_reference(h, _p(None if x_ref is None else _f64(x_ref))), h)


def observables(h, a_ov=0.0, nbins=0, r_max=0.0):
    """dict(msd, mqd, alpha2, f_ov, Z) and, with nbins > 0, the G_s histogram."""
    o = Observables()
    gs = np.zeros(max(nbins, 1))
    _check(lib().observables(h, float(a_ov), int(nbins), float(r_max), C.byref(o),
                             _p(gs) if nbins > 0 else None), h)
    out = {k: getattr(o, k) for k, _ in Observables._fields_}
    if nbins > 0:
        out["G_s"] = gs[:nbins]
    return out


def set_barostat(h, P_target, tau_P, beta=1.0, n_baro=10):
    """Berendsen NPT for later md_steps (tau_P <= 0: fixed box)."""
    _check(lib().set_barostat(h, float(P_target), float(tau_P), float(beta), int(n_baro)), h)


def set_rebuild_rule(h, rule="exact", n_bet=1):
    """List rebuild rule: "exact" (default) or the paper's, every n_bet steps."""
    _check(lib().set_rebuild_rule(h, {"exact": 0, "paper": 1}[rule], int(n_bet)), h)


def get_box(h):
    L = C.c_double()
    _check(lib().get_box(h, C.byref(L)), h)
    return L.value


def set_thermostat(h, T_target, tau):
    """Berendsen NVT for later md_steps (tau <= 0: back to NVE)."""
    _check(lib().set_thermostat(h, float(T_target), float(tau)), h)


def fire_minimize(h, raise_on_fail=False, **params):
    p = dict(FIRE_DEFAULTS)
    p.update(params)
    fp = FireParams(**p)
    r = FireResult()
    st = lib().fire_minimize(h, C.byref(fp), C.byref(r))
    if st not in (0, 5) or (st == 5 and raise_on_fail):
        _check(st, h)
    out = {k: getattr(r, k) for k, _ in FireResult._fields_}
    out["status"] = st
    return out


def swap_sweep(h, T, p=0.1, nsweeps=1, seed=0, pairs=None, uniforms=None):
    acc = C.c_int64(0)
    if pairs is not None:
        pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        u = _f64(uniforms)
        flags = np.zeros(len(pr), dtype=np.uint8)
        _check(lib().swap_sweep(h, 1, float(T), float(p), C.c_uint64(seed), _p(pr), _p(u),
                                len(pr), C.byref(acc), _p(flags)), h)
        return acc.value, flags.astype(bool)
    _check(lib().swap_sweep(h, int(nsweeps), float(T), float(p), C.c_uint64(seed), None, None,
                            0, C.byref(acc), None), h)
    return acc.value, None


def get_info(h):
    i = Info()
    _check(lib().get_info(h, C.byref(i)), h)
    return {k: getattr(i, k) for k, _ in Info._fields_}


def set_tuning(h, lanes_per_atom=0, use_graphs=-1):
    _check(lib().set_tuning(h, int(lanes_per_atom), int(use_graphs)), h)


def profile_kernels(h, reps=50, dt=0.005):
    """Average device ms of (fused MD kernel, full list build, force-only
    kernel, resident MD kernel per step)."""
    out = np.zeros(4)
    _check(lib().profile_kernels(h, int(reps), float(dt), _p(out)), h)
    return dict(step_ms=out[0], rebuild_ms=out[1], force_ms=out[2], resident_step_ms=out[3])


def destroy_system(h):
    if h:
        _check(lib().destroy_system(h))


class System:
    """One resident system: the ABI calls bound to a handle."""

    def __init__(self, d, L, diameters, x=None, v=None, masses=None, eps=1.0, skin=0.3,
                 precision=HDMD_MIXED, stream=None, law="harmonic", a=30.0, eps_scale=False,
                 n=6):
        self.d, self.L = int(d), float(L)
        self.N = int(np.asarray(diameters).shape[0])
        self.h = create_system(self.d, self.N, self.L, diameters, eps, skin, precision, stream,
                               law, a, eps_scale, n)
        if x is not None:
            self.set_state(x, v, masses)

    def set_state(self, x, v=None, masses=None):
        set_state(self.h, x, v, masses)

    def set_diameters(self, diameters):
        set_diameters(self.h, diameters)

    def state(self, **kw):
        return get_state(self.h, self.N, self.d, **kw)

    def state_into(self, x_out, v_out=None):
        get_state_into(self.h, x_out, v_out)

    def build_neighbors(self, force=True):
        return build_neighbors(self.h, force)

    def neighbors(self):
        return get_neighbors(self.h, self.N)

    def forces(self):
        e, w = compute_forces(self.h)
        f = get_state(self.h, self.N, self.d, x=False, v=False, img=False, f=True)["f"]
        return f, e, w

    def md_steps(self, nsteps, dt):
        return md_steps(self.h, nsteps, dt)

    def thermostat(self, T_target, tau):
        set_thermostat(self.h, T_target, tau)

    def barostat(self, P_target, tau_P, beta=1.0, n_baro=10):
        set_barostat(self.h, P_target, tau_P, beta, n_baro)

    def box(self):
        return get_box(self.h)

    def rebuild_rule(self, rule="exact", n_bet=1):
        set_rebuild_rule(self.h, rule, n_bet)

    def list_radius(self, global_radius=False):
        """Per-pair list radius sigma_ij + s, or the paper's sigma_max + s."""
        _check(lib().set_list_radius(self.h, int(bool(global_radius))), self.h)

    def set_reference(self, x_ref=None):
        set_reference(self.h, x_ref)

    def observables(self, a_ov=0.0, nbins=0, r_max=0.0):
        return observables(self.h, a_ov, nbins, r_max)

    def fire(self, **params):
        return fire_minimize(self.h, **params)

    def swap(self, T, **kw):
        return swap_sweep(self.h, T, **kw)

    def info(self):
        return get_info(self.h)

    def tune(self, lanes_per_atom=0, use_graphs=-1):
        set_tuning(self.h, lanes_per_atom, use_graphs)

    def resident(self, on=True):
        """Resident MD kernel on or off (see set_resident in hdmd.h)."""
        _check(lib().set_resident(self.h, 1 if on else 0), self.h)

    def profile(self, reps=50, dt=0.005):
        return profile_kernels(self.h, reps, dt)

    def close(self):
        if self.h:
            destroy_system(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batches
def _bcheck(st, b=None):
    if st != 0:
        raise HDMDError(st, lib().hdmd_batch_last_error(b).decode(errors="replace"))


class Batch:
    """Many independent MD / FIRE jobs advanced by persistent kernels (batch_* ABI)."""

    def __init__(self, pool_bytes=1 << 30, max_jobs=1024, precision=HDMD_MIXED, stream=None):
        self.h = C.c_void_p()
        _bcheck(lib().batch_create(int(pool_bytes), int(max_jobs), int(precision),
                                   stream if stream is not None else default_stream(),
                                   C.byref(self.h)))
        self.meta = {}

    def add(self, kind, d, L, diameters, x, v=None, eps=1.0, skin=0.3, dt=0.005, nsteps=0,
            list_capacity=0, **fire):
        diam = _f64(diameters)
        N = diam.shape[0]
        p = dict(FIRE_DEFAULTS)
        p.update(fire)
        spec = JobSpec(int(kind), int(d), int(N), float(L), float(eps), float(skin), float(dt),
                       int(nsteps), int(list_capacity), FireParams(**p))
        xx = _f64(x)
        vv = None if v is None else _f64(v)
        jid = C.c_int(-1)
        st = lib().batch_add(self.h, C.byref(spec), _p(diam), _p(xx), _p(vv), C.byref(jid))
        if st == 2:
            return None          # no room now (pool or job table)
        _bcheck(st, self.h)
        self.meta[jid.value] = (N, int(d))
        return jid.value

    def run(self, budget=0):
        left = C.c_int(0)
        _bcheck(lib().batch_run(self.h, int(budget), C.byref(left)), self.h)
        return left.value

    def result(self, jid, positions=False):
        r = JobResult()
        N, d = self.meta[jid]
        x = np.empty((N, d)) if positions else None
        _bcheck(lib().batch_result(self.h, int(jid), C.byref(r), _p(x)), self.h)
        out = {k: getattr(r, k) for k, _ in JobResult._fields_}
        if positions:
            out["x"] = x
        return out

    def remove(self, jid):
        _bcheck(lib().batch_remove(self.h, int(jid)), self.h)
        self.meta.pop(jid, None)

    def info(self):
        fb, lj = C.c_int64(0), C.c_int(0)
        lanes = np.zeros(11, dtype=np.int32)
        _bcheck(lib().batch_info(self.h, C.byref(fb), C.byref(lj), _p(lanes)), self.h)
        return dict(free_bytes=fb.value, live_jobs=lj.value, lanes=lanes.tolist())

    def autotune(self, reps=3):
        _bcheck(lib().batch_autotune(self.h, int(reps)), self.h)

    def set_lanes(self, d, lanes):
        _bcheck(lib().batch_set_lanes(self.h, int(d), int(lanes)), self.h)

    def close(self):
        if self.h:
            lib().batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
